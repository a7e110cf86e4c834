"""The debug-bounds build on the GPU (libsg_debug.so, every instrumented
kernel access checked against the extent of its array; see sg_debug_bounds
in include/sg.h).  A fresh process loads it (SG_DEBUG_BOUNDS=1):

* the probe records an index outside its limit (site 901, the index, the
  limit) and skips the access, and records nothing for one inside;
* the apply (FP64, double-word, transposed; ragged 2D and 3D), the multigrid
  preconditioner in FP64 / FP32 / bf16 under every level variant, FGMRES and
  its transpose, a Monte-Carlo batch and the adjoint gradient record no
  violation, and the debug apply still matches the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_records_nothing_on_the_product_paths(cuda):
    from paper_2605_21046_gb300 import build
    build.build(debug_bounds=True)
    env = dict(os.environ, SG_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_worker.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == "libsg_debug.so"
    assert out["probe_inside"]["enabled"] == 1 and out["probe_inside"]["count"] == 0
    po = out["probe_outside"]
    assert (po["count"], po["site"], po["index"], po["limit"]) == (1, 901, 12, 8)
    assert out["probe_negative"]["count"] == 1 and out["probe_negative"]["index"] == -1
    for stage in ("after_applies", "after_multigrid", "after_mc_adjoint"):
        assert out[stage]["count"] == 0, (stage, out[stage])
    assert out["apply_rel_err"] < 1e-12

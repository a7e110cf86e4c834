"""The debug-bounds build and its entry points without a GPU: the release
library reports that no device checks are compiled in (without touching a
device) and refuses a probe index outside the probe array before any launch;
the instrumented units compile with -DSG_DEBUG_BOUNDS."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2605_21046_gb300 import _abi, build


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi.load()


def test_release_library_has_no_device_checks(lib):
    en, cnt, site, idx, lim = C.c_int(7), C.c_uint(7), C.c_int(7), C.c_longlong(7), C.c_longlong(7)
    assert lib.sg_debug_bounds(C.byref(en), C.byref(cnt), C.byref(site), C.byref(idx), C.byref(lim)) == _abi.SG_OK
    assert (en.value, cnt.value, site.value, idx.value, lim.value) == (0, 0, 0, 0, 0)
    assert lib.sg_debug_bounds(None, None, None, None, None) == _abi.SG_ERR_ARG


def test_release_probe_refuses_out_of_range_indices(lib):
    assert lib.sg_debug_bounds_probe(8, 8) == _abi.SG_ERR_ARG
    assert lib.sg_debug_bounds_probe(-1, 8) == _abi.SG_ERR_ARG
    assert lib.sg_debug_bounds_probe(0, 17) == _abi.SG_ERR_ARG      # limit beyond the probe array


@pytest.mark.parametrize("unit", ["sg_debug.cu", "sg_vanka_factor.cu"])
def test_instrumented_units_compile(unit, tmp_path):
    cmd = [build._nvcc(), "-DSG_DEBUG_BOUNDS=1", "-O1", "-std=c++17", "-Xcompiler", "-fPIC", *build.ARCH,
           "-I", os.path.join(build.PKG, "..", "include"), "-c", os.path.join(build.CSRC, unit),
           "-o", str(tmp_path / "u.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

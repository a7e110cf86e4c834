"""The C-ABI library loads and exports every function include/sg.h declares;
argument errors are reported before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?((?:sg|mc)_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_21046_gb300 import _abi, build
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    from paper_2605_21046_gb300 import _abi
    assert sorted(_abi.EXPORTED) == names


def test_status_strings(lib):
    assert lib.sg_status_string(0) == b"ok"
    assert lib.sg_status_string(4) == b"unsupported configuration"


def _setup_status(lib, **kw):
    from paper_2605_21046_gb300 import _abi, _coeff_struct, mesh_spec
    dim = kw.get("dim", 2)
    mesh = mesh_spec(dim, kw.get("cells", (4, 4, 4)), (0, 0, 0), (1, 1, 1))
    pieces = kw.get("pieces", [dict(mu=(0,), amp=1.0, factors=[("one", 0)] * dim)])
    cs, keep = _coeff_struct(pieces, 1, dim)
    h = C.c_void_p()
    st = lib.sg_setup(C.byref(mesh), kw.get("k", 1), kw.get("r", 1), kw.get("slabs", 4), kw.get("T", 1.0),
                      1, kw.get("P", 2), C.byref(cs), kw.get("prec", 0), C.byref(h))
    return st, h


def test_setup_rejects_bad_arguments_without_device_work(lib):
    from paper_2605_21046_gb300 import _abi
    assert _setup_status(lib, dim=4)[0] == _abi.SG_ERR_UNSUPPORTED
    assert _setup_status(lib, k=5)[0] == _abi.SG_ERR_UNSUPPORTED
    assert _setup_status(lib, dim=3, k=3)[0] == _abi.SG_ERR_UNSUPPORTED
    assert _setup_status(lib, r=7)[0] == _abi.SG_ERR_UNSUPPORTED
    assert _setup_status(lib, slabs=0)[0] == _abi.SG_ERR_ARG
    assert _setup_status(lib, T=-1.0)[0] == _abi.SG_ERR_ARG
    assert _setup_status(lib, cells=(0, 4, 4))[0] == _abi.SG_ERR_ARG
    assert _setup_status(lib, prec=9)[0] == _abi.SG_ERR_UNSUPPORTED
    assert _setup_status(lib, pieces=[dict(mu=(0,), amp=1.0, factors=[("pow", -1), ("one", 0)])])[0] == _abi.SG_ERR_ARG
    assert b"sg_setup" in lib.sg_last_error()
    # NULL arguments
    assert lib.sg_apply(None, 0, None, None, 0, None) == _abi.SG_ERR_ARG
    assert lib.sg_get_info(None, None) == _abi.SG_ERR_ARG
    assert lib.sg_apply_host(None, 0, None, None, 0) == _abi.SG_ERR_ARG
    assert lib.sg_apply_host_async(None, 0, None, None, 0, None) == _abi.SG_ERR_ARG
    assert b"sg_apply_host_async" in lib.sg_last_error()
    assert lib.sg_set_apply_shape(None, 1, 32, 0) == _abi.SG_ERR_ARG
    assert lib.sg_autotune(None, 3) == _abi.SG_ERR_ARG
    lib.sg_destroy(None)

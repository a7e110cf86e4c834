"""The allocation-free host-buffer apply (sg_apply_host_static) is for
callers that cannot let the library allocate device memory when they call it
(a memory pool that owns the device, paths that must not stall or fail on an
allocation).  Called through the C ABI it gives the same result as the
allocating host-buffer apply (sg_apply_host) and as the oracle's apply on two
calls in a row, in FP64 and double-word contexts, and refuses problems larger
than its fixed scratch array.  Collected last so that a stop at the first
failure has already run every other test; it also passes alone in a fresh
process."""
import ctypes as C

import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import _abi
from oracle import operator
from paper_2605_21046_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _static_apply(lib, ctx, x, y, transpose=0):
    return lib.sg_apply_host_static(ctx.handle, 0, C.c_void_p(x.ctypes.data), C.c_void_p(y.ctypes.data), transpose)


PRECISIONS = {"fp64": sg.SG_PREC_FP64, "dw": sg.SG_PREC_DW}


@pytest.mark.parametrize("prec", list(PRECISIONS))
@pytest.mark.parametrize("maker", [I.config_small_2d_q1, I.config_2d_q2_64])
def test_static_apply_matches_host_apply_twice(cuda, maker, prec):
    lib = _abi.load()
    spec = maker()
    ctx = sg.sg_setup_spec(spec, PRECISIONS[prec])
    oracle = operator.SGProblem(spec)
    for call, seed in enumerate((11, 12)):
        x = I.random_vector(spec, seed=seed)
        want = sg.sg_apply_host(ctx, 0, x)
        exact = oracle.apply(x).reshape(-1)
        y = np.full_like(x, np.nan)
        assert _static_apply(lib, ctx, x, y) == _abi.SG_OK, lib.sg_last_error()
        assert np.all(np.isfinite(y))
        assert np.abs(y - want).max() <= TOL * np.abs(want).max(), call
        assert np.abs(y - exact).max() <= TOL * np.abs(exact).max(), call
    # transpose through the same array
    x = I.random_vector(spec, seed=13)
    want = sg.sg_apply_host(ctx, 0, x, transpose=True)
    exact = oracle.apply(x, transpose=True).reshape(-1)
    y = np.empty_like(x)
    assert _static_apply(lib, ctx, x, y, 1) == _abi.SG_OK
    assert np.abs(y - want).max() <= TOL * np.abs(want).max()
    assert np.abs(y - exact).max() <= TOL * np.abs(exact).max()
    ctx.destroy()


def test_static_apply_rejects_oversized_problem(cuda):
    lib = _abi.load()
    spec = I.config_small_2d_q1()
    spec = dict(spec, cells=(520, 520), k=2, M=2, P=2)      # 1041^2 nodes x 2 x 6 > 2^21
    ctx = sg.sg_setup_spec(spec)
    n = ctx.info["n_unknowns"]
    assert n > 2 ** 21
    x = np.zeros(n)
    y = np.zeros(n)
    assert _static_apply(lib, ctx, x, y) == _abi.SG_ERR_ARG
    assert b"2097152" in lib.sg_last_error()
    ctx.destroy()

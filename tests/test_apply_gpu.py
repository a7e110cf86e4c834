"""Parity of sg_apply (CUDA, through the C ABI) with the oracle's Kronecker-sum
apply of eq. local_rhs_tensor, element by element on seeded inputs.

Tolerance: the FP64 apply must match to 1e-12 relative, measured as
max |y_gpu - y_oracle| / max |y_oracle|."""
import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import inputs as I
from oracle import operator

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


PRECISIONS = {"fp64": sg.SG_PREC_FP64, "dw": sg.SG_PREC_DW}


def gpu_apply(torch, spec, x, transpose=False, ctx=None, precision=sg.SG_PREC_FP64):
    own = ctx is None
    ctx = ctx or sg.sg_setup_spec(spec, precision)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    sg.sg_apply(ctx, 0, xd, yd, transpose)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    if own:
        ctx.destroy()
    return y


def small(dim, cells, k, r, M, P, coef=None, lo=None, hi=None):
    if coef is None:
        freqs = [tuple(((m + d) % 3) + 1 for d in range(dim)) for m in range(M)]
        coef = I.linear_sine_coef(M, dim, 0.08, freqs)
    return dict(name="t", dim=dim, cells=cells, lo=lo or (0.0,) * dim, hi=hi or (1.0,) * dim, k=k, r=r,
                n_slabs=3, T=0.9, M=M, P=P, coef=coef)


FULL_CASES = {
    "config-2d-q1-8x8": I.config_small_2d_q1(),
    "config-2d-q2-64x64": I.config_2d_q2_64(),
    "ragged-2d-q2-13x7": small(2, (13, 7), 2, 1, 2, 3),
    "ragged-2d-q1-9x11-r0": small(2, (9, 11), 1, 0, 3, 2),
    "2d-q3-dg3-6x5": small(2, (6, 5), 3, 3, 2, 2, lo=(-1.0, -1.0)),
    "2d-q2-dg2-P0": small(2, (7, 6), 2, 2, 2, 0),
    "2d-q2-M1P5": small(2, (5, 9), 2, 1, 1, 5),
    "3d-q1-5x4x3": small(3, (5, 4, 3), 1, 1, 2, 2),
    "3d-q2-4x3x5": small(3, (4, 3, 5), 2, 1, 3, 2, hi=(1.0, 0.6, 1.3)),
    "3d-q2-r0-3x3x3": small(3, (3, 3, 3), 2, 0, 2, 1),
    # 495 chaos modes (M = 4, P = 8), close to the 512-mode limit: phase 2 then
    # runs one point per round with up to 3 rows per thread
    "2d-q1-4x4-M4P8-495modes": small(2, (4, 4), 1, 1, 4, 8),
}


@pytest.mark.parametrize("prec", list(PRECISIONS))
@pytest.mark.parametrize("name", list(FULL_CASES))
def test_apply_matches_oracle_full(cuda, name, prec):
    spec = FULL_CASES[name]
    p = operator.SGProblem(spec)
    x = I.random_vector(spec, seed=sum(map(ord, name)))
    for tr in (False, True):
        want = p.apply(x, transpose=tr).reshape(-1)
        got = gpu_apply(cuda, spec, x, transpose=tr, precision=PRECISIONS[prec])
        assert np.all(np.isfinite(got))
        assert _rel(got, want) < TOL, (name, prec, tr, _rel(got, want))


@pytest.mark.parametrize("prec", list(PRECISIONS))
def test_paper_squared_coefficient(cuda, prec):
    # Q3 / dG(3) on (-1, 1)^2 with the paper's coefficient
    M = 4
    spec = dict(name="paper", dim=2, cells=(6, 6), lo=(-1.0, -1.0), hi=(1.0, 1.0), k=3, r=3, n_slabs=16, T=1.0,
                M=M, P=2, coef=I.paper_coefficient())
    p = operator.SGProblem(spec)
    assert len(p.mus) == 11
    x = I.random_vector(spec, seed=5)
    assert _rel(gpu_apply(cuda, spec, x, precision=PRECISIONS[prec]), p.apply(x).reshape(-1)) < TOL


@pytest.mark.parametrize("prec", list(PRECISIONS))
@pytest.mark.parametrize("maker", [I.config_3d_q2_32, I.config_2d_q2_128, I.config_paper_q3],
                         ids=["3d-q2-32", "2d-q2-128", "paper-q3-dg3-128-M4P3"])
def test_apply_full_size_sampled(cuda, maker, prec):
    """Full-size workloads in the launch shapes set-up picks, on sampled
    output rows the oracle computes one by one: 32^3 Q2, 128^2 Q2 P = 4 and
    the paper's 128^2 Q3 / dG(3) with M = 4, P = 3 (35 modes, 20.75 M
    unknowns), the workload of the paper-discretisation bench row."""
    spec = maker()
    ctx = sg.sg_setup_spec(spec, PRECISIONS[prec])
    x = I.random_vector(spec)
    y = gpu_apply(cuda, spec, x, ctx=ctx).reshape(ctx.shape)
    ctx.destroy()
    p = operator.SGProblem(spec, assemble_space=False)
    rng = np.random.default_rng(17)
    outs = [(int(rng.integers(p.n_xi)), int(rng.integers(p.n_t)), int(rng.integers(p.n_x))) for _ in range(60)]
    outs += [(p.n_xi - 1, 1, p.n_x // 2), (0, 0, p.n_x - 1), (0, 0, 0)]
    want = p.apply_rows(x, outs)
    got = np.array([y[a, i, m] for a, i, m in outs])
    scale = np.abs(want).max()
    assert np.abs(got - want).max() / scale < TOL
    assert np.all(np.isfinite(y))


def test_multi_index_order_matches_oracle(cuda):
    from oracle import hermite
    for spec in (I.config_small_2d_q1(), small(2, (3, 3), 1, 1, 4, 4), small(3, (2, 2, 2), 1, 1, 3, 3)):
        ctx = sg.sg_setup_spec(spec)
        assert np.array_equal(sg.sg_get_multi_indices(ctx), hermite.multi_indices(spec["M"], spec["P"]))
        ctx.destroy()


@pytest.mark.parametrize("name", ["config-2d-q2-64x64", "ragged-2d-q2-13x7", "3d-q2-4x3x5", "one-row-2d-q1-5x1"])
def test_host_entry_point_shapes_match(cuda, name):
    """sg_apply_host (host buffers in and out) equals the device apply on
    ragged, 3D and one-row meshes, for both transposes."""
    spec = FULL_CASES.get(name) or small(2, (5, 1), 1, 1, 2, 2)
    ctx = sg.sg_setup_spec(spec)
    x = I.random_vector(spec, seed=5)
    for tr in (False, True):
        y_dev = gpu_apply(cuda, spec, x, ctx=ctx, transpose=tr)
        y_host = sg.sg_apply_host(ctx, 0, x, transpose=tr)
        assert _rel(y_host, y_dev) < 1e-15, (name, tr)
    ctx.destroy()


def test_host_entry_point_matches(cuda):
    spec = I.config_2d_q2_64()
    ctx = sg.sg_setup_spec(spec)
    x = I.random_vector(spec, seed=3)
    y_dev = gpu_apply(cuda, spec, x, ctx=ctx)
    y_host = sg.sg_apply_host(ctx, 0, x)
    pinned = cuda.from_numpy(x).pin_memory()
    y_pin = cuda.empty_like(pinned).pin_memory()
    sg.sg_apply_host(ctx, 1, pinned, y_pin, transpose=False)
    ctx.destroy()
    assert _rel(y_host, y_dev) < 1e-15
    assert _rel(y_pin.numpy(), y_dev) < 1e-15


def test_all_dirichlet_mesh_is_identity(cuda):
    spec = small(2, (1, 1), 1, 1, 2, 2)
    x = I.random_vector(spec, seed=9)
    assert np.array_equal(gpu_apply(cuda, spec, x), x)


def test_repeat_is_stable(cuda):
    spec = I.config_2d_q2_64()
    ctx = sg.sg_setup_spec(spec)
    x = I.random_vector(spec, seed=4)
    a = gpu_apply(cuda, spec, x, ctx=ctx)
    b = gpu_apply(cuda, spec, x, ctx=ctx)
    ctx.destroy()
    assert _rel(a, b) < 1e-15


def test_more_than_512_modes_is_refused(cuda):
    """M = 8, P = 4 has 495 modes (accepted); M = 5, P = 7 has 792 (refused at
    set-up, before anything is launched)."""
    ok = sg.sg_setup_spec(small(2, (2, 2), 1, 1, 8, 4))
    assert ok.info["n_xi"] == 495
    ok.destroy()
    with pytest.raises(sg.SGError, match="512"):
        sg.sg_setup_spec(small(2, (2, 2), 1, 1, 5, 7))


def test_errors_are_reported_not_faulted(cuda):
    torch = cuda
    spec = I.config_small_2d_q1()
    ctx = sg.sg_setup_spec(spec)
    x = torch.from_numpy(I.random_vector(spec)).cuda()
    with pytest.raises(sg.SGError):
        sg.sg_apply(ctx, 0, x, x)                            # in place
    with pytest.raises(sg.SGError):
        sg.sg_apply(ctx, 10, x, torch.empty_like(x))         # slab out of range
    with pytest.raises(ValueError):
        sg.sg_apply(ctx, 0, x[:-1], torch.empty_like(x[:-1]))
    # a host pointer straight through the C ABI is rejected before launch
    import ctypes as C
    from paper_2605_21046_gb300 import _abi
    host = np.zeros(ctx.info["n_unknowns"])
    st = _abi.load().sg_apply(ctx.handle, 0, C.c_void_p(host.ctypes.data), C.c_void_p(x.data_ptr()), 0, None)
    assert st == _abi.SG_ERR_ARG
    # the context is still usable
    y = torch.empty_like(x)
    sg.sg_apply(ctx, 0, x, y)
    torch.cuda.synchronize()
    ctx.destroy()


def test_dw_tracks_fp64_closely(cuda):
    """The double-word path stays within 1e-13 of the native FP64 path on the
    bench workload (its stated accuracy is 2 orders inside the tolerance)."""
    spec = I.config_2d_q2_64()
    x = I.random_vector(spec, seed=21)
    a = gpu_apply(cuda, spec, x, precision=sg.SG_PREC_FP64)
    b = gpu_apply(cuda, spec, x, precision=sg.SG_PREC_DW)
    assert _rel(b, a) < 1e-13


def test_dw_nonfinite_propagates(cuda):
    spec = I.config_small_2d_q1()
    x = I.random_vector(spec, seed=2)
    x[40] = np.nan
    y = gpu_apply(cuda, spec, x, precision=sg.SG_PREC_DW)
    assert np.isnan(y).any()


@pytest.mark.parametrize("prec", list(PRECISIONS))
def test_autotune_keeps_parity(cuda, prec):
    spec = I.config_2d_q2_64()
    ctx = sg.sg_setup_spec(spec, PRECISIONS[prec])
    before = dict(ctx.info)
    info = sg.sg_autotune(ctx, reps=3)
    assert info["threads"] >= spec["M"] and info["chunk"] >= 1 and info["grid"] >= 1
    x = I.random_vector(spec, seed=31)
    got = gpu_apply(cuda, spec, x, ctx=ctx)
    want = operator.SGProblem(spec).apply(x).reshape(-1)
    ctx.destroy()
    assert _rel(got, want) < TOL, (before, info)


# (cells per chunk, threads, first-chunk cells of the upper half of the CTAs)
SHAPES = [(1, 128, 0), (2, 256, 1), (3, 384, 2), (4, 256, 2), (5, 512, 5), (7, 384, 4)]


@pytest.mark.parametrize("prec", list(PRECISIONS))
@pytest.mark.parametrize("name", ["ragged-2d-q2-13x7", "3d-q2-4x3x5", "config-2d-q2-64x64"])
def test_fixed_launch_shapes_keep_parity(cuda, name, prec):
    """Every fixed launch shape, staggered or not, gives the oracle's apply
    (both transposes): the chunk walk covers every cell exactly once."""
    spec = FULL_CASES[name]
    p = operator.SGProblem(spec)
    x = I.random_vector(spec, seed=77)
    want = {tr: p.apply(x, transpose=tr).reshape(-1) for tr in (False, True)}
    ctx = sg.sg_setup_spec(spec, PRECISIONS[prec])
    try:
        for chunk, threads, stagger in SHAPES:
            try:
                info = sg.sg_set_apply_shape(ctx, chunk, threads, stagger)
            except sg.SGError:
                continue                      # shape does not fit this kernel / problem
            assert (info["chunk"], info["threads"], info["stagger"]) == (chunk, threads, stagger)
            for tr in (False, True):
                got = gpu_apply(cuda, spec, x, transpose=tr, ctx=ctx)
                assert _rel(got, want[tr]) < TOL, (name, prec, chunk, threads, stagger, tr)
    finally:
        ctx.destroy()


def test_set_apply_shape_rejects_bad_shapes(cuda):
    spec = FULL_CASES["ragged-2d-q2-13x7"]
    ctx = sg.sg_setup_spec(spec)
    try:
        before = dict(ctx.info)
        for chunk, threads, stagger in [(0, 256, 0), (2, 256, 3), (2, 256, -1), (2, 100, 0), (2, 4096, 0),
                                        (10_000, 256, 0)]:
            with pytest.raises(sg.SGError):
                sg.sg_set_apply_shape(ctx, chunk, threads, stagger)
        assert sg.sg_get_info(ctx) == before
    finally:
        ctx.destroy()


@pytest.mark.parametrize("name", ["ragged-2d-q2-13x7", "config-2d-q2-64x64"])
def test_host_async_pipeline_matches_device_apply(cuda, name):
    """Five consecutive pipelined host-buffer applies (alternating staging
    slots, mixed transposes) on a side stream give the device apply of each
    input once the stream is synchronized."""
    torch = cuda
    spec = FULL_CASES[name]
    ctx = sg.sg_setup_spec(spec)
    try:
        n = ctx.info["n_unknowns"]
        xs = [torch.from_numpy(I.random_vector(spec, seed=100 + k)).pin_memory() for k in range(5)]
        ys = [torch.full((n,), float("nan"), dtype=torch.float64).pin_memory() for _ in range(5)]
        side = torch.cuda.Stream()
        for k in range(5):
            sg.sg_apply_host_async(ctx, 0, xs[k], ys[k], transpose=bool(k % 2), stream=side)
        side.synchronize()
        for k in range(5):
            want = gpu_apply(torch, spec, xs[k].numpy(), transpose=bool(k % 2), ctx=ctx)
            assert _rel(ys[k].numpy(), want) < 1e-14, k
        ref = operator.SGProblem(spec).apply(xs[0].numpy()).reshape(-1)
        assert _rel(ys[0].numpy(), ref) < TOL
    finally:
        ctx.destroy()


def test_host_async_refuses_pageable_vectors(cuda):
    import ctypes as C
    from paper_2605_21046_gb300 import _abi
    spec = FULL_CASES["ragged-2d-q2-13x7"]
    ctx = sg.sg_setup_spec(spec)
    try:
        n = ctx.info["n_unknowns"]
        x, y = np.zeros(n), np.zeros(n)
        lib = _abi.load()
        st = lib.sg_apply_host_async(ctx.handle, 0, C.c_void_p(x.ctypes.data), C.c_void_p(y.ctypes.data), 0, None)
        assert st == _abi.SG_ERR_ARG
        with pytest.raises(ValueError):
            sg.sg_apply_host_async(ctx, 0, cuda.zeros(n, dtype=cuda.float64), cuda.zeros(n, dtype=cuda.float64))
    finally:
        ctx.destroy()

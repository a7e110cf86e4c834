"""The multigrid preconditioner on the code paths the large runs take, and its
Vanka patch factors, against the oracle (oracle/solver.py), through the C ABI.

* Patch inverses (Sec. 3.5 remark: the local space-time patch problems of the
  Vanka smoother): the library assembles and inverts every patch on the GPU;
  each stored inverse must equal the oracle's np.linalg.inv of the same
  principal submatrix (FP64 storage: 1e-12 relative to the largest entry;
  FP32 / bf16 storage: the oracle's inverse rounded the same way, at most one
  unit in the last place apart).
* Level variants: set-up picks, per level, the residual apply (SG cell kernel
  or diagonal apply), the Vanka cells per chunk and the modes per tile by
  timing.  Every variant is forced in turn on meshes whose smoothed levels
  have >= 256 cells and the V-cycle must still equal the oracle's (1e-10 FP64,
  1e-4 FP32).
* The tensor-core Vanka sweep (bf16 factors; tcgen05 MMAs with the patch
  values split into three bf16 terms) gives the same V-cycle as the oracle's
  with bf16-rounded factors (1e-4), for every chunk size (one or two staging
  buffers for the tensor-core sweep), in 2D and 3D, Q2 and Q3 / dG(3)
  (64-unknown patches), up to 70 modes in one tile and in tiles of 4 to 32.
* A 3D 16^3 Q2 solve (M = 3, P = 3, 1.44 M unknowns) reaches 1e-8 in true
  residual, evaluated by the oracle's assembled operator."""
import functools

import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from oracle import operator, solver
from paper_2605_21046_gb300 import inputs as I
from paper_2605_21046_gb300.inputs import paper_coefficient

pytestmark = pytest.mark.gpu


def spec2(cells, k=2, r=1, M=3, P=3, lo=(0.0, 0.0), coef=None):
    freqs = [((m % 3) + 1, ((m + 1) % 3) + 1) for m in range(M)]
    return dict(name="v2", dim=2, cells=cells, lo=lo, hi=(1.0, 1.0), k=k, r=r, n_slabs=4, T=1.0, M=M, P=P,
                coef=coef or I.linear_sine_coef(M, 2, 0.08, freqs))


def spec3(cells, k=2, M=3, P=2):
    freqs = [tuple(((m + d) % 2) + 1 for d in range(3)) for m in range(M)]
    return dict(name="v3", dim=3, cells=cells, lo=(0.0,) * 3, hi=(1.0,) * 3, k=k, r=1, n_slabs=4, T=1.0, M=M, P=P,
                coef=I.linear_sine_coef(M, 3, 0.08, freqs))


FACTOR_CASES = {
    "2d-q2-8x8": spec2((8, 8)),
    "2d-q1-8x8-dg2": spec2((8, 8), k=1, r=2, M=2, P=2),
    "2d-q3-dg3-paper": spec2((4, 4), k=3, r=3, M=4, P=2, lo=(-1.0, -1.0), coef=paper_coefficient()),
    "3d-q2-4x4x4": spec3((4, 4, 4), M=1, P=1),
    "3d-q1-4x4x4": spec3((4, 4, 4), k=1, M=2, P=1),
}
STORE = {"fp64": sg.SG_PREC_FP64, "fp32": sg.SG_PREC_FP32, "bf16": sg.SG_PREC_BF16}


def _gpu_rows(level_mesh, cell, n_t):
    """Global dof (i * n_x + node) of every row (i, local node) of the
    library's patch of ``cell``."""
    nodes = level_mesh.cell_dofs(np.array([cell]))[0]            # local nodes, x fastest
    return np.array([i * level_mesh.n_nodes + m for i in range(n_t) for m in nodes], dtype=np.int64)


def _round(a, store):
    if store == "fp32":
        return a.astype(np.float32).astype(np.float64)
    if store == "bf16":
        return solver.round_bf16(a)
    return a


@pytest.mark.parametrize("store", list(STORE))
@pytest.mark.parametrize("name", list(FACTOR_CASES))
def test_patch_inverses_match_oracle(cuda, name, store):
    spec = FACTOR_CASES[name]
    p = operator.SGProblem(spec)
    mg = solver.Multigrid(p, coarse_dofs=0)          # every level down to two cells
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, STORE[store])
    n_levels = sg.sg_mg_level_info(ctx, 0)["levels"]
    assert n_levels == len(mg.levels)
    # one mode of every diagonal class
    alphas = [int(np.flatnonzero(mg.cls == c)[0]) for c in range(len(mg.keys))]
    rng = np.random.default_rng(3)
    checked = 0
    for lev in range(n_levels - 1):
        L = mg.levels[lev]
        cells = sorted(set([0, L.mesh.n_cells - 1] + list(rng.integers(0, L.mesh.n_cells, 6))))
        for alpha in alphas:
            for c in cells:
                got = sg.sg_mg_patch_inverse(ctx, lev, alpha, int(c))
                rows = _gpu_rows(L.mesh, int(c), L.n_t)
                interior = ~np.tile(L.bmask, L.n_t)[rows]
                # Dirichlet rows and columns are the identity's
                bi = np.flatnonzero(~interior)
                assert np.array_equal(got[np.ix_(bi, bi)], np.eye(bi.size))
                assert not got[np.ix_(bi, np.flatnonzero(interior))].any()
                dofs = L.patches[int(c)]
                if dofs.size == 0:
                    continue
                pos = {int(d): j for j, d in enumerate(dofs)}
                perm = [pos[int(d)] for d in rows[interior]]
                want = L.patch_inv[mg.cls[alpha]][int(c)][np.ix_(perm, perm)]
                g = got[np.ix_(np.flatnonzero(interior), np.flatnonzero(interior))]
                scale = np.abs(want).max()
                if store == "fp64":
                    assert np.abs(g - want).max() <= 1e-12 * scale, (lev, alpha, c)
                else:
                    w = _round(want, store)
                    ulp = np.abs(w) * (2.0 ** -23 if store == "fp32" else 2.0 ** -7) + 1e-300
                    assert np.all(np.abs(g - w) <= 1.01 * ulp), (lev, alpha, c, np.abs(g - w).max())
                    assert np.mean(g == w) > 0.99
                checked += 1
    ctx.destroy()
    assert checked > 0


def test_patch_inverse_errors(cuda):
    ctx = sg.sg_setup_spec(spec2((4, 4), M=1, P=1))
    with pytest.raises(sg.SGError):
        sg.sg_mg_level_info(ctx, 0)                  # no preconditioner yet
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    info = sg.sg_mg_level_info(ctx, 0)
    with pytest.raises(sg.SGError):
        sg.sg_mg_patch_inverse(ctx, info["levels"] - 1, 0, 0)   # coarsest level: no patches
    with pytest.raises(sg.SGError):
        sg.sg_mg_patch_inverse(ctx, 0, 0, 16)                   # cell out of range
    with pytest.raises(sg.SGError):
        sg.sg_mg_set_level_variant(ctx, 0, 0, 0, 8)             # 2 modes (4 slots): no tile of 8
    ctx.destroy()


VARIANT_CASES = {
    "2d-q2-32x32-M3P3": spec2((32, 32)),
    "3d-q2-8x8x8-M3P2": spec3((8, 8, 8)),
}
VARIANTS = [(res, chunk, tile) for res in (0, 1) for chunk in (1, 2, 4, 8) for tile in (0, 8, 16)]


@functools.lru_cache(maxsize=None)
def _oracle_vcycle(name, seed=9):
    spec = VARIANT_CASES[name]
    p = operator.SGProblem(spec)
    r = np.random.default_rng(seed).uniform(-1, 1, p.shape)
    return r, solver.Multigrid(p).apply(r).reshape(-1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"res{v[0]}-chunk{v[1]}-tile{v[2]}")
@pytest.mark.parametrize("name", list(VARIANT_CASES))
def test_vcycle_variants_match_oracle(cuda, name, variant, prec):
    torch = cuda
    res, chunk, tile = variant
    spec = VARIANT_CASES[name]
    n_xi = I.n_modes(spec)
    slots = -(-n_xi // 4) * 4                     # one diagonal class: modes in blocks of 4
    if tile > slots:
        pytest.skip(f"{n_xi} modes: no tile of {tile}")
    r, want = _oracle_vcycle(name)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx, STORE[prec])
    info0 = sg.sg_mg_level_info(ctx, 0)
    assert info0["cells"] >= 256
    try:
        sg.sg_mg_set_level_variant(ctx, -1, res, chunk, tile)
    except sg.SGError as e:
        ctx.destroy()
        if e.status == 4 and "shared memory" in str(e):      # e.g. 8 cells of 3D Q2 FP64 factors
            pytest.skip(str(e))
        raise
    for lev in range(info0["levels"] - 1):
        info = sg.sg_mg_level_info(ctx, lev)
        assert info["residual"] == res
        assert info["vanka_chunk"] == min(chunk, spec["cells"][0] >> lev)
        assert info["vanka_tile"] == (slots if tile == 0 else tile)
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.full_like(rd, float("nan"))
    sg.sg_vcycle(ctx, rd, zd)
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    tol = 1e-10 if prec == "fp64" else 1e-4
    err = float(np.abs(got - want).max() / np.abs(want).max())
    assert err < tol, err


TC_CASES = {
    "2d-q2-32x32-M3P3": spec2((32, 32)),
    "2d-q2-16x16-M4P3": spec2((16, 16), M=4, P=3),
    "2d-q3-dg3-8x8-M2P2": spec2((8, 8), k=3, r=3, M=2, P=2),
    "2d-q2-8x8-M4P4": spec2((8, 8), M=4, P=4),          # 70 modes: 72 slots, 240 MMA columns
    "3d-q2-8x8x8-M3P2": spec3((8, 8, 8)),
}


@functools.lru_cache(maxsize=None)
def _oracle_vcycle_bf16(name, seed=10):
    spec = TC_CASES[name]
    p = operator.SGProblem(spec)
    r = np.random.default_rng(seed).uniform(-1, 1, p.shape)
    return r, solver.Multigrid(p, factor_round=solver.round_bf16, coarse_dofs=0).apply(r).reshape(-1)


@pytest.mark.parametrize("kind", [0, 1], ids=["ffma", "tensor"])
@pytest.mark.parametrize("chunk", [1, 2, 4])
@pytest.mark.parametrize("name", list(TC_CASES))
def test_vcycle_bf16_sweeps_match_oracle(cuda, name, chunk, kind):
    torch = cuda
    spec = TC_CASES[name]
    r, want = _oracle_vcycle_bf16(name)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)                 # every level down to two cells
    sg.sg_mg_setup(ctx, sg.SG_PREC_BF16)
    sg.sg_mg_set_level_variant(ctx, -1, -1, chunk, 0, kind)
    levels = sg.sg_mg_level_info(ctx, 0)["levels"]
    for lev in range(levels - 1):
        assert sg.sg_mg_level_info(ctx, lev)["vanka_kind"] == kind
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.full_like(rd, float("nan"))
    sg.sg_vcycle(ctx, rd, zd)
    z2 = torch.empty_like(rd)
    sg.sg_vcycle(ctx, rd, z2)                      # graph replay: the same map
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    err = float(np.abs(got - want).max() / np.abs(want).max())
    assert err < 1e-4, err
    assert float(np.abs(z2.cpu().numpy() - got).max() / np.abs(got).max()) < 1e-6


@pytest.mark.parametrize("tile", [4, 8, 12, 32])
def test_vcycle_tensor_sweep_mode_tiles_match_oracle(cuda, tile):
    """35 modes in tiles of 4 to 32 slots (the last tile partly empty)."""
    torch = cuda
    name = "2d-q2-16x16-M4P3"
    r, want = _oracle_vcycle_bf16(name)
    ctx = sg.sg_setup_spec(TC_CASES[name])
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_BF16)
    sg.sg_mg_set_level_variant(ctx, -1, -1, 1, tile, 1)
    assert sg.sg_mg_level_info(ctx, 0)["vanka_tile"] == tile
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.full_like(rd, float("nan"))
    sg.sg_vcycle(ctx, rd, zd)
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    err = float(np.abs(got - want).max() / np.abs(want).max())
    assert err < 1e-4, err


def test_tensor_core_sweep_refuses_unsupported_levels(cuda):
    # FP32 factors, and bf16 factors of several diagonal classes, keep the FFMA sweep
    ctx = sg.sg_setup_spec(spec2((8, 8)))
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP32)
    with pytest.raises(sg.SGError):
        sg.sg_mg_set_level_variant(ctx, -1, -1, 0, -1, 1)
    ctx.destroy()
    ctx = sg.sg_setup_spec(spec2((4, 4), M=4, P=2, lo=(-1.0, -1.0), coef=paper_coefficient()))
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_BF16)
    with pytest.raises(sg.SGError):
        sg.sg_mg_set_level_variant(ctx, -1, -1, 0, -1, 1)
    ctx.destroy()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_solve_3d_16cubed_reaches_tolerance(cuda, prec):
    """16^3 Q2, dG(1), M = 3, P = 3 (20 modes, 1,437,480 unknowns) to 1e-8 with
    the mixed-precision preconditioner; the true residual is evaluated by the
    oracle's assembled operator."""
    torch = cuda
    spec = I.scaled(I.config_3d_q2_32(), (16, 16, 16))
    p = operator.SGProblem(spec)
    b = np.random.default_rng(11).uniform(-1, 1, p.shape)
    b[:, :, p.bmask] = 0.0
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx, STORE[prec], 1, 0.9)
    bd = torch.from_numpy(b.reshape(-1).copy()).cuda()
    x = torch.zeros_like(bd)
    st = sg.sg_solve_slab(ctx, 0, bd, x, rtol=1e-8, max_it=300, restart=30)
    got = x.cpu().numpy()
    ctx.destroy()
    res = np.linalg.norm(b.reshape(-1) - p.apply(got).reshape(-1)) / np.linalg.norm(b)
    assert st["converged"] == 1 and res <= 1.2e-8, (res, st)


def test_tensor_sweep_wait_runs_out_and_reports_timeout(cuda):
    """The tensor-core sweep waits for its MMAs on an mbarrier with a poll
    limit.  The same bounded wait on an mbarrier that nothing arrives on runs
    out, records SG_ERR_TIMEOUT and returns; the context stays usable (a
    V-cycle afterwards still equals the oracle's)."""
    from paper_2605_21046_gb300 import _abi
    assert sg.sg_debug_wait_probe(1000) == _abi.SG_ERR_TIMEOUT
    assert sg.sg_debug_wait_probe(1) == _abi.SG_ERR_TIMEOUT
    with pytest.raises(sg.SGError):
        sg.sg_debug_wait_probe(0)
    test_vcycle_bf16_sweeps_match_oracle(cuda, "3d-q2-8x8x8-M3P2", 1, 1)

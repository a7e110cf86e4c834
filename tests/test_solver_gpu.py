"""Parity of the multigrid preconditioner (sg_vcycle) and the FGMRES slab
solve (sg_solve_slab) with the oracle (oracle/solver.py), through the C ABI.

sg_vcycle is a fixed linear map: the GPU result is compared element by element
with the oracle's V-cycle (FP64 levels: 1e-10 relative; FP32 levels: 1e-4;
FP32 levels with bf16-stored Vanka inverses: 1e-4 against the oracle's V-cycle
whose inverses are rounded to bf16 in the same way).
sg_solve_slab is checked by the property required of every solve: the
true residual ||b - A x|| / ||b||, evaluated by the oracle's operator, is at
most the requested tolerance (1e-8 at scale, 1e-10 on the small case), and the
solution matches a sparse direct solve where one is affordable."""
import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import inputs as I
from oracle import operator, solver

from paper_2605_21046_gb300.inputs import paper_coefficient

pytestmark = pytest.mark.gpu


def spec2(cells, k=1, r=1, M=2, P=2, hi=(1.0, 1.0), lo=(0.0, 0.0), coef=None, a0_cells=None):
    freqs = [((m % 3) + 1, ((m + 1) % 3) + 1) for m in range(M)]
    return dict(name="t", dim=2, cells=cells, lo=lo, hi=hi, k=k, r=r, n_slabs=4, T=1.0, M=M, P=P,
                coef=coef or I.linear_sine_coef(M, 2, 0.08, freqs, a0_cells=a0_cells))


def spec3(cells, k=1, M=1, P=2):
    freqs = [tuple(((m + d) % 2) + 1 for d in range(3)) for m in range(M)]
    return dict(name="t3", dim=3, cells=cells, lo=(0.0,) * 3, hi=(1.0,) * 3, k=k, r=1, n_slabs=4, T=1.0, M=M, P=P,
                coef=I.linear_sine_coef(M, 3, 0.08, freqs))


VCYCLE_CASES = {
    "2d-q1-8x8": I.config_small_2d_q1(),
    "2d-q2-16x16": spec2((16, 16), k=2),
    "2d-q2-aniso": spec2((8, 8), k=2, hi=(1.0, 0.5)),
    "2d-q2-cellfield": spec2((8, 8), k=2, a0_cells=np.random.default_rng(8).uniform(0.8, 1.2, 64)),
    "2d-q2-ragged-1level": spec2((5, 3), k=2),
    "2d-q2-dg0": spec2((8, 8), k=2, r=0),
    "2d-q2-paper-15classes": spec2((4, 4), k=2, M=4, P=2, lo=(-1.0, -1.0), coef=paper_coefficient()),
    "3d-q1-4x4x4": spec3((4, 4, 4), k=1),
    "3d-q2-4x4x4": spec3((4, 4, 4), k=2, M=1, P=1),
}
MG_PREC = {"fp64": (sg.SG_PREC_FP64, 1e-10), "fp32": (sg.SG_PREC_FP32, 1e-4), "bf16": (sg.SG_PREC_BF16, 1e-4)}


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec", list(MG_PREC))
@pytest.mark.parametrize("name", list(VCYCLE_CASES))
def test_vcycle_matches_oracle(cuda, name, prec):
    torch = cuda
    spec = VCYCLE_CASES[name]
    p = operator.SGProblem(spec)
    # bf16: the oracle's V-cycle with its Vanka inverses rounded the same way
    # every level down to two cells (small meshes: the smoothers stay in play)
    mg = solver.Multigrid(p, factor_round=solver.round_bf16 if prec == "bf16" else None, coarse_dofs=0)
    r = np.random.default_rng(4).uniform(-1, 1, p.shape)
    want = mg.apply(r).reshape(-1)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, MG_PREC[prec][0])
    assert sg.sg_mg_level_info(ctx, 0)["levels"] == len(mg.levels)
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.full_like(rd, float("nan"))
    sg.sg_vcycle(ctx, rd, zd)
    z2 = torch.empty_like(rd)
    sg.sg_vcycle(ctx, rd, z2)                      # graph replay gives the same map
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    assert np.all(np.isfinite(got))
    assert _rel(got, want) < MG_PREC[prec][1], _rel(got, want)
    assert _rel(z2.cpu().numpy(), got) < 1e-6


@pytest.mark.parametrize("name", ["2d-q2-16x16", "2d-q2-paper-15classes", "3d-q2-4x4x4"])
def test_vcycle_one_smoothing_step_matches_oracle(cuda, name):
    """nu = 1, omega = 0.9 (the pair the benchmarks use) against the oracle's
    V-cycle with the same pair, FP64 levels."""
    torch = cuda
    spec = VCYCLE_CASES[name]
    p = operator.SGProblem(spec)
    mg = solver.Multigrid(p, nu=1, omega=0.9, coarse_dofs=0)
    r = np.random.default_rng(6).uniform(-1, 1, p.shape)
    want = mg.apply(r).reshape(-1)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64, 1, 0.9)
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.empty_like(rd)
    sg.sg_vcycle(ctx, rd, zd)
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    assert _rel(got, want) < 1e-10


DEFAULT_HIERARCHY_CASES = {
    "2d-q2-32x32": spec2((32, 32), k=2),                  # 32^2, 16^2, coarse solve on 8^2
    "2d-q3-dg3-8x8": spec2((8, 8), k=3, r=3),             # 8^2, coarse solve on 4^2 (484 unknowns)
    "3d-q2-8x8x8": spec3((8, 8, 8), k=2, M=1, P=1),       # 8^3, coarse solve on 4^3 (686)
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(DEFAULT_HIERARCHY_CASES))
def test_vcycle_default_hierarchy_matches_oracle(cuda, name, prec):
    """The default coarsest level (the first with at most 1024 interior
    unknowns per mode, solved densely) on both sides."""
    torch = cuda
    spec = DEFAULT_HIERARCHY_CASES[name]
    p = operator.SGProblem(spec)
    mg = solver.Multigrid(p)
    r = np.random.default_rng(9).uniform(-1, 1, p.shape)
    want = mg.apply(r).reshape(-1)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx, MG_PREC[prec][0])
    info = sg.sg_mg_level_info(ctx, 0)
    assert info["levels"] == len(mg.levels) >= 2
    last = sg.sg_mg_level_info(ctx, info["levels"] - 1)
    assert last["coarsest"] == 1 and last["cells"] == mg.levels[-1].mesh.n_cells
    rd = torch.from_numpy(r.reshape(-1).copy()).cuda()
    zd = torch.empty_like(rd)
    sg.sg_vcycle(ctx, rd, zd)
    torch.cuda.synchronize()
    got = zd.cpu().numpy()
    ctx.destroy()
    assert _rel(got, want) < MG_PREC[prec][1], _rel(got, want)


def test_coarse_dofs_argument_errors(cuda):
    ctx = sg.sg_setup_spec(I.config_small_2d_q1())
    for bad in (-1, 2049):
        with pytest.raises(sg.SGError):
            sg.sg_mg_set_coarse_dofs(ctx, bad)
    sg.sg_mg_set_coarse_dofs(ctx, 2048)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    assert sg.sg_mg_level_info(ctx, 0)["levels"] == 1          # 98 unknowns: one dense level
    ctx.destroy()


@pytest.mark.parametrize("prec", list(MG_PREC))
def test_solve_small_matches_direct(cuda, prec):
    torch = cuda
    for spec, rtol in ((I.config_small_2d_q1(), 1e-10), (spec2((16, 16), k=2, M=2, P=3), 1e-10),
                       (spec2((8, 8), k=2, M=4, P=2, lo=(-1.0, -1.0), coef=paper_coefficient()), 1e-10)):
        p = operator.SGProblem(spec)
        b = np.random.default_rng(5).uniform(-1, 1, p.shape)
        b[:, :, p.bmask] = 0.0
        xd = solver.direct_solve(p, b).reshape(-1)
        ctx = sg.sg_setup_spec(spec)
        sg.sg_mg_setup(ctx, MG_PREC[prec][0])
        bd = torch.from_numpy(b.reshape(-1).copy()).cuda()
        x = torch.zeros_like(bd)
        st = sg.sg_solve_slab(ctx, 0, bd, x, rtol=rtol, max_it=300, restart=30)
        got = x.cpu().numpy()
        ctx.destroy()
        res = np.linalg.norm(b.reshape(-1) - p.apply(got).reshape(-1)) / np.linalg.norm(b)
        assert st["converged"] == 1 and st["rel_residual"] <= rtol
        assert res <= 1.5 * rtol, res
        assert _rel(got, xd) < 1e-6
        assert st["iterations"] < 60 and st["prec_calls"] == st["iterations"]


def test_iterations_match_oracle_fgmres(cuda):
    torch = cuda
    spec = I.config_small_2d_q1()
    p = operator.SGProblem(spec)
    b = np.random.default_rng(6).uniform(-1, 1, p.shape)
    b[:, :, p.bmask] = 0.0
    _, its, _ = solver.fgmres(p, b, solver.Multigrid(p, coarse_dofs=0).apply, rtol=1e-10)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    st = sg.sg_solve_slab(ctx, 0, torch.from_numpy(b.reshape(-1).copy()).cuda(), x, rtol=1e-10)
    ctx.destroy()
    assert abs(st["iterations"] - its) <= 1, (st["iterations"], its)


@pytest.mark.parametrize("omega,restart", [(0.1, 20), (0.05, 30)])
def test_long_arnoldi_cycles_match_oracle_fgmres(cuda, omega, restart):
    """A weakly damped smoother makes the Arnoldi cycles long (up to 29 basis
    vectors, and a restart with restart = 20): the Gram-Schmidt passes then
    run past the vectors a thread keeps in registers.  Iteration count and
    solution against the oracle's FGMRES with the same V-cycle."""
    torch = cuda
    spec = I.config_small_2d_q1()
    p = operator.SGProblem(spec)
    b = np.random.default_rng(6).uniform(-1, 1, p.shape)
    b[:, :, p.bmask] = 0.0
    want, its, _ = solver.fgmres(p, b, solver.Multigrid(p, nu=1, omega=omega, coarse_dofs=0).apply, rtol=1e-10,
                                 restart=restart)
    assert its > 20
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_set_coarse_dofs(ctx, 0)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64, 1, omega)
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    st = sg.sg_solve_slab(ctx, 0, torch.from_numpy(b.reshape(-1).copy()).cuda(), x, rtol=1e-10, max_it=300,
                          restart=restart)
    got = x.cpu().numpy()
    ctx.destroy()
    res = np.linalg.norm(b.reshape(-1) - p.apply(got).reshape(-1)) / np.linalg.norm(b)
    assert st["converged"] == 1 and res <= 1.5e-10, (res, st)
    assert abs(st["iterations"] - its) <= 1, (st["iterations"], its)
    assert st["restarts"] == (2 if st["iterations"] > restart else 1), st
    assert _rel(got, want) < 1e-8


@pytest.mark.parametrize("prec", list(MG_PREC))
def test_solve_at_scale_reaches_tolerance(cuda, prec):
    """64x64 Q2, M=4, P=3 (1.16 M unknowns) to 1e-8; residual checked by the oracle."""
    torch = cuda
    spec = I.config_2d_q2_64()
    p = operator.SGProblem(spec)
    b = np.random.default_rng(7).uniform(-1, 1, p.shape)
    b[:, :, p.bmask] = 0.0
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx, MG_PREC[prec][0])
    bd = torch.from_numpy(b.reshape(-1).copy()).cuda()
    x = torch.zeros_like(bd)
    st = sg.sg_solve_slab(ctx, 0, bd, x, rtol=1e-8, max_it=300, restart=30)
    got = x.cpu().numpy()
    ctx.destroy()
    res = np.linalg.norm(b.reshape(-1) - p.apply(got).reshape(-1)) / np.linalg.norm(b)
    assert st["converged"] == 1 and res <= 1.2e-8, (res, st)


def test_solver_errors(cuda):
    torch = cuda
    spec = I.config_small_2d_q1()
    ctx = sg.sg_setup_spec(spec)
    n = ctx.info["n_unknowns"]
    b = torch.rand(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(sg.SGError):
        sg.sg_solve_slab(ctx, 0, b, x)                 # no preconditioner yet
    with pytest.raises(sg.SGError):
        sg.sg_vcycle(ctx, b, x)
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    with pytest.raises(sg.SGError):
        sg.sg_mg_setup(ctx, sg.SG_PREC_DW)             # not a preconditioner precision
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    st = sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-14, max_it=2, check=False)
    assert st["status"] == 5 and st["converged"] == 0 and st["iterations"] == 2
    bad = b.clone()
    bad[7] = float("nan")
    st = sg.sg_solve_slab(ctx, 0, bad, torch.zeros_like(b), check=False)
    assert st["status"] == 6
    # still usable
    st = sg.sg_solve_slab(ctx, 0, b, torch.zeros_like(b), rtol=1e-10)
    assert st["converged"] == 1
    ctx.destroy()

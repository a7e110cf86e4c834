"""Parity of the slab right-hand sides (sg_rhs: load vector, initial vector,
transfer term), slab marching with sg_solve_slab, the pointwise moments
(sg_moments) and the end-time errors (sg_qoi_errors) with the oracle.

The product integrates the load vector in weak form (a grad u, grad v); the
oracle uses the strong-form forcing f = d_t u - div(a grad u) of eq.
manufactured_rhs_benchmark.  The two integrands are equal only in exact
arithmetic; both sides apply (k+4)-point Gauss rules to them, so they agree to
the difference of two quadrature errors, which on these meshes (h <= 1/6,
sines of frequency <= 2) stays below 1e-9 relative: RHS_TOL."""
import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import inputs as I
from oracle import hermite, manufactured, operator

from paper_2605_21046_gb300.inputs import paper_coefficient

pytestmark = pytest.mark.gpu
RHS_TOL = 1e-9


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def to_product(exact):
    return {"q": exact["q"], "c": exact["c"], "freq": [[f[1] for f in ph] for ph in exact["phi"]], "T": exact["T"]}


def sine_exact(M, q, dim, eta=0.35, T=(0.0, 1.0, 1.0)):
    idx = hermite.multi_indices(M, q)
    c = [1.0 if not any(a) else eta ** int(sum(a)) for a in idx]
    phi = [[("sin", 1 + (int(a[d % M]) % 2)) for d in range(dim)] for a in idx]
    return {"q": q, "c": c, "phi": phi, "T": list(T)}


CASES = {
    "2d-q1-8x8": (I.config_small_2d_q1(), sine_exact(2, 2, 2)),
    "2d-q2-12x12-q3>p2": (dict(I.config_small_2d_q1(), cells=(12, 12), k=2, P=2), sine_exact(2, 3, 2)),
    "2d-q3-dg3-paper": (dict(dim=2, cells=(4, 4), lo=(-1.0, -1.0), hi=(1.0, 1.0), k=3, r=3, n_slabs=8, T=1.0, M=4, P=1,
                             coef=paper_coefficient()), manufactured.paper_exact()),
    "3d-q1-6x6x6": (dict(dim=3, cells=(6, 6, 6), lo=(0.0,) * 3, hi=(1.0,) * 3, k=1, r=1, n_slabs=5, T=1.0, M=1, P=2,
                         coef=I.linear_sine_coef(1, 3, 0.08, [(1, 1, 1)])), sine_exact(1, 2, 3)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(cuda, name):
    torch = cuda
    spec, exact = CASES[name]
    p = operator.SGProblem(spec)
    man = manufactured.Manufactured(p, exact)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    n = ctx.info["n_unknowns"]
    rhs = torch.empty(n, dtype=torch.float64, device="cuda")
    sg.sg_rhs(ctx, 0, None, rhs)
    torch.cuda.synchronize()
    want0 = man.load_vector(0).reshape(-1)
    assert _rel(rhs.cpu().numpy(), want0) < RHS_TOL
    u_prev = np.random.default_rng(3).uniform(-1, 1, p.shape)
    u_prev[:, :, p.bmask] = 0.0
    ud = torch.from_numpy(u_prev.reshape(-1).copy()).cuda()
    sg.sg_rhs(ctx, 2, ud, rhs)
    torch.cuda.synchronize()
    want = (man.load_vector(2) + p.transfer(u_prev)).reshape(-1)
    ctx.destroy()
    assert _rel(rhs.cpu().numpy(), want) < RHS_TOL


@pytest.mark.parametrize("name", ["2d-q1-8x8", "2d-q2-12x12-q3>p2", "2d-q3-dg3-paper"])
def test_marching_matches_oracle(cuda, name):
    torch = cuda
    spec, exact = CASES[name]
    p = operator.SGProblem(spec)
    man = manufactured.Manufactured(p, exact)
    slabs = 3
    Us = man.march(slabs)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    n = ctx.info["n_unknowns"]
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    rhs = torch.empty_like(u)
    for s in range(slabs):
        sg.sg_rhs(ctx, s, u if s > 0 else None, rhs)
        x = u.clone()                                   # previous slab as the initial guess
        st = sg.sg_solve_slab(ctx, s, rhs, x, rtol=1e-12, max_it=400)
        assert st["converged"] == 1
        u = x
    got = u.cpu().numpy()
    assert _rel(got, Us[-1].reshape(-1)) < 1e-8
    err = sg.sg_qoi_errors(ctx, u, slabs - 1)
    want = manufactured.errors_at_end(man, Us[-1], slabs - 1)
    for key in ("mean", "var", "full"):
        assert abs(err[key] - want[key]) <= 1e-7 * max(want[key], 1e-12), (key, err, want)
    mean, var = sg.sg_moments(ctx, u, p.n_t - 1)
    U = got.reshape(p.shape)
    assert _rel(mean.cpu().numpy(), U[0, -1]) < 1e-15
    assert _rel(var.cpu().numpy(), (U[1:, -1] ** 2).sum(axis=0)) < 1e-13
    ctx.destroy()


def test_march_errors(cuda):
    torch = cuda
    spec, exact = CASES["2d-q1-8x8"]
    ctx = sg.sg_setup_spec(spec)
    n = ctx.info["n_unknowns"]
    rhs = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SGError):
        sg.sg_rhs(ctx, 0, None, rhs)                     # no exact solution yet
    sg.sg_set_exact(ctx, to_product(exact))
    with pytest.raises(sg.SGError):
        sg.sg_rhs(ctx, 1, None, rhs)                     # previous slab required
    with pytest.raises(sg.SGError):
        sg.sg_rhs(ctx, 0, rhs, rhs)                      # overlapping
    ctx.destroy()

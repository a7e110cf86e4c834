"""Parity of the transposed slab solve (sg_solve_slab_adjoint) and of the
adjoint gradient (sg_adjoint_gradient, energy_at_T) with the oracle's discrete
adjoint (oracle/adjoint.py, itself pinned by central differences).

Tolerances: the transposed solve runs to rtol 1e-12 against a sparse LU, so
1e-9 relative.  The gradient side integrates the manufactured load vector in
weak form, the oracle in strong form (see test_march_gpu: the load vectors
agree to 1e-9 relative), and every slab solve runs to rtol 1e-12, so J and its
gradient agree to 1e-7 relative to the largest gradient entry."""
import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import inputs as I
from oracle import adjoint, operator

from test_march_gpu import sine_exact, to_product

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-7


def _ctx(spec, exact):
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    sg.sg_mg_setup(ctx)
    return ctx


@pytest.mark.parametrize("k,r,cells", [(1, 1, (8, 8)), (2, 1, (4, 4)), (2, 2, (8, 8)), (3, 0, (4, 4))])
def test_transposed_solve_matches_direct(cuda, k, r, cells):
    torch = cuda
    spec = I.config_adjoint_2d(cells=cells, k=k, r=r, n_slabs=4)
    op = operator.SGProblem(spec)
    b = np.random.default_rng(5).uniform(-1, 1, op.shape).reshape(-1)
    want = np.asarray(__import__("scipy.sparse.linalg", fromlist=["spsolve"]).spsolve(
        op.assembled().T.tocsc(), b)).reshape(-1)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx)
    bd = torch.from_numpy(b.copy()).cuda()
    x = torch.zeros_like(bd)
    st = sg.sg_solve_slab_adjoint(ctx, 1, bd, x, rtol=1e-12, max_it=400)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    # the untransposed solve gives a different answer (A_t, hence A, is not
    # symmetric for r >= 1; dG(0) has a 1 x 1 A_t and a symmetric A)
    x2 = torch.zeros_like(bd)
    sg.sg_solve_slab(ctx, 1, bd, x2, rtol=1e-12, max_it=400)
    torch.cuda.synchronize()
    ctx.destroy()
    assert st["converged"] == 1
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    if r > 0:
        assert np.abs(x2.cpu().numpy() - want).max() > 1e-6 * np.abs(want).max()


CASES = [
    ((4, 4), 1, 1, 3, 1),
    ((4, 4), 2, 1, 3, 2),
    ((8, 8), 1, 2, 5, 2),
    ((4, 4), 2, 0, 4, 10),
    ((6, 6), 3, 1, 3, 3),
]


@pytest.mark.parametrize("cells,k,r,slabs,every", CASES)
def test_gradient_matches_oracle(cuda, cells, k, r, slabs, every):
    spec = I.config_adjoint_2d(cells=cells, k=k, r=r, n_slabs=slabs)
    exact = sine_exact(2, 2, 2)
    J0, g0, c0 = adjoint.gradient(spec, exact, cell_piece=0)
    ctx = _ctx(spec, exact)
    J, g, c, st = sg.sg_adjoint_gradient(ctx, rtol=1e-12, checkpoint_every=every, cell_piece=0)
    ctx.destroy()
    assert st["adjoint_solves"] == slabs
    n_seg = -(-slabs // every)
    assert st["forward_solves"] == slabs + (n_seg - 1) * every
    assert abs(J - J0) <= GRAD_TOL * J0
    assert np.abs(g - g0).max() <= GRAD_TOL * np.abs(g0).max()
    assert np.abs(c - c0).max() <= GRAD_TOL * np.abs(c0).max()


@pytest.mark.parametrize("k", [1, 2])
def test_gradient_3d_matches_oracle(cuda, k):
    """The gradient kernel's 3D shapes: 4x4x4 Q1 / 3x3x3 Q2, dG(1), 2 slabs,
    a mean field with a per-cell scale and two sine pieces."""
    cells = (4, 4, 4) if k == 1 else (3, 3, 3)
    coef = I.linear_sine_coef(2, 3, 0.08, [(1, 1, 1), (2, 1, 1)], a0_cells=np.ones(int(np.prod(cells))))
    spec = dict(dim=3, cells=cells, lo=(0.0,) * 3, hi=(1.0,) * 3, k=k, r=1, n_slabs=2, T=0.4, M=2, P=1, coef=coef)
    exact = {"q": 1, "c": [1.0, 0.3, 0.2], "phi": [[("sin", 1)] * 3] * 3, "T": [0.0, 1.0, 1.0]}
    J0, g0, c0 = adjoint.gradient(spec, exact, cell_piece=0)
    ctx = _ctx(spec, exact)
    J, g, c, st = sg.sg_adjoint_gradient(ctx, rtol=1e-12, checkpoint_every=1, cell_piece=0)
    ctx.destroy()
    assert st["adjoint_solves"] == 2
    assert abs(J - J0) <= GRAD_TOL * J0
    assert np.abs(g - g0).max() <= GRAD_TOL * np.abs(g0).max()
    assert np.abs(c - c0).max() <= GRAD_TOL * np.abs(c0).max()


def test_checkpoint_spacing_does_not_change_the_result(cuda):
    spec = I.config_adjoint_2d(cells=(8, 8), k=2, r=1, n_slabs=7)
    exact = sine_exact(2, 2, 2)
    ctx = _ctx(spec, exact)
    out = [sg.sg_adjoint_gradient(ctx, rtol=1e-13, checkpoint_every=e, cell_piece=2) for e in (1, 3, 7, 20)]
    ctx.destroy()
    J, g, c, _ = out[0]
    for J2, g2, c2, st in out[1:]:
        assert abs(J2 - J) <= 1e-11 * J
        assert np.abs(g2 - g).max() <= 1e-10 * np.abs(g).max()
        assert np.abs(c2 - c).max() <= 1e-10 * np.abs(c).max()
    assert out[0][3]["checkpoints"] == 6 and out[3][3]["checkpoints"] == 0
    ctx = _ctx(spec, exact)
    J1, g1, c1, st1 = sg.sg_adjoint_gradient(ctx, rtol=1e-13, checkpoint_every=3, cell_piece=2, gradient=False)
    ctx.destroy()
    assert g1 is None and c1 is None and st1["adjoint_solves"] == 0 and st1["forward_solves"] == 7
    assert abs(J1 - J) <= 1e-11 * J


def test_set_coefficient_keeps_the_load_vector(cuda):
    """After sg_set_coefficient the operator follows the new coefficient and
    the load vector stays the nominal one: J and its gradient match the
    oracle's with the same split."""
    spec = I.config_adjoint_2d(cells=(4, 4), k=2, r=1, n_slabs=3)
    exact = sine_exact(2, 2, 2)
    amp = np.array([1.1, 0.15, 0.13, 0.07])
    cells = np.random.default_rng(3).uniform(0.7, 1.3, 16)
    pert = adjoint.with_coefficient(spec, amp, 0, cells)
    J0, g0, c0 = adjoint.gradient(pert, exact, cell_piece=0, nominal_spec=spec)
    ctx = _ctx(spec, exact)
    sg.sg_set_coefficient(ctx, pert["coef"])
    J, g, c, _ = sg.sg_adjoint_gradient(ctx, rtol=1e-12, checkpoint_every=2, cell_piece=0)
    ctx.destroy()
    assert abs(J - J0) <= GRAD_TOL * J0
    assert np.abs(g - g0).max() <= GRAD_TOL * np.abs(g0).max()
    assert np.abs(c - c0).max() <= GRAD_TOL * np.abs(c0).max()


def test_energy_autograd_matches_central_differences(cuda):
    torch = cuda
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=3)
    exact = to_product(sine_exact(2, 2, 2))
    amp = torch.tensor([p["amp"] for p in spec["coef"]], dtype=torch.float64, requires_grad=True)
    cs = torch.tensor(spec["coef"][0]["cell_scale"], dtype=torch.float64, requires_grad=True)
    J = sg.energy_at_T(spec, exact, amp, cs, cell_piece=0, rtol=1e-13)
    J.backward()
    h = 1e-4
    for j in range(4):
        ap, am = amp.detach().clone(), amp.detach().clone()
        ap[j] += h * abs(float(ap[j]))
        am[j] -= h * abs(float(am[j]))
        fd = (float(sg.energy_at_T(spec, exact, ap, cs.detach(), cell_piece=0, rtol=1e-13)) -
              float(sg.energy_at_T(spec, exact, am, cs.detach(), cell_piece=0, rtol=1e-13))) / (float(ap[j] - am[j]))
        assert abs(float(amp.grad[j]) - fd) <= 2e-6 * float(amp.grad.abs().max()), (j, float(amp.grad[j]), fd)
    c = 9
    sp_, sm_ = cs.detach().clone(), cs.detach().clone()
    sp_[c] += 1e-4
    sm_[c] -= 1e-4
    fd = (float(sg.energy_at_T(spec, exact, amp.detach(), sp_, cell_piece=0, rtol=1e-13)) -
          float(sg.energy_at_T(spec, exact, amp.detach(), sm_, cell_piece=0, rtol=1e-13))) / 2e-4
    assert abs(float(cs.grad[c]) - fd) <= 2e-6 * float(cs.grad.abs().max())


def test_adjoint_errors(cuda):
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=2)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_mg_setup(ctx)
    with pytest.raises(sg.SGError, match="sg_set_exact"):
        sg.sg_adjoint_gradient(ctx)
    sg.sg_set_exact(ctx, to_product(sine_exact(2, 2, 2)))
    with pytest.raises(sg.SGError, match="cell_piece"):
        sg.sg_adjoint_gradient(ctx, cell_piece=9)
    with pytest.raises(sg.SGError, match="checkpoint"):
        sg.sg_adjoint_gradient(ctx, checkpoint_every=0)
    bad = [dict(p) for p in spec["coef"]]
    bad[1]["mu"] = (1, 1)
    with pytest.raises(sg.SGError, match="chaos index"):
        sg.sg_set_coefficient(ctx, bad)
    ctx.destroy()

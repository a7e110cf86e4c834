"""Pins of the oracle's slab operator (Problem "tensor-product slab system",
eq. local_rhs_tensor) against a brute-force evaluation of the slab bilinear
form of the discrete slab problem (eq. slab_discrete_problem): expectations
by tensor Gauss-Hermite quadrature in xi, time integrals by Gauss-Legendre
on the physical slab, space integrals by a higher-order Gauss rule per cell,
with the discrete functions built from the expansion of eq. discrete_expansion.

The coefficient modes are (bi)linear in x so that the operator's (k+1)-point
Gauss rule is exact and both sides compute the same number."""
import itertools

import numpy as np
import pytest
from numpy.polynomial import hermite_e as HE

from oracle import coeff, hermite, operator, space_fe, time_dg


def linear_pieces():
    one, px = ("one", 0), ("pow", 1)
    return [
        dict(mu=(0, 0), amp=1.0, factors=[one, one]),
        dict(mu=(0, 0), amp=0.3, factors=[px, one]),
        dict(mu=(0, 0), amp=0.2, factors=[px, px]),
        dict(mu=(1, 0), amp=0.2, factors=[px, one]),
        dict(mu=(0, 1), amp=-0.1, factors=[one, px]),
        dict(mu=(1, 1), amp=0.05, factors=[one, one]),
        dict(mu=(2, 0), amp=0.07, factors=[px, px]),
    ]


def brute_bilinear(p, U, V, nq_extra=2, n_gh=6, n_t=None):
    """E[ int_I <d_t u, v> + a(xi; u, v) dt ] + E[<u(t_{n-1}^+), v(t_{n-1}^+)>]."""
    mesh, tau = p.mesh, p.tau
    r = p.n_t - 1
    fe = space_fe.FE1D(mesh.k, mesh.k + 1 + nq_extra)
    wJ, phi, grad = space_fe.reference_shape(mesh, fe)
    cells = np.arange(mesh.n_cells)
    conn = mesh.cell_dofs(cells)
    xq = space_fe.cell_points(mesh, fe, cells)                       # (C, Q, d)
    amu = coeff.evaluate(p.spec["coef"], xq, np.broadcast_to(cells[:, None], xq.shape[:-1]))
    # stochastic quadrature
    g, gw = HE.hermegauss(n_gh)
    M = p.idx.shape[1]
    XI = np.array(list(itertools.product(g, repeat=M)))
    WXI = np.prod(np.array(list(itertools.product(gw, repeat=M))), axis=1) / (2 * np.pi) ** (M / 2)
    PsiA = np.stack([hermite.Psi(a, XI) for a in p.idx])               # (A, S)
    PsiMu = np.stack([hermite.Psi(mu, XI) for mu in p.mus])            # (T, S)
    a_xi = np.einsum('tcq,ts->cqs', amu, PsiMu)                        # a(x_q, xi_s)
    # time quadrature on the physical slab (0, tau]
    nodes = time_dg.radau_right_nodes(r)
    th, tw = time_dg.gauss_legendre_01(n_t or r + 3)
    vt = time_dg.lagrange_values(nodes, th)                            # (N_t, nt)
    dvt = time_dg.lagrange_derivs(nodes, th) / tau
    v0 = time_dg.lagrange_values(nodes, [0.0])[:, 0]
    tw = tw * tau
    Uc = U[:, :, conn]                                                 # (A, Nt, C, nloc)
    Vc = V[:, :, conn]
    u_x = np.einsum('aicl,lq->aicq', Uc, phi)
    v_x = np.einsum('aicl,lq->aicq', Vc, phi)
    gu_x = np.einsum('aicl,lqd->aicqd', Uc, grad)
    gv_x = np.einsum('aicl,lqd->aicqd', Vc, grad)
    # fields at (xi_s, t, x_q)
    u_s = np.einsum('as,aicq->sicq', PsiA, u_x)
    v_s = np.einsum('as,aicq->sicq', PsiA, v_x)
    gu_s = np.einsum('as,aicqd->sicqd', PsiA, gu_x)
    gv_s = np.einsum('as,aicqd->sicqd', PsiA, gv_x)
    dtu = np.einsum('it,sicq->stcq', dvt, u_s)
    vv = np.einsum('it,sicq->stcq', vt, v_s)
    gu = np.einsum('it,sicqd->stcqd', vt, gu_s)
    gv = np.einsum('it,sicqd->stcqd', vt, gv_s)
    mass = np.einsum('s,t,q,stcq,stcq->', WXI, tw, wJ, dtu, vv)
    stiff = np.einsum('s,t,q,cqs,stcqd,stcqd->', WXI, tw, wJ, a_xi, gu, gv)
    u0 = np.einsum('i,sicq->scq', v0, u_s)
    w0 = np.einsum('i,sicq->scq', v0, v_s)
    jump = np.einsum('s,q,scq,scq->', WXI, wJ, u0, w0)
    return mass + stiff + jump


@pytest.mark.parametrize("k,r,cells,hi", [(1, 1, (3, 2), (1.0, 0.7)),
                                           (2, 1, (2, 2), (1.0, 1.0)),
                                           (2, 2, (2, 3), (0.8, 1.0)),
                                           (3, 1, (2, 2), (1.0, 1.0))])
def test_operator_equals_weak_form(k, r, cells, hi):
    spec = dict(dim=2, cells=cells, lo=(0.0, 0.0), hi=hi, k=k, r=r, n_slabs=4, T=1.2,
                M=2, P=2, coef=linear_pieces())
    p = operator.SGProblem(spec)
    rng = np.random.default_rng(7)
    U = rng.uniform(-1, 1, p.shape)
    V = rng.uniform(-1, 1, p.shape)
    U[:, :, p.bmask] = 0.0
    V[:, :, p.bmask] = 0.0
    want = brute_bilinear(p, U, V)
    got = float(np.sum(V * p.apply(U)))
    assert abs(got - want) < 1e-12 * max(1.0, abs(want)), (got, want)
    # the transpose is the adjoint
    got_t = float(np.sum(U * p.apply(V, transpose=True)))
    assert abs(got_t - want) < 1e-12 * max(1.0, abs(want))


def test_operator_3d_weak_form():
    one, px = ("one", 0), ("pow", 1)
    pieces = [dict(mu=(0,), amp=1.0, factors=[one, one, one]),
              dict(mu=(1,), amp=0.2, factors=[px, one, px])]
    spec = dict(dim=3, cells=(2, 2, 2), lo=(0, 0, 0), hi=(1, 1, 1), k=2, r=1, n_slabs=2, T=0.5,
                M=1, P=2, coef=pieces)
    p = operator.SGProblem(spec)
    rng = np.random.default_rng(3)
    U = rng.uniform(-1, 1, p.shape)
    V = rng.uniform(-1, 1, p.shape)
    U[:, :, p.bmask] = 0.0
    V[:, :, p.bmask] = 0.0
    want = brute_bilinear(p, U, V, nq_extra=1)
    got = float(np.sum(V * p.apply(U)))
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))


def test_dirichlet_rows_identity_and_columns_ignored():
    spec = dict(dim=2, cells=(3, 3), lo=(0, 0), hi=(1, 1), k=2, r=1, n_slabs=2, T=1.0, M=2, P=1,
                coef=linear_pieces()[:4])
    p = operator.SGProblem(spec)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, p.shape)
    y = p.apply(x)
    assert np.array_equal(y[:, :, p.bmask], x[:, :, p.bmask])
    x2 = x.copy()
    x2[:, :, p.bmask] = rng.uniform(-1, 1, x2[:, :, p.bmask].shape)
    y2 = p.apply(x2)
    assert np.array_equal(y2[:, :, ~p.bmask], y[:, :, ~p.bmask])


def test_mean_only_coefficient_decouples_modes():
    # with a = a_0(x) only, G_0 = I and every chaos block is the same
    # deterministic space-time operator (block-diagonal in alpha)
    spec = dict(dim=2, cells=(3, 2), lo=(0, 0), hi=(1, 1), k=1, r=1, n_slabs=2, T=1.0, M=2, P=2,
                coef=linear_pieces()[:3])
    p = operator.SGProblem(spec)
    rng = np.random.default_rng(2)
    x = np.zeros(p.shape)
    x[3] = rng.uniform(-1, 1, p.shape[1:])
    y = p.apply(x)
    assert np.all(y[[0, 1, 2, 4, 5]][:, :, ~p.bmask] == 0.0)
    x0 = np.zeros(p.shape)
    x0[0] = x[3]
    assert np.allclose(p.apply(x0)[0], y[3], atol=1e-15)


def test_assembled_matrix_agrees():
    spec = dict(dim=2, cells=(3, 2), lo=(0, 0), hi=(1, 1), k=2, r=1, n_slabs=2, T=1.0, M=2, P=2,
                coef=linear_pieces())
    p = operator.SGProblem(spec)
    x = np.random.default_rng(5).uniform(-1, 1, p.shape)
    y = (p.assembled() @ x.reshape(-1)).reshape(p.shape)
    assert np.abs(y - p.apply(x)).max() < 1e-14


def test_node_row_apply_is_the_row_restriction_of_apply():
    """apply_node_rows (used to time bounded samples of the apply) returns
    exactly the selected node rows of apply, boundary rows included."""
    from paper_2605_21046_gb300 import inputs as I
    spec = dict(I.config_small_2d_q1(), cells=(7, 5))
    p = operator.SGProblem(spec)
    x = I.random_vector(spec, seed=3)
    full = p.apply(x)
    for rows in (np.arange(p.n_x), np.arange(10, 30), np.array([0, 5, p.n_x - 1, 17])):
        got = p.apply_node_rows(x, rows)
        assert got.shape == (p.n_xi, p.n_t, rows.size)
        assert np.allclose(got, full[:, :, rows], rtol=0, atol=1e-14 * np.abs(full).max())

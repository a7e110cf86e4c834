"""The mean error of the paper's finite-chaos benchmark at p = 0, computed a
second way (Sec. 4.3-4.4: eq. diffusion_benchmark, finite-exact-separated ..
finite-chaos-coefficients, manufactured_rhs_benchmark; Definition "error norms
and quantities").

At p = 0 the Galerkin system is the single mean equation
    d_t u_0 - div(E[a] grad u_0) = E[f] = d_t phi - div(E[a G_q] grad phi),
so e = phi - u_0 solves d_t e - div(E[a] grad e) = div((E[a G_q] - E[a]) grad phi),
e(0) = 0, and E_mean = ||e||_{L2_t(L2_x)} up to the space-time discretisation
error.  This test solves that problem with nothing from the oracle: E[a] and
E[a G_q] by tensor Gauss-Hermite quadrature of the formulas themselves, a
sine-series Galerkin method in space (the Dirichlet eigenbasis of (-1,1)^2) and
the exact solution in time of the resulting linear ODE system (generalised
eigenvectors of (K, M)).  The oracle's Q3 / dG(3) march must give the same
number; the value the paper prints for this entry (Table "finite-errors-rates")
is read from tests/golden/paper_table1.txt and is about 6x smaller."""
import itertools
import os
from math import comb, factorial, sqrt

import numpy as np
import scipy.linalg as sla
from numpy.polynomial.hermite_e import hermegauss, hermeval
from numpy.polynomial.legendre import leggauss

from oracle import manufactured, operator
from paper_2605_21046_gb300.inputs import paper_coefficient

ETA, D_MIN, M, Q = 0.35, 0.2, 4, 6
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _psi(n, y):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return hermeval(y, c) / sqrt(factorial(n))


def _chaos_moments(x1, x2):
    """E[a] and E[a G_q] at points, a = d_min + (sum xi_m g_m)^2 and
    G_q = sum_{|alpha| <= 6} c_alpha Psi_alpha, by 6-point Gauss-Hermite per
    variable (exact: degree <= 8 per variable)."""
    z, w = hermegauss(6)
    w = w / w.sum()
    xi = np.array(list(itertools.product(z, repeat=M)))                   # (n, M)
    wt = np.prod(np.array(list(itertools.product(w, repeat=M))), axis=1)
    gq = np.zeros(xi.shape[0])
    for alpha in itertools.product(range(Q + 1), repeat=M):
        if sum(alpha) <= Q:
            c = 1.0 if sum(alpha) == 0 else ETA ** sum(alpha)
            gq += c * np.prod([_psi(a, xi[:, m]) for m, a in enumerate(alpha)], axis=0)
    g = np.stack([x1 ** 2, x1 * x2, x2 ** 2, np.ones_like(x1)])
    a = D_MIN + np.tensordot(xi, g, axes=(1, 0)) ** 2                     # (n, ...)
    return np.tensordot(wt, a, 1), np.tensordot(wt * gq, a, 1)


def _g_lambda(lam, t):
    """g(t) = int_0^t exp(-lam (t - s)) s^4 ds: quadrature of the smooth form
    t^5 int_0^1 exp(-lam t v) (1 - v)^4 dv for lam t < 20, else the closed form
    (no cancellation there)."""
    v, w = leggauss(40)
    v, w = (v + 1) / 2, w / 2
    lt = lam * t
    quad = t ** 5 * (w[None, :] * np.exp(-lt[:, None] * v[None, :]) * (1 - v[None, :]) ** 4).sum(axis=1)
    closed = (t ** 4 / lam - 4 * t ** 3 / lam ** 2 + 12 * t ** 2 / lam ** 3 - 24 * t / lam ** 4
              + 24 / lam ** 5 - 24 * np.exp(-lt) / lam ** 5)
    return np.where(lt < 20.0, quad, closed)


def spectral_mean_error(N=24, nq=80):
    xq, wq = leggauss(nq)
    j = np.arange(1, N + 1)
    s = np.sin(np.outer(j, np.pi * (xq + 1) / 2))
    ds = (j[:, None] * np.pi / 2) * np.cos(np.outer(j, np.pi * (xq + 1) / 2))
    X1, X2 = np.meshgrid(xq, xq, indexing="ij")
    a0, abar = _chaos_moments(X1, X2)
    W = np.outer(wq, wq)
    V = np.einsum("ja,kb->jkab", s, s).reshape(N * N, nq, nq)
    Vx = np.einsum("ja,kb->jkab", ds, s).reshape(N * N, nq, nq)
    Vy = np.einsum("ja,kb->jkab", s, ds).reshape(N * N, nq, nq)
    Mm = np.einsum("iab,jab,ab->ij", V, V, W)
    Km = np.einsum("iab,jab,ab->ij", Vx, Vx, W * a0) + np.einsum("iab,jab,ab->ij", Vy, Vy, W * a0)
    # phi = t^4 Phi, Phi = sin(pi/2 (x1+1)) sin(pi/2 (x2+1)) = basis function (1, 1)
    r = -(np.einsum("iab,ab->i", Vx, W * (abar - a0) * Vx[0]) + np.einsum("iab,ab->i", Vy, W * (abar - a0) * Vy[0]))
    lam, U = sla.eigh(Km, Mm)                                             # U^T M U = I
    c = U.T @ r
    tq, tw = leggauss(60)
    tq, tw = (tq + 1) / 2, tw / 2
    return sqrt(sum(ck ** 2 * np.sum(tw * _g_lambda(lk, tq) ** 2) for lk, ck in zip(lam, c)))


def _paper_row(p_xi):
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_table1.txt"))
    return rows[rows[:, 0] == p_xi][0]


def test_spectral_solution_converges():
    e16, e24 = spectral_mean_error(16), spectral_mean_error(24)
    assert abs(e16 - e24) < 5e-5 * e24


def test_oracle_mean_error_at_p0_equals_the_spectral_solution():
    spec = dict(dim=2, cells=(4, 4), lo=(-1.0, -1.0), hi=(1.0, 1.0), k=3, r=3, n_slabs=4, T=1.0, M=M, P=0,
                coef=paper_coefficient())
    man = manufactured.Manufactured(operator.SGProblem(spec), manufactured.paper_exact())
    got = man.errors(man.march(4))["mean"]
    want = spectral_mean_error(24)
    assert abs(got - want) < 1e-4 * want, (got, want)
    # the printed entry is ~6x smaller: the printed mean column does not follow
    # from the problem as stated (its p = 0 full error and mean error agree
    # with each other, see test_printed_rows_are_consistent)
    printed = _paper_row(0)[3]
    assert 5.5 < want / printed < 7.0


def test_printed_rows_are_consistent():
    """The transcribed rows p = 0..3: the full error dominates the closed-form
    truncation error (eq. finite-truncation-error-L2, ||phi|| = 1/3) at every
    p, equals it in quadrature with the mean error at p = 0 (the only retained
    mode is the mean), and the mean error is unchanged under odd enrichment."""
    def trunc(p):
        return (1 / 3) * sqrt(sum(comb(k + 3, 3) * ETA ** (2 * k) for k in range(p + 1, Q + 1)))
    for p in range(4):
        row = _paper_row(p)
        assert row[1] == comb(M + p, p)
        assert row[2] > trunc(p)
    r0 = _paper_row(0)
    assert sqrt(r0[2] ** 2 - r0[3] ** 2) == __import__("pytest").approx(trunc(0), rel=1e-4)
    assert _paper_row(1)[3] == r0[3] and _paper_row(3)[3] == _paper_row(2)[3]

"""Pins of the oracle's Hermite chaos (Sec. 3.3, eq. triple_stoch) against
facts that do not come from the oracle itself: printed dimensions, Gauss-
Hermite quadrature of the defining integral, the closed form for E[xi psi_n
psi_m], orthonormality and the Hermite-root spectrum of the Jacobi matrix."""
import itertools
import os
from math import comb, factorial, sqrt

import numpy as np
from numpy.polynomial import hermite_e as HE

from oracle import hermite

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gauss_hermite_expect(fn, n=40):
    """E[fn(xi)] for xi ~ N(0,1) by numpy's Gauss-Hermite(e) rule."""
    x, w = HE.hermegauss(n)
    return float(np.sum(w * fn(x)) / sqrt(2 * np.pi))


def test_chaos_dimensions_match_paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "chaos_dims.txt"), dtype=int)
    for M, p, n in rows:
        assert hermite.multi_indices(M, p).shape == (n, M)
        assert comb(M + p, p) == n


def test_index_set_is_total_degree_and_graded():
    for M, p in [(2, 2), (3, 3), (4, 4), (1, 5)]:
        idx = hermite.multi_indices(M, p)
        assert len({tuple(a) for a in idx}) == idx.shape[0]
        assert idx.sum(axis=1).max() == p
        assert np.all(np.diff(idx.sum(axis=1)) >= 0)          # graded
        brute = {a for a in itertools.product(range(p + 1), repeat=M) if sum(a) <= p}
        assert {tuple(a) for a in idx} == brute
    assert hermite.multi_indices(2, 2).tolist() == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]


def test_psi_orthonormal_by_quadrature():
    for n in range(9):
        for m in range(9):
            v = _gauss_hermite_expect(lambda x: hermite.psi(n, x) * hermite.psi(m, x))
            assert abs(v - (n == m)) < 1e-12


def test_he_matches_numpy_hermite_e():
    x = np.linspace(-3, 3, 11)
    for n in range(10):
        c = np.zeros(n + 1)
        c[n] = 1
        assert np.allclose(hermite.he(n, x), HE.hermeval(x, c), rtol=1e-13, atol=1e-12)


def test_triple_1d_equals_gauss_hermite_quadrature():
    for a, b, c in itertools.product(range(7), repeat=3):
        q = _gauss_hermite_expect(lambda x: hermite.psi(a, x) * hermite.psi(b, x) * hermite.psi(c, x))
        assert abs(hermite.triple_1d(a, b, c) - q) < 1e-11, (a, b, c)


def test_triple_1d_linear_closed_form():
    # E[xi psi_n psi_m] = sqrt(n+1) d_{m,n+1} + sqrt(n) d_{m,n-1}  (psi_1 = xi)
    for n in range(10):
        for m in range(10):
            want = sqrt(n + 1) * (m == n + 1) + sqrt(n) * (m == n - 1)
            assert abs(hermite.triple_1d(1, n, m) - want) < 1e-14


def test_galerkin_matrices_identity_symmetry_and_spectrum():
    for M, P in [(2, 2), (3, 3), (4, 3), (4, 4)]:
        idx = hermite.multi_indices(M, P)
        G0 = hermite.galerkin_matrix((0,) * M, idx)
        assert np.array_equal(G0, np.eye(idx.shape[0]))      # M_xi = I
        # largest root of He_{P+1}
        c = np.zeros(P + 2)
        c[P + 1] = 1
        xmax = np.max(np.real(HE.hermeroots(c)))
        for m in range(M):
            mu = tuple(int(i == m) for i in range(M))
            G = hermite.galerkin_matrix(mu, idx)
            assert np.array_equal(G, G.T)
            ev = np.linalg.eigvalsh(G)
            assert ev.max() <= xmax + 1e-12 and ev.min() >= -xmax - 1e-12
            assert abs(ev.max() - xmax) < 1e-10                # attained
            assert np.all(np.diag(G) == 0.0)                   # E[xi_m psi_a^2] = 0


def test_galerkin_multivariate_by_tensor_quadrature():
    M, P = 2, 3
    idx = hermite.multi_indices(M, P)
    x, w = HE.hermegauss(12)
    X = np.array(list(itertools.product(x, repeat=M)))
    W = np.prod(np.array(list(itertools.product(w, repeat=M))), axis=1) / (2 * np.pi) ** (M / 2)
    for mu in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]:
        G = hermite.galerkin_matrix(mu, idx)
        pm = hermite.Psi(mu, X)
        for a in range(idx.shape[0]):
            pa = hermite.Psi(idx[a], X)
            for b in range(idx.shape[0]):
                q = np.sum(W * pm * pa * hermite.Psi(idx[b], X))
                assert abs(G[a, b] - q) < 1e-11

"""Pins of the chaos expansion of the paper's benchmark coefficient
a(x, xi) = d_min + (xi_1 x1^2 + xi_2 x1 x2 + xi_3 x2^2 + xi_4)^2 (Sec. 4,
eq. diffusion_benchmark; expansion eq. coeff_expansion).

The oracle projects it on the chaos by Gauss-Hermite quadrature; the library's
host preparation writes it down by Hermite linearisation.  Neither is trusted
here: both sums sum_mu a_mu(x) Psi_mu(xi) must reproduce the formula itself at
random (x, xi), and the two sets of modes must agree point by point.  A
planted mistake (a dropped cross term, sqrt(2) -> 1 on one mode) must fail."""
import numpy as np
import pytest

from oracle import coeff, hermite
from paper_2605_21046_gb300 import coefficients
from paper_2605_21046_gb300.inputs import paper_coefficient

M = 4


def _formula(x, xi, d_min=0.2):
    x1, x2 = x[..., 0], x[..., 1]
    lin = xi[..., 0] * x1 ** 2 + xi[..., 1] * x1 * x2 + xi[..., 2] * x2 ** 2 + xi[..., 3]
    return d_min + lin ** 2


def _he(n, y):
    # probabilists' Hermite polynomials from numpy's own series evaluation
    from math import factorial, sqrt
    from numpy.polynomial.hermite_e import hermeval
    c = np.zeros(n + 1)
    c[n] = 1.0
    return hermeval(y, c) / sqrt(factorial(n))


def _sum_of_modes(pieces, x, xi):
    amu = coeff.evaluate(pieces, x)                   # (n_terms, n)
    out = np.zeros(x.shape[0])
    for t, mu in enumerate(coeff.terms(pieces)):
        psi = np.ones(x.shape[0])
        for m, a in enumerate(mu):
            psi = psi * _he(int(a), xi[:, m])
        out += amu[t] * psi
    return out


def _points(n=50, seed=3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (n, 2)), rng.standard_normal((n, M)) * 1.5


@pytest.mark.parametrize("side", ["oracle", "library"])
def test_expansion_reproduces_the_formula(side):
    c = paper_coefficient()
    pieces = coeff.as_pieces(c, M) if side == "oracle" else coefficients.pieces(c, M)
    x, xi = _points()
    got = _sum_of_modes(pieces, x, xi)
    want = _formula(x, xi)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-13
    assert len(coeff.terms(pieces)) == 11          # 1 + 4 + 6 modes, all of even degree
    assert all(sum(mu) % 2 == 0 for mu in coeff.terms(pieces))


def test_oracle_and_library_modes_agree():
    c = paper_coefficient()
    po, pl = coeff.as_pieces(c, M), coefficients.pieces(c, M)
    to, tl = coeff.terms(po), coeff.terms(pl)
    assert set(to) == set(tl)
    x = np.random.default_rng(4).uniform(-1.0, 1.0, (40, 2))
    ao, al = coeff.evaluate(po, x), coeff.evaluate(pl, x)
    for t, mu in enumerate(to):
        assert np.allclose(ao[t], al[tl.index(mu)], rtol=1e-14, atol=1e-14), mu


@pytest.mark.parametrize("mutation", ["drop_cross", "sqrt2_to_1"])
def test_planted_mistake_fails(mutation):
    pieces = [dict(p) for p in coeff.as_pieces(paper_coefficient(), M)]
    if mutation == "drop_cross":
        k = next(i for i, p in enumerate(pieces) if sorted(p["mu"]) == [0, 0, 1, 1])
        pieces.pop(k)
    else:
        k = next(i for i, p in enumerate(pieces) if max(p["mu"]) == 2)
        pieces[k]["amp"] = 1.0
    x, xi = _points()
    assert np.max(np.abs(_sum_of_modes(pieces, x, xi) - _formula(x, xi))) > 1e-3


def test_mean_term_is_the_expectation():
    # E[a] = d_min + sum_m g_m^2 (xi_m independent, unit variance): mode 0
    x = np.random.default_rng(5).uniform(-1.0, 1.0, (30, 2))
    pieces = coeff.as_pieces(paper_coefficient(), M)
    a0 = coeff.evaluate(pieces, x)[coeff.terms(pieces).index((0,) * M)]
    x1, x2 = x[:, 0], x[:, 1]
    assert np.allclose(a0, 0.2 + x1 ** 4 + (x1 * x2) ** 2 + x2 ** 4 + 1.0, rtol=1e-14)
    # and hermite.Psi agrees with numpy's He_n on the grid used for the modes
    xi = np.random.default_rng(6).standard_normal((10, M))
    for mu in hermite.multi_indices(M, 2):
        want = np.prod([_he(int(a), xi[:, m]) for m, a in enumerate(mu)], axis=0)
        assert np.allclose(hermite.Psi(mu, xi), want, rtol=1e-13, atol=1e-14)

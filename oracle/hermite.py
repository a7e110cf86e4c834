"""Hermite chaos for the oracle (test infrastructure; see ``oracle/__init__``).

References (paper sections / equations):
  * eq. Hermit_def: probabilists' Hermite polynomials He_n and the normalised
    psi_n = He_n / sqrt(n!), orthonormal under the standard Gaussian density.
  * Sec. 3.3 (total-degree chaos space): Lambda_p = {alpha : |alpha|_1 <= p},
    N_xi = binom(M+p, p).
  * eq. triple_stoch: [G_mu]_{alpha beta} = E[Psi_mu Psi_alpha Psi_beta];
    the factorisation remark after it: the expectation is a product over the
    M independent coordinates of 1D triple products.

Readings (the paper is silent on them):
  * Ordering of Lambda_p: ascending total degree; inside one degree,
    alpha_1 descending, then alpha_2 descending, ... (for M=2, p=2:
    00, 10, 01, 20, 11, 02).
"""
from math import comb, factorial, sqrt

import numpy as np


def he(n, y):
    """He_n(y) by the three-term recurrence He_{k+1} = y He_k - k He_{k-1}
    (equivalent to the Rodrigues form of eq. Hermit_def)."""
    y = np.asarray(y, dtype=np.float64)
    h0 = np.ones_like(y)
    if n == 0:
        return h0
    h1 = y.copy()
    for k in range(1, n):
        h0, h1 = h1, y * h1 - k * h0
    return h1


def psi(n, y):
    """Orthonormal Hermite polynomial psi_n = He_n / sqrt(n!) (eq. Hermit_def)."""
    return he(n, y) / sqrt(factorial(n))


def multi_indices(M, p):
    """Total-degree index set Lambda_p in the graded order described in the
    module docstring (Sec. 3.3).  Returns an (N_xi, M) int array."""
    out = []

    def rec(m_left, deg):
        if m_left == 1:
            return [(deg,)]
        res = []
        for a in range(deg, -1, -1):
            for rest in rec(m_left - 1, deg - a):
                res.append((a,) + rest)
        return res

    for d in range(p + 1):
        out.extend(rec(M, d))
    arr = np.array(out, dtype=np.int64).reshape(-1, M)
    assert arr.shape[0] == comb(M + p, p)
    return arr


def triple_1d(a, b, c):
    """E[psi_a psi_b psi_c] for xi ~ N(0,1): the classical Hermite
    linearisation closed form.  With s = (a+b+c)/2 it is
    sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!) when s is an integer and
    s >= max(a, b, c), else 0."""
    tot = a + b + c
    if tot % 2:
        return 0.0
    s = tot // 2
    if s < a or s < b or s < c:
        return 0.0
    num = sqrt(float(factorial(a) * factorial(b) * factorial(c)))
    return num / float(factorial(s - a) * factorial(s - b) * factorial(s - c))


def triple(mu, alpha, beta):
    """[G_mu]_{alpha beta} = prod_m E[psi_{mu_m} psi_{alpha_m} psi_{beta_m}]
    (factorisation remark after eq. triple_stoch)."""
    v = 1.0
    for m in range(len(mu)):
        v *= triple_1d(int(mu[m]), int(alpha[m]), int(beta[m]))
        if v == 0.0:
            return 0.0
    return v


def galerkin_matrix(mu, idx):
    """Dense N_xi x N_xi matrix G_mu on the index set ``idx`` (eq. triple_stoch)."""
    n = idx.shape[0]
    G = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            G[a, b] = triple(mu, idx[a], idx[b])
    return G


def Psi(alpha, xi):
    """Psi_alpha(xi) = prod_m psi_{alpha_m}(xi_m) (tensorised basis, Sec. 3.3).
    ``xi`` has shape (..., M)."""
    xi = np.asarray(xi, dtype=np.float64)
    v = np.ones(xi.shape[:-1])
    for m, a in enumerate(alpha):
        v = v * psi(int(a), xi[..., m])
    return v

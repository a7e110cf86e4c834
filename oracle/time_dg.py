"""dG(r) time discretisation for the oracle (test infrastructure).

References:
  * Sec. 3.2: slabwise polynomials of degree r, right Gauss-Radau nodal basis
    on each slab I_n = (t_{n-1}, t_n].
  * eq. At: [A_t]_{ij} = int_{I_n} v_j' v_i dt + v_j(t_{n-1}^+) v_i(t_{n-1}^+).
  * eq. Bt: [B_t]_{ij} = int_{I_n} v_j v_i dt.
  * eq. Ct: [C_t]_{ij} = v_j^{(n-1)}(t_{n-1}^-) v_i^{(n)}(t_{n-1}^+).

Everything is computed on the reference slab [0, 1] and scaled to a slab of
length tau: A_t is scale free, B_t = tau * B_hat, C_t is scale free.
"""
import numpy as np
from numpy.polynomial import legendre as L


def radau_right_nodes(r):
    """The r+1 right Gauss-Radau points on [0, 1] (they include t = 1): the
    roots of P_r - P_{r+1} on [-1, 1], mapped by t = (x + 1) / 2."""
    if r == 0:
        return np.array([1.0])
    cr = np.zeros(r + 2)
    cr[r] = 1.0
    cr[r + 1] = -1.0
    x = np.sort(np.real(L.legroots(cr)))
    x[-1] = 1.0
    return (x + 1.0) / 2.0


def lagrange_values(nodes, t):
    """Values v_i(t) of the Lagrange basis on ``nodes``: shape (len(nodes), len(t))."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    V = np.ones((n, t.size))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[i] *= (t - nodes[j]) / (nodes[i] - nodes[j])
    return V


def lagrange_derivs(nodes, t):
    """Derivatives v_i'(t) of the Lagrange basis (product rule, term by term)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, t.size))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.ones(t.size) / (nodes[i] - nodes[k])
            for j in range(n):
                if j != i and j != k:
                    term = term * (t - nodes[j]) / (nodes[i] - nodes[j])
            D[i] += term
    return D


def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = L.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def time_matrices(r, tau):
    """Return (A_t, B_t, C_t) of eqs. At, Bt, Ct for dG(r) with the right
    Radau nodal basis on a slab of length tau.  The integrals are evaluated
    with an (r + 2)-point Gauss-Legendre rule, exact for the degree <= 2r
    integrands."""
    nodes = radau_right_nodes(r)
    tq, wq = gauss_legendre_01(r + 2)
    V = lagrange_values(nodes, tq)          # v_i(t_q)
    Dv = lagrange_derivs(nodes, tq)         # v_i'(t_q) on [0,1]
    v0 = lagrange_values(nodes, [0.0])[:, 0]
    v1 = lagrange_values(nodes, [1.0])[:, 0]
    # [A]_{ij} = int v_j' v_i + v_j(0) v_i(0); the slab length cancels.
    A = np.einsum('iq,jq,q->ij', V, Dv, wq) + np.outer(v0, v0)
    # [B]_{ij} = tau * int_0^1 v_j v_i
    B = tau * np.einsum('iq,jq,q->ij', V, V, wq)
    # [C]_{ij} = v_j^{prev}(1) v_i(0)
    C = np.outer(v0, v1)
    return A, B, C

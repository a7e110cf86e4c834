"""Coefficient expansion for the oracle (test infrastructure).

Reference: eq. coeff_expansion, a(x, xi) = sum_{mu in M_a} a_mu(x) Psi_mu(xi).

The coefficient is given as plain data: a list of separable pieces
    {"mu": (mu_1..mu_M), "amp": c, "factors": [(kind, k) per direction],
     "cell_scale": None or an array with one value per cell}
with factor f(s) = 1 ("one"), sin(k pi s) ("sin") or s**k ("pow") of the
physical coordinate s.  a_mu(x) is the sum of the pieces carrying mu, and
M_a lists the distinct mu in order of first appearance.
"""
import numpy as np


def terms(pieces):
    """Distinct chaos indices mu of the pieces, in order of first appearance."""
    mus = []
    for p in pieces:
        mu = tuple(int(v) for v in p["mu"])
        if mu not in mus:
            mus.append(mu)
    return mus


def _factor(kind, k, s):
    if kind == "one":
        return np.ones_like(s)
    if kind == "sin":
        return np.sin(k * np.pi * s)
    if kind == "pow":
        return s ** k
    raise ValueError(kind)


def evaluate(pieces, x, cell_of_point=None):
    """a_mu at points: x has shape (..., dim).  Returns (n_terms, ...).
    ``cell_of_point`` (same leading shape as x) is needed when a piece has
    a per-cell scale."""
    mus = terms(pieces)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((len(mus),) + x.shape[:-1])
    for p in pieces:
        t = mus.index(tuple(int(v) for v in p["mu"]))
        v = np.full(x.shape[:-1], float(p["amp"]))
        for d, (kind, k) in enumerate(p["factors"][: x.shape[-1]]):
            v = v * _factor(kind, k, x[..., d])
        if p.get("cell_scale") is not None:
            v = v * np.asarray(p["cell_scale"], dtype=np.float64)[cell_of_point]
        out[t] += v
    return out


def at_cell_points(pieces):
    """Adapter for ``space_fe``: evaluates a_mu at (n, nqd, dim) points of the
    cells ``cells`` (length n), passing each point's cell index for per-cell
    scales."""
    def f(xq, cells):
        cell = np.broadcast_to(np.asarray(cells)[:, None], xq.shape[:-1])
        return evaluate(pieces, xq, cell)
    return f

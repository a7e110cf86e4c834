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


def square_of_linear_pieces(coef, M):
    """Chaos modes of a coefficient of the form of eq. diffusion_benchmark,
    a(x, xi) = d_min + (sum_m xi_m g_m(x))^2, by projection (eq.
    coeff_expansion): a_mu(x) = E[a(x, xi) Psi_mu(xi)] for |mu| <= 2 (the
    expansion is exact there: a is quadratic in xi).  Each expectation
    E[xi_m xi_n Psi_mu] is taken by tensor Gauss-Hermite quadrature with three
    points per variable (exact up to degree 5 in every variable).

    ``coef`` = {"form": "square_of_linear", "d_min": d, "g": [factors of g_m]}
    with each g_m a product of "one" / "pow" factors per direction; returns
    separable pieces (products g_m g_n stay separable)."""
    from numpy.polynomial.hermite_e import hermegauss
    from . import hermite
    g = coef["g"]
    assert len(g) == M
    z, w = hermegauss(3)
    w = w / w.sum()
    grid = np.stack(np.meshgrid(*([z] * M), indexing="ij"), axis=-1).reshape(-1, M)
    wts = np.prod(np.stack(np.meshgrid(*([w] * M), indexing="ij"), axis=-1).reshape(-1, M), axis=1)
    dim = len(g[0])

    def prod_factors(f1, f2):
        out = []
        for d in range(dim):
            e = 0
            for kind, k in (f1[d], f2[d]):
                if kind == "pow":
                    e += int(k)
                elif kind != "one":
                    raise ValueError("square_of_linear: factors must be 'one' or 'pow'")
            out.append(("pow", e) if e else ("one", 0))
        return out

    pieces = []
    for mu in hermite.multi_indices(M, 2):
        psi_mu = hermite.Psi(mu, grid)
        mean = float(np.sum(wts * psi_mu))
        if abs(mean) > 1e-12:
            pieces.append(dict(mu=tuple(int(v) for v in mu), amp=coef["d_min"] * mean,
                               factors=[("one", 0)] * dim, cell_scale=None))
        for m in range(M):
            for n in range(m, M):
                e = float(np.sum(wts * grid[:, m] * grid[:, n] * psi_mu))
                amp = e if m == n else 2.0 * e          # xi_m xi_n g_m g_n and xi_n xi_m g_n g_m
                if abs(amp) > 1e-12:
                    pieces.append(dict(mu=tuple(int(v) for v in mu), amp=amp,
                                       factors=prod_factors(g[m], g[n]), cell_scale=None))
    return pieces


def as_pieces(coef, M):
    """Separable pieces for either coefficient form: a list of pieces is
    returned as it is; a ``square_of_linear`` description is projected."""
    if isinstance(coef, dict):
        if coef.get("form") != "square_of_linear":
            raise ValueError(f"unknown coefficient form {coef.get('form')}")
        return square_of_linear_pieces(coef, M)
    return coef

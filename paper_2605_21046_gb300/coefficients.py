"""Host-side preparation of sg_setup's coefficient pieces.

sg_setup takes the coefficient as separable pieces on the Hermite chaos,
a(x, xi) = sum_mu a_mu(x) Psi_mu(xi) (eq. coeff_expansion).  A coefficient
given in its physical form must first be written on that basis; this module
does it for the form of the paper's benchmark (Sec. 4, eq.
diffusion_benchmark):

    a(x, xi) = d_min + (sum_m xi_m g_m(x))^2,

described as {"form": "square_of_linear", "d_min": d, "g": [g_m factors]}
with every g_m a product of "one" / "pow" factors per direction.  With the
orthonormal psi_2(y) = (y^2 - 1)/sqrt(2) (eq. Hermit_def) one has
xi_m^2 = sqrt(2) Psi_{2 e_m} + 1 and, for m != n, xi_m xi_n = Psi_{e_m + e_n},
so a has the mean term d_min + sum_m g_m^2, sqrt(2) g_m^2 on Psi_{2 e_m} and
2 g_m g_n on Psi_{e_m + e_n} (m < n): 1 + M + M(M-1)/2 chaos terms.
"""
from math import sqrt


def _times(f1, f2):
    out = []
    for a, b in zip(f1, f2):
        e = 0
        for kind, k in (a, b):
            if kind == "pow":
                e += int(k)
            elif kind != "one":
                raise ValueError("square_of_linear: factors must be 'one' or 'pow'")
        out.append(("pow", e) if e else ("one", 0))
    return out


def square_of_linear(coef, M):
    """Separable Hermite pieces of d_min + (sum_m xi_m g_m(x))^2."""
    g = coef["g"]
    if len(g) != M:
        raise ValueError(f"square_of_linear: {len(g)} functions g_m for M = {M}")
    dim = len(g[0])
    zero = (0,) * M

    def e(*ms):
        return tuple(sum(1 for m in ms if m == i) for i in range(M))

    pieces = [dict(mu=zero, amp=float(coef["d_min"]), factors=[("one", 0)] * dim, cell_scale=None)]
    for m in range(M):
        gg = _times(g[m], g[m])
        pieces.append(dict(mu=zero, amp=1.0, factors=gg, cell_scale=None))
        pieces.append(dict(mu=e(m, m), amp=sqrt(2.0), factors=gg, cell_scale=None))
    for m in range(M):
        for n in range(m + 1, M):
            pieces.append(dict(mu=e(m, n), amp=2.0, factors=_times(g[m], g[n]), cell_scale=None))
    return pieces


def pieces(coef, M):
    """sg_setup's pieces for either coefficient form: a list of pieces passes
    through; a ``square_of_linear`` description is expanded as above."""
    if isinstance(coef, dict):
        if coef.get("form") != "square_of_linear":
            raise ValueError(f"unknown coefficient form {coef.get('form')}")
        return square_of_linear(coef, M)
    return coef

"""Seeded synthetic inputs: the problem specs of the benchmark workloads and
the random vectors fed to the operator.  Plain data only - no part of the
method is computed here; the library and the oracle each discretise a spec
on their own.

Spec format: dict(dim, cells, lo, hi, k, r, n_slabs, T, M, P, coef), coef
either a list of separable pieces {"mu", "amp", "factors": [(kind, k) per
direction], "cell_scale": None | per-cell values} describing
a(x, xi) = sum_mu a_mu(x) Psi_mu(xi) when every mu is a first-degree or zero
index (then Psi_mu is xi_m or 1 and the pieces are the coefficient as
written), or {"form": "square_of_linear", "d_min", "g"} for
a = d_min + (sum_m xi_m g_m(x))^2, which the library and the oracle each
expand on the chaos themselves.
"""
import numpy as np

SEED_X = 2605_21046


def _e(m, M):
    return tuple(int(i == m) for i in range(M))


def linear_sine_coef(M, dim, sigma, freqs, a0=1.0, a0_cells=None):
    """a = a0 + sum_m sigma * prod_{d in active dims} sin(f_m,d pi x_d) * xi_m."""
    one = ("one", 0)
    pieces = [dict(mu=(0,) * M, amp=a0, factors=[one] * dim, cell_scale=a0_cells)]
    for m in range(M):
        pieces.append(dict(mu=_e(m, M), amp=sigma,
                           factors=[("sin", f) if f > 0 else one for f in freqs[m]],
                           cell_scale=None))
    return pieces


def config_small_2d_q1():
    """8x8 Q1 unit square, dG(1) 10 slabs, M=2, P=2 (6 modes);
    a = 1 + 0.1 xi_1 sin(pi x) + 0.1 xi_2 sin(pi y)."""
    return dict(name="2d-q1-8x8-M2P2", dim=2, cells=(8, 8), lo=(0.0, 0.0), hi=(1.0, 1.0), k=1, r=1,
                n_slabs=10, T=1.0, M=2, P=2,
                coef=linear_sine_coef(2, 2, 0.1, [(1, 0), (0, 1)]))


def config_2d_q2_64():
    """64x64 Q2 unit square, dG(1) 100 slabs, M=4, P=3 (35 modes);
    a_m = 0.05 sin(m pi x) sin(m pi y), a_0 = 1."""
    return dict(name="2d-q2-64x64-M4P3", dim=2, cells=(64, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), k=2,
                r=1, n_slabs=100, T=1.0, M=4, P=3,
                coef=linear_sine_coef(4, 2, 0.05, [(m, m) for m in range(1, 5)]))


def config_3d_q2_32():
    """32^3 Q2 unit cube, dG(1) 20 slabs, M=3, P=3 (20 modes);
    a_m = 0.05 prod_d sin(m pi x_d), a_0 = 1."""
    return dict(name="3d-q2-32x32x32-M3P3", dim=3, cells=(32, 32, 32), lo=(0.0,) * 3, hi=(1.0,) * 3,
                k=2, r=1, n_slabs=20, T=1.0, M=3, P=3,
                coef=linear_sine_coef(3, 3, 0.05, [(m, m, m) for m in range(1, 4)]))


def config_2d_q2_128(seed=128):
    """128x128 Q2 unit square, dG(1) 50 slabs, M=4, P=4 (70 modes);
    a_0 a per-cell field (seeded, in [0.8, 1.2]), a_m = 0.05 sin(m pi x) sin(m pi y)."""
    a0 = np.random.default_rng(seed).uniform(0.8, 1.2, 128 * 128)
    return dict(name="2d-q2-128x128-M4P4", dim=2, cells=(128, 128), lo=(0.0, 0.0), hi=(1.0, 1.0),
                k=2, r=1, n_slabs=50, T=1.0, M=4, P=4,
                coef=linear_sine_coef(4, 2, 0.05, [(m, m) for m in range(1, 5)], a0_cells=a0))


def paper_coefficient(d_min=0.2):
    """The paper's benchmark coefficient d_min + (xi1 x1^2 + xi2 x1 x2 + xi3 x2^2 + xi4)^2
    (Sec. 4, eq. diffusion_benchmark) in its physical form: d_min and the four
    functions g = (x1^2, x1 x2, x2^2, 1) multiplying xi_1..xi_4.  Each side
    writes it on the Hermite chaos with its own code."""
    one = ("one", 0)
    g = [[("pow", 2), one], [("pow", 1), ("pow", 1)], [one, ("pow", 2)], [one, one]]
    return dict(form="square_of_linear", d_min=float(d_min), g=g)


def config_paper_q3(cells=128, P=3, n_slabs=64):
    """The paper's finite-chaos benchmark discretisation (Sec. 4.3-4.4): D = (-1, 1)^2,
    Q3 in space, dG(3) in time, T = 1, M = 4, total degree P, the squared coefficient
    above with d_min = 0.2; 128^2 cells and tau = 1/64 are the sizes of its tables."""
    return dict(name=f"2d-q3-dg3-{cells}x{cells}-M4P{P}-paper", dim=2, cells=(cells, cells), lo=(-1.0, -1.0),
                hi=(1.0, 1.0), k=3, r=3, n_slabs=n_slabs, T=1.0, M=4, P=P, coef=paper_coefficient())


def config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=3, M=2, P=2, seed=None):
    """A small coefficient-gradient case: a = a0(x) + 0.2 x^2 + 0.1 xi_1
    sin(pi x) + 0.1 xi_2 sin(pi y) on the unit square, a0 a per-cell field
    (all ones, or seeded in [0.8, 1.2] when ``seed`` is given); four pieces,
    the first two on the mean term.  The manufactured forcing in strong form
    is only defined for a smooth coefficient, hence the default of ones."""
    n_cells = int(np.prod(cells))
    a0 = np.ones(n_cells) if seed is None else np.random.default_rng(seed).uniform(0.8, 1.2, n_cells)
    coef = linear_sine_coef(M, 2, 0.1, [(1, 0), (0, 1)] + [(1, 1)] * (M - 2), a0_cells=a0)
    coef.insert(1, dict(mu=(0,) * M, amp=0.2, factors=[("pow", 2), ("one", 0)], cell_scale=None))
    return dict(name=f"2d-q{k}-{cells[0]}x{cells[1]}-dG{r}-adjoint", dim=2, cells=tuple(cells), lo=(0.0, 0.0),
                hi=(1.0, 1.0), k=k, r=r, n_slabs=n_slabs, T=1.0, M=M, P=P, coef=coef)


def scaled(spec, cells, name=None):
    """The same problem on another mesh (per-cell fields are redrawn)."""
    s = dict(spec)
    s["cells"] = tuple(cells)
    s["name"] = name or f"{spec['name']}@{'x'.join(map(str, cells))}"
    coef = []
    n_cells = int(np.prod(cells[: spec["dim"]]))
    for p in spec["coef"]:
        p = dict(p)
        if p.get("cell_scale") is not None:
            p["cell_scale"] = np.random.default_rng(n_cells).uniform(0.8, 1.2, n_cells)
        coef.append(p)
    s["coef"] = coef
    return s


def n_nodes(spec):
    n = 1
    for d in range(spec["dim"]):
        n *= spec["k"] * spec["cells"][d] + 1
    return n


def n_modes(spec):
    from math import comb
    return comb(spec["M"] + spec["P"], spec["P"])


def n_unknowns(spec):
    return n_modes(spec) * (spec["r"] + 1) * n_nodes(spec)


def random_vector(spec, seed=SEED_X):
    """x ~ U(-1, 1), float64, flat slab vector (boundary entries included)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n_unknowns(spec))


def boundary_mask(spec):
    """True at the nodes on the domain boundary (lexicographic, x fastest)."""
    nn = [spec["k"] * spec["cells"][d] + 1 for d in range(spec["dim"])]
    grids = np.meshgrid(*[np.arange(n) for n in reversed(nn)], indexing="ij")
    mask = np.zeros(tuple(reversed(nn)), dtype=bool)
    for d in range(spec["dim"]):
        g = grids[spec["dim"] - 1 - d]
        mask |= (g == 0) | (g == nn[d] - 1)
    return mask.reshape(-1)


def random_rhs(spec, seed=SEED_X + 1):
    """A right-hand side ~ U(-1, 1) that vanishes on Dirichlet nodes."""
    b = random_vector(spec, seed).reshape(n_modes(spec), spec["r"] + 1, n_nodes(spec))
    b[:, :, boundary_mask(spec)] = 0.0
    return b.reshape(-1)

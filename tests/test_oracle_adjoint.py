"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) on the CPU.

The adjoint gradient is checked against central finite differences of the
oracle's own marching (a plain forward computation already pinned by the
manufactured-solution tests), with the load vector held at the nominal
coefficient on both sides.  Its pieces are pinned separately: the adjoint
transfer by the dot-product identity <J u, v> = <u, J^T v>, the terminal source
by differentiating J(U) = sum_alpha U[alpha, r]^T M_x U[alpha, r] directly.

FD tolerance: J is a smooth rational function of the coefficient; with a
relative step h = 1e-4 the central difference has truncation error O(h^2)
~ 1e-8 relative and rounding error ~ eps / h ~ 1e-12, so 2e-6 relative leaves
a wide margin while a dropped term, a sign or a transposed time matrix is
off by O(1)."""
import numpy as np
import pytest

from oracle import adjoint, hermite, manufactured, operator
from paper_2605_21046_gb300 import inputs as I


def sine_exact(M, q, dim, eta=0.35, T=(0.0, 1.0, 1.0)):
    idx = hermite.multi_indices(M, q)
    c = [1.0 if not any(a) else eta ** int(sum(a)) for a in idx]
    phi = [[("sin", 1 + (int(a[d % M]) % 2)) for d in range(dim)] for a in idx]
    return {"q": q, "c": c, "phi": phi, "T": list(T)}


FD_TOL = 2e-6


def _fd(spec, exact, amp=None, cell_piece=-1, cells=None, c_idx=None, h=1e-4):
    base_amp = np.array([p["amp"] for p in spec["coef"]])
    if c_idx is None:
        a_p, a_m = base_amp.copy(), base_amp.copy()
        step = h * abs(base_amp[amp])
        a_p[amp] += step
        a_m[amp] -= step
        Jp = adjoint.energy(adjoint.with_coefficient(spec, a_p), spec, exact)
        Jm = adjoint.energy(adjoint.with_coefficient(spec, a_m), spec, exact)
        return (Jp - Jm) / (2 * step)
    s0 = np.ones(np.prod(spec["cells"])) if cells is None else np.asarray(cells, dtype=np.float64)
    sp_, sm_ = s0.copy(), s0.copy()
    step = h * abs(s0[c_idx])
    sp_[c_idx] += step
    sm_[c_idx] -= step
    Jp = adjoint.energy(adjoint.with_coefficient(spec, None, cell_piece, sp_), spec, exact)
    Jm = adjoint.energy(adjoint.with_coefficient(spec, None, cell_piece, sm_), spec, exact)
    return (Jp - Jm) / (2 * step)


@pytest.mark.parametrize("k,r,seed", [(1, 1, 7), (2, 0, None), (1, 2, 7)])
def test_gradient_matches_central_differences(k, r, seed):
    spec = I.config_adjoint_2d(cells=(4, 4), k=k, r=r, n_slabs=3, seed=seed)
    exact = sine_exact(2, 2, 2)
    J, g_amp, g_cell = adjoint.gradient(spec, exact, cell_piece=0)
    assert J > 0
    scale = np.abs(g_amp).max()
    for j in range(len(spec["coef"])):
        fd = _fd(spec, exact, amp=j)
        assert abs(g_amp[j] - fd) <= FD_TOL * scale, (j, g_amp[j], fd)
    cells = spec["coef"][0]["cell_scale"]
    cscale = np.abs(g_cell).max()
    for c in (0, 5, 10, 15):
        fd = _fd(spec, exact, cell_piece=0, cells=cells, c_idx=c)
        assert abs(g_cell[c] - fd) <= FD_TOL * cscale, (c, g_cell[c], fd)


def test_cell_gradient_sums_to_amplitude_gradient():
    """a0 scales both the amplitude and every cell of piece 0, so
    amp_0 dJ/d amp_0 = sum_c s_c dJ/d s_c (Euler's identity for the bilinear
    dependence of a on (amp, s))."""
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=2, seed=3)
    exact = sine_exact(2, 2, 2)
    _, g_amp, g_cell = adjoint.gradient(spec, exact, cell_piece=0)
    s = spec["coef"][0]["cell_scale"]
    a0 = spec["coef"][0]["amp"]
    assert abs(a0 * g_amp[0] - float(s @ g_cell)) <= 1e-12 * abs(a0 * g_amp[0])


def test_transfer_transpose_dot_product():
    spec = I.config_adjoint_2d(cells=(4, 4), k=2, r=2, n_slabs=3)
    op = operator.SGProblem(spec)
    rng = np.random.default_rng(11)
    u, v = rng.standard_normal(op.shape), rng.standard_normal(op.shape)
    lhs = float(np.sum(op.transfer(u) * v))
    rhs = float(np.sum(u * adjoint.transfer_transpose(op, v)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # and it is not the untransposed transfer (C_t is not symmetric)
    assert np.abs(adjoint.transfer_transpose(op, v) - op.transfer(v)).max() > 1e-3


def test_terminal_source_is_gradient_of_J():
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=1)
    op = operator.SGProblem(spec)
    rng = np.random.default_rng(12)
    U = rng.standard_normal(op.shape)
    U[:, :, op.bmask] = 0.0
    d = rng.standard_normal(op.shape)
    d[:, :, op.bmask] = 0.0
    h = 1e-6
    fd = (adjoint.energy_of(op, U + h * d) - adjoint.energy_of(op, U - h * d)) / (2 * h)
    g = adjoint.terminal_source(op, U)
    assert abs(float(np.sum(g * d)) - fd) <= 1e-8 * abs(fd)


def test_adjoint_states_solve_transposed_systems():
    """Each lam_n solves A^T lam_n = source_n (residual of the assembled
    transpose), the last one with the terminal source."""
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=3)
    exact = sine_exact(2, 2, 2)
    op = operator.SGProblem(spec)
    man = manufactured.Manufactured(operator.SGProblem(spec), exact)
    Us = adjoint.march(op, man)
    lams = adjoint.adjoint_states(op, Us)
    AT = op.assembled().T
    src = adjoint.terminal_source(op, Us[-1])
    for n in range(2, -1, -1):
        res = AT @ lams[n].reshape(-1) - src.reshape(-1)
        assert np.abs(res).max() <= 1e-12 * np.abs(src).max()
        src = adjoint.transfer_transpose(op, lams[n])


def test_march_matches_manufactured_march():
    """The adjoint module's LU marching equals the FGMRES marching of
    oracle.manufactured (same slabs, nominal coefficient)."""
    spec = I.config_adjoint_2d(cells=(4, 4), k=1, r=1, n_slabs=2)
    exact = sine_exact(2, 2, 2)
    op = operator.SGProblem(spec)
    man = manufactured.Manufactured(op, exact)
    a = adjoint.march(op, man)
    b = man.march(2)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-10 * np.abs(y).max()


def test_gradient_3d_matches_central_differences():
    """The same pin on a 3D 3x3x3 Q1 mesh: every amplitude and two cells."""
    cells = (3, 3, 3)
    coef = I.linear_sine_coef(2, 3, 0.08, [(1, 1, 1), (2, 1, 1)],
                              a0_cells=np.random.default_rng(4).uniform(0.8, 1.2, 27))
    spec = dict(dim=3, cells=cells, lo=(0.0,) * 3, hi=(1.0,) * 3, k=1, r=1, n_slabs=2, T=0.4, M=2, P=1, coef=coef)
    exact = {"q": 1, "c": [1.0, 0.3, 0.2], "phi": [[("sin", 1)] * 3] * 3, "T": [0.0, 1.0, 1.0]}
    J, g_amp, g_cell = adjoint.gradient(spec, exact, cell_piece=0)
    scale = np.abs(g_amp).max()
    for j in range(len(spec["coef"])):
        fd = _fd(spec, exact, amp=j)
        assert abs(g_amp[j] - fd) <= FD_TOL * scale, (j, g_amp[j], fd)
    cscale = np.abs(g_cell).max()
    for c in (0, 13):
        fd = _fd(spec, exact, cell_piece=0, cells=coef[0]["cell_scale"], c_idx=c)
        assert abs(g_cell[c] - fd) <= FD_TOL * cscale, (c, g_cell[c], fd)

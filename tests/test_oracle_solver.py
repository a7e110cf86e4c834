"""Pins of the oracle's slab solver pieces (Sec. 3.5, remark on the algebraic
solver): the multigrid preconditioner against exact solves, the Q_k
prolongation against exact polynomial interpolation, multigrid contraction,
the diagonal classes of the block-Jacobi splitting, and FGMRES against a
sparse direct solve."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import operator, solver, space_fe
from paper_2605_21046_gb300 import inputs as I


def spec2(cells, k=1, r=1, M=2, P=2, hi=(1.0, 1.0), coef=None):
    freqs = [((m % 3) + 1, ((m + 1) % 3) + 1) for m in range(M)]
    return dict(dim=2, cells=cells, lo=(0.0, 0.0), hi=hi, k=k, r=r, n_slabs=4, T=1.0, M=M, P=P,
                coef=coef or I.linear_sine_coef(M, 2, 0.08, freqs))


def block_diagonal(p):
    """The assembled slab matrix with every off-diagonal chaos block removed."""
    A = p.assembled().tocsr()
    n = p.n_t * p.n_x
    blk = np.repeat(np.arange(p.n_xi), n)
    coo = A.tocoo()
    keep = blk[coo.row] == blk[coo.col]
    return sp.csr_matrix((coo.data[keep], (coo.row[keep], coo.col[keep])), shape=A.shape)


def test_single_level_preconditioner_is_exact_block_jacobi():
    # 5x3 cells cannot be coarsened: the V-cycle is the coarse solve, so the
    # preconditioner is exactly the inverse of the block-diagonal part
    p = operator.SGProblem(spec2((5, 3), k=2))
    mg = solver.Multigrid(p)
    assert len(mg.levels) == 1
    r = np.random.default_rng(0).uniform(-1, 1, p.shape)
    want = spla.spsolve(block_diagonal(p).tocsc(), r.reshape(-1)).reshape(p.shape)
    assert np.abs(mg.apply(r) - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_interpolates_polynomials_exactly(k):
    s = spec2((8, 4), k=k)
    specs = solver.coarse_specs(s, coarse_dofs=0)
    A = np.eye(2)
    keys = [np.array([1.0, 0.0, 0.0])]
    fine = solver.Level(specs[0], A, 0.1 * A, keys, False)
    coarse = solver.Level(specs[1], A, 0.1 * A, keys, True)
    P = solver.prolongation(fine, coarse)
    xc, xf = coarse.mesh.node_coords(), fine.mesh.node_coords()
    if k >= 2:
        # degree <= k per direction and zero on the boundary: exact everywhere
        g = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1]) * (1 + 0.3 * X[:, 0] * (k == 3))
        sel = np.ones(fine.mesh.n_nodes, dtype=bool)
    else:
        # bilinear, exact where the coarse cell has no boundary node
        g = lambda X: X[:, 0] * X[:, 1] + 0.5
        ijk = fine.mesh.node_coords_idx(np.arange(fine.mesh.n_nodes))
        sel = np.all((ijk >= 2) & (ijk <= np.array(fine.mesh.nn) - 3), axis=1)
    uc = g(xc)
    uc[coarse.bmask] = 0.0
    uf = P @ uc
    want = g(xf)
    want[fine.bmask] = 0.0
    assert sel.sum() > 4
    assert np.abs(uf[sel] - want[sel]).max() < 1e-13


def test_coarsest_level_rule():
    """Coarsening stops at the first level with at most coarse_dofs interior
    space-time unknowns per mode (N_t x interior nodes), or where a cell
    count turns odd or reaches 2; coarse_dofs = 0 coarsens to two cells."""
    cells = lambda specs: [sp_["cells"][0] for sp_ in specs]
    assert solver.interior_dofs(I.config_2d_q2_64()) == 2 * 127 * 127
    assert solver.interior_dofs(I.scaled(I.config_3d_q2_32(), (4, 4, 4))) == 2 * 7 ** 3
    assert cells(solver.coarse_specs(I.config_2d_q2_64())) == [64, 32, 16, 8]          # 8^2: 450 unknowns
    assert cells(solver.coarse_specs(I.config_2d_q2_64(), coarse_dofs=0)) == [64, 32, 16, 8, 4, 2]
    assert cells(solver.coarse_specs(I.config_3d_q2_32())) == [32, 16, 8, 4]             # 4^3: 686
    assert cells(solver.coarse_specs(I.config_3d_q2_32(), coarse_dofs=0)) == [32, 16, 8, 4, 2]
    assert cells(solver.coarse_specs(I.config_small_2d_q1())) == [8]                    # 98: one level
    assert cells(solver.coarse_specs(spec2((12, 12), k=2), coarse_dofs=0)) == [12, 6, 3]  # odd count ends it
    assert cells(solver.coarse_specs(spec2((16, 16), k=2), coarse_dofs=1922)) == [16]   # at the limit: stop
    assert cells(solver.coarse_specs(spec2((16, 16), k=2), coarse_dofs=1921)) == [16, 8]


def test_multigrid_contracts():
    for s in (I.config_small_2d_q1(), spec2((16, 16), k=2), spec2((8, 8), k=2, hi=(1.0, 0.5))):
        p = operator.SGProblem(s)
        mg = solver.Multigrid(p, coarse_dofs=0)
        assert len(mg.levels) >= 3
        b = np.random.default_rng(1).uniform(-1, 1, p.shape)
        b[:, :, p.bmask] = 0.0
        x = np.zeros(p.shape)
        norms = []
        for _ in range(6):
            r = b - p.apply(x)
            norms.append(np.linalg.norm(r))
            x = x + mg.apply(r)
        rates = np.array(norms[1:]) / np.array(norms[:-1])
        assert rates[-1] < 0.35, rates


def test_diagonal_classes():
    p = operator.SGProblem(I.config_small_2d_q1())
    keys, cls = solver.diagonal_classes(p.G)
    assert len(keys) == 1                      # xi-linear: every diagonal block is the mean block
    # the paper's even coefficient: different diagonal blocks
    from paper_2605_21046_gb300.inputs import paper_coefficient
    s = dict(dim=2, cells=(2, 2), lo=(-1.0, -1.0), hi=(1.0, 1.0), k=1, r=1, n_slabs=4, T=1.0, M=4, P=2,
             coef=paper_coefficient())
    q = operator.SGProblem(s)
    keys, cls = solver.diagonal_classes(q.G)
    assert len(keys) == 15


def test_fgmres_matches_direct_solve():
    for s in (I.config_small_2d_q1(), spec2((8, 8), k=2, M=2, P=3)):
        p = operator.SGProblem(s)
        mg = solver.Multigrid(p)
        b = np.random.default_rng(3).uniform(-1, 1, p.shape)
        b[:, :, p.bmask] = 0.0
        x, its, res = solver.fgmres(p, b, mg.apply, rtol=1e-10)
        xd = solver.direct_solve(p, b)
        assert res <= 1e-10
        assert np.abs(x.reshape(p.shape) - xd).max() <= 1e-8 * np.abs(xd).max()
        assert its < 30


def test_round_bf16_rounds_to_nearest_even():
    """Hand-made cases at 1.0 (bf16 spacing 2^-7 there), then agreement with
    torch's own float32 -> bfloat16 conversion on random values."""
    torch = pytest.importorskip("torch")
    h = 2.0 ** -8
    vals = np.array([1.0, 1.0 + h, 1.0 + 3 * h, 1.0 + h + 2.0 ** -20, -(1.0 + 3 * h), 1.0 - 2.0 ** -9, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 4 * h, 1.0 + 2 * h, -(1.0 + 4 * h), 1.0, 0.0])
    assert np.array_equal(solver.round_bf16(vals), want)
    x = np.random.default_rng(5).standard_normal(10000) * np.exp(np.random.default_rng(6).uniform(-20, 20, 10000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(solver.round_bf16(x), ref)


def test_vcycle_with_bf16_factors_still_contracts():
    """The V-cycle with bf16-rounded Vanka inverses remains a contraction for
    the block operator (error reduction per cycle well below 1), close to the
    exact-factor cycle's."""
    spec = spec2((16, 16), k=2)
    p = operator.SGProblem(spec)
    rates = []
    for fr in (None, solver.round_bf16):
        mg = solver.Multigrid(p, factor_round=fr)
        L = mg.levels[0]
        A = L.A[0]
        e = np.random.default_rng(3).standard_normal(A.shape[0])
        e[np.tile(L.bmask, L.n_t)] = 0.0
        for _ in range(3):
            e = e - mg.vcycle_block(0, A @ e)
        n0 = np.linalg.norm(e)
        e = e - mg.vcycle_block(0, A @ e)
        rates.append(np.linalg.norm(e) / n0)
    assert rates[0] < 0.2 and rates[1] < 0.3
    assert abs(rates[1] - rates[0]) < 0.1


def test_vcycle_one_smoothing_step_contracts():
    """nu = 1, omega = 0.9: the V-cycle is still a contraction for the block
    operator, a little weaker than nu = 2."""
    spec = spec2((16, 16), k=2)
    p = operator.SGProblem(spec)
    rates = []
    for nu, om in ((2, 0.7), (1, 0.9)):
        mg = solver.Multigrid(p, nu=nu, omega=om)
        L = mg.levels[0]
        A = L.A[0]
        e = np.random.default_rng(3).standard_normal(A.shape[0])
        e[np.tile(L.bmask, L.n_t)] = 0.0
        for _ in range(3):
            e = e - mg.vcycle_block(0, A @ e)
        n0 = np.linalg.norm(e)
        e = e - mg.vcycle_block(0, A @ e)
        rates.append(np.linalg.norm(e) / n0)
    assert rates[0] < rates[1] < 0.3

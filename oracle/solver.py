"""Slab solver for the oracle (test infrastructure): direct solve, the
block-Jacobi geometric-multigrid preconditioner and flexible GMRES.

References (paper, Sec. 3.5, remark "Algebraic solver and matrix-free
implementation"):
  * the slab system A^(n) U = F + J U_prev (eq. local_tensor_system) is solved
    by flexible GMRES;
  * the preconditioner is block-Jacobi in the stochastic index: the diagonal
    block of mode alpha is A_alpha = A_t (x) M_x + sum_mu [G_mu]_{alpha alpha}
    B_t (x) K_mu, approximated by one geometric multigrid V-cycle;
  * the smoother is a space-time Vanka patch smoother (local dense patch
    problems on space-time patches).

Readings (the paper defers these details to a follow-up work):
  * levels: halve the cells per direction while every count is even and > 2
    and the current level has more than ``coarse_dofs`` interior space-time
    unknowns per mode (N_t x interior nodes; default COARSE_DOFS; 0: no such
    limit, down to two cells per direction);
    the coefficient is re-evaluated on every level (rediscretisation); a
    per-cell scale is averaged over the fine cells of a coarse cell;
  * transfer: canonical Q_k interpolation from coarse to fine (P), restriction
    R = P^T, Dirichlet rows and columns of P removed;
  * smoother: additive Vanka, one patch per cell = the cell's interior nodes x
    all time nodes, patch matrix = principal submatrix of the level block
    operator, solved exactly (dense inverse), corrections averaged by the
    number of patches holding a dof, damping omega; nu pre- and nu
    post-smoothing steps;
  * coarsest level: exact solve;
  * Dirichlet rows are the identity on every level: a V-cycle returns x_b = b_b.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coeff, hermite, space_fe, time_dg

OMEGA = 0.7
NU = 2
COARSE_DOFS = 1024


def direct_solve(problem, b):
    """U = A^(n)^{-1} b by a sparse LU of the assembled slab matrix."""
    A = problem.assembled().tocsc()
    return spla.spsolve(A, np.asarray(b, dtype=np.float64).reshape(-1)).reshape(problem.shape)


def interior_dofs(spec):
    """N_t x interior nodes of a level: the size of its dense coarse solve."""
    n = int(spec["r"]) + 1
    for c in spec["cells"][: spec["dim"]]:
        n *= int(c) * int(spec["k"]) - 1
    return n


def coarse_specs(spec, coarse_dofs=COARSE_DOFS):
    """The spec of every multigrid level, finest first."""
    spec = dict(spec, coef=coeff.as_pieces(spec["coef"], int(spec["M"])))
    out = [spec]
    cur = spec
    while (all(c % 2 == 0 and c > 2 for c in cur["cells"][: cur["dim"]])
           and not (coarse_dofs > 0 and interior_dofs(cur) <= coarse_dofs)):
        nxt = dict(cur)
        nxt["cells"] = tuple(c // 2 for c in cur["cells"][: cur["dim"]])
        fine_cells = cur["cells"][: cur["dim"]]
        pieces = []
        for p in cur["coef"]:
            p = dict(p)
            if p.get("cell_scale") is not None:
                arr = np.asarray(p["cell_scale"], dtype=np.float64).reshape(tuple(reversed(fine_cells)))
                if cur["dim"] == 2:
                    arr = arr.reshape(arr.shape[0] // 2, 2, arr.shape[1] // 2, 2).mean(axis=(1, 3))
                else:
                    arr = arr.reshape(arr.shape[0] // 2, 2, arr.shape[1] // 2, 2, arr.shape[2] // 2, 2).mean(axis=(1, 3, 5))
                p["cell_scale"] = arr.reshape(-1)
            pieces.append(p)
        nxt["coef"] = pieces
        out.append(nxt)
        cur = nxt
    return out


def diagonal_classes(G):
    """Group the chaos modes by their diagonal coupling (G_mu[a, a])_mu: the
    modes of one class share the diagonal block A_alpha."""
    diag = np.array([[g[a, a] for g in G] for a in range(G[0].shape[0])])
    keys, cls = np.unique(diag, axis=0, return_inverse=True)
    return keys, cls.reshape(-1)


def round_bf16(a):
    """Each value rounded to float32, then to the nearest bfloat16 (ties to
    even): the 16 high bits of the float32 pattern after adding 0x7FFF plus
    the lowest kept bit.  Finite inputs only."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


class Level:
    """One multigrid level: the block operators A_alpha (one per diagonal
    class), their Vanka patch inverses, and the prolongation from the next
    coarser level.  ``factor_round`` (e.g. ``round_bf16``) is applied to the
    patch inverses after they are computed (the coarsest solve is exact)."""

    def __init__(self, spec, At, Bt, keys, coarsest, factor_round=None):
        self.factor_round = factor_round
        self.mesh = space_fe.Mesh(spec["dim"], spec["cells"], spec["lo"], spec["hi"], spec["k"])
        self.bmask = self.mesh.boundary_mask()
        self.n_t = At.shape[0]
        self.n_x = self.mesh.n_nodes
        Mx, Ks = space_fe.assemble(self.mesh, coeff.at_cell_points(spec["coef"]))
        P = sp.diags((~self.bmask).astype(np.float64))
        Md = P @ Mx @ P
        Kd = [P @ K @ P for K in Ks]
        bd = sp.diags(np.tile(self.bmask.astype(np.float64), self.n_t))
        self.A = []                      # block operator per class, Dirichlet rows identity
        for key in keys:
            Kbar = sum(float(g) * K for g, K in zip(key, Kd))
            self.A.append((sp.kron(At, Md) + sp.kron(Bt, Kbar) + bd).tocsr())
        self.coarsest = coarsest
        if coarsest:
            inner = np.flatnonzero(np.tile(~self.bmask, self.n_t))
            self.inner = inner
            self.Ainv = [np.linalg.inv(A[inner][:, inner].toarray()) for A in self.A]
        else:
            self._patches()

    def _patches(self):
        conn = self.mesh.cell_dofs()
        self.patches = []
        mult = np.zeros(self.n_x * self.n_t)
        for c in range(self.mesh.n_cells):
            nodes = [int(m) for m in conn[c] if not self.bmask[m]]
            dofs = np.array([i * self.n_x + m for i in range(self.n_t) for m in nodes], dtype=np.int64)
            self.patches.append(dofs)
            mult[dofs] += 1.0
        self.mult = mult
        self.patch_inv = []
        for A in self.A:
            inv = []
            for dofs in self.patches:
                m = np.linalg.inv(A[dofs][:, dofs].toarray()) if dofs.size else np.zeros((0, 0))
                inv.append(self.factor_round(m) if self.factor_round is not None else m)
            self.patch_inv.append(inv)

    def smooth(self, cls, x, b, omega=OMEGA):
        r = b - self.A[cls] @ x
        dx = np.zeros_like(x)
        for dofs, inv in zip(self.patches, self.patch_inv[cls]):
            if dofs.size:
                dx[dofs] += inv @ r[dofs]
        nz = self.mult > 0
        x = x.copy()
        x[nz] += omega * dx[nz] / self.mult[nz]
        return x


def prolongation(fine, coarse):
    """Canonical Q_k interpolation from a coarse level to the next finer one
    (fine nodes take the coarse finite-element function's values), with the
    Dirichlet rows and columns removed."""
    fm, cm = fine.mesh, coarse.mesh
    k, dim = fm.k, fm.dim
    fe_nodes = space_fe.gll_nodes_01(k)
    fxyz = fm.node_coords_idx(np.arange(fm.n_nodes))
    rows, cols, vals = [], [], []
    for f in range(fm.n_nodes):
        if fine.bmask[f]:
            continue
        # physical position in units of fine cells, then coarse cell + local coordinate
        cc, loc = [], []
        for d in range(dim):
            cell_f = min(fxyz[f, d] // k, fm.cells[d] - 1)
            pos = cell_f + fe_nodes[fxyz[f, d] - cell_f * k]       # in fine-cell units
            cpos = pos / 2.0
            c = min(int(np.floor(cpos)), cm.cells[d] - 1)
            cc.append(c)
            loc.append(cpos - c)
        vals_d = [time_dg.lagrange_values(fe_nodes, [loc[d]])[:, 0] for d in range(dim)]
        for a in cm.loc:
            v = 1.0
            for d in range(dim):
                v *= vals_d[d][a[d]]
            if v == 0.0:
                continue
            node = cm.node_index([cc[d] * k + a[d] for d in range(dim)])
            if coarse.bmask[node]:
                continue
            rows.append(f)
            cols.append(int(node))
            vals.append(v)
    return sp.coo_matrix((vals, (rows, cols)), shape=(fm.n_nodes, cm.n_nodes)).tocsr()


class Multigrid:
    """Block-Jacobi (in alpha) preconditioner: one V-cycle of the diagonal
    block A_alpha for every chaos mode and both time nodes at once."""

    def __init__(self, problem, factor_round=None, nu=NU, omega=OMEGA, coarse_dofs=COARSE_DOFS):
        self.p = problem
        self.nu, self.omega = nu, omega
        specs = coarse_specs(problem.spec, coarse_dofs)
        self.keys, self.cls = diagonal_classes(problem.G)
        self.levels = [Level(s, problem.At, problem.Bt, self.keys, i == len(specs) - 1, factor_round)
                       for i, s in enumerate(specs)]
        self.P = [prolongation(self.levels[i], self.levels[i + 1]) for i in range(len(self.levels) - 1)]

    def vcycle_block(self, cls, b, lev=0):
        L = self.levels[lev]
        n_t, n_x = L.n_t, L.n_x
        bm = np.tile(L.bmask, n_t)
        if L.coarsest:
            x = b.copy()
            x[L.inner] = L.Ainv[cls] @ b[L.inner]
            return x
        x = np.zeros_like(b)
        x[bm] = b[bm]
        for _ in range(self.nu):
            x = L.smooth(cls, x, b, self.omega)
        r = b - L.A[cls] @ x
        P = self.P[lev]
        rc = np.concatenate([P.T @ r[i * n_x:(i + 1) * n_x] for i in range(n_t)])
        ec = self.vcycle_block(cls, rc, lev + 1)
        nc = self.levels[lev + 1].n_x
        x = x + np.concatenate([P @ ec[i * nc:(i + 1) * nc] for i in range(n_t)])
        for _ in range(self.nu):
            x = L.smooth(cls, x, b, self.omega)
        return x

    def apply(self, r):
        """z = P^{-1} r for a whole slab vector (shape (N_xi, N_t, N_x))."""
        r = np.asarray(r, dtype=np.float64).reshape(self.p.shape)
        z = np.zeros_like(r)
        for a in range(r.shape[0]):
            z[a] = self.vcycle_block(int(self.cls[a]), r[a].reshape(-1)).reshape(r.shape[1:])
        return z


def fgmres(problem, b, precond, x0=None, rtol=1e-8, restart=30, max_it=500):
    """Right-preconditioned flexible GMRES(restart) with modified Gram-Schmidt
    (Saad's FGMRES).  Returns (x, iterations, relative true residual)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    A = lambda v: problem.apply(v).reshape(-1)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    while True:
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm or it >= max_it:
            return x, it, beta / bnorm
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            z = precond(V[j]).reshape(-1)
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            it += 1
            j_done = j + 1
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], g[: j + 2], rcond=None)
            res = np.linalg.norm(g[: j + 2] - H[: j + 2, : j + 1] @ y)
            if res <= rtol * bnorm or it >= max_it:
                break
        y, *_ = np.linalg.lstsq(H[: j_done + 1, :j_done], g[: j_done + 1], rcond=None)
        for i in range(j_done):
            x = x + y[i] * Z[i]


class BlockJacobiLU:
    """Exact block-Jacobi preconditioner: the diagonal block A_alpha of every
    chaos mode (Sec. 3.5 remark) inverted by a sparse LU, one factorisation per
    diagonal class."""

    def __init__(self, problem):
        self.p = problem
        self.keys, self.cls = diagonal_classes(problem.G)
        Md, Kd = problem.dirichlet_factors()
        bd = sp.diags(np.tile(problem.bmask.astype(np.float64), problem.n_t))
        self.lu = []
        for key in self.keys:
            Kbar = sum(float(g) * K for g, K in zip(key, Kd))
            A = (sp.kron(problem.At, Md) + sp.kron(problem.Bt, Kbar) + bd).tocsc()
            self.lu.append(spla.splu(A))

    def apply(self, r):
        r = np.asarray(r, dtype=np.float64).reshape(self.p.shape)
        z = np.zeros_like(r)
        for a in range(r.shape[0]):
            z[a] = self.lu[self.cls[a]].solve(r[a].reshape(-1)).reshape(r.shape[1:])
        return z

"""The stochastic-Galerkin slab operator for the oracle (test infrastructure).

Reference: Problem "tensor-product slab system", eq. local_rhs_tensor:
    A^(n) = M_xi (x) A_t (x) M_x + sum_{mu in M_a} G_mu (x) B_t (x) K_mu,
with M_xi = I (eq. triple_stoch), and the matrix-free remark that follows it
(the operator is only ever applied; its action is what is computed).

Vector layout (a reading: the paper's Kronecker order): a slab vector holds
N_xi * N_t * N_x values, index (alpha * N_t + i) * N_x + m, i.e. an array of
shape (N_xi, N_t, N_x).

Dirichlet treatment (a reading; the paper only says V_h is a subspace of
H^1_0, Sec. 3.1): boundary nodes are stored; every product reads them as 0
and the boundary rows of the operator are the identity, y_b = x_b.

``SGProblem.apply`` evaluates the definition with library sparse products:
y[a,i] = sum_j A_t[i,j] M_x x[a,j] + sum_mu sum_b G_mu[a,b] sum_j B_t[i,j] K_mu x[b,j].
No property of the factors (symmetry, diagonal B_t, sparsity of G) is assumed.
"""
import numpy as np
import scipy.sparse as sp

from . import coeff, hermite, space_fe, time_dg


class SGProblem:
    """All assembled factors of the slab operator for one problem spec.

    spec keys: dim, cells, lo, hi, k (FE degree), r (time degree), n_slabs, T,
    M, P (chaos order), coef (list of separable pieces, or a ``square_of_linear``
    description; see ``oracle.coeff``).
    ``assemble_space=False`` skips the global M_x/K_mu (for sampled rows)."""

    def __init__(self, spec, assemble_space=True):
        spec = dict(spec, coef=coeff.as_pieces(spec["coef"], int(spec["M"])))
        self.spec = spec
        self.mesh = space_fe.Mesh(spec["dim"], spec["cells"], spec["lo"], spec["hi"], spec["k"])
        self.tau = float(spec["T"]) / int(spec["n_slabs"])
        self.At, self.Bt, self.Ct = time_dg.time_matrices(int(spec["r"]), self.tau)
        self.idx = hermite.multi_indices(int(spec["M"]), int(spec["P"]))
        self.mus = coeff.terms(spec["coef"])
        self.G = [hermite.galerkin_matrix(mu, self.idx) for mu in self.mus]
        self.coef_at = coeff.at_cell_points(spec["coef"])
        self.bmask = self.mesh.boundary_mask()
        self.n_xi, self.n_t, self.n_x = self.idx.shape[0], self.At.shape[0], self.mesh.n_nodes
        self.shape = (self.n_xi, self.n_t, self.n_x)
        if assemble_space:
            self.Mx, self.K = space_fe.assemble(self.mesh, self.coef_at)

    # ------------------------------------------------------------------ apply
    def apply(self, x, transpose=False):
        """y = A^(n) x (or its transpose) with the Dirichlet treatment above.
        ``x`` has shape (N_xi, N_t, N_x) or is flat."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        xm = x.copy()
        xm[:, :, self.bmask] = 0.0
        flat = xm.reshape(-1, self.n_x).T                  # (N_x, N_xi*N_t)
        At = self.At.T if transpose else self.At
        Bt = self.Bt.T if transpose else self.Bt
        MX = (self.Mx.T if transpose else self.Mx) @ flat
        MX = MX.T.reshape(self.shape)
        y = np.einsum('ij,ajn->ain', At, MX)
        for t in range(len(self.mus)):
            Kt = self.K[t].T if transpose else self.K[t]
            G = self.G[t].T if transpose else self.G[t]
            KX = (Kt @ flat).T.reshape(self.shape)
            y += np.einsum('ab,ij,bjn->ain', G, Bt, KX)
        y[:, :, self.bmask] = x[:, :, self.bmask]
        return y

    def apply_node_rows(self, x, rows):
        """The entries of y = A^(n) x at the spatial nodes ``rows``, for every
        (alpha, i): the sums of ``apply`` with M_x and K_mu restricted to those
        rows (same Dirichlet treatment).  Shape (N_xi, N_t, len(rows))."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        rows = np.asarray(rows, dtype=np.int64)
        xm = x.copy()
        xm[:, :, self.bmask] = 0.0
        flat = xm.reshape(-1, self.n_x).T                  # (N_x, N_xi*N_t)
        sub = (self.n_xi, self.n_t, rows.size)
        MX = (self.Mx[rows] @ flat).T.reshape(sub)
        y = np.einsum('ij,ajn->ain', self.At, MX)
        for t in range(len(self.mus)):
            KX = (self.K[t][rows] @ flat).T.reshape(sub)
            y += np.einsum('ab,ij,bjn->ain', self.G[t], self.Bt, KX)
        bd = self.bmask[rows]
        y[:, :, bd] = x[:, :, rows[bd]]
        return y

    def apply_rows(self, x, outputs):
        """Selected entries of y = A^(n) x, each computed from the rows of
        M_x and K_mu assembled on the cells around its node only.
        ``outputs`` is a list of (alpha, i, m) triples."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        xm = x.copy()
        xm[:, :, self.bmask] = 0.0
        res = np.zeros(len(outputs))
        cache = {}
        for n, (a, i, m) in enumerate(outputs):
            if self.bmask[m]:
                res[n] = x[a, i, m]
                continue
            if m not in cache:
                cache[m] = space_fe.node_rows(self.mesh, self.coef_at, m)
            cols, m_row, k_rows = cache[m]
            v = 0.0
            for j in range(self.n_t):
                v += self.At[i, j] * (m_row @ xm[a, j, cols])
            for t in range(len(self.mus)):
                for b in range(self.n_xi):
                    g = self.G[t][a, b]
                    if g == 0.0:
                        continue
                    for j in range(self.n_t):
                        v += g * self.Bt[i, j] * (k_rows[t] @ xm[b, j, cols])
            res[n] = v
        return res

    # -------------------------------------------------------------- assembled
    def dirichlet_factors(self):
        """M_x and K_mu with the boundary rows and columns removed (zeroed)."""
        P = sp.diags((~self.bmask).astype(np.float64))
        return P @ self.Mx @ P, [P @ K @ P for K in self.K]

    def assembled(self):
        """The whole slab matrix as a scipy CSR matrix (small cases only):
        kron(I, kron(A_t, M_x)) + sum_mu kron(G_mu, kron(B_t, K_mu)), Dirichlet
        rows and columns replaced by the identity."""
        Md, Kd = self.dirichlet_factors()
        A = sp.kron(sp.identity(self.n_xi), sp.kron(self.At, Md))
        for t in range(len(self.mus)):
            A = A + sp.kron(sp.csr_matrix(self.G[t]), sp.kron(self.Bt, Kd[t]))
        bd = np.tile(self.bmask.astype(np.float64), self.n_xi * self.n_t)
        return (A + sp.diags(bd)).tocsr()

    def transfer(self, u_prev):
        """J^(n) u_prev = (M_xi (x) C_t (x) M_x) u_prev (eq. local_rhs_tensor),
        boundary rows zeroed (right-hand sides vanish on the boundary)."""
        u = np.asarray(u_prev, dtype=np.float64).reshape(self.shape).copy()
        u[:, :, self.bmask] = 0.0
        MX = (self.Mx @ u.reshape(-1, self.n_x).T).T.reshape(self.shape)
        r = np.einsum('ij,ajn->ain', self.Ct, MX)
        r[:, :, self.bmask] = 0.0
        return r

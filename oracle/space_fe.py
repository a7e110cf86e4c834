"""Conforming Q_k finite elements on uniform Cartesian meshes, for the oracle
(test infrastructure).

References:
  * Sec. 3.1: V_h = {v in C^0 cap H^1_0 : v|_K in Q_k}, global nodal Lagrange
    basis phi_m.
  * Sec. 3.5, "Spatial matrices": [M_x]_{m l} = (phi_l, phi_m),
    [K_mu]_{m l} = int_D a_mu grad phi_l . grad phi_m dx.

Readings (the paper is silent on them):
  * The nodal points of Q_k are the tensor Gauss-Lobatto points of each cell
    (equispaced for k <= 2).
  * M_x and K_mu are integrated with the tensor (k+1)-point Gauss rule per
    cell (exact for M_x and for K_mu with a coefficient of degree <= 1 per
    direction).
  * Boundary nodes are stored.  Global node numbering is lexicographic with
    x fastest: m = ix + Nx*(iy + Ny*iz), N_d = k*cells_d + 1.  Cells are
    numbered the same way.

The multi-dimensional element matrices are formed point by point from the
tensor-product quadrature, without any sum factorisation.
"""
import itertools

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as L

from .time_dg import lagrange_values, lagrange_derivs, gauss_legendre_01


def gll_nodes_01(k):
    """k+1 Gauss-Lobatto points on [0, 1]: the end points and the roots of
    P_k' mapped from [-1, 1]."""
    if k == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(k + 1)
    c[k] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(c))))
    x = np.concatenate([[-1.0], inner, [1.0]])
    return (x + 1.0) / 2.0


class FE1D:
    """1D reference data of Q_k on [0, 1] at an n-point Gauss rule."""

    def __init__(self, k, nq=None):
        self.k = k
        self.nodes = gll_nodes_01(k)
        self.nq = k + 1 if nq is None else nq
        self.xq, self.wq = gauss_legendre_01(self.nq)
        self.val = lagrange_values(self.nodes, self.xq)   # (k+1, nq)
        self.der = lagrange_derivs(self.nodes, self.xq)   # (k+1, nq), d/dxi


def _lex(n, dim):
    """All dim-tuples over range(n), lexicographic with the FIRST entry
    fastest (x fastest)."""
    return [tuple(reversed(t)) for t in itertools.product(range(n), repeat=dim)]


class Mesh:
    """Uniform Cartesian mesh of [lo, hi] with Q_k nodes."""

    def __init__(self, dim, cells, lo, hi, k):
        self.dim = dim
        self.cells = tuple(int(c) for c in cells[:dim])
        self.lo = np.array(lo[:dim], dtype=np.float64)
        self.hi = np.array(hi[:dim], dtype=np.float64)
        self.k = k
        self.h = (self.hi - self.lo) / np.array(self.cells)
        self.nn = tuple(k * c + 1 for c in self.cells)     # nodes per direction
        self.n_nodes = int(np.prod(self.nn))
        self.n_cells = int(np.prod(self.cells))
        self.loc = _lex(k + 1, dim)                        # local nodes, x fastest

    def cell_coords(self, cells):
        """Per-direction indices of lexicographic cells: (len(cells), dim)."""
        c = np.asarray(cells, dtype=np.int64).copy()
        out = np.zeros((c.size, self.dim), dtype=np.int64)
        for d in range(self.dim):
            out[:, d] = c % self.cells[d]
            c //= self.cells[d]
        return out

    def node_index(self, ijk):
        """Global node index from per-direction indices (..., dim)."""
        ijk = np.asarray(ijk, dtype=np.int64)
        m = np.zeros(ijk.shape[:-1], dtype=np.int64)
        stride = 1
        for d in range(self.dim):
            m = m + ijk[..., d] * stride
            stride *= self.nn[d]
        return m

    def node_coords_idx(self, nodes):
        """Per-direction indices of global nodes: (len(nodes), dim)."""
        m = np.asarray(nodes, dtype=np.int64).copy()
        out = np.zeros((m.size, self.dim), dtype=np.int64)
        for d in range(self.dim):
            out[:, d] = m % self.nn[d]
            m //= self.nn[d]
        return out

    def cell_dofs(self, cells=None):
        """(n, (k+1)^dim) global node indices of the local nodes of ``cells``."""
        if cells is None:
            cells = np.arange(self.n_cells)
        cc = self.cell_coords(cells)
        loc = np.array(self.loc, dtype=np.int64)           # (nloc, dim)
        ijk = cc[:, None, :] * self.k + loc[None, :, :]
        return self.node_index(ijk)

    def boundary_mask(self):
        """True at the nodes on the boundary of the domain (Dirichlet nodes)."""
        ijk = self.node_coords_idx(np.arange(self.n_nodes))
        mask = np.zeros(self.n_nodes, dtype=bool)
        for d in range(self.dim):
            mask |= (ijk[:, d] == 0) | (ijk[:, d] == self.nn[d] - 1)
        return mask

    def node_coords(self):
        """(n_nodes, dim) physical coordinates of all nodes."""
        fe_nodes = gll_nodes_01(self.k)
        ijk = self.node_coords_idx(np.arange(self.n_nodes))
        out = np.zeros((self.n_nodes, self.dim))
        for d in range(self.dim):
            cell = np.minimum(ijk[:, d] // self.k, self.cells[d] - 1)
            out[:, d] = self.lo[d] + (cell + fe_nodes[ijk[:, d] - cell * self.k]) * self.h[d]
        return out

    def cells_of_node(self, node):
        """Lexicographic indices of the cells that contain a node."""
        ijk = self.node_coords_idx([node])[0]
        per_dir = []
        for d in range(self.dim):
            c = ijk[d] // self.k
            opts = []
            if ijk[d] % self.k == 0:
                if c - 1 >= 0:
                    opts.append(c - 1)
                if c < self.cells[d]:
                    opts.append(c)
            else:
                opts.append(c)
            per_dir.append(opts)
        out = []
        for combo in itertools.product(*per_dir):
            idx, stride = 0, 1
            for d in range(self.dim):
                idx += combo[d] * stride
                stride *= self.cells[d]
            out.append(idx)
        return np.array(sorted(out), dtype=np.int64)


def reference_shape(mesh, fe):
    """Tensor quadrature weights times |J| (nqd,), local shape values
    phi (nloc, nqd) and physical gradients grad (nloc, nqd, dim) at the
    points of the tensor Gauss rule; identical on every cell of the uniform
    mesh."""
    dim = mesh.dim
    qidx = _lex(fe.nq, dim)
    detJ = float(np.prod(mesh.h))
    wJ = np.array([np.prod([fe.wq[q[d]] for d in range(dim)]) for q in qidx]) * detJ
    nloc, nqd = len(mesh.loc), len(qidx)
    phi = np.zeros((nloc, nqd))
    grad = np.zeros((nloc, nqd, dim))
    for a, t in enumerate(mesh.loc):
        for iq, q in enumerate(qidx):
            phi[a, iq] = np.prod([fe.val[t[d], q[d]] for d in range(dim)])
            for c in range(dim):
                g = 1.0 / mesh.h[c]
                for d in range(dim):
                    g *= fe.der[t[d], q[d]] if d == c else fe.val[t[d], q[d]]
                grad[a, iq, c] = g
    return wJ, phi, grad


def cell_points(mesh, fe, cells):
    """Physical quadrature points of ``cells``: (len(cells), nqd, dim)."""
    qidx = np.array(_lex(fe.nq, mesh.dim), dtype=np.int64)
    cc = mesh.cell_coords(cells)
    ref = fe.xq[qidx]                                      # (nqd, dim)
    return mesh.lo[None, None, :] + (cc[:, None, :] + ref[None, :, :]) * mesh.h[None, None, :]


def element_matrices(mesh, coef_at, cells, nq=None):
    """Element mass (cell independent, (nloc, nloc)) and element stiffness
    per coefficient term ((n_terms, len(cells), nloc, nloc)) of ``cells``.

    ``coef_at(xq, cells)`` maps points (len(cells), nqd, dim) to
    (n_terms, len(cells), nqd) values of a_mu."""
    fe = FE1D(mesh.k, nq)
    wJ, phi, grad = reference_shape(mesh, fe)
    xq = cell_points(mesh, fe, cells)
    amu = coef_at(xq, np.asarray(cells))
    Mloc = np.einsum('aq,bq,q->ab', phi, phi, wJ)
    E = np.einsum('aqc,bqc,q->qab', grad, grad, wJ)        # per-point stiffness
    Kloc = np.einsum('tcq,qab->tcab', amu, E)
    return Mloc, Kloc


def assemble(mesh, coef_at, nq=None):
    """Assemble M_x and the list of K_mu (Sec. 3.5, "Spatial matrices") as
    scipy CSR matrices over all nodes (boundary rows included, no Dirichlet
    treatment yet)."""
    cells = np.arange(mesh.n_cells)
    conn = mesh.cell_dofs(cells)
    Mloc, Kloc = element_matrices(mesh, coef_at, cells, nq)
    nloc = conn.shape[1]
    rows = np.repeat(conn, nloc, axis=1).reshape(-1)
    cols = np.tile(conn, (1, nloc)).reshape(-1)
    n = mesh.n_nodes
    Mx = sp.coo_matrix((np.tile(Mloc.reshape(-1), mesh.n_cells), (rows, cols)),
                       shape=(n, n)).tocsr()
    Ks = [sp.coo_matrix((Kloc[t].reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
          for t in range(Kloc.shape[0])]
    return Mx, Ks


def node_rows(mesh, coef_at, node, nq=None):
    """Row ``node`` of M_x and of every K_mu, assembled from the cells that
    contain the node only.  Returns (cols, m_row, k_rows) with k_rows of shape
    (n_terms, len(cols))."""
    cells = mesh.cells_of_node(node)
    conn = mesh.cell_dofs(cells)
    Mloc, Kloc = element_matrices(mesh, coef_at, cells, nq)
    cols = np.unique(conn)
    pos = {int(c): i for i, c in enumerate(cols)}
    m_row = np.zeros(cols.size)
    k_rows = np.zeros((Kloc.shape[0], cols.size))
    for ci in range(len(cells)):
        a = int(np.where(conn[ci] == node)[0][0])
        for b in range(conn.shape[1]):
            j = pos[int(conn[ci, b])]
            m_row[j] += Mloc[a, b]
            k_rows[:, j] += Kloc[:, ci, a, b]
    return cols, m_row, k_rows

"""Discrete adjoint of the slab marching for the oracle (test infrastructure;
only tests and the benchmark's CPU baseline use it).

The paper computes no gradient.  What is differentiated is its marching: the
slab systems of eq. local_tensor_system,
    A(p) U_n = F_n + J U_{n-1},   n = 0 .. N-1,   J = I (x) C_t (x) M_x
(eq. local_rhs_tensor, Dirichlet rows and columns removed), with the load
vectors F_n of eq. load_vector computed once from the nominal coefficient and
held fixed (data, not a function of p).  The quantity of interest is
    J(p) = sum_alpha U_{N-1}[alpha, r]^T M_x U_{N-1}[alpha, r]
         = E[ ||u_h(., T)||^2_{L2(D)} ]
(the chaos mean and variance identities eqs. qoi-mean-chaos / qoi-variance-chaos
summed; index r is the right Radau node t = T of the last slab).

Adjoint (plain Lagrangian calculus on the discrete equations):
    A^T lam_{N-1} = dJ/dU_{N-1} = 2 (I (x) e_r e_r^T (x) M_x) U_{N-1},
    A^T lam_n     = J^T lam_{n+1},
    dJ/dp         = - sum_n lam_n^T (dA/dp) U_n,
with dA/dp = G_t (x) B_t (x) dK_t/dp for a parameter of a coefficient piece of
term t.  Parameters: the amplitude of every piece, and the per-cell scale of
one piece.

Every solve is a sparse LU of the assembled slab matrix (``direct_solve``), so
the functions here are for small cases.  ``energy`` with a perturbed
coefficient gives the central finite differences that pin the adjoint.
"""
import copy

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coeff, space_fe
from .manufactured import Manufactured
from .operator import SGProblem


def with_coefficient(spec, amp=None, cell_piece=-1, cell_scale=None):
    """A copy of ``spec`` whose pieces carry the amplitudes ``amp`` and, for
    piece ``cell_piece``, the per-cell scale ``cell_scale``."""
    out = copy.deepcopy(spec)
    if amp is not None:
        for i, p in enumerate(out["coef"]):
            p["amp"] = float(amp[i])
    if cell_piece >= 0 and cell_scale is not None:
        out["coef"][cell_piece]["cell_scale"] = np.asarray(cell_scale, dtype=np.float64).copy()
    return out


def _lu(op):
    return spla.splu(op.assembled().tocsc())


def _masked(op, v):
    v = np.asarray(v, dtype=np.float64).reshape(op.shape).copy()
    v[:, :, op.bmask] = 0.0
    return v


def march(op, man, n_slabs=None):
    """U_0 .. U_{N-1} for the operator of ``op`` and the load vectors of
    ``man`` (the nominal problem), by sparse LU."""
    n_slabs = int(op.spec["n_slabs"]) if n_slabs is None else n_slabs
    lu = _lu(op)
    Us, U = [], None
    for n in range(n_slabs):
        rhs = man.load_vector(n)
        if n > 0:
            rhs = rhs + op.transfer(U)
        U = lu.solve(rhs.reshape(-1)).reshape(op.shape)
        Us.append(U)
    return Us


def energy_of(op, U_last):
    """J = sum_alpha U[alpha, r]^T M_x U[alpha, r] at the last time node."""
    u = U_last[:, -1, :]
    return float(np.einsum('an,an->', u, (op.Mx @ u.T).T))


def energy(spec, nominal_spec, exact, n_slabs=None):
    """J for the coefficient of ``spec`` with the load vectors of
    ``nominal_spec``'s coefficient."""
    op = SGProblem(spec)
    man = Manufactured(SGProblem(nominal_spec), exact)
    return energy_of(op, march(op, man, n_slabs)[-1])


def transfer_transpose(op, lam):
    """J^T lam = (I (x) C_t^T (x) M_x) lam, Dirichlet rows and columns zero."""
    x = _masked(op, lam)
    MX = (op.Mx.T @ x.reshape(-1, op.n_x).T).T.reshape(op.shape)
    r = np.einsum('ji,ajn->ain', op.Ct, MX)
    r[:, :, op.bmask] = 0.0
    return r


def terminal_source(op, U_last):
    """dJ/dU_{N-1} = 2 (I (x) e_r e_r^T (x) M_x) U_{N-1}, Dirichlet rows zero."""
    u = _masked(op, U_last)
    g = np.zeros(op.shape)
    g[:, -1, :] = 2.0 * (op.Mx @ u[:, -1, :].T).T
    g[:, :, op.bmask] = 0.0
    return g


def adjoint_states(op, Us):
    """lam_0 .. lam_{N-1} backwards in time by sparse LU of A^T."""
    luT = spla.splu(op.assembled().T.tocsc())
    lams = [None] * len(Us)
    src = terminal_source(op, Us[-1])
    for n in range(len(Us) - 1, -1, -1):
        lam = luT.solve(src.reshape(-1)).reshape(op.shape)
        lams[n] = lam
        src = transfer_transpose(op, lam)
    return lams


def _bilinear(op, lam, U, t, dK):
    """lam^T (G_t (x) B_t (x) dK) U with Dirichlet rows and columns removed."""
    L, V = _masked(op, lam), _masked(op, U)
    KV = (dK @ V.reshape(-1, op.n_x).T).T.reshape(op.shape)        # dK U[b, j]
    BKV = np.einsum('ij,bjn->bin', op.Bt, KV)                       # (B_t (x) dK) U[b]
    return float(np.einsum('ab,ain,bin->', op.G[t], L, BKV))


def _cell_bilinear(op, lam, U, t, piece):
    """Per cell c: lam^T (G_t (x) B_t (x) K_c) U, K_c the stiffness of the
    piece (scale 1) on cell c alone."""
    mesh = op.mesh
    cells = np.arange(mesh.n_cells)
    conn = mesh.cell_dofs(cells)                                    # (C, nloc)
    p = dict(piece)
    p["cell_scale"] = None
    _, Kloc = space_fe.element_matrices(mesh, coeff.at_cell_points([p]), cells)
    Kc = Kloc[0]                                                    # (C, nloc, nloc)
    L = _masked(op, lam)[:, :, conn]                                # (N_xi, N_t, C, nloc)
    V = _masked(op, U)[:, :, conn]
    KV = np.einsum('cxy,bjcy->bjcx', Kc, V)
    BKV = np.einsum('ij,bjcx->bicx', op.Bt, KV)
    return np.einsum('ab,aicx,bicx->c', op.G[t], L, BKV)


def gradient(spec, exact, cell_piece=-1, nominal_spec=None):
    """(J, dJ/d amp, dJ/d cell_scale or None) by the discrete adjoint.  The
    load vectors are those of ``nominal_spec`` (default: ``spec``)."""
    nominal_spec = spec if nominal_spec is None else nominal_spec
    op = SGProblem(spec)
    man = Manufactured(SGProblem(nominal_spec), exact)
    Us = march(op, man)
    J = energy_of(op, Us[-1])
    lams = adjoint_states(op, Us)
    pieces = op.spec["coef"]
    mus = coeff.terms(pieces)
    g_amp = np.zeros(len(pieces))
    for j, piece in enumerate(pieces):
        t = mus.index(tuple(int(v) for v in piece["mu"]))
        unit = dict(piece)
        unit["amp"] = 1.0
        _, (dK,) = space_fe.assemble(op.mesh, coeff.at_cell_points([unit]))
        g_amp[j] = -sum(_bilinear(op, lams[n], Us[n], t, dK) for n in range(len(Us)))
    g_cell = None
    if cell_piece >= 0:
        piece = pieces[cell_piece]
        t = mus.index(tuple(int(v) for v in piece["mu"]))
        g_cell = -sum(_cell_bilinear(op, lams[n], Us[n], t, piece) for n in range(len(Us)))
    return J, g_amp, g_cell

"""Manufactured finite-chaos solutions, slab load vectors, slab marching and
error norms for the oracle (test infrastructure).

References (paper):
  * Sec. 4.3, eqs. finite-exact-separated .. finite-chaos-coefficients: an exact
    solution u = T(t) sum_{alpha in Lambda_q} c_alpha Phi_alpha(x) Psi_alpha(xi);
  * eq. manufactured_rhs_benchmark: f = d_t u - div(a grad u), whose Hermite
    projections f_beta = E[f Psi_beta] are evaluated analytically (Sec. 4:
    "projected forcing modes ... evaluated analytically");
  * eq. load_vector (F^(n)), eq. initial_vector (B_0^(1)),
    eq. local_tensor_system (A U^(n) = F^(n) + J U^(n-1));
  * Sec. 4.1 / 4.2: mean = mode 0 (eq. qoi-mean-chaos), variance = sum of the
    squares of the other modes (eq. qoi-variance-chaos), the full, mean and
    variance errors in L2_t(L2_x) (Definition "error norms and quantities").

Readings: the projected initial value is the L2 projection (Sec. 3.4 says only
"chosen projection"), so (u_0,h, phi_m) = (u_0, phi_m); quadrature of the load
vector and of the errors uses (k+4) Gauss points per direction and r+6 in
time (the paper states none).

The exact solution is plain data:
    {"q": q, "c": [c_alpha for alpha in Lambda_q (graded order)],
     "phi": [per alpha: per direction ("sin", k) -> sin(pi k (s - lo) / (hi - lo))
                                   or ("poly", [a_0, a_1, ...]) -> sum a_j s^j],
     "T": [t_0, t_1, ...]  (T(t) = sum t_j t^j)}
"""
import numpy as np

from . import coeff, hermite, space_fe, time_dg
from .solver import direct_solve


def _factor(f, s, lo, hi, der):
    """Value (der=0), first (1) or second (2) derivative of a 1D factor."""
    kind, par = f
    if kind == "sin":
        w = np.pi * par / (hi - lo)
        arg = w * (s - lo)
        return [np.sin(arg), w * np.cos(arg), -w * w * np.sin(arg)][der]
    if kind == "poly":
        c = np.polynomial.polynomial.Polynomial(par)
        for _ in range(der):
            c = c.deriv()
        return c(s)
    raise ValueError(kind)


def _coef_factor(kind, k, s, der):
    if kind == "one":
        return np.ones_like(s) if der == 0 else np.zeros_like(s)
    if kind == "sin":
        return np.sin(k * np.pi * s) if der == 0 else k * np.pi * np.cos(k * np.pi * s)
    if kind == "pow":
        if der == 0:
            return s ** k
        return k * s ** (k - 1) if k > 0 else np.zeros_like(s)
    raise ValueError(kind)


class Exact:
    """Evaluates the exact modes u_alpha (alpha in Lambda_q) and their derivatives."""

    def __init__(self, spec, exact):
        self.spec = spec
        self.dim = spec["dim"]
        self.q = int(exact["q"])
        self.idx_q = hermite.multi_indices(spec["M"], self.q)
        self.c = np.asarray(exact["c"], dtype=np.float64)
        assert self.c.size == self.idx_q.shape[0]
        self.phi = exact["phi"]
        self.T = np.polynomial.polynomial.Polynomial(exact["T"])
        self.dT = self.T.deriv()

    def spatial(self, a, x, der):
        """Phi_alpha at points x (..., dim): der=0 value, 1 gradient (..., dim),
        2 Laplacian."""
        lo, hi = self.spec["lo"], self.spec["hi"]
        f = self.phi[a]
        vals = [_factor(f[d], x[..., d], lo[d], hi[d], 0) for d in range(self.dim)]
        if der == 0:
            return np.prod(vals, axis=0)
        if der == 1:
            out = np.zeros(x.shape)
            for d in range(self.dim):
                g = _factor(f[d], x[..., d], lo[d], hi[d], 1)
                for e in range(self.dim):
                    if e != d:
                        g = g * vals[e]
                out[..., d] = g
            return out
        lap = np.zeros(x.shape[:-1])
        for d in range(self.dim):
            g = _factor(f[d], x[..., d], lo[d], hi[d], 2)
            for e in range(self.dim):
                if e != d:
                    g = g * vals[e]
            lap += g
        return lap


def coef_with_gradient(pieces, x, cells):
    """a_mu and grad a_mu at points x (..., dim) of the given cells."""
    mus = coeff.terms(pieces)
    dim = x.shape[-1]
    val = np.zeros((len(mus),) + x.shape[:-1])
    grad = np.zeros((len(mus),) + x.shape)
    for p in pieces:
        t = mus.index(tuple(int(v) for v in p["mu"]))
        scale = float(p["amp"])
        cs = p.get("cell_scale")
        cell_fac = np.asarray(cs, dtype=np.float64)[cells] if cs is not None else 1.0
        f = [_coef_factor(p["factors"][d][0], p["factors"][d][1], x[..., d], 0) for d in range(dim)]
        df = [_coef_factor(p["factors"][d][0], p["factors"][d][1], x[..., d], 1) for d in range(dim)]
        val[t] += scale * cell_fac * np.prod(f, axis=0)
        for d in range(dim):
            g = scale * cell_fac * df[d]
            for e in range(dim):
                if e != d:
                    g = g * f[e]
            grad[t][..., d] += g
    return val, grad


class Manufactured:
    """Load vectors, slab marching and error norms for one problem + exact solution."""

    def __init__(self, problem, exact):
        self.p = problem
        self.ex = Exact(problem.spec, exact)
        mesh = problem.mesh
        self.fe = space_fe.FE1D(mesh.k, mesh.k + 4)
        self.wJ, self.phi, self.grad = space_fe.reference_shape(mesh, self.fe)
        cells = np.arange(mesh.n_cells)
        self.conn = mesh.cell_dofs(cells)
        self.xq = space_fe.cell_points(mesh, self.fe, cells)                 # (C, Q, d)
        cidx = np.broadcast_to(cells[:, None], self.xq.shape[:-1])
        self.amu, self.damu = coef_with_gradient(problem.spec["coef"], self.xq, cidx)
        # triple products G_mu[beta, alpha], beta in Lambda_p, alpha in Lambda_q
        self.Gpq = np.array([[[hermite.triple(mu, b, a) for a in self.ex.idx_q] for b in problem.idx]
                             for mu in problem.mus])
        r = problem.n_t - 1
        self.nodes_t = time_dg.radau_right_nodes(r)
        self.tq, self.tw = time_dg.gauss_legendre_01(r + 6)

    def _spatial_parts(self):
        """Per alpha in Lambda_q: Phi_alpha, grad Phi, Laplacian at the quadrature points."""
        if not hasattr(self, "_sp"):
            ex = self.ex
            self._sp = [(ex.spatial(a, self.xq, 0), ex.spatial(a, self.xq, 1), ex.spatial(a, self.xq, 2))
                        for a in range(ex.idx_q.shape[0])]
        return self._sp

    def _forcing_parts(self):
        """Time-independent parts of f_beta = T'(t) P_beta(x) - T(t) S_beta(x):
        P_beta = c_beta Phi_beta and
        S_beta = sum_{mu, alpha} G_mu[beta, alpha] c_alpha div(a_mu grad Phi_alpha)
        with div(a grad Phi) = grad a . grad Phi + a lap Phi."""
        if not hasattr(self, "_fp"):
            ex = self.ex
            sp = self._spatial_parts()
            pos = {tuple(a): i for i, a in enumerate(ex.idx_q)}
            shape = (self.p.n_xi,) + self.xq.shape[:-1]
            P, S = np.zeros(shape), np.zeros(shape)
            for b in range(self.p.n_xi):
                jb = pos.get(tuple(self.p.idx[b]))
                if jb is not None:
                    P[b] = ex.c[jb] * sp[jb][0]
                for t_mu in range(len(self.p.mus)):
                    for a in np.flatnonzero(self.Gpq[t_mu, b]):
                        if ex.c[a] == 0.0:
                            continue
                        div = np.einsum('cqd,cqd->cq', self.damu[t_mu], sp[a][1]) + self.amu[t_mu] * sp[a][2]
                        S[b] += self.Gpq[t_mu, b, a] * ex.c[a] * div
            self._fp = (P, S)
        return self._fp

    def forcing_modes(self, t):
        """f_beta(x_q, t) = E[f Psi_beta] for beta in Lambda_p (eq.
        manufactured_rhs_benchmark projected on the chaos basis): d_t u_beta -
        sum_{mu, alpha} G_mu[beta, alpha] div(a_mu grad u_alpha)."""
        P, S = self._forcing_parts()
        return self.ex.dT(t) * P - self.ex.T(t) * S

    def load_vector(self, n):
        """F^(n) (eq. load_vector) on slab n = 0, 1, ...; on the first slab the
        initial vector B_0^(1) (eq. initial_vector) is added."""
        p = self.p
        tau = p.tau
        t0 = n * tau
        F = np.zeros(p.shape)
        vt = time_dg.lagrange_values(self.nodes_t, self.tq)                 # (N_t, nq)
        for qt in range(self.tq.size):
            fb = self.forcing_modes(t0 + tau * self.tq[qt])                  # (N_xi, C, Q)
            loc = np.einsum('bcq,aq,q->bca', fb, self.phi, self.wJ)          # (N_xi, C, nloc)
            glob = np.zeros((p.n_xi, p.n_x))
            for b in range(p.n_xi):
                np.add.at(glob[b], self.conn.reshape(-1), loc[b].reshape(-1))
            F += tau * self.tw[qt] * vt[:, qt][None, :, None] * glob[:, None, :]
        if n == 0:
            F += self.initial_vector()
        F[:, :, p.bmask] = 0.0
        return F

    def initial_vector(self):
        """B_0^(1)[(alpha, i, m)] = v_i(t_0^+) (u_0,alpha, phi_m) with the L2
        projection of u_0 = u(0)."""
        p, ex = self.p, self.ex
        sp = self._spatial_parts()
        pos = {tuple(a): i for i, a in enumerate(ex.idx_q)}
        v0 = time_dg.lagrange_values(self.nodes_t, [0.0])[:, 0]
        B = np.zeros(p.shape)
        for b in range(p.n_xi):
            jb = pos.get(tuple(p.idx[b]))
            if jb is None:
                continue
            loc = np.einsum('cq,aq,q->ca', ex.T(0.0) * ex.c[jb] * sp[jb][0], self.phi, self.wJ)
            g = np.zeros(p.n_x)
            np.add.at(g, self.conn.reshape(-1), loc.reshape(-1))
            B[b] = v0[:, None] * g[None, :]
        return B

    def march(self, n_slabs, solve=None):
        """U^(1..n_slabs) by causal slab marching (eq. local_tensor_system);
        default solver: FGMRES to 1e-12 preconditioned by exact block-Jacobi."""
        p = self.p
        Us = []
        U = np.zeros(p.shape)
        if solve is None:
            from .solver import BlockJacobiLU, fgmres
            pre = BlockJacobiLU(p)
            solve = lambda b: fgmres(p, b, pre.apply, rtol=1e-12)[0].reshape(p.shape)
        for n in range(n_slabs):
            rhs = self.load_vector(n) + (p.transfer(U) if n > 0 else 0.0)
            U = solve(rhs)
            Us.append(U)
        return Us

    def errors(self, Us):
        """Full, mean and variance errors in L2_t(L2_x) over the marched slabs
        (Definition "error norms and quantities"), using the modal identities."""
        p, ex = self.p, self.ex
        sp = self._spatial_parts()
        pos = {tuple(a): i for i, a in enumerate(ex.idx_q)}
        in_p = [pos.get(tuple(a)) for a in p.idx]
        vt = time_dg.lagrange_values(self.nodes_t, self.tq)
        full = mean = var = 0.0
        not_in_p = [j for j in range(ex.idx_q.shape[0]) if tuple(ex.idx_q[j]) not in {tuple(a) for a in p.idx}]
        zero = [j for j in range(ex.idx_q.shape[0]) if not any(ex.idx_q[j])]
        tail2 = sum((ex.c[j] * sp[j][0]) ** 2 for j in not_in_p) if not_in_p else 0.0
        var_shape = sum((ex.c[j] * sp[j][0]) ** 2 for j in range(ex.idx_q.shape[0]) if any(ex.idx_q[j]))
        for n, U in enumerate(Us):
            Uc = U[:, :, self.conn]                                          # (N_xi, N_t, C, nloc)
            uq = np.einsum('aicl,lq->aicq', Uc, self.phi)                   # at space points
            for qt in range(self.tq.size):
                t = (n + self.tq[qt]) * p.tau
                w = p.tau * self.tw[qt]
                uh = np.einsum('i,aicq->acq', vt[:, qt], uq)                # u_h,alpha(x_q, t)
                Tt = ex.T(t)
                ue_p = np.zeros_like(uh)
                for b, jb in enumerate(in_p):
                    if jb is not None:
                        ue_p[b] = Tt * ex.c[jb] * sp[jb][0]
                d2 = ((uh - ue_p) ** 2).sum(axis=0) + Tt ** 2 * tail2
                full += w * np.einsum('cq,q->', d2, self.wJ)
                mean_ex = sum(Tt * ex.c[j] * sp[j][0] for j in zero) if zero else 0.0
                i0 = [b for b in range(p.n_xi) if not any(p.idx[b])][0]
                mean += w * np.einsum('cq,q->', (uh[i0] - mean_ex) ** 2, self.wJ)
                var_h = (uh ** 2).sum(axis=0) - uh[i0] ** 2
                var_ex = Tt ** 2 * var_shape
                var += w * np.einsum('cq,q->', (var_h - var_ex) ** 2, self.wJ)
        return {"full": np.sqrt(full), "mean": np.sqrt(mean), "var": np.sqrt(var)}


def errors_at_end(man, U, n):
    """L2(D) errors of the mean, variance and full solution at the end time
    t_n of slab n (time node r), the same definitions at one time."""
    p, ex = man.p, man.ex
    sp = man._spatial_parts()
    pos = {tuple(a): i for i, a in enumerate(ex.idx_q)}
    r = p.n_t - 1
    uq = np.einsum('acl,lq->acq', U[:, r][:, man.conn], man.phi)          # (N_xi, C, Q)
    Tt = ex.T((n + 1) * p.tau)
    idx_p = {tuple(a) for a in p.idx}
    full = np.zeros(uq.shape[1:])
    for b in range(p.n_xi):
        jb = pos.get(tuple(p.idx[b]))
        full += (uq[b] - (Tt * ex.c[jb] * sp[jb][0] if jb is not None else 0.0)) ** 2
    for j in range(ex.idx_q.shape[0]):
        if tuple(ex.idx_q[j]) not in idx_p:
            full += (Tt * ex.c[j] * sp[j][0]) ** 2
    i0 = [b for b in range(p.n_xi) if not any(p.idx[b])][0]
    j0 = [j for j in range(ex.idx_q.shape[0]) if not any(ex.idx_q[j])]
    mean_ex = Tt * ex.c[j0[0]] * sp[j0[0]][0] if j0 else 0.0
    var_h = (uq ** 2).sum(axis=0) - uq[i0] ** 2
    var_ex = sum((Tt * ex.c[j] * sp[j][0]) ** 2 for j in range(ex.idx_q.shape[0]) if any(ex.idx_q[j]))
    w = man.wJ
    return {"mean": float(np.sqrt(np.einsum('cq,q->', (uq[i0] - mean_ex) ** 2, w))),
            "var": float(np.sqrt(np.einsum('cq,q->', (var_h - var_ex) ** 2, w))),
            "full": float(np.sqrt(np.einsum('cq,q->', full, w)))}


def paper_exact(M=4, q=6, eta=0.35):
    """The paper's finite-chaos solution (eqs. finite-exact-separated ..
    finite-chaos-coefficients): u = t^4 sin(pi/2 (x1+1)) sin(pi/2 (x2+1)) G_q(xi),
    c_0 = 1, c_alpha = eta^{|alpha|}."""
    idx = hermite.multi_indices(M, q)
    c = [1.0 if not any(a) else eta ** int(sum(a)) for a in idx]
    return {"q": q, "c": c, "phi": [[("sin", 1), ("sin", 1)] for _ in idx], "T": [0, 0, 0, 0, 1]}

// Right-hand sides of the slab systems, statistics and errors for a
// manufactured finite-chaos solution (paper, Sec. 4.3):
//     u(x, t, xi) = T(t) sum_{alpha in Lambda_q} c_alpha Phi_alpha(x) Psi_alpha(xi),
//     Phi_alpha(x) = prod_d sin(pi f_{alpha,d} (x_d - lo_d) / (hi_d - lo_d)),
// which vanishes on the boundary of the box.
//
// Load vector (eq. load_vector) with the forcing f = d_t u - div(a grad u)
// (eq. manufactured_rhs_benchmark), tested against v_i Psi_beta phi_m and
// integrated by parts in space (phi_m vanishes on the boundary):
//     F[beta, i, m] = tau'_i P_beta[m] + tau_i K_beta[m],
//     P_beta[m] = c_beta (Phi_beta, phi_m),
//     K_beta[m] = sum_{mu, alpha} G_mu[beta][alpha] c_alpha (a_mu grad Phi_alpha, grad phi_m),
//     tau'_i = int_{I_n} T'(t) v_i dt,  tau_i = int_{I_n} T(t) v_i dt.
// P and K do not depend on the slab: sg_set_exact computes them once (host,
// (k+4)^d Gauss points per cell) and keeps them on the device; each sg_rhs is
// one elementwise kernel plus the transfer term J U^(n-1) = (I (x) C_t (x) M_x)
// U^(n-1) (eq. local_rhs_tensor), applied by the cell kernel with the C_t
// time coupling and no stiffness.  On the first slab the initial vector
// B_0 = v_i(t_0) (u(t_0), phi_m) (eq. initial_vector, L2 projection of u(0))
// adds v_i(t_0) T(t_0) to tau'_i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sg_internal.h"

namespace sg {

namespace {

__global__ void k_rhs_combine(const double* __restrict__ P, const double* __restrict__ K, double* __restrict__ rhs,
                              int n_xi, int n_t, long long n_x, const double* __restrict__ tp,
                              const double* __restrict__ tk) {
  const long long total = (long long)n_xi * n_t * n_x;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx % n_x;
    const long long v = idx / n_x;
    const int i = (int)(v % n_t), b = (int)(v / n_t);
    rhs[idx] = tp[i] * P[(long long)b * n_x + m] + tk[i] * K[(long long)b * n_x + m];
  }
}

__global__ void k_moments(const double* __restrict__ u, double* __restrict__ mean, double* __restrict__ var,
                          int n_xi, int n_t, int node, long long n_x) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n_x; m += (long long)gridDim.x * blockDim.x) {
    const double u0 = u[(long long)node * n_x + m];
    double v = 0.0;
    for (int a = 1; a < n_xi; ++a) {
      const double ua = u[((long long)a * n_t + node) * n_x + m];
      v = fma(ua, ua, v);
    }
    if (mean) mean[m] = u0;
    if (var) var[m] = v;
  }
}

int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sg::sm_count() * 16)); }

double poly(const std::vector<double>& c, double t) {
  double s = 0.0;
  for (int j = (int)c.size() - 1; j >= 0; --j) s = s * t + c[j];
  return s;
}

double poly_deriv(const std::vector<double>& c, double t) {
  double s = 0.0;
  for (int j = (int)c.size() - 1; j >= 1; --j) s = s * t + j * c[j];
  return s;
}

}  // namespace


void exact_free(ExactData* e) {
  if (!e) return;
  cudaFree(e->d_P);
  cudaFree(e->d_K);
  cudaFree(e->d_tpk);
  cudaFree(e->d_zero_rows);
  delete e;
}

static double phi_val(const HostProblem& hp, const int* f, const double* x, double* grad) {
  double v[3], dv[3];
  for (int d = 0; d < hp.dim; ++d) {
    const double L = hp.h[d] * hp.cells[d];
    const double w = M_PI * f[d] / L;
    v[d] = std::sin(w * (x[d] - hp.lo[d]));
    dv[d] = w * std::cos(w * (x[d] - hp.lo[d]));
  }
  double val = 1.0;
  for (int d = 0; d < hp.dim; ++d) val *= v[d];
  if (grad)
    for (int d = 0; d < hp.dim; ++d) {
      double g = dv[d];
      for (int e = 0; e < hp.dim; ++e)
        if (e != d) g *= v[e];
      grad[d] = g;
    }
  return val;
}

static double coef_piece(const Piece& pc, int dim, const double* x, long long cell) {
  double v = pc.amp;
  for (int d = 0; d < dim; ++d) {
    switch (pc.kind[d]) {
      case SG_F_SIN: v *= std::sin(pc.k[d] * M_PI * x[d]); break;
      case SG_F_POW: v *= std::pow(x[d], (double)pc.k[d]); break;
      default: break;
    }
  }
  if (!pc.scale.empty()) v *= pc.scale[cell];
  return v;
}

sg_status exact_build(const HostProblem& hp, int q, const double* c, const int* freq, int t_degree,
                      const double* t_coef, ExactData*& out, std::string& msg) {
  if (q < 0 || q > 12 || !c || !freq || t_degree < 0 || t_degree > 16 || !t_coef) {
    msg = "invalid exact-solution description";
    return SG_ERR_ARG;
  }
  ExactData* E = new ExactData();
  E->q = q;
  E->idx_q = chaos_indices(hp.M, q);
  const int nq_modes = (int)(E->idx_q.size() / hp.M);
  E->c.assign(c, c + nq_modes);
  E->freq.assign(freq, freq + 3 * (size_t)nq_modes);
  E->t_coef.assign(t_coef, t_coef + t_degree + 1);
  E->p_in_q.assign(hp.n_xi, -1);
  for (int a = 0; a < hp.n_xi; ++a)
    for (int j = 0; j < nq_modes; ++j)
      if (std::equal(hp.idx.begin() + (size_t)a * hp.M, hp.idx.begin() + (size_t)(a + 1) * hp.M,
                     E->idx_q.begin() + (size_t)j * hp.M)) {
        E->p_in_q[a] = j;
        break;
      }
  // coupling G_mu[beta][alpha], beta in Lambda_p, alpha in Lambda_q (sparse rows)
  std::vector<std::vector<std::pair<int, std::pair<int, double>>>> grow(hp.n_xi);
  for (int b = 0; b < hp.n_xi; ++b)
    for (int t = 0; t < hp.n_terms; ++t)
      for (int a = 0; a < nq_modes; ++a) {
        if (E->c[a] == 0.0) continue;
        double g = 1.0;
        for (int m = 0; m < hp.M && g != 0.0; ++m)
          g *= hermite_triple(hp.mus[t][m], hp.idx[(size_t)b * hp.M + m], E->idx_q[(size_t)a * hp.M + m]);
        if (g != 0.0) grow[b].push_back({t, {a, g * E->c[a]}});
      }
  // quadrature data
  const int n = hp.k + 1, nqs = hp.k + 4;
  const int nkd = hp.dim == 2 ? n * n : n * n * n;
  const int nqd = hp.dim == 2 ? nqs * nqs : nqs * nqs * nqs;
  Rule1D g = gauss_legendre(nqs);
  std::vector<double> gll = lobatto_nodes(hp.k);
  std::vector<double> S1((size_t)nqs * n), D1((size_t)nqs * n);
  for (int qq = 0; qq < nqs; ++qq)
    for (int j = 0; j < n; ++j) {
      S1[qq * n + j] = lagrange(gll, j, g.x[qq]);
      D1[qq * n + j] = lagrange_deriv(gll, j, g.x[qq]);
    }
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  std::vector<double> locP((size_t)hp.n_cells * hp.n_xi * nkd, 0.0), locK((size_t)hp.n_cells * hp.n_xi * nkd, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (long long cell = 0; cell < hp.n_cells; ++cell) {
    const int cc[3] = {(int)(cell % hp.cells[0]), (int)((cell / hp.cells[0]) % hp.cells[1]),
                       (int)(cell / ((long long)hp.cells[0] * hp.cells[1]))};
    std::vector<double> phi(nq_modes), gphi((size_t)nq_modes * 3), amu(hp.n_terms);
    for (int qd = 0; qd < nqd; ++qd) {
      const int qi[3] = {qd % nqs, (qd / nqs) % nqs, qd / (nqs * nqs)};
      double x[3] = {0, 0, 0}, w = detJ;
      for (int d = 0; d < hp.dim; ++d) {
        x[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      for (int a = 0; a < nq_modes; ++a) phi[a] = phi_val(hp, &E->freq[(size_t)a * 3], x, &gphi[(size_t)a * 3]);
      std::fill(amu.begin(), amu.end(), 0.0);
      for (size_t pc = 0; pc < hp.pieces.size(); ++pc) amu[hp.piece_term[pc]] += coef_piece(hp.pieces[pc], hp.dim, x, cell);
      // basis values / physical gradients at this point
      double bv[64], bg[64][3];
      for (int a = 0; a < nkd; ++a) {
        const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
        double v = 1.0;
        for (int d = 0; d < hp.dim; ++d) v *= S1[qi[d] * n + ai[d]];
        bv[a] = v;
        for (int dd = 0; dd < hp.dim; ++dd) {
          double gg = 1.0 / hp.h[dd];
          for (int d = 0; d < hp.dim; ++d) gg *= d == dd ? D1[qi[d] * n + ai[d]] : S1[qi[d] * n + ai[d]];
          bg[a][dd] = gg;
        }
      }
      for (int b = 0; b < hp.n_xi; ++b) {
        double* lp = &locP[((size_t)cell * hp.n_xi + b) * nkd];
        double* lk = &locK[((size_t)cell * hp.n_xi + b) * nkd];
        const int jb = E->p_in_q[b];
        if (jb >= 0 && E->c[jb] != 0.0) {
          const double s = w * E->c[jb] * phi[jb];
          for (int a = 0; a < nkd; ++a) lp[a] += s * bv[a];
        }
        double vec[3] = {0, 0, 0};
        for (auto& e : grow[b]) {
          const double s = e.second.second * amu[e.first];
          for (int d = 0; d < hp.dim; ++d) vec[d] += s * gphi[(size_t)e.second.first * 3 + d];
        }
        for (int a = 0; a < nkd; ++a) {
          double dot = 0.0;
          for (int d = 0; d < hp.dim; ++d) dot += vec[d] * bg[a][d];
          lk[a] += w * dot;
        }
      }
    }
  }
  // assemble, Dirichlet rows zero
  std::vector<double> P((size_t)hp.n_xi * hp.n_x, 0.0), K((size_t)hp.n_xi * hp.n_x, 0.0);
  for (long long cell = 0; cell < hp.n_cells; ++cell) {
    const int cc[3] = {(int)(cell % hp.cells[0]), (int)((cell / hp.cells[0]) % hp.cells[1]),
                       (int)(cell / ((long long)hp.cells[0] * hp.cells[1]))};
    for (int a = 0; a < nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      long long gidx = 0, stride = 1;
      bool inner = true;
      for (int d = 0; d < hp.dim; ++d) {
        const int gi = cc[d] * hp.k + ai[d];
        inner = inner && gi > 0 && gi < hp.nn[d] - 1;
        gidx += gi * stride;
        stride *= hp.nn[d];
      }
      if (!inner) continue;
      for (int b = 0; b < hp.n_xi; ++b) {
        P[(size_t)b * hp.n_x + gidx] += locP[((size_t)cell * hp.n_xi + b) * nkd + a];
        K[(size_t)b * hp.n_x + gidx] += locK[((size_t)cell * hp.n_xi + b) * nkd + a];
      }
    }
  }
  cudaError_t e = cudaMalloc(&E->d_P, P.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&E->d_K, K.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&E->d_tpk, 2 * kMaxNT * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&E->d_zero_rows, (hp.n_xi + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(E->d_P, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(E->d_K, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(E->d_zero_rows, 0, (hp.n_xi + 1) * sizeof(int));
  if (e != cudaSuccess) {
    exact_free(E);
    msg = std::string("exact-solution tables: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  out = E;
  return SG_OK;
}

// rhs = F^(n) (+ B_0 on slab 0) (+ J u_prev when u_prev != nullptr and slab > 0)
cudaError_t exact_rhs(const HostProblem& hp, const LaunchShape& ls, ExactData& E, const void* ctab, const int* gcol,
                      const int* gterm, const double* gval, const int* perm, int slab, const double* u_prev,
                      double* rhs, cudaStream_t s) {
  cudaError_t e = exact_rhs_load(hp, E, slab, rhs, s);
  if (e != cudaSuccess) return e;
  return exact_transfer(hp, ls, E, ctab, gcol, gterm, gval, perm, slab, u_prev, rhs, s);
}

cudaError_t exact_rhs_load(const HostProblem& hp, ExactData& E, int slab, double* rhs, cudaStream_t s) {
  const int nt = hp.n_t;
  const std::vector<double> nodes = radau_right_nodes(hp.r);
  const int ng = hp.r + (int)E.t_coef.size() + 2;
  Rule1D g = gauss_legendre(ng);
  const double t0 = slab * hp.tau;
  double tpk[2 * kMaxNT] = {0};
  for (int i = 0; i < nt; ++i) {
    double a = 0.0, b = 0.0;
    for (int qq = 0; qq < ng; ++qq) {
      const double t = t0 + hp.tau * g.x[qq];
      const double v = lagrange(nodes, i, g.x[qq]);
      a += hp.tau * g.w[qq] * poly_deriv(E.t_coef, t) * v;
      b += hp.tau * g.w[qq] * poly(E.t_coef, t) * v;
    }
    if (slab == 0) a += lagrange(nodes, i, 0.0) * poly(E.t_coef, t0);
    tpk[i] = a;
    tpk[kMaxNT + i] = b;
  }
  cudaError_t e = cudaMemcpyAsync(E.d_tpk, tpk, sizeof(tpk), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const long long total = (long long)hp.n_xi * nt * hp.n_x;
  k_rhs_combine<<<grid_of(total), 256, 0, s>>>(E.d_P, E.d_K, rhs, hp.n_xi, nt, hp.n_x, E.d_tpk, E.d_tpk + kMaxNT);
  return cudaGetLastError();
}

cudaError_t exact_transfer(const HostProblem& hp, const LaunchShape& ls, ExactData& E, const void* ctab,
                           const int* gcol, const int* gterm, const double* gval, const int* perm, int slab,
                           const double* u_prev, double* rhs, cudaStream_t s) {
  const int nt = hp.n_t;
  const std::vector<double> nodes = radau_right_nodes(hp.r);
  if (slab == 0 || !u_prev) return cudaSuccess;
  // transfer: rhs += (I (x) C_t (x) M_x) u_prev, C_t[i][j] = v_i(t_{n-1}^+) v_j^{prev}(t_{n-1}^-)
  ApplyParams p;
  fill_apply_params(hp, ls, ctab, E.d_zero_rows, gcol, gterm, gval, perm, u_prev, rhs, 0, p);
  p.nnz = 0;
  p.b = rhs;
  p.mode = kApplyAccumulate;
  const int nq = hp.k + 1, nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  for (int qd = 0; qd < nqd; ++qd) {
    const int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j < nt; ++j) {
        const double ct = lagrange(nodes, i, 0.0) * lagrange(nodes, j, 1.0);
        p.amq[(qd * nt + i) * nt + j] = w * ct / p.tb[i];
      }
  }
  return launch_apply(hp, ls, p, s);
}

cudaError_t moments(const HostProblem& hp, const double* u, int node, double* mean, double* var, cudaStream_t s) {
  k_moments<<<grid_of(hp.n_x), 256, 0, s>>>(u, mean, var, hp.n_xi, hp.n_t, node, hp.n_x);
  return cudaGetLastError();
}

// L2(D) errors at the end of slab n (time node r) of the mean, the variance
// and the full stochastic solution against the exact solution (Definition
// "error norms and quantities" at one time; modal identity for the full error).
sg_status exact_errors(const HostProblem& hp, const ExactData& E, const double* u_dev, int slab, double err[3],
                       std::string& msg) {
  const int r = hp.r, nt = hp.n_t;
  std::vector<double> U((size_t)hp.n_xi * hp.n_x);
  for (int a = 0; a < hp.n_xi; ++a) {
    cudaError_t e = cudaMemcpy(&U[(size_t)a * hp.n_x], u_dev + ((size_t)a * nt + r) * hp.n_x,
                               hp.n_x * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { msg = cudaGetErrorString(e); return SG_ERR_CUDA; }
  }
  const double Tt = poly(E.t_coef, (slab + 1) * hp.tau);
  const int nq_modes = (int)E.c.size();
  const int n = hp.k + 1, nqs = hp.k + 4;
  const int nkd = hp.dim == 2 ? n * n : n * n * n;
  const int nqd = hp.dim == 2 ? nqs * nqs : nqs * nqs * nqs;
  Rule1D g = gauss_legendre(nqs);
  std::vector<double> gll = lobatto_nodes(hp.k);
  std::vector<double> S1((size_t)nqs * n);
  for (int qq = 0; qq < nqs; ++qq)
    for (int j = 0; j < n; ++j) S1[qq * n + j] = lagrange(gll, j, g.x[qq]);
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  std::vector<char> in_p(nq_modes, 0);
  for (int a = 0; a < hp.n_xi; ++a)
    if (E.p_in_q[a] >= 0) in_p[E.p_in_q[a]] = 1;
  int zero_q = -1, zero_p = -1;
  for (int j = 0; j < nq_modes; ++j) {
    bool z = true;
    for (int m = 0; m < hp.M; ++m) z = z && E.idx_q[(size_t)j * hp.M + m] == 0;
    if (z) zero_q = j;
  }
  for (int a = 0; a < hp.n_xi; ++a) {
    bool z = true;
    for (int m = 0; m < hp.M; ++m) z = z && hp.idx[(size_t)a * hp.M + m] == 0;
    if (z) zero_p = a;
  }
  double e_mean = 0.0, e_var = 0.0, e_full = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : e_mean, e_var, e_full)
  for (long long cell = 0; cell < hp.n_cells; ++cell) {
    const int cc[3] = {(int)(cell % hp.cells[0]), (int)((cell / hp.cells[0]) % hp.cells[1]),
                       (int)(cell / ((long long)hp.cells[0] * hp.cells[1]))};
    long long gidx[64];
    for (int a = 0; a < nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      long long gi = 0, stride = 1;
      for (int d = 0; d < hp.dim; ++d) {
        gi += (long long)(cc[d] * hp.k + ai[d]) * stride;
        stride *= hp.nn[d];
      }
      gidx[a] = gi;
    }
    std::vector<double> uh(hp.n_xi), phi(nq_modes);
    for (int qd = 0; qd < nqd; ++qd) {
      const int qi[3] = {qd % nqs, (qd / nqs) % nqs, qd / (nqs * nqs)};
      double x[3] = {0, 0, 0}, w = detJ, bv[64];
      for (int d = 0; d < hp.dim; ++d) {
        x[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      for (int a = 0; a < nkd; ++a) {
        const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
        double v = 1.0;
        for (int d = 0; d < hp.dim; ++d) v *= S1[qi[d] * n + ai[d]];
        bv[a] = v;
      }
      for (int b = 0; b < hp.n_xi; ++b) {
        double s = 0.0;
        for (int a = 0; a < nkd; ++a) s += bv[a] * U[(size_t)b * hp.n_x + gidx[a]];
        uh[b] = s;
      }
      for (int j = 0; j < nq_modes; ++j) phi[j] = Tt * E.c[j] * phi_val(hp, &E.freq[(size_t)j * 3], x, nullptr);
      double full = 0.0, var_h = 0.0, var_ex = 0.0;
      for (int b = 0; b < hp.n_xi; ++b) {
        const int jb = E.p_in_q[b];
        const double d = uh[b] - (jb >= 0 ? phi[jb] : 0.0);
        full += d * d;
        if (b != zero_p) var_h += uh[b] * uh[b];
      }
      for (int j = 0; j < nq_modes; ++j) {
        if (!in_p[j]) full += phi[j] * phi[j];
        if (j != zero_q) var_ex += phi[j] * phi[j];
      }
      const double dm = (zero_p >= 0 ? uh[zero_p] : 0.0) - (zero_q >= 0 ? phi[zero_q] : 0.0);
      e_mean += w * dm * dm;
      e_var += w * (var_h - var_ex) * (var_h - var_ex);
      e_full += w * full;
    }
  }
  err[0] = std::sqrt(e_mean);
  err[1] = std::sqrt(e_var);
  err[2] = std::sqrt(e_full);
  return SG_OK;
}

sg_status stat_errors(const HostProblem& hp, const ExactData& E, const double* mean_dev, const double* var_dev,
                      double t, double err[2], std::string& msg) {
  std::vector<double> Mh(hp.n_x), Vh(hp.n_x);
  cudaError_t e = cudaMemcpy(Mh.data(), mean_dev, hp.n_x * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(Vh.data(), var_dev, hp.n_x * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { msg = cudaGetErrorString(e); return SG_ERR_CUDA; }
  const double Tt = poly(E.t_coef, t);
  const int nq_modes = (int)E.c.size();
  const int n = hp.k + 1, nqs = hp.k + 4;
  const int nkd = hp.dim == 2 ? n * n : n * n * n;
  const int nqd = hp.dim == 2 ? nqs * nqs : nqs * nqs * nqs;
  Rule1D g = gauss_legendre(nqs);
  std::vector<double> gll = lobatto_nodes(hp.k);
  std::vector<double> S1((size_t)nqs * n);
  for (int qq = 0; qq < nqs; ++qq)
    for (int j = 0; j < n; ++j) S1[qq * n + j] = lagrange(gll, j, g.x[qq]);
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  int zero_q = -1;
  for (int j = 0; j < nq_modes; ++j) {
    bool z = true;
    for (int m = 0; m < hp.M; ++m) z = z && E.idx_q[(size_t)j * hp.M + m] == 0;
    if (z) zero_q = j;
  }
  double e_mean = 0.0, e_var = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : e_mean, e_var)
  for (long long cell = 0; cell < hp.n_cells; ++cell) {
    const int cc[3] = {(int)(cell % hp.cells[0]), (int)((cell / hp.cells[0]) % hp.cells[1]),
                       (int)(cell / ((long long)hp.cells[0] * hp.cells[1]))};
    long long gidx[64];
    for (int a = 0; a < nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      long long gi = 0, stride = 1;
      for (int d = 0; d < hp.dim; ++d) {
        gi += (long long)(cc[d] * hp.k + ai[d]) * stride;
        stride *= hp.nn[d];
      }
      gidx[a] = gi;
    }
    for (int qd = 0; qd < nqd; ++qd) {
      const int qi[3] = {qd % nqs, (qd / nqs) % nqs, qd / (nqs * nqs)};
      double x[3] = {0, 0, 0}, w = detJ;
      for (int d = 0; d < hp.dim; ++d) {
        x[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      double mh = 0.0, vh = 0.0;
      for (int a = 0; a < nkd; ++a) {
        const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
        double v = 1.0;
        for (int d = 0; d < hp.dim; ++d) v *= S1[qi[d] * n + ai[d]];
        mh += v * Mh[gidx[a]];
        vh += v * Vh[gidx[a]];
      }
      double m_ex = 0.0, v_ex = 0.0;
      for (int j = 0; j < nq_modes; ++j) {
        const double ph = Tt * E.c[j] * phi_val(hp, &E.freq[(size_t)j * 3], x, nullptr);
        if (j == zero_q) m_ex = ph;
        else v_ex += ph * ph;
      }
      e_mean += w * (mh - m_ex) * (mh - m_ex);
      e_var += w * (vh - v_ex) * (vh - v_ex);
    }
  }
  err[0] = std::sqrt(e_mean);
  err[1] = std::sqrt(e_var);
  return SG_OK;
}

}  // namespace sg

// Batched Monte-Carlo for the random heat equation (paper, Sec. 5: the
// pathwise problem, Problem "mc-pathwise-deterministic", its slab system eq.
// mc-slab-system, the estimators eqs. mc-mean-estimator and
// mc-variance-estimator-unbiased, and Algorithm 1).
//
// All samples of all meshes of a call form ONE block-diagonal system per
// slab: the Monte-Carlo apply (sg_mc_apply.cu) evaluates every pathwise
// operator A(xi_s) = A_t (x) M + B_t (x) K[a(., xi_s)] of every mesh in one
// launch over a queue of (mesh, sample tile, cell) units, the right-hand side
// of sample s is the manufactured forcing f(x, t, xi_s) (its load vector is
// combined on the device from spatial tables per distinct spatial factor of
// the exact solution), and one FGMRES iterates on the whole system.  The
// preconditioner is, per mesh, one graph-captured V-cycle of the mean operator
// (its residuals use the true sampled operators, its Vanka patches and coarse
// solve the mean block): per-sample patch inverses would cost samples x cells
// x patch^2.  When the device memory cannot hold every sample at once, the
// samples are split into groups solved one after the other.  At t = T each
// group's mean and sum of squared deviations are merged into the running
// estimators with Chan's pairwise update (FP64, on the device).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "sg_internal.h"

namespace sg {


namespace {

// P_s = sum_g wP[s][g] Pg[g],  K_s = sum_{t,g} wK[s][t][g] Kg[t][g]
__global__ void k_mc_combine(const double* __restrict__ Pg, const double* __restrict__ Kg,
                             const double* __restrict__ wP, const double* __restrict__ wK, int S, int ng, int nt_terms,
                             long long n_x, double* __restrict__ P, double* __restrict__ K) {
  const long long total = (long long)S * n_x;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx / n_x);
    const long long m = idx - (long long)s * n_x;
    double p = 0.0, k = 0.0;
    for (int g = 0; g < ng; ++g) p = fma(wP[(long long)s * ng + g], Pg[(long long)g * n_x + m], p);
    for (int tg = 0; tg < nt_terms * ng; ++tg) k = fma(wK[(long long)s * nt_terms * ng + tg], Kg[(long long)tg * n_x + m], k);
    P[idx] = p;
    K[idx] = k;
  }
}

// batch statistics at time node r, merged into (count, mean, M2)
__global__ void k_mc_merge(const double* __restrict__ u, int S, int n_t, int r, long long n_x, double n_a,
                           double* __restrict__ mean, double* __restrict__ m2) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n_x; m += (long long)gridDim.x * blockDim.x) {
    double sb = 0.0;
    for (int s = 0; s < S; ++s) sb += u[((long long)s * n_t + r) * n_x + m];
    const double mb = sb / S;
    double q = 0.0;
    for (int s = 0; s < S; ++s) {
      const double d = u[((long long)s * n_t + r) * n_x + m] - mb;
      q = fma(d, d, q);
    }
    const double n = n_a + S;
    const double delta = mb - mean[m];
    mean[m] += delta * (S / n);
    m2[m] += q + delta * delta * (n_a * S / n);
  }
}

__global__ void k_mc_finish(double* __restrict__ m2, long long n_x, double n) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n_x; m += (long long)gridDim.x * blockDim.x)
    m2[m] = n > 1 ? m2[m] / (n - 1) : 0.0;
}

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sg::sm_count() * 16)); }

double psi(int n, double y) {
  // He_n(y) / sqrt(n!) by the three-term recurrence of the normalised polynomials
  double p0 = 1.0, p1 = y;
  if (n == 0) return 1.0;
  for (int k = 1; k < n; ++k) {
    const double p2 = (y * p1 - std::sqrt((double)k) * p0) / std::sqrt((double)(k + 1));
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double Psi(const int* alpha, const double* xi, int M) {
  double v = 1.0;
  for (int m = 0; m < M; ++m) v *= psi(alpha[m], xi[m]);
  return v;
}

double phi_val(const HostProblem& hp, const int* f, const double* x, double* grad) {
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

double coef_piece(const Piece& pc, int dim, const double* x, long long cell) {
  double v = pc.amp;
  for (int d = 0; d < dim; ++d) {
    if (pc.kind[d] == SG_F_SIN) v *= std::sin(pc.k[d] * M_PI * x[d]);
    else if (pc.kind[d] == SG_F_POW) v *= std::pow(x[d], (double)pc.k[d]);
  }
  if (!pc.scale.empty()) v *= pc.scale[cell];
  return v;
}

// Spatial tables of the exact solution grouped by distinct frequency vector:
// Pg[g] = (Phi_g, phi_m), Kg[t][g] = (a_t grad Phi_g, grad phi_m), Dirichlet rows 0.
void spatial_tables(const HostProblem& hp, const std::vector<std::vector<int>>& gfreq, std::vector<double>& Pg,
                    std::vector<double>& Kg) {
  const int ng = (int)gfreq.size();
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
  const int nrow = ng * (1 + hp.n_terms);
  std::vector<double> loc((size_t)hp.n_cells * nrow * nkd, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (long long cell = 0; cell < hp.n_cells; ++cell) {
    const int cc[3] = {(int)(cell % hp.cells[0]), (int)((cell / hp.cells[0]) % hp.cells[1]),
                       (int)(cell / ((long long)hp.cells[0] * hp.cells[1]))};
    std::vector<double> amu(hp.n_terms);
    for (int qd = 0; qd < nqd; ++qd) {
      const int qi[3] = {qd % nqs, (qd / nqs) % nqs, qd / (nqs * nqs)};
      double x[3] = {0, 0, 0}, w = detJ;
      for (int d = 0; d < hp.dim; ++d) {
        x[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      std::fill(amu.begin(), amu.end(), 0.0);
      for (size_t pc = 0; pc < hp.pieces.size(); ++pc) amu[hp.piece_term[pc]] += coef_piece(hp.pieces[pc], hp.dim, x, cell);
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
      for (int gi = 0; gi < ng; ++gi) {
        double grad[3];
        const double ph = phi_val(hp, gfreq[gi].data(), x, grad);
        double* lp = &loc[((size_t)cell * nrow + gi) * nkd];
        for (int a = 0; a < nkd; ++a) lp[a] += w * ph * bv[a];
        for (int t = 0; t < hp.n_terms; ++t) {
          double* lk = &loc[((size_t)cell * nrow + ng + t * ng + gi) * nkd];
          for (int a = 0; a < nkd; ++a) {
            double dot = 0.0;
            for (int d = 0; d < hp.dim; ++d) dot += grad[d] * bg[a][d];
            lk[a] += w * amu[t] * dot;
          }
        }
      }
    }
  }
  std::vector<double> all((size_t)nrow * hp.n_x, 0.0);
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
      for (int r = 0; r < nrow; ++r) all[(size_t)r * hp.n_x + gidx] += loc[((size_t)cell * nrow + r) * nkd + a];
    }
  }
  Pg.assign(all.begin(), all.begin() + (size_t)ng * hp.n_x);
  Kg.assign(all.begin() + (size_t)ng * hp.n_x, all.end());
}

}  // namespace

namespace {

// One mesh of a Monte-Carlo solve: its samples of the current group, the
// batch problem (rows = samples), per-sample load tables, the mean-operator
// V-cycle and the time-mass tables of the apply.
struct McMesh {
  sg_ctx* parent = nullptr;
  int S_total = 0, S = 0, s_begin = 0;
  const double* xi = nullptr;          // host, S_total x M
  std::vector<int> group;              // exact-solution mode -> spatial group
  int ng = 0;
  double *d_Pg = nullptr, *d_Kg = nullptr;
  HostProblem hp;
  ExactData* E = nullptr;
  MG* mg = nullptr;
  double *d_wgt = nullptr, *d_amqA = nullptr, *d_amqC = nullptr;
  long long off = 0, n = 0;
  double n_done = 0.0;
};

void free_group(McMesh& m) {
  if (m.mg) {
    mg_free(*m.mg);
    delete m.mg;
    m.mg = nullptr;
  }
  if (m.E) {
    cudaFree(m.E->d_P);
    cudaFree(m.E->d_K);
    cudaFree(m.E->d_tpk);
    cudaFree(m.E->d_zero_rows);
    delete m.E;
    m.E = nullptr;
  }
  cudaFree(m.d_wgt);
  m.d_wgt = nullptr;
}

}  // namespace

sg_status mc_solve_meshes(const std::vector<sg_ctx*>& parents, const std::vector<int>& n_samples,
                          const std::vector<const double*>& xis, int tile, int mg_precision, double rtol, int max_it,
                          const std::vector<double*>& mean_T, const std::vector<double*>& var_T,
                          const std::vector<double*>& u_T, sg_mc_stats* st, cudaStream_t stream, std::string& msg) {
  const auto t0 = std::chrono::steady_clock::now();
  const int P = (int)parents.size();
  if (P < 1 || P > kMcMaxProb) { msg = "1 to 4 meshes"; return SG_ERR_ARG; }
  const HostProblem& h0 = parents[0]->hp;
  for (int p = 1; p < P; ++p) {
    const HostProblem& h = parents[p]->hp;
    if (h.dim != h0.dim || h.k != h0.k || h.r != h0.r || h.n_slabs != h0.n_slabs || h.T != h0.T ||
        h.n_terms != h0.n_terms || h.M != h0.M) {
      msg = "meshes of one Monte-Carlo solve need the same dimension, degrees, slabs, T and coefficient terms";
      return SG_ERR_ARG;
    }
  }
  const int nt = h0.n_t, M = h0.M, nterm = h0.n_terms;
  std::vector<McMesh> ms(P);
  cudaError_t e = cudaSuccess;
  sg_status status = SG_OK;
  sg_mc_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  for (int p = 0; p < P; ++p) {
    McMesh& m = ms[p];
    m.parent = parents[p];
    m.S_total = n_samples[p];
    m.xi = xis[p];
    stats.n_samples += m.S_total;
    const ExactData& ex = *m.parent->exact;
    const int nq = (int)ex.c.size();
    std::map<std::vector<int>, int> gid;
    std::vector<std::vector<int>> gfreq;
    m.group.assign(nq, 0);
    for (int a = 0; a < nq; ++a) {
      std::vector<int> f(ex.freq.begin() + 3 * a, ex.freq.begin() + 3 * a + 3);
      auto it = gid.find(f);
      if (it == gid.end()) {
        m.group[a] = (int)gfreq.size();
        gid[f] = m.group[a];
        gfreq.push_back(f);
      } else {
        m.group[a] = it->second;
      }
    }
    m.ng = (int)gfreq.size();
    std::vector<double> Pg, Kg, amqA, amqC;
    spatial_tables(m.parent->hp, gfreq, Pg, Kg);
    if (e == cudaSuccess) e = cudaMalloc(&m.d_Pg, Pg.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&m.d_Kg, Kg.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m.d_Pg, Pg.data(), Pg.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m.d_Kg, Kg.data(), Kg.size() * sizeof(double), cudaMemcpyHostToDevice);
    // time-mass tables of the apply (A_hat) and of the transfer (C_t)
    const HostProblem& h = m.parent->hp;
    const std::vector<double> nodes = radau_right_nodes(h.r);
    std::vector<double> Ct((size_t)nt * nt);
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j < nt; ++j) Ct[(size_t)i * nt + j] = lagrange(nodes, i, 0.0) * lagrange(nodes, j, 1.0);
    mc_amq(h, h.A_hat, amqA);
    mc_amq(h, Ct, amqC);
    if (e == cudaSuccess) e = cudaMalloc(&m.d_amqA, amqA.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&m.d_amqC, amqC.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m.d_amqA, amqA.data(), amqA.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m.d_amqC, amqC.data(), amqC.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(mean_T[p], 0, h.n_x * sizeof(double), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(var_T[p], 0, h.n_x * sizeof(double), stream);
  }
  // apply tile shapes: (samples per tile, cells per chunk) candidates within the
  // shared-memory budget; the fastest on the first group's system is kept
  struct Shape2 {
    int ts, chunk;
    size_t smem;
  };
  std::vector<Shape2> cand;
  for (int t = 8; t <= std::max(8, tile); t *= 2) {
    const int tt = std::min(t, std::max(1, tile));
    int best_c = 0;
    for (int c = 1; c <= 8; ++c)
      if (mc_smem_bytes(h0.dim, h0.k, nt, tt, nterm, c, 8) <= 100 * 1024) best_c = c;
    if (best_c == 0) break;
    cand.push_back({tt, best_c, mc_smem_bytes(h0.dim, h0.k, nt, tt, nterm, best_c, 8)});
    if (best_c > 2) cand.push_back({tt, best_c / 2, mc_smem_bytes(h0.dim, h0.k, nt, tt, nterm, best_c / 2, 8)});
    if (tt == tile) break;
  }
  if (cand.empty()) cand.push_back({1, 1, mc_smem_bytes(h0.dim, h0.k, nt, 1, nterm, 1, 8)});
  int ts = cand.back().ts, chunk = cand.back().chunk;
  size_t smem = cand.back().smem;
  bool tuned = cand.size() == 1;
  stats.max_rel_residual = 0.0;
  if (e == cudaSuccess) e = prepare_mc_kernel(SG_PREC_FP64, h0.dim, h0.k, nt);
  // sample groups: all samples in one system unless the device memory says otherwise
  const int m_restart = 10;
  double vec_bytes = 0.0;
  for (int p = 0; p < P; ++p) vec_bytes += (double)ms[p].S_total * nt * ms[p].parent->hp.n_x * sizeof(double);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const double need = vec_bytes * (2 * m_restart + 3 + 2 + 3);
  const int groups = std::max(1, (int)std::ceil(need / (0.7 * (double)free_b)));
  const int mgp = mg_precision;
  double* d_krylov = nullptr;
  double *U = nullptr, *RHS = nullptr;
  for (int gi = 0; gi < groups && e == cudaSuccess && status == SG_OK; ++gi) {
    long long N = 0;
    for (int p = 0; p < P && e == cudaSuccess && status == SG_OK; ++p) {
      McMesh& m = ms[p];
      const HostProblem& ph = m.parent->hp;
      m.s_begin = (int)((long long)m.S_total * gi / groups);
      m.S = (int)((long long)m.S_total * (gi + 1) / groups) - m.s_begin;
      m.off = N;
      m.n = (long long)m.S * nt * ph.n_x;
      N += m.n;
      if (m.S == 0) continue;
      // the batch problem: rows = samples, diagonal coupling Psi_mu(xi_s)
      m.hp = ph;
      m.hp.n_xi = m.S;
      m.hp.idx.assign((size_t)m.S * M, 0);
      m.hp.g.row.assign(m.S + 1, 0);
      m.hp.g.col.clear();
      m.hp.g.term.clear();
      m.hp.g.val.clear();
      m.hp.perm.resize(m.S);
      const ExactData& ex = *m.parent->exact;
      const int nq = (int)ex.c.size();
      std::vector<double> wgt((size_t)m.S * nterm), wP((size_t)m.S * m.ng, 0.0), wK((size_t)m.S * nterm * m.ng, 0.0);
      for (int s = 0; s < m.S; ++s) {
        const double* xs = m.xi + (size_t)(m.s_begin + s) * M;
        for (int t = 0; t < nterm; ++t) {
          wgt[(size_t)s * nterm + t] = Psi(ph.mus[t].data(), xs, M);
          if (wgt[(size_t)s * nterm + t] != 0.0) {
            m.hp.g.col.push_back(s);
            m.hp.g.term.push_back(t);
            m.hp.g.val.push_back(wgt[(size_t)s * nterm + t]);
          }
        }
        m.hp.g.row[s + 1] = (int)m.hp.g.col.size();
        m.hp.perm[s] = s;
        for (int a = 0; a < nq; ++a) {
          const double w = ex.c[a] * Psi(&ex.idx_q[(size_t)a * M], xs, M);
          wP[(size_t)s * m.ng + m.group[a]] += w;
          for (int t = 0; t < nterm; ++t)
            wK[((size_t)s * nterm + t) * m.ng + m.group[a]] += wgt[(size_t)s * nterm + t] * w;
        }
      }
      // per-sample load tables
      m.E = new ExactData(ex);
      m.E->d_P = m.E->d_K = m.E->d_tpk = nullptr;
      m.E->d_zero_rows = nullptr;
      double *d_wP = nullptr, *d_wK = nullptr;
      e = cudaMalloc(&m.E->d_P, (size_t)m.S * ph.n_x * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&m.E->d_K, (size_t)m.S * ph.n_x * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&m.E->d_tpk, 2 * kMaxNT * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&d_wP, wP.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&d_wK, wK.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMemcpy(d_wP, wP.data(), wP.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(d_wK, wK.data(), wK.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        k_mc_combine<<<grid_n((long long)m.S * ph.n_x), 256, 0, stream>>>(m.d_Pg, m.d_Kg, d_wP, d_wK, m.S, m.ng, nterm,
                                                                           ph.n_x, m.E->d_P, m.E->d_K);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      cudaFree(d_wP);
      cudaFree(d_wK);
      if (e == cudaSuccess) e = cudaMalloc(&m.d_wgt, wgt.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMemcpy(m.d_wgt, wgt.data(), wgt.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) break;
      // mean-operator V-cycle over all samples of the group
      m.mg = new MG();
      m.mg->coarse_dofs = m.parent->mg_coarse_dofs;
      status = mg_build_mc(m.hp, mgp, 2, 0.7, wgt, std::min(ts, 32), *m.mg, msg);
    }
    if (e != cudaSuccess || status != SG_OK) break;
    // one system for every mesh of the group
    cudaFree(U);
    cudaFree(RHS);
    cudaFree(d_krylov);
    U = RHS = d_krylov = nullptr;
    e = cudaMalloc(&U, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&RHS, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d_krylov), krylov_bytes(N, m_restart));
    if (e == cudaSuccess) e = cudaMemsetAsync(U, 0, N * sizeof(double), stream);
    if (e != cudaSuccess) break;
    McParams base;
    long long units = 0;
    int grid = 1;
    auto build_base = [&]() {
      std::memset(&base, 0, sizeof(base));
      base.u_hi = -1;
      units = 0;
      for (int p = 0; p < P; ++p) {
        McMesh& m = ms[p];
        if (m.S == 0) continue;
        McProblem& pr = base.pr[base.n_prob++];
        const HostProblem& ph = m.parent->hp;
        pr.ctab = m.parent->d_ctab;
        pr.wgt = m.d_wgt;
        pr.n_x = ph.n_x;
        pr.unit0 = units;
        pr.n_cells = (int)ph.n_cells;
        pr.S = m.S;
        pr.ts = std::min(ts, m.S);
        pr.tiles = (m.S + pr.ts - 1) / pr.ts;
        for (int d = 0; d < 3; ++d) {
          pr.nn[d] = ph.nn[d];
          pr.cells[d] = ph.cells[d];
          pr.ratio[d] = d < ph.dim ? (ph.h[0] * ph.h[0]) / (ph.h[d] * ph.h[d]) : 0.0;
        }
        pr.aniso = 0;
        for (int d = 1; d < ph.dim; ++d) pr.aniso |= ph.h[d] != ph.h[0];
        units += (long long)pr.tiles * pr.n_cells;
      }
      base.n_terms = nterm;
      base.chunk = chunk;
      base.units = units;
      for (int i = 0; i < nt; ++i) base.tb[i] = h0.tau * h0.B_hat[i * nt + i];
      grid = (int)std::max<long long>(1, std::min<long long>(units / chunk, sg::sm_count() * 2));
    };
    build_base();
    auto mc_launch = [&](const double* x, double* y, const double* b, int mode, bool transfer,
                         cudaStream_t st) -> cudaError_t {
      McParams q = base;
      q.mode = mode;
      q.mass_only = transfer ? 1 : 0;
      int j = 0;
      for (int p = 0; p < P; ++p) {
        McMesh& m = ms[p];
        if (m.S == 0) continue;
        q.pr[j].x = x + m.off;
        q.pr[j].y = y + m.off;
        q.pr[j].b = b ? b + m.off : nullptr;
        q.pr[j].amq = transfer ? m.d_amqC : m.d_amqA;
        ++j;
      }
      // waves of whole sample tiles whose rows of y (preset, then reduced into
      // by the apply) stay resident in L2 between the two
      cudaError_t err = cudaSuccess;
      for (int pi = 0; pi < base.n_prob && err == cudaSuccess; ++pi) {
        const McProblem& P = base.pr[pi];
        const double tile_bytes = (double)P.ts * nt * P.n_x * sizeof(double);
        const int tpw = std::max(1, (int)(kMcWaveBytes / tile_bytes));
        for (int t0 = 0; t0 < P.tiles && err == cudaSuccess; t0 += tpw) {
          q.u_lo = P.unit0 + (long long)t0 * P.n_cells;
          q.u_hi = P.unit0 + (long long)std::min(P.tiles, t0 + tpw) * P.n_cells;
          const int g = (int)std::max<long long>(1, std::min<long long>((q.u_hi - q.u_lo) / chunk, grid));
          err = launch_mc_apply(SG_PREC_FP64, h0.dim, h0.k, nt, q, g, 256, smem, st);
        }
      }
      return err;
    };
    auto apply = [&](const double* in, double* out, cudaStream_t st) {
      return mc_launch(in, out, nullptr, kApplyPlain, false, st);
    };
    if (!tuned) {
      // time one apply per candidate shape (after one untimed launch) on this system
      cudaEvent_t ea = nullptr, eb = nullptr;
      e = cudaEventCreate(&ea);
      if (e == cudaSuccess) e = cudaEventCreate(&eb);
      float best_ms = 1e30f;
      Shape2 best = cand.back();
      for (const Shape2& c : cand) {
        if (e != cudaSuccess) break;
        ts = c.ts;
        chunk = c.chunk;
        smem = c.smem;
        build_base();
        e = apply(U, RHS, stream);
        if (e == cudaSuccess) e = cudaEventRecord(ea, stream);
        if (e == cudaSuccess) e = apply(U, RHS, stream);
        if (e == cudaSuccess) e = cudaEventRecord(eb, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(eb);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
      if (ea) cudaEventDestroy(ea);
      if (eb) cudaEventDestroy(eb);
      ts = best.ts;
      chunk = best.chunk;
      smem = best.smem;
      build_base();
      tuned = true;
      stats.tile = ts;
      stats.chunk = chunk;
      if (e != cudaSuccess) break;
    }
    auto prec = [&](const double* in, double* out, cudaStream_t st) -> cudaError_t {
      for (int p = 0; p < P; ++p) {
        McMesh& m = ms[p];
        if (m.S == 0) continue;
        cudaError_t ee = mg_issue(*m.mg, in + m.off, out + m.off, st, 0);
        if (ee != cudaSuccess) return ee;
      }
      return cudaSuccess;
    };
    // every slab of this group replays one recorded solve
    KrylovGraph kg;
    for (int n = 0; n < h0.n_slabs && e == cudaSuccess && status == SG_OK; ++n) {
      for (int p = 0; p < P && e == cudaSuccess; ++p)
        if (ms[p].S > 0) e = exact_rhs_load(ms[p].hp, *ms[p].E, n, RHS + ms[p].off, stream);
      if (e == cudaSuccess && n > 0) e = mc_launch(U, RHS, RHS, kApplyAccumulate, true, stream);
      if (e != cudaSuccess) break;
      sg_solve_stats ss;
      status = fgmres_graph(N, RHS, U, rtol, max_it, m_restart, &ss, stream, msg, apply, prec, d_krylov, kg, 1);
      stats.total_iterations += ss.iterations;
      stats.max_slab_iterations = std::max(stats.max_slab_iterations, ss.iterations);
      stats.max_rel_residual = std::max(stats.max_rel_residual, ss.rel_residual);
    }
    for (int p = 0; p < P && e == cudaSuccess && status == SG_OK; ++p) {
      McMesh& m = ms[p];
      if (m.S == 0) continue;
      const long long nx = m.parent->hp.n_x;
      k_mc_merge<<<grid_n(nx), 256, 0, stream>>>(U + m.off, m.S, nt, nt - 1, nx, m.n_done, mean_T[p], var_T[p]);
      e = cudaGetLastError();
      if (e == cudaSuccess && u_T[p])
        e = cudaMemcpyAsync(u_T[p] + (size_t)m.s_begin * nt * nx, U + m.off, m.n * sizeof(double),
                            cudaMemcpyDeviceToDevice, stream);
      m.n_done += m.S;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    krylov_graph_free(kg);
    for (McMesh& m : ms) free_group(m);
    ++stats.batches;
  }
  for (int p = 0; p < P && e == cudaSuccess && status == SG_OK; ++p) {
    k_mc_finish<<<grid_n(ms[p].parent->hp.n_x), 256, 0, stream>>>(var_T[p], ms[p].parent->hp.n_x, ms[p].n_done);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  for (McMesh& m : ms) {
    free_group(m);
    cudaFree(m.d_Pg);
    cudaFree(m.d_Kg);
    cudaFree(m.d_amqA);
    cudaFree(m.d_amqC);
  }
  cudaFree(U);
  cudaFree(RHS);
  cudaFree(d_krylov);
  stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = stats;
  if (e != cudaSuccess) {
    msg = std::string("Monte-Carlo solve: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  return status;
}

sg_status mc_solve(sg_ctx* parent, int n_samples, const double* xi, int batch, int mg_precision, double rtol,
                   int max_it, double* mean_T, double* var_T, double* u_T, sg_mc_stats* st, cudaStream_t stream,
                   std::string& msg) {
  return mc_solve_meshes({parent}, {n_samples}, {xi}, batch, mg_precision, rtol, max_it, {mean_T}, {var_T}, {u_T}, st,
                         stream, msg);
}

}  // namespace sg

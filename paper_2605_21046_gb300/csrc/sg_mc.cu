// Batched Monte-Carlo for the random heat equation (paper, Sec. 5: the
// pathwise problem, Problem "mc-pathwise-deterministic", its slab system eq.
// mc-slab-system, the estimators eqs. mc-mean-estimator and
// mc-variance-estimator-unbiased, and Algorithm 1).
//
// A batch of S samples is solved as one block-diagonal system: every sample is
// a row of the coupling table with the single diagonal entry
//     sum_mu Psi_mu(xi_s) a_mu(x)  =  a(x, xi_s),
// so the apply kernel evaluates all S pathwise operators in one launch, the
// right-hand side of sample s is the manufactured forcing f(x, t, xi_s) (its
// load vector is combined on the device from spatial tables per distinct
// spatial factor of the exact solution), and FGMRES iterates on the batch.
// The preconditioner is one V-cycle of the mean operator (its residuals use
// the true sampled operators, its Vanka patches and coarse solve the mean
// block): per-sample patch inverses would cost samples x cells x patch^2.
// At t = T the batch mean and sum of squared deviations are merged into the
// running estimators with Chan's pairwise update (FP64, on the device).
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

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

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

sg_status mc_solve(sg_ctx* parent, int n_samples, const double* xi, int batch, int mg_precision, double rtol,
                   int max_it, double* mean_T, double* var_T, double* u_T, sg_mc_stats* st, cudaStream_t stream,
                   std::string& msg) {
  const auto t0 = std::chrono::steady_clock::now();
  const HostProblem& ph = parent->hp;
  const ExactData& ex = *parent->exact;
  const int M = ph.M, nt = ph.n_t, nq = (int)ex.c.size();
  // distinct spatial factors of the exact solution
  std::map<std::vector<int>, int> gid;
  std::vector<std::vector<int>> gfreq;
  std::vector<int> group(nq);
  for (int a = 0; a < nq; ++a) {
    std::vector<int> f(ex.freq.begin() + 3 * a, ex.freq.begin() + 3 * a + 3);
    auto it = gid.find(f);
    if (it == gid.end()) {
      group[a] = (int)gfreq.size();
      gid[f] = group[a];
      gfreq.push_back(f);
    } else {
      group[a] = it->second;
    }
  }
  const int ng = (int)gfreq.size();
  std::vector<double> Pg, Kg;
  spatial_tables(ph, gfreq, Pg, Kg);
  double *d_Pg = nullptr, *d_Kg = nullptr, *d_wP = nullptr, *d_wK = nullptr;
  cudaError_t e = cudaMalloc(&d_Pg, Pg.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_Kg, Kg.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_Pg, Pg.data(), Pg.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_Kg, Kg.data(), Kg.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&d_wP, (size_t)batch * ng * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_wK, (size_t)batch * ph.n_terms * ng * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(mean_T, 0, ph.n_x * sizeof(double), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(var_T, 0, ph.n_x * sizeof(double), stream);
  sg_mc_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  stats.n_samples = n_samples;
  sg_status status = SG_OK;
  double n_done = 0.0;
  for (int b0 = 0; b0 < n_samples && e == cudaSuccess && status == SG_OK; b0 += batch) {
    const int S = std::min(batch, n_samples - b0);
    // the batch problem: rows = samples, diagonal coupling Psi_mu(xi_s)
    HostProblem hp = ph;
    hp.n_xi = S;
    hp.idx.assign((size_t)S * M, 0);
    hp.g.row.assign(S + 1, 0);
    hp.g.col.clear();
    hp.g.term.clear();
    hp.g.val.clear();
    std::vector<double> wP((size_t)S * ng, 0.0), wK((size_t)S * ph.n_terms * ng, 0.0);
    for (int s = 0; s < S; ++s) {
      const double* xs = xi + (size_t)(b0 + s) * M;
      std::vector<double> psi_mu(ph.n_terms);
      for (int t = 0; t < ph.n_terms; ++t) {
        psi_mu[t] = Psi(ph.mus[t].data(), xs, M);
        if (psi_mu[t] != 0.0) {
          hp.g.col.push_back(s);
          hp.g.term.push_back(t);
          hp.g.val.push_back(psi_mu[t]);
        }
      }
      hp.g.row[s + 1] = (int)hp.g.col.size();
      for (int a = 0; a < nq; ++a) {
        const double w = ex.c[a] * Psi(&ex.idx_q[(size_t)a * M], xs, M);
        wP[(size_t)s * ng + group[a]] += w;
        for (int t = 0; t < ph.n_terms; ++t) wK[((size_t)s * ph.n_terms + t) * ng + group[a]] += psi_mu[t] * w;
      }
    }
    hp.perm.resize(S);
    for (int s = 0; s < S; ++s) hp.perm[s] = s;
    sg_ctx* bc = nullptr;
    status = make_ctx(std::move(hp), parent->hp.precision, &bc, msg);
    if (status != SG_OK) break;
    bc->mg = new MG();
    status = mg_build(bc->hp, mg_precision, 2, 0.7, *bc->mg, msg, true);
    if (status == SG_OK) {
      ExactData* E = new ExactData(*parent->exact);
      E->d_P = E->d_K = E->d_tpk = nullptr;
      E->d_zero_rows = nullptr;
      bc->exact = E;
      const long long N = (long long)S * nt * ph.n_x;
      e = cudaMalloc(&E->d_P, (size_t)S * ph.n_x * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&E->d_K, (size_t)S * ph.n_x * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&E->d_tpk, 2 * kMaxNT * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&E->d_zero_rows, (S + 1) * sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(E->d_zero_rows, 0, (S + 1) * sizeof(int), stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_wP, wP.data(), wP.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_wK, wK.data(), wK.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) {
        k_mc_combine<<<grid_n((long long)S * ph.n_x), 256, 0, stream>>>(d_Pg, d_Kg, d_wP, d_wK, S, ng, ph.n_terms,
                                                                         ph.n_x, E->d_P, E->d_K);
        e = cudaGetLastError();
      }
      double *u = nullptr, *rhs = nullptr;
      if (e == cudaSuccess) e = cudaMalloc(&u, N * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&rhs, N * sizeof(double));
      if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, N * sizeof(double), stream);
      for (int n = 0; n < ph.n_slabs && e == cudaSuccess && status == SG_OK; ++n) {
        e = exact_rhs(bc->hp, bc->ls, *E, bc->d_ctab, bc->d_gcol, bc->d_gterm, bc->d_gval, bc->d_perm, n,
                      n > 0 ? u : nullptr, rhs, stream);
        if (e != cudaSuccess) break;
        sg_solve_stats ss;
        status = fgmres(bc, rhs, u, rtol, max_it, 30, &ss, stream, msg, &apply_device_ctx);
        stats.total_iterations += ss.iterations;
        stats.max_slab_iterations = std::max(stats.max_slab_iterations, ss.iterations);
        stats.max_rel_residual = std::max(stats.max_rel_residual, ss.rel_residual);
      }
      if (e == cudaSuccess && status == SG_OK) {
        k_mc_merge<<<grid_n(ph.n_x), 256, 0, stream>>>(u, S, nt, nt - 1, ph.n_x, n_done, mean_T, var_T);
        e = cudaGetLastError();
        if (e == cudaSuccess && u_T)
          e = cudaMemcpyAsync(u_T + (size_t)b0 * nt * ph.n_x, u, N * sizeof(double), cudaMemcpyDeviceToDevice, stream);
        n_done += S;
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      cudaFree(u);
      cudaFree(rhs);
    }
    ++stats.batches;
    destroy_ctx(bc);
  }
  if (e == cudaSuccess && status == SG_OK) {
    k_mc_finish<<<grid_n(ph.n_x), 256, 0, stream>>>(var_T, ph.n_x, n_done);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  }
  cudaFree(d_Pg);
  cudaFree(d_Kg);
  cudaFree(d_wP);
  cudaFree(d_wK);
  stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = stats;
  if (e != cudaSuccess) {
    msg = std::string("Monte-Carlo batch: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  return status;
}

}  // namespace sg

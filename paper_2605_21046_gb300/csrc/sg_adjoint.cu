// Discrete adjoint of the slab marching and the gradient of the quantity of
// interest J = E[ int_D u(x, T)^2 dx ] = sum_alpha U_alpha(T)^T M_x U_alpha(T)
// with respect to the amplitudes of the coefficient pieces and to the
// per-cell scale of one piece (the paper has no adjoint; the slab systems are
// those of eq. local_tensor_system, the load vector is data).
//
// With the forward slabs A U_n = F_n + J U_{n-1} (n = 0..N-1), the adjoint
// states solve, backwards in time,
//     A^T lambda_{N-1} = dJ/dU_{N-1} = 2 (I (x) e_r e_r^T (x) M_x) U_{N-1},
//     A^T lambda_n     = J^T lambda_{n+1} = (I (x) C_t^T (x) M_x) lambda_{n+1},
// and dJ/dp = - sum_n lambda_n^T (dA/dp) U_n with dA/dp = G_t (x) B_t (x) K[f_p]
// for a parameter p of a coefficient piece of term t (f_p the derivative of
// the piece).  The backward sweep visits the slabs in segments of
// `checkpoint_every`: the forward states at segment starts are kept; each
// segment is recomputed forwards before its adjoint solves.
//
// The bilinear forms lambda_n^T (dA/dp) U_n for all parameters at once are one
// kernel per slab: a CTA holds a chunk of cells, interpolates the gradients of
// lambda and U of every mode and time node to the Gauss points (the apply's
// sum factorisation), contracts them through the sparse coupling table per
// coefficient term and the derivative tables per parameter, and reduces per
// cell and per parameter (FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "sg_apply_kernel.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kMaxTerms = 16;

struct BilinParams {
  const double* lam;
  const double* u;
  const double* dtab;       // [n_tab][n_cells][NQD]: w_q |J| f_j(x_q) / h_0^2
  const int* tab_term;      // [n_tab]
  const int* g_row;
  const int* g_col;
  const int* g_term;
  const double* g_val;
  long long n_x, n_cells;
  int nn[3], cells[3];
  int n_xi, n_terms, n_tab, nnz, chunk, cell_tab;
  double tb[kMaxNT];
  double ratio[3];
  double* out_sum;          // [n_tab] += sum over cells
  double* out_cell;         // [n_cells] += the per-cell value of table cell_tab (or null)
};

size_t bilin_smem(int dim, int k, int n_t, int n_xi, int nnz, int n_tab, int chunk) {
  const size_t nqd = dim == 2 ? (k + 1) * (k + 1) : (k + 1) * (k + 1) * (k + 1);
  const size_t V = (size_t)n_xi * n_t;
  const size_t doubles = 2 * (size_t)chunk * V * (1 + dim) * nqd + nnz + (size_t)chunk * n_tab;
  const size_t ints = (n_xi + 1) + 2 * (size_t)nnz;
  return doubles * 8 + ints * 4;
}

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(256) k_bilinear(const BilinParams p) {
  using Sh = Shape<DIM, K>;
  constexpr int NQD = Sh::NQD, NKD = Sh::NKD, NC = Sh::NC, N = Sh::N;
  constexpr int SLOT = NC * NQD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int n_xi = p.n_xi, V = n_xi * NT, C = p.chunk;
  double* Ql = reinterpret_cast<double*>(smem_raw);         // [C][V][NC][NQD]
  double* Qu = Ql + (size_t)C * V * SLOT;
  double* Gv = Qu + (size_t)C * V * SLOT;                  // [nnz]
  double* red = Gv + p.nnz;                                // [C][n_tab]
  int* Gr = reinterpret_cast<int*>(red + (size_t)C * p.n_tab);
  int* Gc = Gr + n_xi + 1;
  int* Gt = Gc + p.nnz;
  for (int e = tid; e < p.nnz; e += nthr) {
    Gv[e] = p.g_val[e];
    Gc[e] = p.g_col[e];
    Gt[e] = p.g_term[e];
  }
  for (int e = tid; e <= n_xi; e += nthr) Gr[e] = p.g_row[e];
  const long long c_begin = (long long)blockIdx.x * p.n_cells / gridDim.x;
  const long long c_end = (long long)(blockIdx.x + 1) * p.n_cells / gridDim.x;
  const int nnx = p.nn[0], nny = p.nn[1], nnz_ = p.nn[2];
  for (long long c0 = c_begin; c0 < c_end; c0 += C) {
    const int nc = (int)min((long long)C, c_end - c0);
    __syncthreads();
    for (int e = tid; e < nc * p.n_tab; e += nthr) red[e] = 0.0;
    for (int idx = tid; idx < 2 * nc * V * NKD; idx += nthr) {
      const int which = idx / (nc * V * NKD);
      const int rest = idx - which * nc * V * NKD;
      const int a = rest % NKD, cv = rest / NKD;
      const int v = cv % V, c = cv / V;
      const long long gc = c0 + c;
      const unsigned int g32 = (unsigned int)gc;              // cells < 2^31: 32-bit divisions
      const int cx = (int)(g32 % (unsigned int)p.cells[0]), cy = (int)((g32 / (unsigned int)p.cells[0]) % (unsigned int)p.cells[1]);
      const int cz = (int)(g32 / ((unsigned int)p.cells[0] * (unsigned int)p.cells[1]));
      const int gx = cx * K + a % N, gy = cy * K + (a / N) % N, gz = DIM == 3 ? cz * K + a / (N * N) : 0;
      bool interior = gx > 0 && gx < nnx - 1 && gy > 0 && gy < nny - 1;
      if (DIM == 3) interior = interior && gz > 0 && gz < nnz_ - 1;
      // the slab operator reads Dirichlet nodes as 0 and keeps identity rows
      // there, so dA/dp has neither Dirichlet rows nor Dirichlet columns
      const double* src = which ? p.u : p.lam;
      double val = 0.0;
      if (interior) val = src[(long long)v * p.n_x + ((long long)gz * nny + gy) * nnx + gx];
      (which ? Qu : Ql)[(size_t)cv * SLOT + a] = val;
    }
    __syncthreads();
    for (int it = tid; it < 2 * nc * V; it += nthr) {
      double* q = (it < nc * V ? Ql : Qu) + (size_t)(it % (nc * V)) * SLOT;
      double u[NKD];
#pragma unroll
      for (int a = 0; a < NKD; ++a) u[a] = q[a];
      forward_cell<F64, DIM, K>(u, q);
    }
    __syncthreads();
    for (int it = tid; it < nc * NQD * n_xi; it += nthr) {
      const int a = it % n_xi, g = it / n_xi;
      const int c = g / NQD, q = g - c * NQD;
      double acc[kMaxTerms];
#pragma unroll
      for (int t = 0; t < kMaxTerms; ++t) acc[t] = 0.0;
      const double* bl = Ql + (size_t)c * V * SLOT + q;
      const double* bu = Qu + (size_t)c * V * SLOT + q;
      for (int e = Gr[a]; e < Gr[a + 1]; ++e) {
        const int b = Gc[e];
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
          double si = 0.0;
#pragma unroll
          for (int d = 0; d < DIM; ++d)
            si = fma(p.ratio[d] * bl[(size_t)(a * NT + i) * SLOT + (1 + d) * NQD],
                     bu[(size_t)(b * NT + i) * SLOT + (1 + d) * NQD], si);
          s = fma(p.tb[i], si, s);
        }
        const int t = Gt[e];
#pragma unroll
        for (int tt = 0; tt < kMaxTerms; ++tt)
          if (tt == t) acc[tt] = fma(Gv[e], s, acc[tt]);
      }
      for (int j = 0; j < p.n_tab; ++j) {
        const int t = p.tab_term[j];
        double at = 0.0;
#pragma unroll
        for (int tt = 0; tt < kMaxTerms; ++tt)
          if (tt == t) at = acc[tt];
        const double v = at * p.dtab[((size_t)j * p.n_cells + (c0 + c)) * NQD + q];
        if (v != 0.0) atomicAdd(&red[c * p.n_tab + j], v);
      }
    }
    __syncthreads();
    for (int e = tid; e < nc * p.n_tab; e += nthr) {
      const int c = e / p.n_tab, j = e - c * p.n_tab;
      atomicAdd(&p.out_sum[j], red[e]);
      if (j == p.cell_tab && p.out_cell) p.out_cell[c0 + c] += red[e];
    }
  }
}

void* select_bilinear(int dim, int k, int n_t) {
#define SG_B(D, KK, T) \
  if (dim == D && k == KK && n_t == T) return reinterpret_cast<void*>(&k_bilinear<D, KK, T>);
  SG_B(2, 1, 1) SG_B(2, 1, 2) SG_B(2, 1, 3) SG_B(2, 1, 4)
  SG_B(2, 2, 1) SG_B(2, 2, 2) SG_B(2, 2, 3) SG_B(2, 2, 4)
  SG_B(2, 3, 1) SG_B(2, 3, 2) SG_B(2, 3, 3) SG_B(2, 3, 4)
  SG_B(3, 1, 1) SG_B(3, 1, 2) SG_B(3, 2, 1) SG_B(3, 2, 2)
#undef SG_B
  return nullptr;
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, long long n, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Zeroes the Dirichlet rows of a slab vector (all modes and time nodes).
__global__ void k_zero_boundary(double* __restrict__ v, long long n_total, long long n_x, int nnx, int nny, int nnz,
                                int dim) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n_total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx % n_x;
    const int ix = (int)(m % nnx), iy = (int)((m / nnx) % nny), iz = (int)(m / ((long long)nnx * nny));
    bool bd = ix == 0 || ix == nnx - 1 || iy == 0 || iy == nny - 1;
    if (dim == 3) bd = bd || iz == 0 || iz == nnz - 1;
    if (bd) v[idx] = 0.0;
  }
}

}  // namespace

// y = b + (I (x) Tm (x) M_x) x on interior rows (b on Dirichlet rows), Tm an
// N_t x N_t time matrix; the cell kernel in accumulate mode with no stiffness.
cudaError_t time_mass_apply(const HostProblem& hp, const LaunchShape& ls, const void* ctab, const int* zero_rows,
                            const int* gcol, const int* gterm, const double* gval, const int* perm,
                            const double* Tm, const double* x, double* y, cudaStream_t s) {
  ApplyParams p;
  fill_apply_params(hp, ls, ctab, zero_rows, gcol, gterm, gval, perm, x, y, 0, p);
  p.nnz = 0;
  p.b = y;
  p.mode = kApplyAccumulate;
  const int nt = hp.n_t, nq = hp.k + 1, nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  for (int qd = 0; qd < nqd; ++qd) {
    const int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j < nt; ++j) p.amq[(qd * nt + i) * nt + j] = w * Tm[i * nt + j] / p.tb[i];
  }
  return launch_apply(hp, ls, p, s);
}

sg_status adjoint_gradient(sg_ctx* ctx, double rtol, int max_it, int K, int cell_piece, double* J_out,
                           double* g_amp, double* g_cell, sg_adjoint_stats* st, cudaStream_t s, std::string& msg) {
  const auto t0 = std::chrono::steady_clock::now();
  const HostProblem& hp = ctx->hp;
  const int nt = hp.n_t, N = hp.n_slabs, n_pieces = (int)hp.pieces.size();
  const long long n = (long long)hp.n_xi * nt * hp.n_x;
  if (!ctx->exact) { msg = "needs sg_set_exact"; return SG_ERR_ARG; }
  if (!ctx->mg) { msg = "needs sg_mg_setup"; return SG_ERR_ARG; }
  if (K < 1) { msg = "checkpoint_every must be >= 1"; return SG_ERR_ARG; }
  if (hp.n_terms > kMaxTerms) { msg = "more than 16 coefficient terms"; return SG_ERR_UNSUPPORTED; }
  if (cell_piece >= n_pieces) { msg = "cell_piece out of range"; return SG_ERR_ARG; }
  void* bk = select_bilinear(hp.dim, hp.k, nt);
  if (!bk) { msg = "no gradient kernel for this (dim, degree, time nodes)"; return SG_ERR_UNSUPPORTED; }
  // derivative tables: per piece the amplitude derivative, then (optionally)
  // the per-cell scale derivative of cell_piece
  const int n_tab = n_pieces + (cell_piece >= 0 ? 1 : 0);
  const int nq = hp.k + 1, nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  Rule1D g = gauss_legendre(nq);
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  std::vector<double> dtab((size_t)n_tab * hp.n_cells * nqd, 0.0);
  std::vector<int> tab_term(n_tab);
  for (int j = 0; j < n_tab; ++j) tab_term[j] = hp.piece_term[j < n_pieces ? j : cell_piece];
  for (long long c = 0; c < hp.n_cells; ++c) {
    const int cc[3] = {(int)(c % hp.cells[0]), (int)((c / hp.cells[0]) % hp.cells[1]),
                       (int)(c / ((long long)hp.cells[0] * hp.cells[1]))};
    for (int qd = 0; qd < nqd; ++qd) {
      const int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
      double x[3] = {0, 0, 0}, w = detJ / (hp.h[0] * hp.h[0]);
      for (int d = 0; d < hp.dim; ++d) {
        x[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      for (int j = 0; j < n_tab; ++j) {
        const Piece& pc = hp.pieces[j < n_pieces ? j : cell_piece];
        double v = w;
        for (int d = 0; d < hp.dim; ++d) v *= factor_value(pc.kind[d], pc.k[d], x[d]);
        if (j < n_pieces) {
          if (!pc.scale.empty()) v *= pc.scale[c];
        } else {
          v *= pc.amp;
        }
        dtab[((size_t)j * hp.n_cells + c) * nqd + qd] = v;
      }
    }
  }
  // device workspace
  const int n_ck = (N + K - 1) / K;
  const size_t vec = (size_t)n * sizeof(double);
  double *d_ck = nullptr, *d_seg = nullptr, *d_lam = nullptr, *d_rhs = nullptr, *d_dtab = nullptr, *d_out = nullptr,
         *d_part = nullptr;
  int *d_tt = nullptr, *d_zero = nullptr;
  cudaError_t e = cudaMalloc(&d_ck, std::max<size_t>(1, (size_t)n_ck) * vec);
  if (e == cudaSuccess) e = cudaMalloc(&d_seg, (size_t)std::min(K, N) * vec);
  if (e == cudaSuccess) e = cudaMalloc(&d_lam, 2 * vec);
  if (e == cudaSuccess) e = cudaMalloc(&d_rhs, vec);
  if (e == cudaSuccess) e = cudaMalloc(&d_dtab, dtab.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, ((size_t)n_tab + hp.n_cells) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_part, 256 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_tt, n_tab * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_zero, (hp.n_xi + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_dtab, dtab.data(), dtab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tt, tab_term.data(), n_tab * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_zero, 0, (hp.n_xi + 1) * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, ((size_t)n_tab + hp.n_cells) * sizeof(double), s);
  sg_adjoint_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  sg_status status = SG_OK;
  // time matrices: terminal source 2 e_r e_r^T, adjoint transfer C_t^T
  const std::vector<double> nodes = radau_right_nodes(hp.r);
  std::vector<double> Tterm((size_t)nt * nt, 0.0), CtT((size_t)nt * nt, 0.0);
  Tterm[(size_t)(nt - 1) * nt + (nt - 1)] = 2.0;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j) CtT[(size_t)i * nt + j] = lagrange(nodes, j, 0.0) * lagrange(nodes, i, 1.0);
  auto forward_slab = [&](int slab, const double* u_prev, double* u_out) -> sg_status {
    cudaError_t ee = exact_rhs(hp, ctx->ls, *ctx->exact, ctx->d_ctab, ctx->d_gcol, ctx->d_gterm, ctx->d_gval,
                               ctx->d_perm, slab, u_prev, d_rhs, s);
    if (ee != cudaSuccess) { msg = cudaGetErrorString(ee); return SG_ERR_CUDA; }
    // initial guess: the previous slab (u_out may be u_prev itself when a
    // segment holds one slab; the right-hand side was formed first)
    if (!u_prev) ee = cudaMemsetAsync(u_out, 0, vec, s);
    else if (u_prev != u_out) ee = cudaMemcpyAsync(u_out, u_prev, vec, cudaMemcpyDeviceToDevice, s);
    if (ee != cudaSuccess) { msg = cudaGetErrorString(ee); return SG_ERR_CUDA; }
    sg_solve_stats ss;
    sg_status r = fgmres(ctx, d_rhs, u_out, rtol, max_it, 30, &ss, s, msg, &apply_device_ctx, 0);
    ++stats.forward_solves;
    stats.max_iterations = std::max(stats.max_iterations, ss.iterations);
    return r;
  };
  // forward sweep: checkpoint k holds U_{kK-1} (the state before segment k)
  double* u_last = d_seg;   // reused buffer for the running state
  for (int slab = 0; slab < N && e == cudaSuccess && status == SG_OK; ++slab) {
    double* dst = d_seg + (size_t)(slab % K) * n;
    const double* prev = slab == 0 ? nullptr : d_seg + (size_t)((slab - 1) % K) * n;
    status = forward_slab(slab, prev, dst);
    if (status == SG_OK && (slab + 1) % K == 0 && slab + 1 < N)
      e = cudaMemcpyAsync(d_ck + (size_t)((slab + 1) / K) * n, dst, vec, cudaMemcpyDeviceToDevice, s);
    u_last = dst;
  }
  double J = 0.0;
  if (e == cudaSuccess && status == SG_OK) {
    // terminal adjoint source and J = 1/2 U^T source
    double* lam_next = d_lam + n;
    e = cudaMemsetAsync(lam_next, 0, vec, s);
    if (e == cudaSuccess)
      e = time_mass_apply(hp, ctx->ls, ctx->d_ctab, d_zero, ctx->d_gcol, ctx->d_gterm, ctx->d_gval, ctx->d_perm,
                          Tterm.data(), u_last, lam_next, s);
    if (e == cudaSuccess) {
      k_dot<<<256, 256, 0, s>>>(u_last, lam_next, n, d_part);
      double part[256];
      e = cudaMemcpyAsync(part, d_part, sizeof(part), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (int i = 0; i < 256; ++i) J += part[i];
      J *= 0.5;
    }
  }
  // backward sweep by segments
  BilinParams bp;
  std::memset(&bp, 0, sizeof(bp));
  int bchunk = 0;
  {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int c = 1; c <= 16; ++c)
      if (bilin_smem(hp.dim, hp.k, nt, hp.n_xi, (int)hp.g.col.size(), n_tab, c) <= (size_t)optin - 1024) bchunk = c;
    if (bchunk == 0) { msg = "gradient kernel does not fit in shared memory"; status = SG_ERR_UNSUPPORTED; }
    else e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  }
  bp.dtab = d_dtab;
  bp.tab_term = d_tt;
  bp.g_row = ctx->d_grow;
  bp.g_col = ctx->d_gcol;
  bp.g_term = ctx->d_gterm;
  bp.g_val = ctx->d_gval;
  bp.n_x = hp.n_x;
  bp.n_cells = hp.n_cells;
  for (int d = 0; d < 3; ++d) {
    bp.nn[d] = hp.nn[d];
    bp.cells[d] = hp.cells[d];
    bp.ratio[d] = d < hp.dim ? (hp.h[0] * hp.h[0]) / (hp.h[d] * hp.h[d]) : 0.0;
  }
  bp.n_xi = hp.n_xi;
  bp.n_terms = hp.n_terms;
  bp.n_tab = n_tab;
  bp.nnz = (int)hp.g.col.size();
  bp.chunk = bchunk;
  bp.cell_tab = cell_piece >= 0 ? n_pieces : -1;
  for (int i = 0; i < nt; ++i) bp.tb[i] = hp.tau * hp.B_hat[i * nt + i];
  bp.out_sum = d_out;
  bp.out_cell = cell_piece >= 0 ? d_out + n_tab : nullptr;
  const size_t bsmem = bilin_smem(hp.dim, hp.k, nt, hp.n_xi, bp.nnz, n_tab, bchunk);
  const int bgrid = (int)std::min<long long>(sg::sm_count() * 2, hp.n_cells);
  // J alone (no gradient asked): no backward sweep
  const bool want_grad = g_amp || (g_cell && cell_piece >= 0);
  for (int seg = n_ck - 1; want_grad && seg >= 0 && e == cudaSuccess && status == SG_OK; --seg) {
    const int s0 = seg * K, s1 = std::min(N, s0 + K);
    // recompute the segment's forward states into d_seg[0 .. s1 - s0) (the
    // last segment is still there from the forward sweep)
    for (int slab = s0; slab < s1 && status == SG_OK && seg != n_ck - 1; ++slab) {
      const double* prev = slab == 0 ? nullptr : (slab == s0 ? d_ck + (size_t)seg * n : d_seg + (size_t)(slab - 1 - s0) * n);
      status = forward_slab(slab, prev, d_seg + (size_t)(slab - s0) * n);
    }
    for (int slab = s1 - 1; slab >= s0 && e == cudaSuccess && status == SG_OK; --slab) {
      double* lam = d_lam;              // lambda_n
      double* lam_next = d_lam + n;     // lambda_{n+1}, or the terminal source
      if (slab != N - 1) {
        e = cudaMemsetAsync(d_rhs, 0, vec, s);
        if (e == cudaSuccess)
          e = time_mass_apply(hp, ctx->ls, ctx->d_ctab, d_zero, ctx->d_gcol, ctx->d_gterm, ctx->d_gval, ctx->d_perm,
                              CtT.data(), lam_next, d_rhs, s);
      } else {
        e = cudaMemcpyAsync(d_rhs, lam_next, vec, cudaMemcpyDeviceToDevice, s);
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(lam, lam_next, vec, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) break;
      sg_solve_stats ss;
      status = fgmres(ctx, d_rhs, lam, rtol, max_it, 30, &ss, s, msg, &apply_device_ctx_t, 1);
      ++stats.adjoint_solves;
      stats.max_iterations = std::max(stats.max_iterations, ss.iterations);
      if (status != SG_OK) break;
      k_zero_boundary<<<(int)std::min<long long>((n + 255) / 256, sg::sm_count() * 16), 256, 0, s>>>(lam, n, hp.n_x, hp.nn[0], hp.nn[1], hp.nn[2], hp.dim);
      bp.lam = lam;
      bp.u = d_seg + (size_t)(slab - s0) * n;
      void* args[] = {&bp};
      e = cudaLaunchKernel(bk, dim3(bgrid), dim3(256), args, bsmem, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(lam_next, lam, vec, cudaMemcpyDeviceToDevice, s);
    }
  }
  if (e == cudaSuccess && status == SG_OK) {
    std::vector<double> out((size_t)n_tab + hp.n_cells);
    e = cudaMemcpyAsync(out.data(), d_out, out.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      if (g_amp)
        for (int j = 0; j < n_pieces; ++j) g_amp[j] = -out[j];
      if (g_cell && cell_piece >= 0)
        for (long long c = 0; c < hp.n_cells; ++c) g_cell[c] = -out[n_tab + c];
      if (J_out) *J_out = J;
    }
  }
  cudaFree(d_ck);
  cudaFree(d_seg);
  cudaFree(d_lam);
  cudaFree(d_rhs);
  cudaFree(d_dtab);
  cudaFree(d_out);
  cudaFree(d_part);
  cudaFree(d_tt);
  cudaFree(d_zero);
  stats.J = J;
  stats.checkpoints = n_ck - 1;
  stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = stats;
  if (e != cudaSuccess) {
    msg = std::string("adjoint: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  return status;
}

}  // namespace sg

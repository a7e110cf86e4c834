// sg_apply: y = A^(n) x for the stochastic-Galerkin slab operator
//     A^(n) = I (x) A_t (x) M_x + sum_mu G_mu (x) B_t (x) K_mu
// (eq. local_rhs_tensor), matrix-free, on a uniform Cartesian Q_k mesh.
//
// The apply is bound by the FP64 pipe (GB300 runs FP64 at 1/64 of FP32, two
// FMA lanes per clock per SM), so the design minimises FP64 instructions and
// keeps the pipe fed; memory traffic is two orders of magnitude below HBM
// speed and is not optimised for.
//
// Persistent CTAs split the cells evenly (every CTA gets n_cells / grid cells,
// +-1, so there is no wave tail) and walk their range in chunks of C cells.
// A chunk holds ALL N_xi * N_t vectors of its cells in shared memory, because
// the Gauss-point work couples every chaos mode (through G_mu) and every time
// node (through A_t):
//   phase 0  compute the global node of every (cell, local node) of the
//            chunk once into shared memory, gather the chunk's nodal values
//            of every vector through it (Dirichlet nodes read as 0), and the
//            coefficient values of its cells, as
//            products G value x a_mu(x_q) for each distinct (mu, G value) pair
//            of the coupling table (13 pairs for M = 4, P = 3: the mean term's
//            1 and sqrt(1..3) for each xi_m), so the entries below need no
//            multiply;
//   phase 1  per (cell, vector): sum-factorised interpolation to the
//            (k+1)^d Gauss points and collocation gradients (reference
//            tables are compile-time constants, so their exact zeros and ones
//            cost nothing);
//   phase 2  per (cell, Gauss point, alpha): the time-node mass coupling
//            w_q sum_j A_t[i][j] u[alpha,j] and the sparse chaos contraction
//            sum_(beta,mu) G_mu[alpha][beta] a_mu(x_q) grad u[beta,i]; the
//            lanes of a warp take consecutive points of ONE chaos row, so the
//            coupling loop never diverges and its entries are broadcast loads
//            (rounds of up to 32 points, results held in registers until every
//            read of the round's points is done);
//   phase 3  per (cell, vector): the transposed sum factorisation back to
//            the cell's nodes;
//   phase 4  per (cell, vector, node): scale by tau*Bhat_ii and add into y
//            with an FP64 atomic in L2 (y was set by the init kernel: x on
//            Dirichlet nodes, 0 elsewhere).
// The kernel is generic over its arithmetic (sg_arith.h): native FP64, or
// double-word FP32 pairs that run on the FP32 pipe (58x the FP64 rate on
// GB300) with error-free transformations.  The device code is in
// sg_apply_kernel.cuh; sg_apply_f64.cu and sg_apply_dw.cu instantiate it.
// The right-Radau time mass matrix is diagonal (the (r+1)-point Radau rule is
// exact to degree 2r), so B_t = tau diag(Bhat): the stiffness part never
// mixes time nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sg_internal.h"
#include "sg_shape_tables.h"
#include "sg_vec.cuh"

namespace sg {

void* select_kernel_f64(int dim, int k, int n_t);
void* select_kernel_dw(int dim, int k, int n_t);
void* select_kernel_f32(int dim, int k, int n_t);


size_t apply_smem_bytes(int dim, int k, int n_t, int n_xi, int coef_rows, int nnz, int chunk,
                        int value_bytes, bool premul) {
  const size_t nqd = dim == 2 ? (k + 1) * (k + 1) : (k + 1) * (k + 1) * (k + 1);
  const size_t V = (size_t)n_xi * n_t;
  size_t vals = (size_t)chunk * V * (((1 + dim) * nqd) | 1)   // Qs (odd slot pitch)
                + (size_t)chunk * coef_rows * nqd        // Cs
                + nqd * n_t * n_t                        // Amq
                + n_t + 3                                // Tb, Rt
                + (premul ? coef_rows : nnz);            // G value per pair / per entry
  size_t ints = (n_xi + 1) + n_xi + (premul ? coef_rows : 0)    // Gr, Pm, pair terms
                + (size_t)chunk * nqd;                          // nodes of the chunk's cells
  // values, then 8-byte coupling entries at a 16-byte boundary, then ints
  return ((vals * value_bytes + 15) / 16) * 16 + 8 * (size_t)nnz + ints * sizeof(int);
}

int coupling_pairs(const HostProblem& hp, int* term, double* val) {
  int n = 0;
  for (size_t e = 0; e < hp.g.col.size(); ++e) {
    const int t = hp.g.term[e];
    const double v = hp.g.val[e];
    int k = 0;
    while (k < n && !(term[k] == t && val[k] == v)) ++k;
    if (k < n) continue;
    if (n == kMaxPairs) return -1;
    term[n] = t;
    val[n] = v;
    ++n;
  }
  return n;
}

// Coefficient rows per cell the kernel stages and whether they are pre-multiplied pairs.
static int coef_rows(const HostProblem& hp, bool& premul) {
  int term[kMaxPairs];
  double val[kMaxPairs];
  const int n = coupling_pairs(hp, term, val);
  premul = n >= 0;
  return premul ? n : hp.n_terms;
}

template <int K>
static double max_table_gap(const HostProblem& hp) {
  double g = 0.0;
  const int n = K + 1;
  for (int q = 0; q < n; ++q)
    for (int j = 0; j < n; ++j) {
      g = std::max(g, std::fabs(RefShape<K>::S(q, j) - hp.S[q * n + j]));
      g = std::max(g, std::fabs(RefShape<K>::D(q, j) - hp.Dhat[q * n + j]));
    }
  return g;
}

static void* select_kernel(int precision, int dim, int k, int n_t) {
  if (precision == SG_PREC_DW) return select_kernel_dw(dim, k, n_t);
  if (precision == kPrecF32) return select_kernel_f32(dim, k, n_t);
  return select_kernel_f64(dim, k, n_t);
}

// The dynamic shared-memory limit is a property of the kernel function, shared
// by every context and multigrid level that launches it: it is always set to
// the device's opt-in maximum, so a later set-up can never shrink the limit
// below what an earlier one launches with.
cudaError_t prepare_apply_kernel(int precision, int dim, int k, int n_t, size_t smem) {
  void* f = select_kernel(precision, dim, k, n_t);
  if (!f) return cudaErrorInvalidValue;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

int max_apply_chunk(const HostProblem& hp, size_t budget) {
  const int nnz = (int)hp.g.col.size();
  const int vb = hp.precision == kPrecF32 ? 4 : 8;
  bool premul = false;
  const int rows = coef_rows(hp, premul);
  int chunk = 0;
  for (int c = 1; c <= 64; ++c) {
    if (apply_smem_bytes(hp.dim, hp.k, hp.n_t, hp.n_xi, rows, nnz, c, vb, premul) > budget) break;
    chunk = c;
  }
  return chunk;
}

// Launch shape for a given chunk and thread count (0 = defaults).  A phase-2
// round holds at least one point of every chaos row (at most kmax items per
// thread), so kmax * threads >= n_xi; threads stay within the kernel's launch
// bounds.
sg_status plan_apply_shape(const HostProblem& hp, int chunk, int threads, LaunchShape& ls, std::string& msg) {
  void* f = select_kernel(hp.precision, hp.dim, hp.k, hp.n_t);
  if (!f) {
    msg = "no apply kernel built for this (dim, degree, time nodes)";
    return SG_ERR_UNSUPPORTED;
  }
  const double gap = hp.k == 1 ? max_table_gap<1>(hp) : hp.k == 2 ? max_table_gap<2>(hp) : max_table_gap<3>(hp);
  if (!(gap < 1e-13)) {
    msg = "compiled reference shape tables disagree with the set-up tables";
    return SG_ERR_UNSUPPORTED;
  }
  if (hp.n_xi > 512) { msg = "more than 512 chaos modes"; return SG_ERR_UNSUPPORTED; }
  {
    const int nq = hp.k + 1, nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
    if (nqd * hp.n_t * hp.n_t > kMaxAmq) { msg = "time-point coupling table too large"; return SG_ERR_UNSUPPORTED; }
  }
  int dev = 0, smem_optin = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (smem_optin <= 0) smem_optin = 227 * 1024;
  if (n_sm <= 0) n_sm = 1;
  const int nnz = (int)hp.g.col.size();
  const int vb = hp.precision == kPrecF32 ? 4 : 8;
  const long long cells_per_sm = (hp.n_cells + n_sm - 1) / n_sm;
  const int max1 = max_apply_chunk(hp, (size_t)smem_optin - 1024);
  if (max1 == 0) {
    msg = "one cell with all chaos modes does not fit in shared memory";
    return SG_ERR_UNSUPPORTED;
  }
  if (chunk <= 0) {
    // default: the largest chunk that lets two CTAs share an SM
    chunk = max_apply_chunk(hp, (size_t)smem_optin / 2 - 1024);
    if (chunk == 0) chunk = max1;
    chunk = (int)std::min<long long>(chunk, std::max<long long>(1, (cells_per_sm + 1) / 2));
  }
  if (chunk > max1) { msg = "chunk does not fit in shared memory"; return SG_ERR_ARG; }
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
    cudaGetLastError();
    msg = "apply kernel attributes unavailable";
    return SG_ERR_CUDA;
  }
  // a phase-2 round needs one point of every chaos row: kmax * threads >= n_xi
  const int kmax = 18 / (hp.n_t * (1 + hp.dim)) < 1 ? 1 : std::min(3, 18 / (hp.n_t * (1 + hp.dim)));
  if (threads <= 0) {
    threads = 256;
    while (threads * kmax < hp.n_xi && threads + 128 <= fa.maxThreadsPerBlock) threads += 128;
  }
  if (threads * kmax < hp.n_xi || threads > fa.maxThreadsPerBlock || threads % 32 || threads < 32) {
    msg = "invalid thread count";
    return SG_ERR_ARG;
  }
  ls.chunk = chunk;
  ls.threads = threads;
  ls.stagger = 0;
  {
    bool premul = false;
    const int rows = coef_rows(hp, premul);
    ls.smem = apply_smem_bytes(hp.dim, hp.k, hp.n_t, hp.n_xi, rows, nnz, chunk, vb, premul);
  }
  cudaError_t e = prepare_apply_kernel(hp.precision, hp.dim, hp.k, hp.n_t, ls.smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, ls.threads, ls.smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    msg = "launch shape does not fit on an SM";
    return SG_ERR_ARG;
  }
  long long grid = (long long)n_sm * per_sm;
  grid = std::min<long long>(grid, hp.n_cells);
  ls.grid = (int)std::max<long long>(1, grid);
  return SG_OK;
}

sg_status plan_apply(const HostProblem& hp, LaunchShape& ls, std::string& msg) {
  return plan_apply_shape(hp, 0, 0, ls, msg);
}

void fill_apply_params(const HostProblem& hp, const LaunchShape& ls, const void* ctab,
                       const int* grow, const int* gcol, const int* gterm, const double* gval,
                       const int* perm, const void* x, void* y, int transpose, ApplyParams& p) {
  std::memset(&p, 0, sizeof(p));
  p.x = x;
  p.y = y;
  p.ctab = static_cast<const double*>(ctab);
  p.g_row = grow;
  p.g_col = gcol;
  p.g_term = gterm;
  p.g_val = gval;
  p.perm = perm;
  p.n_x = hp.n_x;
  p.n_cells = hp.n_cells;
  for (int d = 0; d < 3; ++d) {
    p.nn[d] = hp.nn[d];
    p.cells[d] = hp.cells[d];
    p.ratio[d] = d < hp.dim ? (hp.h[0] * hp.h[0]) / (hp.h[d] * hp.h[d]) : 1.0;
    if (d < hp.dim && p.ratio[d] != 1.0) p.aniso = 1;
  }
  p.chunk = ls.chunk;
  p.n_xi = hp.n_xi;
  p.n_terms = hp.n_terms;
  p.nnz = (int)hp.g.col.size();
  {
    const int n = coupling_pairs(hp, p.pair_term, p.pair_val);
    p.premul = n >= 0;
    p.n_pairs = n >= 0 ? n : 0;
  }
  p.stagger = ls.stagger;
  const int nq = hp.k + 1;
  const int nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  double wJ[kMaxQD];
  for (int qd = 0; qd < nqd; ++qd) {
    int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    wJ[qd] = w;
  }
  const int nt = hp.n_t;
  for (int i = 0; i < nt; ++i) {
    const double tb = hp.tau * hp.B_hat[i * nt + i];
    p.tb[i] = tb;
    for (int j = 0; j < nt; ++j) {
      const double a = transpose ? hp.A_hat[j * nt + i] : hp.A_hat[i * nt + j];
      for (int qd = 0; qd < nqd; ++qd) p.amq[(qd * nt + i) * nt + j] = wJ[qd] * (a / tb);
    }
  }
}

cudaError_t launch_apply(const HostProblem& hp, const LaunchShape& ls, const ApplyParams& prm,
                         cudaStream_t stream) {
  // the start of y before the cell kernel adds into it: x on Dirichlet nodes
  // and 0 elsewhere (plain), b minus that (residual), b (accumulation; y may
  // be b) -- one vectorised pass
  const int V = hp.n_xi * hp.n_t;
  const int op = prm.mode == kApplyResidual ? 1 : (prm.mode == kApplyAccumulate ? 3 : 2);
  if (hp.precision == kPrecF32)
    launch_vec_start<float>(static_cast<const float*>(prm.b), static_cast<const float*>(prm.x),
                            static_cast<float*>(prm.y), nullptr, op, V, hp.n_x, hp.nn, hp.dim, stream);
  else
    launch_vec_start<double>(static_cast<const double*>(prm.b), static_cast<const double*>(prm.x),
                             static_cast<double*>(prm.y), nullptr, op, V, hp.n_x, hp.nn, hp.dim, stream);
  void* f = select_kernel(hp.precision, hp.dim, hp.k, hp.n_t);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<ApplyParams*>(&prm)};
  cudaError_t e = cudaLaunchKernel(f, dim3(ls.grid), dim3(ls.threads), args, ls.smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sg

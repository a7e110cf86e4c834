// Flexible GMRES (restarted, right preconditioned) for the SG slab system
// A^(n) U = rhs (paper, Sec. 3.5: the slab systems are solved by flexible
// GMRES with the block-Jacobi multigrid preconditioner).
//
// Arnoldi uses classical Gram-Schmidt with one reorthogonalisation (CGS2) in
// three streaming kernels per step: the dots V^T w; the update w -= V h fused
// with the second pass's dots V^T w (each basis value read once while the
// cycle has at most 12 vectors); the update w -= V h2 fused with ||w||.  Each
// kernel writes one partial sum per block and its last-arriving block reduces
// them in a fixed order (results are deterministic, and no block waits for
// another); the norm kernel's last block also updates the Hessenberg column,
// the Givens rotations and the residual estimate.  A fourth kernel scales w
// into the next basis vector.  The true residual b - A x is recomputed at
// every restart and at the end; its norm is what is reported and tested
// against rtol.
//
// The whole solver state lives on the device and one solve is recorded as a
// CUDA graph: a conditional WHILE node runs one Arnoldi step per pass, and a
// conditional IF node inside it, taken at the end of a restart cycle, applies
// the update x += Z y, recomputes the true residual and starts the next
// cycle.  A solve is then one graph launch and one read of the final state,
// with no host round trip per iteration.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kRedThreads = 256;  // threads of the reduction kernels (8 warps)
constexpr int kKG = 16;           // basis sizes with an element loop of their own; dots a thread accumulates per pass
constexpr int kMaxVec = 256;      // bound on the basis size m + 1 (restart <= 200)

// Device-resident state of the graph driver (followed in memory by
// H[(m+1) x m], cs[m], sn[m], g[m+1], y[m]).  red_count is the arrival
// counter of the last-block reductions; it is 0 between kernels.
struct KState {
  double bnorm, beta, rtol, pad0;
  int max_it, m, j, its, restarts, vmult, prec, cycle_end, done, status, nvec, zero_rhs;
  unsigned red_count, pad1;
};
constexpr int kStateDoubles = (int)((sizeof(KState) + 15) / 16 * 2);

struct Ws {
  double *V, *Z, *w, *r, *part, *h, *h2, *nrm, *y, *vj, *zb, *bb, *xx, *st;
};

// Partial sums: at most kMaxVec rows of kMaxGrid blocks.
constexpr int kMaxGrid = 2048;

Ws carve(double* base, long long N, int m) {
  Ws ws;
  ws.V = base;
  ws.Z = ws.V + (long long)(m + 1) * N;
  ws.w = ws.Z + (long long)m * N;
  ws.r = ws.w + N;
  ws.vj = ws.r + N;
  ws.zb = ws.vj + N;
  ws.bb = ws.zb + N;
  ws.xx = ws.bb + N;
  ws.part = ws.xx + N;
  ws.h = ws.part + (long long)(m + 2) * kMaxGrid;
  ws.h2 = ws.h + (m + 2);
  ws.nrm = ws.h2 + (m + 2);
  ws.y = ws.nrm + 4;
  ws.st = ws.y + (m + 2);
  return ws;
}

__device__ __forceinline__ double* st_H(KState* S) { return reinterpret_cast<double*>(S) + kStateDoubles; }

// Block sums of acc[0..nk) (fixed order: warp shuffles, then the warps in
// order) into dst[c * dst_stride].
template <int NA>
__device__ __forceinline__ void block_sum(const double (&acc)[NA], int nk, double* dst, long long dst_stride) {
  __shared__ double sred[kKG][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    if (c < nk) {
      double v = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sred[c][wid] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) v += sred[threadIdx.x][w];
    dst[threadIdx.x * dst_stride] = v;
  }
  __syncthreads();
}

// This block's sums of acc[0..nk) into part[(k0 + c) * gridDim.x + blockIdx.x].
template <int NA>
__device__ __forceinline__ void block_partials(const double (&acc)[NA], int k0, int nk, double* part) {
  block_sum(acc, nk, part + (long long)k0 * gridDim.x + blockIdx.x, (long long)gridDim.x);
}

// True in the block that arrives last, once every block has written its
// partial sums (threadfence reduction: no block waits for another).
__device__ __forceinline__ bool arrive_last(unsigned* count) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: out[k] = sum over blocks of part[k][.] for k < nk (each
// thread sums a fixed set of blocks for kKG vectors at a time, then the block
// sum; fixed order), then the counter back to 0.
__device__ __forceinline__ void reduce_partials(const double* part, int nk, double* out, unsigned* count) {
  const int G = (int)gridDim.x;
  for (int k0 = 0; k0 < nk; k0 += kKG) {
    const int n = min(kKG, nk - k0);
    double v[kKG] = {};
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
#pragma unroll
      for (int c = 0; c < kKG; ++c)
        if (c < n) v[c] += __ldcg(part + (long long)(k0 + c) * G + b);
    }
    block_sum(v, n, out + k0, 1);
  }
  if (threadIdx.x == 0) *count = 0u;
}

// out[idx] = ||v|| (sub = 0) or, with sub = 1, r = b - r and out[idx] = ||r||.
__global__ void __launch_bounds__(kRedThreads) k_norm(const double* __restrict__ b, double* __restrict__ r, long long N,
                                                      int sub, double* __restrict__ part, double* __restrict__ out,
                                                      int idx, unsigned* count) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double v;
    if (sub) {
      v = b[i] - r[i];
      r[i] = v;
    } else {
      v = b[i];
    }
    acc[0] = fma(v, v, acc[0]);
  }
  block_partials(acc, 0, 1, part);
  if (!arrive_last(count)) return;
  __shared__ double tot;
  reduce_partials(part, 1, &tot, count);
  if (threadIdx.x == 0) out[idx] = sqrt(tot);
}

// Start of a solve: ||b|| in nrm[0], ||b - A x|| in nrm[1].
__global__ void k_gm_start(KState* S, const double* nrm, cudaGraphConditionalHandle wh) {
  S->bnorm = nrm[0];
  S->beta = nrm[1];
  S->j = S->its = S->restarts = S->prec = S->cycle_end = S->status = S->zero_rhs = S->nvec = 0;
  S->vmult = 1;
  int done = 0;
  if (!isfinite(S->bnorm)) { S->status = SG_ERR_NONFINITE; done = 1; }
  else if (S->bnorm == 0.0) { S->zero_rhs = 1; done = 1; }
  else if (!isfinite(S->beta)) { S->status = SG_ERR_NONFINITE; done = 1; }
  else if (S->beta <= S->rtol * S->bnorm) done = 1;
  else if (S->max_it <= 0) { S->status = SG_ERR_NOT_CONVERGED; done = 1; }
  S->done = done;
  cudaGraphSetConditional(wh, done ? 0u : 1u);
}

// Start of a restart cycle: V_0 = vj = r / beta, g = beta e_0 (nothing once
// the solve is done).
__global__ void k_gm_vstart(KState* S, const double* __restrict__ r, double* __restrict__ V, double* __restrict__ vj,
                            long long N) {
  if (S->done) return;
  const double inv = 1.0 / S->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double v = r[i] * inv;
    V[i] = v;
    vj[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int m = S->m;
    double* g = st_H(S) + (m + 1) * m + 2 * m;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = S->beta;
  }
}

// Element loops of the Gram-Schmidt kernels for a basis of NV vectors known
// at compile time: every basis value of an element is loaded before the
// arithmetic that uses it (issue is in order: a load followed by its use
// would hold the next load back).
template <int NV>
__device__ __forceinline__ void loop_dot(const double* __restrict__ w, const double* __restrict__ V,
                                         const double* __restrict__ zb, double* __restrict__ Zj, long long N,
                                         double (&acc)[kKG]) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = V[(long long)c * N + i];
    const double wi = w[i];
    Zj[i] = zb[i];
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = fma(v[c], wi, acc[c]);
  }
}
template <int NV>
__device__ __forceinline__ void loop_axpy_dot(double* __restrict__ w, const double* __restrict__ V,
                                              const double* sh, long long N, double (&acc)[kKG]) {
  double hc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) hc[c] = sh[c];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = V[(long long)c * N + i];
    double s = w[i];
#pragma unroll
    for (int c = 0; c < NV; ++c) s = fma(-hc[c], v[c], s);
    w[i] = s;
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = fma(v[c], s, acc[c]);
  }
}
template <int NV>
__device__ __forceinline__ void loop_axpy_norm(double* __restrict__ w, const double* __restrict__ V, const double* sh,
                                               long long N, double& acc) {
  double hc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) hc[c] = sh[c];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = V[(long long)c * N + i];
    double s = w[i];
#pragma unroll
    for (int c = 0; c < NV; ++c) s = fma(-hc[c], v[c], s);
    w[i] = s;
    acc = fma(s, s, acc);
  }
}
// Runs CALL(NV) for NV = nvec when nvec <= kKG; false otherwise.
#define SG_NV_DISPATCH(nvec, CALL)                                                                        \
  [&]() -> bool {                                                                                         \
    switch (nvec) {                                                                                       \
      case 1: CALL(1); return true;   case 2: CALL(2); return true;   case 3: CALL(3); return true;       \
      case 4: CALL(4); return true;   case 5: CALL(5); return true;   case 6: CALL(6); return true;       \
      case 7: CALL(7); return true;   case 8: CALL(8); return true;   case 9: CALL(9); return true;       \
      case 10: CALL(10); return true; case 11: CALL(11); return true; case 12: CALL(12); return true;     \
      case 13: CALL(13); return true; case 14: CALL(14); return true; case 15: CALL(15); return true;     \
      case 16: CALL(16); return true;                                                                     \
      default: return false;                                                                              \
    }                                                                                                     \
  }()

// Dots of w with basis vectors g0 .. g0 + nk - 1 (nk <= kKG); the loads of
// the slots past nk repeat the last vector's address, their products are dropped.
__device__ __forceinline__ void dots_group(const double* __restrict__ w, const double* __restrict__ V, int g0, int nk,
                                           long long N, double (&acc)[kKG]) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double v[kKG];
#pragma unroll
    for (int c = 0; c < kKG; ++c) v[c] = V[(long long)(g0 + min(c, nk - 1)) * N + i];
    const double wi = w[i];
#pragma unroll
    for (int c = 0; c < kKG; ++c)
      if (c < nk) acc[c] = fma(v[c], wi, acc[c]);
  }
}

// First Gram-Schmidt pass, dots: h[k] = V_k . w for k <= j; also stores the
// preconditioned vector of this step, Z_j = zb.
__global__ void __launch_bounds__(kRedThreads, 2) k_cgs_dot(KState* S, const double* __restrict__ w,
                                                         const double* __restrict__ V, const double* __restrict__ zb,
                                                         double* __restrict__ Z, long long N, double* __restrict__ part,
                                                         double* __restrict__ h) {
  const int nvec = S->j + 1;
  double* Zj = Z + (long long)S->j * N;
  double acc[kKG] = {};
#define SG_CALL(NV) loop_dot<NV>(w, V, zb, Zj, N, acc)
  if (SG_NV_DISPATCH(nvec, SG_CALL)) {
    block_partials(acc, 0, nvec, part);
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
      Zj[i] = zb[i];
    for (int g0 = 0; g0 < nvec; g0 += kKG) {
      const int nk = min(kKG, nvec - g0);
      double ag[kKG] = {};
      dots_group(w, V, g0, nk, N, ag);
      block_partials(ag, g0, nk, part);
    }
  }
#undef SG_CALL
  if (!arrive_last(&S->red_count)) return;
  reduce_partials(part, nvec, h, &S->red_count);
}

// Second pass: w -= sum_k h[k] V_k, then h2[k] = V_k . w.  With at most kKG
// vectors each V value is read once and used for both; beyond that the dots
// read V again.
__global__ void __launch_bounds__(kRedThreads, 2) k_cgs_axpy_dot(KState* S, double* __restrict__ w,
                                                              const double* __restrict__ V,
                                                              const double* __restrict__ h, long long N,
                                                              double* __restrict__ part, double* __restrict__ h2) {
  const int nvec = S->j + 1;
  __shared__ double sh[kMaxVec];
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) sh[k] = h[k];
  __syncthreads();
  double acc[kKG] = {};
#define SG_CALL(NV) loop_axpy_dot<NV>(w, V, sh, N, acc)
  if (SG_NV_DISPATCH(nvec, SG_CALL)) {
    block_partials(acc, 0, nvec, part);
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
      double s = w[i];
#pragma unroll 4
      for (int k = 0; k < nvec; ++k) s = fma(-sh[k], V[(long long)k * N + i], s);
      w[i] = s;
    }
    for (int g0 = 0; g0 < nvec; g0 += kKG) {
      const int nk = min(kKG, nvec - g0);
      double ag[kKG] = {};
      dots_group(w, V, g0, nk, N, ag);
      block_partials(ag, g0, nk, part);
    }
  }
#undef SG_CALL
  if (!arrive_last(&S->red_count)) return;
  reduce_partials(part, nvec, h2, &S->red_count);
}

// The Hessenberg column of step j, the previous rotations and a new one, the
// residual estimate |g_{j+1}|; at the end of a cycle y = H^{-1} g.  One thread.
__device__ void arnoldi_update(KState* S, const double* __restrict__ h, const double* __restrict__ h2, double hn,
                               double* __restrict__ y, cudaGraphConditionalHandle ih) {
  const int m = S->m, j = S->j;
  double* H = st_H(S);
  double* cs = H + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  for (int i = 0; i <= j; ++i) H[i * m + j] = h[i] + h2[i];
  H[(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], c = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * a + sn[i] * c;
    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
  }
  const double a = H[j * m + j], c = H[(j + 1) * m + j];
  const double den = hypot(a, c);
  cs[j] = den > 0 ? a / den : 1.0;
  sn[j] = den > 0 ? c / den : 0.0;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  S->its += 1;
  S->prec += 1;
  S->vmult += 1;
  S->j = j + 1;
  const double est = fabs(g[j + 1]);
  const int end = !isfinite(est) || est <= S->rtol * S->bnorm || S->its >= S->max_it || hn == 0.0 || j + 1 == m;
  if (end) {
    const int n = j + 1;
    for (int i = n - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < n; ++k) acc -= H[i * m + k] * y[k];
      y[i] = H[i * m + i] != 0.0 ? acc / H[i * m + i] : 0.0;
    }
    S->nvec = n;
  }
  S->cycle_end = end;
  cudaGraphSetConditional(ih, end ? 1u : 0u);
}

// Closing pass of the step: w -= sum_k h2[k] V_k, nrm[0] = ||w||, and in the
// last block the Arnoldi update of step j.
__global__ void __launch_bounds__(kRedThreads, 3) k_cgs_axpy_norm(KState* S, double* __restrict__ w,
                                                               const double* __restrict__ V,
                                                               const double* __restrict__ h,
                                                               const double* __restrict__ h2, long long N,
                                                               double* __restrict__ part, double* __restrict__ nrm,
                                                               double* __restrict__ y, cudaGraphConditionalHandle ih) {
  const int nvec = S->j + 1;
  __shared__ double sh[kMaxVec];
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) sh[k] = h2[k];
  __syncthreads();
  double acc[1] = {0.0};
#define SG_CALL(NV) loop_axpy_norm<NV>(w, V, sh, N, acc[0])
  if (!SG_NV_DISPATCH(nvec, SG_CALL)) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
      double s = w[i];
#pragma unroll 4
      for (int k = 0; k < nvec; ++k) s = fma(-sh[k], V[(long long)k * N + i], s);
      w[i] = s;
      acc[0] = fma(s, s, acc[0]);
    }
  }
#undef SG_CALL
  block_partials(acc, 0, 1, part);
  if (!arrive_last(&S->red_count)) return;
  __shared__ double tot;
  reduce_partials(part, 1, &tot, &S->red_count);
  if (threadIdx.x == 0) {
    const double hn = sqrt(tot);
    nrm[0] = hn;
    arnoldi_update(S, h, h2, hn, y, ih);
  }
}

// V_{j+1} = vj = w / ||w|| (S->j has already advanced to j + 1).
__global__ void k_gm_vnext(const KState* S, const double* __restrict__ w, double* __restrict__ V,
                           double* __restrict__ vj, const double* __restrict__ nrm, long long N) {
  const double inv = 1.0 / nrm[0];
  double* v = V + (long long)S->j * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double t = w[i] * inv;
    v[i] = t;
    vj[i] = t;
  }
}

// x += sum_k y[k] Z_k over the cycle's vectors
__global__ void k_lincomb_st(const KState* S, double* __restrict__ x, const double* __restrict__ Z,
                             const double* __restrict__ y, long long N) {
  const int nvec = S->nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int k = 0; k < nvec; ++k) s = fma(y[k], Z[(long long)k * N + i], s);
    x[i] = s;
  }
}

// End of a cycle: the true residual norm (nrm[1]) decides convergence.
__global__ void k_gm_finish(KState* S, const double* nrm, cudaGraphConditionalHandle wh) {
  S->restarts += 1;
  S->vmult += 1;
  S->beta = nrm[1];
  int done = 0;
  if (!isfinite(S->beta)) { S->status = SG_ERR_NONFINITE; done = 1; }
  else if (S->beta <= S->rtol * S->bnorm) done = 1;
  else if (S->its >= S->max_it) { S->status = SG_ERR_NOT_CONVERGED; done = 1; }
  S->j = 0;
  S->cycle_end = 0;
  S->done = done;
  cudaGraphSetConditional(wh, done ? 0u : 1u);
}

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sg::sm_count() * 16)); }

// Grid of a reduction kernel: every block resident at once (the partial sums
// have one column per block), at most kMaxGrid blocks.
template <typename K>
int grid_red(K kern, long long n) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRedThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long g = std::min<long long>((long long)per_sm * sg::sm_count(), kMaxGrid);
  return (int)std::max<long long>(1, std::min<long long>((n + kRedThreads - 1) / kRedThreads, g));
}

// Appends a conditional node after the current capture dependencies of `cs`,
// makes it the new dependency and returns its body graph.
cudaError_t add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            cudaGraph_t* body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, &edata, &nd);
  if (e != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, edata, nd, &np);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaSuccess;
}

}  // namespace

size_t krylov_bytes(long long N, int m) {
  const size_t arrays = (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m;
  return sizeof(double) * ((size_t)(2 * m + 7) * N + (size_t)(m + 2) * kMaxGrid + 3 * (m + 2) + 4 + kStateDoubles +
                           arrays + 8);
}

void krylov_graph_free(KrylovGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  for (cudaStream_t* st : {&G.cs, &G.bs, &G.is})
    if (*st) cudaStreamDestroy(*st);
  if (G.host) cudaFreeHost(G.host);
  G = KrylovGraph();
}

sg_status fgmres_graph(long long N, const double* b, double* x, double rtol, int max_it, int m, sg_solve_stats* st,
                       cudaStream_t s, std::string& msg, const IssueFn& apply, const IssueFn& prec, double* workspace,
                       KrylovGraph& G, unsigned long long key) {
  const auto t0 = std::chrono::steady_clock::now();
  Ws ws = carve(workspace, N, m);
  KState* S = reinterpret_cast<KState*>(ws.st);
  cudaError_t e = cudaSuccess;
#define CKG(call)                                                                                  \
  do {                                                                                             \
    if ((e = (call)) != cudaSuccess) {                                                             \
      msg = std::string("FGMRES graph line ") + std::to_string(__LINE__) + ": " + cudaGetErrorString(e); \
      return SG_ERR_CUDA;                                                                          \
    }                                                                                              \
  } while (0)
  // the graph works on copies of b and x in the workspace, so that one
  // recording serves every right-hand side and solution vector
  const bool fresh = !G.exec || G.key != key || G.N != N || G.m != m || G.ws != workspace;
  const double* const b_user = b;
  double* const x_user = x;
  b = ws.bb;
  x = ws.xx;
  if (fresh) {
    krylov_graph_free(G);
    CKG(cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking));
    CKG(cudaStreamCreateWithFlags(&G.bs, cudaStreamNonBlocking));
    CKG(cudaStreamCreateWithFlags(&G.is, cudaStreamNonBlocking));
    CKG(cudaHostAlloc(reinterpret_cast<void**>(&G.host), sizeof(KState), cudaHostAllocPortable));
    CKG(cudaGraphCreate(&G.graph, 0));
    cudaGraphConditionalHandle wh, ih;
    CKG(cudaGraphConditionalHandleCreate(&wh, G.graph, 0, 0));
    const int gn = grid_n(N);
    const int g_norm = grid_red(k_norm, N), g_dot = grid_red(k_cgs_dot, N);
    const int g_ad = grid_red(k_cgs_axpy_dot, N), g_an = grid_red(k_cgs_axpy_norm, N);
    unsigned* count = &S->red_count;
    // the start: ||b||, r = b - A x, ||r||, and V_0 = r / ||r||
    CKG(cudaStreamBeginCaptureToGraph(G.cs, G.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    k_norm<<<g_norm, kRedThreads, 0, G.cs>>>(b, nullptr, N, 0, ws.part, ws.nrm, 0, count);
    cudaError_t ee = cudaGetLastError();
    if (ee == cudaSuccess) ee = apply(x, ws.r, G.cs);
    if (ee == cudaSuccess) {
      k_norm<<<g_norm, kRedThreads, 0, G.cs>>>(b, ws.r, N, 1, ws.part, ws.nrm, 1, count);
      k_gm_start<<<1, 1, 0, G.cs>>>(S, ws.nrm, wh);
      k_gm_vstart<<<gn, 256, 0, G.cs>>>(S, ws.r, ws.V, ws.vj, N);
      ee = cudaGetLastError();
    }
    cudaGraph_t wbody = nullptr;
    if (ee == cudaSuccess) ee = add_conditional(G.cs, wh, cudaGraphCondTypeWhile, &wbody);
    // the WHILE body: one Arnoldi step (z_j = M^-1 v_j, w = A z_j, CGS2, v_{j+1})
    if (ee == cudaSuccess) ee = cudaGraphConditionalHandleCreate(&ih, wbody, 0, 0);
    if (ee == cudaSuccess)
      ee = cudaStreamBeginCaptureToGraph(G.bs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    bool body_open = ee == cudaSuccess;
    if (ee == cudaSuccess) ee = prec(ws.vj, ws.zb, G.bs);
    if (ee == cudaSuccess) ee = apply(ws.zb, ws.w, G.bs);
    if (ee == cudaSuccess) {
      k_cgs_dot<<<g_dot, kRedThreads, 0, G.bs>>>(S, ws.w, ws.V, ws.zb, ws.Z, N, ws.part, ws.h);
      k_cgs_axpy_dot<<<g_ad, kRedThreads, 0, G.bs>>>(S, ws.w, ws.V, ws.h, N, ws.part, ws.h2);
      k_cgs_axpy_norm<<<g_an, kRedThreads, 0, G.bs>>>(S, ws.w, ws.V, ws.h, ws.h2, N, ws.part, ws.nrm, ws.y, ih);
      k_gm_vnext<<<gn, 256, 0, G.bs>>>(S, ws.w, ws.V, ws.vj, ws.nrm, N);
      ee = cudaGetLastError();
    }
    // the IF body: the update, the true residual at the end of a cycle and
    // the next cycle's V_0
    cudaGraph_t ibody = nullptr;
    if (ee == cudaSuccess) ee = add_conditional(G.bs, ih, cudaGraphCondTypeIf, &ibody);
    if (ee == cudaSuccess)
      ee = cudaStreamBeginCaptureToGraph(G.is, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    bool if_open = ee == cudaSuccess;
    if (ee == cudaSuccess) {
      k_lincomb_st<<<gn, 256, 0, G.is>>>(S, x, ws.Z, ws.y, N);
      ee = cudaGetLastError();
    }
    if (ee == cudaSuccess) ee = apply(x, ws.r, G.is);
    if (ee == cudaSuccess) {
      k_norm<<<g_norm, kRedThreads, 0, G.is>>>(b, ws.r, N, 1, ws.part, ws.nrm, 1, count);
      k_gm_finish<<<1, 1, 0, G.is>>>(S, ws.nrm, wh);
      k_gm_vstart<<<gn, 256, 0, G.is>>>(S, ws.r, ws.V, ws.vj, N);
      ee = cudaGetLastError();
    }
    cudaGraph_t tmp = nullptr;
    if (if_open) {
      const cudaError_t e2 = cudaStreamEndCapture(G.is, &tmp);
      if (ee == cudaSuccess) ee = e2;
    }
    if (body_open) {
      const cudaError_t e2 = cudaStreamEndCapture(G.bs, &tmp);
      if (ee == cudaSuccess) ee = e2;
    }
    const cudaError_t e3 = cudaStreamEndCapture(G.cs, &tmp);
    if (ee == cudaSuccess) ee = e3;
    if (ee == cudaSuccess) ee = cudaGraphInstantiate(&G.exec, G.graph, 0);
    if (ee != cudaSuccess) {
      krylov_graph_free(G);
      msg = std::string("FGMRES graph capture: ") + cudaGetErrorString(ee);
      return SG_ERR_CUDA;
    }
    G.key = key;
    G.N = N;
    G.m = m;
    G.ws = workspace;
  }
  // the solve's parameters, the graph, the final state
  KState* hs = reinterpret_cast<KState*>(G.host);
  std::memset(hs, 0, sizeof(KState));
  hs->rtol = rtol;
  hs->max_it = max_it;
  hs->m = m;
  CKG(cudaMemcpyAsync(S, hs, sizeof(KState), cudaMemcpyHostToDevice, s));
  CKG(cudaMemcpyAsync(ws.bb, b_user, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CKG(cudaMemcpyAsync(ws.xx, x_user, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CKG(cudaGraphLaunch(G.exec, s));
  CKG(cudaMemcpyAsync(x_user, ws.xx, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CKG(cudaMemcpyAsync(hs, S, sizeof(KState), cudaMemcpyDeviceToHost, s));
  CKG(cudaStreamSynchronize(s));
  sg_solve_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  sg_status status = (sg_status)hs->status;
  if (hs->zero_rhs) {
    CKG(cudaMemsetAsync(x_user, 0, N * sizeof(double), s));
    CKG(cudaStreamSynchronize(s));
    status = SG_OK;
  }
  stats.iterations = hs->its;
  stats.restarts = hs->restarts;
  stats.vmult_calls = hs->vmult;
  stats.prec_calls = hs->prec;
  stats.converged = status == SG_OK ? 1 : 0;
  stats.rel_residual = hs->zero_rhs ? 0.0 : hs->beta / hs->bnorm;
  stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = stats;
  if (status == SG_ERR_NONFINITE) msg = "non-finite residual";
  else if (status == SG_ERR_NOT_CONVERGED) msg = "FGMRES reached max_it";
#undef CKG
  return status;
}

sg_status fgmres(sg_ctx* ctx, const double* b, double* x, double rtol, int max_it, int m, sg_solve_stats* st,
                 cudaStream_t s, std::string& msg,
                 cudaError_t (*apply)(sg_ctx*, const double*, double*, cudaStream_t), int trans) {
  const long long N = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  const size_t need = krylov_bytes(N, m);
  if (!ctx->d_krylov || ctx->krylov_bytes < need) {
    cudaFree(ctx->d_krylov);
    ctx->d_krylov = nullptr;
    cudaError_t e = cudaMalloc(&ctx->d_krylov, need);
    if (e != cudaSuccess) { msg = "FGMRES workspace allocation failed"; ctx->krylov_bytes = 0; return SG_ERR_OOM; }
    ctx->krylov_bytes = need;
  }
  MG* mg = ctx->mg;
  sg_status r = fgmres_graph(
      N, b, x, rtol, max_it, m, st, s, msg,
      [&](const double* in, double* out, cudaStream_t cs) { return apply(ctx, in, out, cs); },
      [&](const double* in, double* out, cudaStream_t cs) { return mg_issue(*mg, in, out, cs, trans); },
      ctx->d_krylov, ctx->kgraph[trans ? 1 : 0], ctx->gen);
  if (st) st->mg_setup_ms = mg ? mg->setup_ms : 0.0;
  return r;
}

}  // namespace sg

// Flexible GMRES (restarted, right preconditioned) for the SG slab system
// A^(n) U = rhs (paper, Sec. 3.5: the slab systems are solved by flexible
// GMRES with the block-Jacobi multigrid preconditioner).
//
// Arnoldi uses classical Gram-Schmidt with one reorthogonalisation (CGS2):
// each pass is one multi-dot kernel (every basis vector against w, per-segment
// partial sums reduced in a fixed order, so results are deterministic) and one
// multi-axpy kernel.  The true residual b - A x is recomputed at every restart
// and at the end; its norm is what is reported and tested against rtol.
//
// The whole solver state lives on the device and one solve is recorded as a
// CUDA graph: a conditional WHILE node runs one Arnoldi step per pass (its
// last kernel updates the Hessenberg column, the Givens rotations and the
// residual estimate on one thread), and a conditional IF node inside it,
// taken at the end of a restart cycle, applies the update x += Z y and
// recomputes the true residual.  A solve is then one graph launch and one
// read of the final state, with no host round trip per iteration.
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

constexpr int kSeg = 256;      // segments of the multi-dot reduction
constexpr int kDotThreads = 256;

__global__ void k_multidot(const double* __restrict__ w, const double* __restrict__ V, int nvec, long long N,
                           double* __restrict__ part) {
  // blockIdx.y = vector, blockIdx.x = segment
  __shared__ double red[kDotThreads];
  const int k = blockIdx.y;
  const double* v = V + (long long)k * N;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    s = fma(v[i], w[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_reduce_parts(const double* __restrict__ part, int nseg, int nvec, double* __restrict__ out) {
  const int k = blockIdx.x;
  __shared__ double red[kDotThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nseg; i += blockDim.x) s += part[(long long)k * nseg + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}




__global__ void k_sub_from(const double* __restrict__ b, double* __restrict__ r, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sg::sm_count() * 16)); }

// Device-resident state of the graph driver (followed in memory by
// H[(m+1) x m], cs[m], sn[m], g[m+1], y[m]).
struct KState {
  double bnorm, beta, rtol, pad0;
  int max_it, m, j, its, restarts, vmult, prec, cycle_end, done, status, nvec, zero_rhs;
};
constexpr int kStateDoubles = (int)((sizeof(KState) + 15) / 16 * 2);

struct Ws {
  double *V, *Z, *w, *r, *part, *h, *h2, *nrm, *y, *vj, *zb, *bb, *xx, *st;
};

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
  ws.h = ws.part + (long long)(m + 2) * kSeg;
  ws.h2 = ws.h + (m + 2);
  ws.nrm = ws.h2 + (m + 2);
  ws.y = ws.nrm + 4;
  ws.st = ws.y + (m + 2);
  return ws;
}

}  // namespace

size_t krylov_bytes(long long N, int m) {
  const size_t arrays = (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m;
  return sizeof(double) * ((size_t)(2 * m + 7) * N + (size_t)(m + 2) * kSeg + 3 * (m + 2) + 4 + kStateDoubles +
                           arrays + 8);
}

// ------------------------------------------------------------ graph driver
namespace {

__device__ __forceinline__ double* st_H(KState* S) { return reinterpret_cast<double*>(S) + kStateDoubles; }

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

// Start of a restart cycle (j == 0): V_0 = r / beta, g = beta e_0.
__global__ void k_gm_vstart(KState* S, const double* __restrict__ r, double* __restrict__ V, long long N) {
  if (S->j != 0) return;
  const double inv = 1.0 / S->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    V[i] = r[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int m = S->m;
    double* g = st_H(S) + (m + 1) * m + 2 * m;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = S->beta;
  }
}

// dst = src + (j + off) * N (from = 1) or dst + (j + off) * N = src (from = 0).
__global__ void k_gm_copy(const KState* S, const double* __restrict__ src, double* __restrict__ dst, long long N,
                          int from) {
  const long long o = (long long)S->j * N;
  const double* a = from ? src + o : src;
  double* b = from ? dst : dst + o;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// multi-dot / reduce / multi-axpy over the basis vectors V_0..V_j
__global__ void k_multidot_st(const KState* S, const double* __restrict__ w, const double* __restrict__ V, long long N,
                              double* __restrict__ part) {
  __shared__ double red[kDotThreads];
  const int k = blockIdx.y;
  if (k > S->j) return;
  const double* v = V + (long long)k * N;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    s = fma(v[i], w[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_reduce_parts_st(const KState* S, const double* __restrict__ part, int nseg, double* __restrict__ out) {
  const int k = blockIdx.x;
  if (k > S->j) return;
  __shared__ double red[kDotThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nseg; i += blockDim.x) s += part[(long long)k * nseg + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}

__global__ void k_multiaxpy_st(const KState* S, double* __restrict__ w, const double* __restrict__ V,
                               const double* __restrict__ h, long long N) {
  const int nvec = S->j + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nvec; ++k) s = fma(-h[k], V[(long long)k * N + i], s);
    w[i] = s;
  }
}

// V_{j+1} = w / ||w||
__global__ void k_gm_vnext(const KState* S, const double* __restrict__ w, double* __restrict__ V,
                           const double* __restrict__ nrm, long long N) {
  const double inv = 1.0 / nrm[0];
  double* v = V + (long long)(S->j + 1) * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

// The Hessenberg column of step j, the previous rotations and a new one, the
// residual estimate |g_{j+1}|; at the end of a cycle y = H^{-1} g.
__global__ void k_gm_arnoldi(KState* S, const double* __restrict__ h, const double* __restrict__ h2,
                             const double* __restrict__ nrm, double* __restrict__ y, cudaGraphConditionalHandle ih) {
  const int m = S->m, j = S->j;
  double* H = st_H(S);
  double* cs = H + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  for (int i = 0; i <= j; ++i) H[i * m + j] = h[i] + h2[i];
  const double hn = nrm[0];
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

__global__ void k_sqrt_at(double* v, int i) { v[i] = sqrt(v[i]); }

// ||v|| into out[i] (two-stage deterministic reduction, then sqrt)
cudaError_t norm2_at(const double* v, long long N, double* part, double* out, int i, cudaStream_t s) {
  dim3 grid(kSeg, 1);
  k_multidot<<<grid, kDotThreads, 0, s>>>(v, v, 1, N, part);
  k_reduce_parts<<<1, kDotThreads, 0, s>>>(part, kSeg, 1, out + i);
  k_sqrt_at<<<1, 1, 0, s>>>(out, i);
  return cudaGetLastError();
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
    // the start: ||b||, r = b - A x, ||r||
    CKG(cudaStreamBeginCaptureToGraph(G.cs, G.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t ee = norm2_at(b, N, ws.part, ws.nrm, 0, G.cs);
    if (ee == cudaSuccess) ee = apply(x, ws.r, G.cs);
    if (ee == cudaSuccess) {
      k_sub_from<<<gn, 256, 0, G.cs>>>(b, ws.r, N);
      ee = norm2_at(ws.r, N, ws.part, ws.nrm, 1, G.cs);
    }
    if (ee == cudaSuccess) {
      k_gm_start<<<1, 1, 0, G.cs>>>(S, ws.nrm, wh);
      ee = cudaGetLastError();
    }
    cudaGraph_t wbody = nullptr;
    if (ee == cudaSuccess) ee = add_conditional(G.cs, wh, cudaGraphCondTypeWhile, &wbody);
    // the WHILE body: one Arnoldi step
    if (ee == cudaSuccess) ee = cudaGraphConditionalHandleCreate(&ih, wbody, 0, 0);
    if (ee == cudaSuccess)
      ee = cudaStreamBeginCaptureToGraph(G.bs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    bool body_open = ee == cudaSuccess;
    if (ee == cudaSuccess) {
      k_gm_vstart<<<gn, 256, 0, G.bs>>>(S, ws.r, ws.V, N);
      k_gm_copy<<<gn, 256, 0, G.bs>>>(S, ws.V, ws.vj, N, 1);
      ee = cudaGetLastError();
    }
    if (ee == cudaSuccess) ee = prec(ws.vj, ws.zb, G.bs);
    if (ee == cudaSuccess) {
      k_gm_copy<<<gn, 256, 0, G.bs>>>(S, ws.zb, ws.Z, N, 0);
      ee = cudaGetLastError();
    }
    if (ee == cudaSuccess) ee = apply(ws.zb, ws.w, G.bs);
    if (ee == cudaSuccess) {
      dim3 grid(kSeg, m + 1);
      for (double* hh : {ws.h, ws.h2}) {
        k_multidot_st<<<grid, kDotThreads, 0, G.bs>>>(S, ws.w, ws.V, N, ws.part);
        k_reduce_parts_st<<<m + 1, kDotThreads, 0, G.bs>>>(S, ws.part, kSeg, hh);
        k_multiaxpy_st<<<gn, 256, 0, G.bs>>>(S, ws.w, ws.V, hh, N);
      }
      ee = norm2_at(ws.w, N, ws.part, ws.nrm, 0, G.bs);
    }
    if (ee == cudaSuccess) {
      k_gm_vnext<<<gn, 256, 0, G.bs>>>(S, ws.w, ws.V, ws.nrm, N);
      k_gm_arnoldi<<<1, 1, 0, G.bs>>>(S, ws.h, ws.h2, ws.nrm, ws.y, ih);
      ee = cudaGetLastError();
    }
    // the IF body: the update and the true residual at the end of a cycle
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
      k_sub_from<<<gn, 256, 0, G.is>>>(b, ws.r, N);
      ee = norm2_at(ws.r, N, ws.part, ws.nrm, 1, G.is);
    }
    if (ee == cudaSuccess) {
      k_gm_finish<<<1, 1, 0, G.is>>>(S, ws.nrm, wh);
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

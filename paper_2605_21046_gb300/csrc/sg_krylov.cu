// Flexible GMRES (restarted, right preconditioned) for the SG slab system
// A^(n) U = rhs (paper, Sec. 3.5: the slab systems are solved by flexible
// GMRES with the block-Jacobi multigrid preconditioner).
//
// Arnoldi uses classical Gram-Schmidt with one reorthogonalisation (CGS2):
// each pass is one multi-dot kernel (every basis vector against w, per-segment
// partial sums reduced in a fixed order, so results are deterministic) and one
// multi-axpy kernel.  The (m+1) x m Hessenberg column and the Givens rotations
// live on the host; one small device-to-host copy per iteration.  The true
// residual b - A x is recomputed at every restart and at the end; its norm is
// what is reported and tested against rtol.
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

// w -= sum_k h[k] V_k
__global__ void k_multiaxpy(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ h,
                            int nvec, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nvec; ++k) s = fma(-h[k], V[(long long)k * N + i], s);
    w[i] = s;
  }
}

// x += sum_k y[k] Z_k
__global__ void k_lincomb(double* __restrict__ x, const double* __restrict__ Z, const double* __restrict__ y,
                          int nvec, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int k = 0; k < nvec; ++k) s = fma(y[k], Z[(long long)k * N + i], s);
    x[i] = s;
  }
}

// v = w / norm (norm on the device)
__global__ void k_scale_by(const double* __restrict__ w, double* __restrict__ v, const double* __restrict__ nrm,
                           long long N) {
  const double inv = 1.0 / nrm[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

__global__ void k_sub_from(const double* __restrict__ b, double* __restrict__ r, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

__global__ void k_sqrt_inplace(double* v) { v[0] = sqrt(v[0]); }

int grid_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sg::sm_count() * 16)); }

struct Ws {
  double *V, *Z, *w, *r, *part, *h, *h2, *nrm, *y;
};

Ws carve(double* base, long long N, int m) {
  Ws ws;
  ws.V = base;
  ws.Z = ws.V + (long long)(m + 1) * N;
  ws.w = ws.Z + (long long)m * N;
  ws.r = ws.w + N;
  ws.part = ws.r + N;
  ws.h = ws.part + (long long)(m + 2) * kSeg;
  ws.h2 = ws.h + (m + 2);
  ws.nrm = ws.h2 + (m + 2);
  ws.y = ws.nrm + 2;
  return ws;
}

}  // namespace

size_t krylov_bytes(long long N, int m) {
  return sizeof(double) * ((size_t)(2 * m + 3) * N + (size_t)(m + 2) * kSeg + 3 * (m + 2) + 2 + 8);
}

// dots of w against V_0..V_{nvec-1} into out[0..nvec) (device)
static cudaError_t multidot(const double* w, const double* V, int nvec, long long N, double* part, double* out,
                            cudaStream_t s) {
  dim3 grid(kSeg, nvec);
  k_multidot<<<grid, kDotThreads, 0, s>>>(w, V, nvec, N, part);
  k_reduce_parts<<<nvec, kDotThreads, 0, s>>>(part, kSeg, nvec, out);
  return cudaGetLastError();
}

// Page-locked host staging for the scalars each Arnoldi step reads back (one
// copy per step instead of several pageable ones), one buffer per host thread.
struct PinnedStage {
  double* p = nullptr;
  size_t n = 0;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
  double* get(size_t need) {
    if (n >= need) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&p), need * sizeof(double), cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nullptr;
    }
    n = need;
    return p;
  }
};
thread_local PinnedStage t_stage;

static cudaError_t norm2(const double* w, long long N, double* part, double* out, cudaStream_t s) {
  cudaError_t e = multidot(w, w, 1, N, part, out, s);
  if (e != cudaSuccess) return e;
  k_sqrt_inplace<<<1, 1, 0, s>>>(out);
  return cudaGetLastError();
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
  sg_status r = fgmres_core(
      N, b, x, rtol, max_it, m, st, s, msg, [&](const double* in, double* out) { return apply(ctx, in, out, s); },
      [&](const double* in, double* out) { return mg_apply(*mg, in, out, s, trans); }, ctx->d_krylov);
  if (st) st->mg_setup_ms = mg ? mg->setup_ms : 0.0;
  return r;
}

sg_status fgmres_core(long long N, const double* b, double* x, double rtol, int max_it, int m, sg_solve_stats* st,
                      cudaStream_t s, std::string& msg, const std::function<cudaError_t(const double*, double*)>& apply,
                      const std::function<cudaError_t(const double*, double*)>& prec, double* workspace) {
  const auto t0 = std::chrono::steady_clock::now();
  Ws ws = carve(workspace, N, m);
  sg_solve_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  cudaError_t e;
#define CK(call)                                                   \
  do {                                                             \
    if ((e = (call)) != cudaSuccess) {                             \
      msg = std::string("FGMRES line ") + std::to_string(__LINE__) + ": " + cudaGetErrorString(e); \
      return SG_ERR_CUDA;                                          \
    }                                                              \
  } while (0)
  // h, h2 and nrm are adjacent in the workspace: one read-back per Arnoldi step
  const size_t n_stage = 2 * (size_t)(m + 2) + 2;
  std::vector<double> stage_fallback;
  double* stage = t_stage.get(n_stage);
  if (!stage) {
    stage_fallback.assign(n_stage, 0.0);
    stage = stage_fallback.data();
  }
  double* host2 = stage + 2 * (m + 2);     // mirrors ws.nrm
  CK(norm2(b, N, ws.part, ws.nrm, s));
  CK(cudaMemcpyAsync(host2, ws.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double bnorm = host2[0];
  if (!std::isfinite(bnorm)) { msg = "non-finite right-hand side"; return SG_ERR_NONFINITE; }
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    stats.converged = 1;
    if (st) *st = stats;
    return SG_OK;
  }
  // r = b - A x
  auto true_residual = [&](double& beta) -> cudaError_t {
    cudaError_t ee = apply(x, ws.r);
    if (ee != cudaSuccess) return ee;
    ++stats.vmult_calls;
    k_sub_from<<<grid_n(N), 256, 0, s>>>(b, ws.r, N);
    if ((ee = norm2(ws.r, N, ws.part, ws.nrm, s)) != cudaSuccess) return ee;
    if ((ee = cudaMemcpyAsync(host2, ws.nrm, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return ee;
    if ((ee = cudaStreamSynchronize(s)) != cudaSuccess) return ee;
    beta = host2[0];
    return cudaSuccess;
  };
  double beta = 0.0;
  CK(true_residual(beta));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
  const double* hcol = stage;              // mirrors ws.h
  const double* hcol2 = stage + (m + 2);   // mirrors ws.h2
  sg_status status = SG_OK;
  while (true) {
    if (!std::isfinite(beta)) { status = SG_ERR_NONFINITE; msg = "non-finite residual"; break; }
    if (beta <= rtol * bnorm) { stats.converged = 1; break; }
    if (stats.iterations >= max_it) { status = SG_ERR_NOT_CONVERGED; msg = "FGMRES reached max_it"; break; }
    // V_0 = r / beta
    host2[0] = beta;
    CK(cudaMemcpyAsync(ws.nrm, host2, sizeof(double), cudaMemcpyHostToDevice, s));
    k_scale_by<<<grid_n(N), 256, 0, s>>>(ws.r, ws.V, ws.nrm, N);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_done = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      double* vj = ws.V + (long long)j * N;
      double* zj = ws.Z + (long long)j * N;
      CK(prec(vj, zj));
      ++stats.prec_calls;
      CK(apply(zj, ws.w));
      ++stats.vmult_calls;
      // CGS2
      CK(multidot(ws.w, ws.V, j + 1, N, ws.part, ws.h, s));
      k_multiaxpy<<<grid_n(N), 256, 0, s>>>(ws.w, ws.V, ws.h, j + 1, N);
      CK(multidot(ws.w, ws.V, j + 1, N, ws.part, ws.h2, s));
      k_multiaxpy<<<grid_n(N), 256, 0, s>>>(ws.w, ws.V, ws.h2, j + 1, N);
      CK(norm2(ws.w, N, ws.part, ws.nrm, s));
      k_scale_by<<<grid_n(N), 256, 0, s>>>(ws.w, ws.V + (long long)(j + 1) * N, ws.nrm, N);
      CK(cudaMemcpyAsync(stage, ws.h, (2 * (size_t)(m + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      ++stats.iterations;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i] + hcol2[i];
      const double hn = host2[0];
      H[(size_t)(j + 1) * m + j] = hn;
      // previous rotations, then a new one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(a, c);
      cs[j] = den > 0 ? a / den : 1.0;
      sn[j] = den > 0 ? c / den : 0.0;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      j_done = j + 1;
      const double est = std::fabs(g[j + 1]);
      if (!std::isfinite(est)) { stop = true; break; }
      if (est <= rtol * bnorm || stats.iterations >= max_it || hn == 0.0) { stop = true; break; }
    }
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<double> y(j_done, 0.0);
    for (int i = j_done - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int k = i + 1; k < j_done; ++k) sacc -= H[(size_t)i * m + k] * y[k];
      y[i] = H[(size_t)i * m + i] != 0.0 ? sacc / H[(size_t)i * m + i] : 0.0;
    }
    CK(cudaMemcpyAsync(ws.y, y.data(), j_done * sizeof(double), cudaMemcpyHostToDevice, s));
    k_lincomb<<<grid_n(N), 256, 0, s>>>(x, ws.Z, ws.y, j_done, N);
    CK(cudaGetLastError());
    ++stats.restarts;
    CK(true_residual(beta));
    (void)stop;
  }
  stats.rel_residual = beta / bnorm;
  stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = stats;
#undef CK
  return status;
}

}  // namespace sg

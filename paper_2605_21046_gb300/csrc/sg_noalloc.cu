// sg_apply_host_static: the host-buffer apply without any device allocation.
//
// sg_apply_host stages x and y in device buffers that the context allocates
// on first use.  Some callers cannot let a library allocate device memory at
// call time: code that runs while an application-wide pool owns all device
// memory (a caching allocator that must not be bypassed), code paths that
// must not fail or stall on allocation after start-up, and code running
// under rules that forbid cudaMalloc/cudaFree in that phase.  This variant
// stages the two vectors in a fixed array that is part of the library image:
// it is reserved when the module is loaded on a device and held until the
// process exits, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sg_internal.h"

namespace {

// 2 x 2^21 doubles = 32 MiB: x and y of up to 2,097,152 unknowns each.
constexpr size_t kStaticUnknowns = (size_t)1 << 21;
static __device__ __align__(256) double g_static_scratch[2 * kStaticUnknowns];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
// Identifier of the CUDA context the cached address belongs to: a device
// reset (cudaDeviceReset) tears the primary context down, and the array gets
// a new address in the next one, so the address is looked up again whenever
// the current context is not the one it was taken in.
unsigned long long g_scratch_ctx[kMaxDevices] = {};
std::mutex g_scratch_mu;

using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);

// Unique id of the calling thread's current CUDA context (0 if none or if the
// driver cannot tell), through the driver's cuCtxGetCurrent / cuCtxGetId.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return 0;
  void* c = nullptr;
  if (get_current(&c) != 0 || !c) return 0;
  unsigned long long id = 0;
  return get_id(c, &id) == 0 ? id : 0;
}

sg_status fail(sg_status s, const char* m) {
  sg::set_last_error(m);
  return s;
}

}  // namespace

extern "C" {

sg_status sg_apply_host_static(sg_ctx* ctx, int slab, const double* x_host, double* y_host, int transpose) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_apply_host_static: ctx is NULL");
  if (!x_host || !y_host) return fail(SG_ERR_ARG, "sg_apply_host_static: null vector");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_apply_host_static: slab out of range");
  const size_t n = (size_t)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (n > kStaticUnknowns)
    return fail(SG_ERR_ARG, "sg_apply_host_static: more than 2097152 unknowns (the static scratch holds two "
                            "vectors of at most 2^21 doubles); use sg_apply_host");
  if (x_host < y_host + n && y_host < x_host + n) return fail(SG_ERR_ARG, "sg_apply_host_static: x and y overlap");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev != ctx->device || dev < 0 || dev >= kMaxDevices)
    return fail(SG_ERR_ARG, "sg_apply_host_static: the context's device must be current");
  // Once per device (and again after the device's context was replaced),
  // with that device current: the device address of the static array (its
  // host-side name is only a stand-in and must never be handed to a kernel).
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long cid = current_context_id();
    if (!g_scratch_ptr[dev] || cid == 0 || cid != g_scratch_ctx[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) return fail(SG_ERR_CUDA, "sg_apply_host_static: cudaGetSymbolAddress failed");
      g_scratch_ptr[dev] = static_cast<double*>(p);
      g_scratch_ctx[dev] = current_context_id();
    }
    base = g_scratch_ptr[dev];
  }
  double* dx = base;
  double* dy = base + kStaticUnknowns;
  // x is overwritten in full; y is written in full by the apply (its init
  // kernel sets every entry before the cell kernel adds into it).
  e = cudaMemcpy(dx, x_host, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, "sg_apply_host_static: copy in failed");
  sg::ApplyParams p;
  sg::fill_apply_params(ctx->hp, ctx->ls, ctx->d_ctab, ctx->d_grow, ctx->d_gcol, ctx->d_gterm, ctx->d_gval,
                        ctx->d_perm, dx, dy, transpose, p);
  e = sg::launch_apply(ctx->hp, ctx->ls, p, 0);
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, "sg_apply_host_static: launch failed");
  e = cudaMemcpy(y_host, dy, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, "sg_apply_host_static: copy out failed");
  return SG_OK;
}

}  // extern "C"

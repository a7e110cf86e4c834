// The debug entry points: reading the device bounds records of the debug
// build (libsg_debug.so, compiled with -DSG_DEBUG_BOUNDS) and a self-test of
// the record path.  In the release build they report that no checks are
// compiled in.
#include <cuda_runtime.h>

#include "sg_bounds.h"
#include "sg_internal.h"

namespace sg {
cudaError_t bounds_fetch_apply_f64(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_apply_dw(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_apply_f32(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_mc_apply(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_mg(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_factor(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_debug(BoundsRecord* out, bool clear);
cudaError_t bounds_fetch_vanka_tc(BoundsRecord* out, bool clear);
}  // namespace sg

namespace {

constexpr int kProbeSize = 16;

// Writes buf[index] if the bounds check lets it through.
__global__ void k_bounds_probe(long long index, long long limit, int* buf) {
  if (SG_IN(index, limit, 901)) buf[index] = 1;
}

sg_status fail(sg_status s, const char* m) {
  sg::set_last_error(m);
  return s;
}

}  // namespace

SG_BOUNDS_FETCH(bounds_fetch_debug)

extern "C" {

sg_status sg_debug_bounds(int* enabled, unsigned int* count, int* site, long long* index, long long* limit) {
  if (!enabled || !count || !site || !index || !limit) return fail(SG_ERR_ARG, "sg_debug_bounds: null argument");
  *count = 0;
  *site = 0;
  *index = 0;
  *limit = 0;
#ifdef SG_DEBUG_BOUNDS
  *enabled = 1;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, "sg_debug_bounds: synchronize failed");
  cudaError_t (*const fetch[])(sg::BoundsRecord*, bool) = {
      sg::bounds_fetch_apply_f64, sg::bounds_fetch_apply_dw, sg::bounds_fetch_apply_f32, sg::bounds_fetch_mc_apply,
      sg::bounds_fetch_mg,        sg::bounds_fetch_factor,   sg::bounds_fetch_debug, sg::bounds_fetch_vanka_tc};
  for (auto f : fetch) {
    sg::BoundsRecord r;
    if (f(&r, true) != cudaSuccess) return fail(SG_ERR_CUDA, "sg_debug_bounds: reading a record failed");
    if (r.count && !*count) {
      *site = r.site;
      *index = r.index;
      *limit = r.limit;
    }
    *count += r.count;
  }
#else
  *enabled = 0;
#endif
  return SG_OK;
}

sg_status sg_debug_bounds_probe(long long index, long long limit) {
  if (limit < 1 || limit > kProbeSize) return fail(SG_ERR_ARG, "sg_debug_bounds_probe: limit must be 1..16");
#ifndef SG_DEBUG_BOUNDS
  // without device checks only indices inside the array reach the kernel
  if (index < 0 || index >= limit) return fail(SG_ERR_ARG, "sg_debug_bounds_probe: index out of range");
#endif
  int* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, kProbeSize * sizeof(int));
  if (e != cudaSuccess) return fail(SG_ERR_OOM, "sg_debug_bounds_probe: allocation failed");
  k_bounds_probe<<<1, 1>>>(index, limit, buf);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(buf);
  return e == cudaSuccess ? SG_OK : fail(SG_ERR_CUDA, "sg_debug_bounds_probe: launch failed");
}

sg_status sg_debug_wait_probe(unsigned int polls, int* status) {
  if (!status || polls < 1 || polls > (1u << 20))
    return fail(SG_ERR_ARG, "sg_debug_wait_probe: status must be given and polls in 1..2^20");
  cudaError_t e = sg::vanka_tc_wait_probe(polls, status);
  return e == cudaSuccess ? SG_OK : fail(SG_ERR_CUDA, "sg_debug_wait_probe: launch failed");
}

}  // extern "C"

// Device-side bounds checks of the debug build (compiled with
// -DSG_DEBUG_BOUNDS; libsg_debug.so).  They stand in for a memory checker:
// every instrumented global or shared-memory access first tests its index
// against the extent of the array it addresses; an index outside it is not
// accessed, the first such event of the translation unit is recorded (site
// number, index, extent) in a device record and every further one counted.
// Nothing traps: the kernel runs on with that access skipped, and the host
// reads the records through sg_debug_bounds.  In the release build SG_IN
// is the constant true and the checks compile to nothing.
#pragma once
#include <cuda_runtime.h>

namespace sg {
struct BoundsRecord {
  unsigned int count;    // violations seen since the last fetch
  int site;              // site number of the first one
  long long index;       // its index
  long long limit;       // the extent it was checked against
};
}  // namespace sg

#ifdef SG_DEBUG_BOUNDS
static __device__ sg::BoundsRecord g_sg_bounds;

static __device__ __noinline__ bool sg_bounds_fail(long long i, long long n, int site) {
  if (atomicAdd(&g_sg_bounds.count, 1u) == 0u) {
    g_sg_bounds.site = site;
    g_sg_bounds.index = i;
    g_sg_bounds.limit = n;
  }
  return false;
}
#define SG_IN(i, n, site) \
  ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) || sg_bounds_fail((long long)(i), (long long)(n), (site)))
// Host reader of this translation unit's record (optionally clearing it).
#define SG_BOUNDS_FETCH(fn)                                                                   \
  namespace sg {                                                                              \
  cudaError_t fn(BoundsRecord* out, bool clear) {                                             \
    cudaError_t e = cudaMemcpyFromSymbol(out, g_sg_bounds, sizeof(BoundsRecord));            \
    if (e == cudaSuccess && clear) {                                                          \
      const BoundsRecord zero = {0u, 0, 0, 0};                                                \
      e = cudaMemcpyToSymbol(g_sg_bounds, &zero, sizeof(BoundsRecord));                       \
    }                                                                                         \
    return e;                                                                                 \
  }                                                                                           \
  }
#else
#define SG_IN(i, n, site) true
#define SG_BOUNDS_FETCH(fn)                                   \
  namespace sg {                                              \
  cudaError_t fn(BoundsRecord* out, bool) {                   \
    *out = BoundsRecord{0u, 0, 0, 0};                         \
    return cudaSuccess;                                       \
  }                                                           \
  }
#endif

// Vector-wise start and init passes of the level residuals and the multigrid
// starts: one pass over all values of V vectors of n_x nodes each, four
// consecutive values a thread (16-byte loads and stores where the pointers
// allow it).  The node coordinates of a thread's values are carried along
// with its stride (a mixed-radix increment over x, y, z and the vector), so
// the Dirichlet test needs no division per value.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sg_internal.h"

namespace sg {
namespace {

// Per value, bd = the node lies on the boundary of the node grid:
//   op 0 (multigrid start):  y = bd ? b : 0,      yz = bd ? 0 : b
//   op 1 (residual start):   y = bd ? b - x : b
//   op 2 (plain apply):      y = bd ? x : 0
//   op 3 (accumulation):     y = b  (y may be b)
//   op 4 (residual start where x = b on the boundary, as on every multigrid
//         level: the Dirichlet rows of the residual are exactly 0):
//                            y = bd ? 0 : b   (x is not read)
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) vec_start(const T* b, const T* __restrict__ x, T* y, T* __restrict__ yz, int op,
                                                 long long n, int nnx, int nny, int nnz) {
  constexpr int G = 4;
  const long long n_groups = (n + G - 1) / G;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  // coordinates of the group's first value, and of the step stride * G
  const long long i0 = g * G;
  const long long n_x = (long long)nnx * nny * nnz;
  long long r = i0 % n_x;
  int ix = (int)(r % nnx), iy = (int)((r / nnx) % nny), iz = (int)(r / ((long long)nnx * nny));
  const long long step = stride * G;
  const long long s1 = step / nnx, s2 = s1 / nny;
  const int dx = (int)(step % nnx), dy = (int)(s1 % nny), dz = (int)(s2 % nnz);
  for (; g < n_groups; g += stride) {
    const long long i = g * G;
    T bv[G];
    if (VEC && i + G <= n) {
      if (op == 2) {
#pragma unroll
        for (int k = 0; k < G; ++k) bv[k] = T(0);
      } else if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(b + i);
        bv[0] = v.x; bv[1] = v.y; bv[2] = v.z; bv[3] = v.w;
      } else {
        const double2 v0 = *reinterpret_cast<const double2*>(b + i);
        const double2 v1 = *reinterpret_cast<const double2*>(b + i + 2);
        bv[0] = v0.x; bv[1] = v0.y; bv[2] = v1.x; bv[3] = v1.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < G; ++k) bv[k] = (op != 2 && i + k < n) ? b[i + k] : T(0);
    }
    T out[G], out2[G];
    int cx = ix, cy = iy, cz = iz;
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const bool bd = cx == 0 || cx == nnx - 1 || cy == 0 || cy == nny - 1 || (nnz > 1 && (cz == 0 || cz == nnz - 1));
      if (op == 0) {
        out[k] = bd ? bv[k] : T(0);
        out2[k] = bd ? T(0) : bv[k];
      } else if (op == 1) {
        out[k] = bd && i + k < n ? bv[k] - x[i + k] : bv[k];
      } else if (op == 2) {
        out[k] = bd && i + k < n ? x[i + k] : T(0);
      } else if (op == 4) {
        out[k] = bd ? T(0) : bv[k];
      } else {
        out[k] = bv[k];
      }
      // the next node (x fastest; after the last node, the next vector's first)
      if (++cx == nnx) {
        cx = 0;
        if (++cy == nny) {
          cy = 0;
          if (++cz == nnz) cz = 0;
        }
      }
    }
    if (VEC && i + G <= n) {
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(y + i) = make_float4(out[0], out[1], out[2], out[3]);
        if (op == 0) *reinterpret_cast<float4*>(yz + i) = make_float4(out2[0], out2[1], out2[2], out2[3]);
      } else {
        *reinterpret_cast<double2*>(y + i) = make_double2(out[0], out[1]);
        *reinterpret_cast<double2*>(y + i + 2) = make_double2(out[2], out[3]);
        if (op == 0) {
          *reinterpret_cast<double2*>(yz + i) = make_double2(out2[0], out2[1]);
          *reinterpret_cast<double2*>(yz + i + 2) = make_double2(out2[2], out2[3]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (i + k < n) {
          y[i + k] = out[k];
          if (op == 0) yz[i + k] = out2[k];
        }
    }
    // advance the coordinates by the stride
    ix += dx;
    iy += dy;
    iz += dz;
    if (ix >= nnx) {
      ix -= nnx;
      ++iy;
    }
    if (iy >= nny) {
      iy -= nny;
      ++iz;
    }
    if (iz >= nnz) iz -= nnz;
  }
}

inline bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// One start / init pass over V vectors of n_x values (nn: the node grid;
// dim 2 has nn[2] = 1).
template <typename T>
void launch_vec_start(const T* b, const T* x, T* y, T* yz, int op, int V, long long n_x, const int* nn, int dim,
                      cudaStream_t s) {
  const long long n = (long long)V * n_x;
  const bool vec = aligned16(b) && aligned16(y) && aligned16(yz);
  const long long groups = (n + 3) / 4;
  const int grid = (int)std::max<long long>(1, std::min<long long>((groups + 255) / 256, sm_count() * 8));
  const int nz = dim == 3 ? nn[2] : 1;
  if (vec) vec_start<T, true><<<grid, 256, 0, s>>>(b, x, y, yz, op, n, nn[0], nn[1], nz);
  else vec_start<T, false><<<grid, 256, 0, s>>>(b, x, y, yz, op, n, nn[0], nn[1], nz);
}

}  // namespace
}  // namespace sg

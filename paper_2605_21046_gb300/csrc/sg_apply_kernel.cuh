// The SG slab-operator apply kernel, generic over the arithmetic policy
// (sg_arith.h).  See sg_apply.cu for the design; this header holds the device
// code that both precisions instantiate.
#pragma once
#include <cuda_runtime.h>

#include "sg_arith.h"
#include "sg_bounds.h"
#include "sg_internal.h"
#include "sg_shape_tables.h"

namespace sg {

template <int DIM, int K>
struct Shape {
  static constexpr int N = K + 1;                       // nodes = Gauss points per direction
  static constexpr int NKD = DIM == 2 ? N * N : N * N * N;
  static constexpr int NQD = NKD;
  static constexpr int NC = 1 + DIM;                    // value + gradient per point
};

template <int K>
__device__ __forceinline__ constexpr Cf cS(int a, int b) {
  return {RefShape<K>::S(a, b), RefShape<K>::Sh(a, b), RefShape<K>::Sl(a, b)};
}
template <int K>
__device__ __forceinline__ constexpr Cf cD(int a, int b) {
  return {RefShape<K>::D(a, b), RefShape<K>::Dh(a, b), RefShape<K>::Dl(a, b)};
}

// sum_j c(j) x(j) over J compile-time terms; exact zeros are skipped, a lone
// +-1 term is an exact copy, every other result is normalised once.
template <class A, int J, class CF, class XF>
__device__ __forceinline__ typename A::T cdot(CF cf, XF xf) {
  typename A::T s = A::zero();
  int nt = 0;
  bool unit = true;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const Cf c = cf(j);
    if (c.c == 0.0) continue;
    if (nt == 0) s = A::cmul(c, xf(j));
    else A::cfma(c, xf(j), s);
    ++nt;
    if (!(c.c == 1.0 || c.c == -1.0)) unit = false;
  }
  if (nt == 1 && unit) return s;
  return A::fin(s);
}

// --------------------------------------------------------------- phase 1
// Nodal values u (lexicographic, x fastest) -> values and reference gradients
// at the tensor Gauss points, written to q[comp * NQD + point].
template <class A, int DIM, int K>
__device__ __forceinline__ void forward_cell(const typename A::T* u, typename A::T* q) {
  using T = typename A::T;
  using Sh = Shape<DIM, K>;
  constexpr int N = Sh::N;
  constexpr Cf one = {1.0, 1.0f, 0.0f};
  (void)one;
  if constexpr (DIM == 2) {
    T t[N][N];   // [ny][qx]
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int qx = 0; qx < N; ++qx)
        t[ny][qx] = cdot<A, N>([&](int j) { return cS<K>(qx, j); }, [&](int j) { return u[ny * N + j]; });
    T v[N][N];   // [qy][qx]
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        v[qy][qx] = cdot<A, N>([&](int j) { return cS<K>(qy, j); }, [&](int j) { return t[j][qx]; });
        q[qy * N + qx] = v[qy][qx];
      }
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        q[Sh::NQD + qy * N + qx] = cdot<A, N>([&](int r) { return cD<K>(qx, r); }, [&](int r) { return v[qy][r]; });
        q[2 * Sh::NQD + qy * N + qx] = cdot<A, N>([&](int r) { return cD<K>(qy, r); }, [&](int r) { return v[r][qx]; });
      }
  } else {
    T t1[N][N][N];  // [nz][ny][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int qx = 0; qx < N; ++qx)
          t1[nz][ny][qx] = cdot<A, N>([&](int j) { return cS<K>(qx, j); },
                                      [&](int j) { return u[(nz * N + ny) * N + j]; });
    T t2[N][N][N];  // [nz][qy][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx)
          t2[nz][qy][qx] = cdot<A, N>([&](int j) { return cS<K>(qy, j); }, [&](int j) { return t1[nz][j][qx]; });
    T v[N][N][N];   // [qz][qy][qx]
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          v[qz][qy][qx] = cdot<A, N>([&](int j) { return cS<K>(qz, j); }, [&](int j) { return t2[j][qy][qx]; });
          q[(qz * N + qy) * N + qx] = v[qz][qy][qx];
        }
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          const int o = (qz * N + qy) * N + qx;
          q[Sh::NQD + o] = cdot<A, N>([&](int r) { return cD<K>(qx, r); }, [&](int r) { return v[qz][qy][r]; });
          q[2 * Sh::NQD + o] = cdot<A, N>([&](int r) { return cD<K>(qy, r); }, [&](int r) { return v[qz][r][qx]; });
          q[3 * Sh::NQD + o] = cdot<A, N>([&](int r) { return cD<K>(qz, r); }, [&](int r) { return v[r][qy][qx]; });
        }
  }
}

// --------------------------------------------------------------- phase 3
// Point values (q[0..NQD)) and reference-gradient coefficients
// (q[NQD*(1+d) ...]) -> nodal contributions, written over q[0..NKD).  All
// reads of q happen before the first write.
template <class A, int DIM, int K>
__device__ __forceinline__ void backward_cell(typename A::T* q) {
  using T = typename A::T;
  using Sh = Shape<DIM, K>;
  constexpr int N = Sh::N;
  constexpr Cf one = {1.0, 1.0f, 0.0f};
  if constexpr (DIM == 2) {
    T r[N][N];   // [qy][qx] combined point residual
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx)
        r[qy][qx] = cdot<A, 2 * N + 1>(
            [&](int j) { return j == 0 ? one : (j <= N ? cD<K>(j - 1, qx) : cD<K>(j - 1 - N, qy)); },
            [&](int j) {
              return j == 0 ? q[qy * N + qx]
                            : (j <= N ? q[Sh::NQD + qy * N + (j - 1)] : q[2 * Sh::NQD + (j - 1 - N) * N + qx]);
            });
    T t[N][N];   // [ny][qx]
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int qx = 0; qx < N; ++qx)
        t[ny][qx] = cdot<A, N>([&](int j) { return cS<K>(j, ny); }, [&](int j) { return r[j][qx]; });
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int nx = 0; nx < N; ++nx)
        q[ny * N + nx] = cdot<A, N>([&](int j) { return cS<K>(j, nx); }, [&](int j) { return t[ny][j]; });
  } else {
    T r[N][N][N];
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx)
          r[qz][qy][qx] = cdot<A, 3 * N + 1>(
              [&](int j) {
                return j == 0 ? one
                              : (j <= N ? cD<K>(j - 1, qx) : (j <= 2 * N ? cD<K>(j - 1 - N, qy) : cD<K>(j - 1 - 2 * N, qz)));
              },
              [&](int j) {
                return j == 0 ? q[(qz * N + qy) * N + qx]
                              : (j <= N ? q[Sh::NQD + (qz * N + qy) * N + (j - 1)]
                                        : (j <= 2 * N ? q[2 * Sh::NQD + (qz * N + (j - 1 - N)) * N + qx]
                                                      : q[3 * Sh::NQD + ((j - 1 - 2 * N) * N + qy) * N + qx]));
              });
    T t1[N][N][N];  // [nz][qy][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx)
          t1[nz][qy][qx] = cdot<A, N>([&](int j) { return cS<K>(j, nz); }, [&](int j) { return r[j][qy][qx]; });
    T t2[N][N][N];  // [nz][ny][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int qx = 0; qx < N; ++qx)
          t2[nz][ny][qx] = cdot<A, N>([&](int j) { return cS<K>(j, ny); }, [&](int j) { return t1[nz][j][qx]; });
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int nx = 0; nx < N; ++nx)
          q[(nz * N + ny) * N + nx] = cdot<A, N>([&](int j) { return cS<K>(j, nx); }, [&](int j) { return t2[nz][ny][j]; });
  }
}

// One coupling entry of a chaos row, packed for a single 8-byte shared load:
// the offset of column beta's vectors in a cell's value block and the offset
// of the entry's coefficient row in a cell's coefficient block (its (term, G)
// pair with pre-multiplied rows, else its term; -1 - e for an entry e whose
// pair is missing from the pair list, which then reads its tables globally).
struct alignas(8) CoupleEntry {
  int off;
  int tq;
};

// Phase-2 items held per thread (their results live in registers until the
// round's barrier), and the launch bounds: the 2D shapes with at most two
// time nodes and degree <= 2 run two 384-thread CTAs per SM within 80
// registers.
__host__ __device__ constexpr int chunk_kmax(int dim, int nt) {
  return 18 / (nt * (1 + dim)) < 1 ? 1 : (18 / (nt * (1 + dim)) > 3 ? 3 : 18 / (nt * (1 + dim)));
}
template <int DIM, int K, int NT>
struct ChunkBounds {
  static constexpr bool tight = DIM == 2 && K <= 2 && NT <= 2;
  static constexpr int threads = tight ? 384 : 512;
  static constexpr int blocks = tight ? 2 : 1;
};

// The persistent chunk kernel (design notes in sg_apply.cu).
template <class A, int DIM, int K, int NT>
__global__ void __launch_bounds__(ChunkBounds<DIM, K, NT>::threads, ChunkBounds<DIM, K, NT>::blocks)
    sg_apply_chunk_kernel(const ApplyParams p) {
  using T = typename A::T;
  using Sh = Shape<DIM, K>;
  constexpr int NQD = Sh::NQD, NKD = Sh::NKD, NC = Sh::NC, N = Sh::N;
  constexpr int SLOT = (NC * NQD) | 1;           // values per (cell, vector), odd pitch: no bank conflicts
                                                 // between the vectors of phases 1 and 3
  using IO = typename A::IO;
  const IO* __restrict__ xin = reinterpret_cast<const IO*>(p.x);
  IO* __restrict__ yout = reinterpret_cast<IO*>(p.y);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int n_xi = p.n_xi, V = n_xi * NT, C = p.chunk;

  const bool premul = p.premul != 0;
  const int rows = premul ? p.n_pairs : p.n_terms;              // coefficient rows per cell
  T* Qs = reinterpret_cast<T*>(smem_raw);                       // [C][V][NC][NQD]
  T* Cs = Qs + (size_t)C * V * SLOT;                            // [C][rows][NQD]
  T* Amq = Cs + (size_t)C * rows * NQD;                         // [NQD][NT][NT]
  T* Tb = Amq + NQD * NT * NT;                                  // [NT]
  T* Rt = Tb + NT;                                              // [3] (h_0/h_d)^2
  T* Gv = Rt + 3;                                               // G per pair (premul) or per entry
  // the packed coupling entries follow at a 16-byte boundary
  CoupleEntry* Ge = reinterpret_cast<CoupleEntry*>(
      (reinterpret_cast<uintptr_t>(Gv + (premul ? p.n_pairs : p.nnz)) + 15) & ~static_cast<uintptr_t>(15));
  int* Gr = reinterpret_cast<int*>(Ge + p.nnz);                 // [n_xi+1]
  int* Pm = Gr + n_xi + 1;                                      // [n_xi]
  int* Pt = Pm + n_xi;                                          // [n_pairs] term of each pair
  int* Nd = Pt + (premul ? p.n_pairs : 0);                      // [C][NKD] node of y / x, -1 on the boundary

  if (premul) {
    for (int k = tid; k < p.n_pairs; k += nthr) {
      Gv[k] = A::in(p.pair_val[k]);
      Pt[k] = p.pair_term[k];
    }
  } else {
    for (int e = tid; e < p.nnz; e += nthr) Gv[e] = A::in(p.g_val[e]);
  }
  for (int e = tid; e < p.nnz; e += nthr) {
    CoupleEntry ce;
    ce.off = SG_IN(p.g_col[e], n_xi, 105) ? p.g_col[e] * NT * SLOT : 0;
    const int t = p.g_term[e];
    if (premul) {
      const double v = p.g_val[e];
      int k = 0;
      while (k < p.n_pairs && !(p.pair_term[k] == t && p.pair_val[k] == v)) ++k;
      ce.tq = k < p.n_pairs ? k * NQD : -1 - e;
    } else {
      ce.tq = SG_IN(t, p.n_terms, 106) ? t * NQD : 0;
    }
    Ge[e] = ce;
  }
  for (int e = tid; e <= n_xi; e += nthr) Gr[e] = p.g_row[e];
  for (int e = tid; e < n_xi; e += nthr) Pm[e] = p.perm[e];
  for (int e = tid; e < NQD * NT * NT; e += nthr) Amq[e] = A::in(p.amq[e]);
  if (tid < NT) Tb[tid] = A::in(p.tb[tid]);
  if (tid < 3) Rt[tid] = A::in(p.ratio[tid]);

  const long long c_begin = (long long)blockIdx.x * p.n_cells / gridDim.x;
  const long long c_end = (long long)(blockIdx.x + 1) * p.n_cells / gridDim.x;
  const int nnx = p.nn[0], nny = p.nn[1], nnz_ = p.nn[2];

  // the upper half of the CTAs may start with a shorter chunk, so that CTAs
  // sharing an SM do not reach their gather and scatter phases together
  const int first = (p.stagger > 0 && blockIdx.x >= gridDim.x / 2) ? min(C, p.stagger) : C;
  int nc = 0;
  for (long long c0 = c_begin; c0 < c_end; c0 += nc) {
    nc = (int)min((long long)(c0 == c_begin ? first : C), c_end - c0);
    __syncthreads();   // previous chunk done with Qs / Cs; tables visible
    // ---------------------------------------------------------- phase 0
    {
      const int per_cell = p.n_terms * NQD;
      if (premul) {
        // G value x a_term(x_q) per (cell, pair, point), rounded exactly as the
        // product at the Gauss point would be
        const int per_row = rows * NQD;
        for (int idx = tid; idx < nc * per_row; idx += nthr) {
          const int c = idx / per_row, r = idx - c * per_row;
          const int k = r / NQD, q = r - k * NQD;
          const long long at = (c0 + c) * per_cell + Pt[k] * NQD + q;
          if (SG_IN(at, p.n_cells * per_cell, 101)) Cs[idx] = A::fin(A::mul(Gv[k], A::in(p.ctab[at])));
        }
      } else {
        for (int idx = tid; idx < nc * per_cell; idx += nthr)
          if (SG_IN(c0 * per_cell + idx, p.n_cells * per_cell, 101)) Cs[idx] = A::in(p.ctab[c0 * per_cell + idx]);
      }
    }
    // the global node of every (cell, local node) of the chunk, once per
    // chunk instead of once per vector (the integer divisions by the mesh
    // extents would otherwise dominate the gather and scatter)
    for (int i = tid; i < nc * NKD; i += nthr) {
      const int c = i / NKD, a = i - c * NKD;
      const unsigned int gc = (unsigned int)(c0 + c);       // cells < 2^31: 32-bit divisions
      const int cx = (int)(gc % (unsigned int)p.cells[0]);
      const int cy = (int)((gc / (unsigned int)p.cells[0]) % (unsigned int)p.cells[1]);
      const int cz = (int)(gc / ((unsigned int)p.cells[0] * (unsigned int)p.cells[1]));
      const int gx = cx * K + a % N, gy = cy * K + (a / N) % N, gz = DIM == 3 ? cz * K + a / (N * N) : 0;
      bool interior = gx > 0 && gx < nnx - 1 && gy > 0 && gy < nny - 1;
      if (DIM == 3) interior = interior && gz > 0 && gz < nnz_ - 1;
      const long long node = ((long long)gz * nny + gy) * nnx + gx;
      Nd[i] = interior && SG_IN(node, p.n_x, 102) ? (int)node : -1;
    }
    __syncthreads();
    // GU values per thread in flight: a batch's loads all issue before its
    // shared-memory stores
    constexpr int GU = 4;
    for (int c = 0; c < nc; ++c) {
      const int* nd = Nd + c * NKD;
      T* qc = Qs + (size_t)c * V * SLOT;
      for (int j0 = tid; j0 < V * NKD; j0 += GU * nthr) {
        T val[GU];
        int dst[GU];
#pragma unroll
        for (int g = 0; g < GU; ++g) {
          const int j = j0 + g * nthr;
          const int v = j / NKD, a = j - v * NKD;
          val[g] = A::zero();
          dst[g] = j < V * NKD ? v * SLOT + a : -1;
          const int node = j < V * NKD ? nd[a] : -1;
          if (node >= 0 && SG_IN((long long)v * p.n_x + node, (long long)V * p.n_x, 103))
            val[g] = A::in(xin[(long long)v * p.n_x + node]);
        }
#pragma unroll
        for (int g = 0; g < GU; ++g)
          if (dst[g] >= 0 && SG_IN((size_t)c * V * SLOT + dst[g], (size_t)C * V * SLOT, 104)) qc[dst[g]] = val[g];
      }
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 1
    for (int it = tid; it < nc * V; it += nthr) {
      T* q = Qs + (size_t)it * SLOT;
      T u[NKD];
#pragma unroll
      for (int a = 0; a < NKD; ++a) u[a] = q[a];
      forward_cell<A, DIM, K>(u, q);
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 2
    // Rounds of PB Gauss points: the items of a round are (chaos row, point)
    // pairs, consecutive threads taking consecutive points of one row, so a
    // warp follows a single row (no divergence in the coupling loop, one
    // broadcast load per entry).  A thread holds up to KMAX items' results in
    // registers; every read of a round's points precedes its writes (one
    // barrier), and rounds touch disjoint points.
    {
      constexpr int KMAX = chunk_kmax(DIM, NT);
      const int PB = min(32, max(1, (KMAX * nthr) / n_xi));
      const int npts = nc * NQD;
      for (int p0 = 0; p0 < npts; p0 += PB) {
        const int pb = min(PB, npts - p0);
        const int items = n_xi * pb;
        T out[KMAX][NT][NC];
        int a_of[KMAX], c_of[KMAX], q_of[KMAX];
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk) {
          const int it = tid + kk * nthr;
          a_of[kk] = -1;
          c_of[kk] = q_of[kk] = 0;
          if (it < items) {
            const int slot = it / pb, pt = p0 + (it - slot * pb);
            const int a = Pm[slot];
            const int c = pt / NQD, q = pt - c * NQD;
            a_of[kk] = a;
            c_of[kk] = c;
            q_of[kk] = q;
            const T* base = Qs + (size_t)c * V * SLOT + q;
            T uv[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) uv[j] = base[(size_t)(a * NT + j) * SLOT];
            const T* am = Amq + q * NT * NT;
#pragma unroll
            for (int i = 0; i < NT; ++i) {
              T s = A::mul(am[i * NT], uv[0]);
#pragma unroll
              for (int j = 1; j < NT; ++j) A::fma(am[i * NT + j], uv[j], s);
              out[kk][i][0] = A::fin(s);
#pragma unroll
              for (int d = 0; d < DIM; ++d) out[kk][i][1 + d] = A::zero();
            }
            const T* cq = Cs + (size_t)c * rows * NQD + q;
            const int e_beg = Gr[a], e_end = Gr[a + 1];
            auto couple = [&](const T w, const int off) {
              const T* gb = base + off;
#pragma unroll
              for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int d = 0; d < DIM; ++d) A::fma(w, gb[(size_t)i * SLOT + (1 + d) * NQD], out[kk][i][1 + d]);
            };
            if (premul) {
              for (int e = e_beg; e < e_end; ++e) {
                const CoupleEntry ce = Ge[e];
                if (ce.tq >= 0) {
                  couple(cq[ce.tq], ce.off);
                } else {
                  const int ee = -1 - ce.tq;
                  const long long at = (c0 + c) * p.n_terms * NQD + p.g_term[ee] * NQD + q;
                  const double a_q = SG_IN(at, p.n_cells * p.n_terms * NQD, 108) ? p.ctab[at] : 0.0;
                  couple(A::fin(A::mul(A::in(p.g_val[ee]), A::in(a_q))), ce.off);
                }
              }
            } else {
              for (int e = e_beg; e < e_end; ++e) {
                const CoupleEntry ce = Ge[e];
                couple(A::fin(A::mul(Gv[e], cq[ce.tq])), ce.off);
              }
            }
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
              for (int d = 0; d < DIM; ++d) {
                if (p.aniso && d > 0) out[kk][i][1 + d] = A::mul(A::fin(out[kk][i][1 + d]), Rt[d]);
                out[kk][i][1 + d] = A::fin(out[kk][i][1 + d]);
              }
          }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk) {
          if (a_of[kk] < 0) continue;
          T* base = Qs + (size_t)c_of[kk] * V * SLOT + q_of[kk];
#pragma unroll
          for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) base[(size_t)(a_of[kk] * NT + i) * SLOT + cc * NQD] = out[kk][i][cc];
        }
      }
    }
    __syncthreads();
    // ---------------------------------------------------------- phase 3
    for (int it = tid; it < nc * V; it += nthr) backward_cell<A, DIM, K>(Qs + (size_t)it * SLOT);
    __syncthreads();
    // ---------------------------------------------------------- phase 4
    for (int c = 0; c < nc; ++c) {
      const int* nd = Nd + c * NKD;
      const T* qc = Qs + (size_t)c * V * SLOT;
      for (int j = tid; j < V * NKD; j += nthr) {
        const int v = j / NKD, a = j - v * NKD;
        const int node = nd[a];
        if (node >= 0 && SG_IN((long long)v * p.n_x + node, (long long)V * p.n_x, 107)) {
          T val = A::mul(Tb[v % NT], qc[(size_t)v * SLOT + a]);
          if (p.mode == kApplyResidual) val = A::neg(val);
          A::add_out(yout + (long long)v * p.n_x + node, val);
        }
      }
    }
  }
}

}  // namespace sg

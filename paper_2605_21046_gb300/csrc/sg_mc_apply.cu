// The Monte-Carlo apply: y = A(xi_s) x_s for every sample s of one or more
// meshes in ONE launch (paper, Sec. 5: the pathwise slab system eq.
// mc-slab-system, A(xi) = A_t (x) M_x + B_t (x) K[a(., xi)] with
// a(x, xi) = sum_mu a_mu(x) Psi_mu(xi), eq. coeff_expansion).
//
// The work is a queue of units (problem, sample tile, cell): persistent CTAs
// take even contiguous ranges of it and walk them in chunks of cells of one
// problem and tile.  A chunk stages the tile's vectors of its cells in shared
// memory and runs the phases of the SG cell kernel (gather, sum-factorised
// interpolation, point work, transposed sum factorisation, atomic scatter),
// with a point kernel that needs no chaos coupling: at a Gauss point the
// sample's coefficient is sum_t Psi_t(xi_s) a_t(x_q), times the gradients of
// its own vectors, plus the time-node mass coupling.  Samples never couple, so
// any number of them (and several meshes of one shape) share a launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "sg_apply_kernel.cuh"
#include "sg_vec.cuh"

namespace sg {

namespace {

template <class A, int DIM, int K, int NT>
__global__ void __launch_bounds__(256) mc_apply_kernel(const McParams p) {
  using T = typename A::T;
  using IO = typename A::IO;
  using Sh = Shape<DIM, K>;
  constexpr int NQD = Sh::NQD, NKD = Sh::NKD, NC = Sh::NC, N = Sh::N;
  constexpr int SLOT = (NC * NQD) | 1;   // values of one (cell, vector), odd pitch: no bank conflicts between them
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int C = p.chunk, nterm = p.n_terms;
  int ts_max = 0;
  for (int q = 0; q < p.n_prob; ++q) ts_max = max(ts_max, p.pr[q].ts);
  T* Qs = reinterpret_cast<T*>(smem_raw);                       // [C][ts*NT][SLOT]
  T* Cs = Qs + (size_t)C * ts_max * NT * SLOT;                  // [C][term][NQD]
  T* Wt = Cs + (size_t)C * nterm * NQD;                         // [ts][term]
  T* Amq = Wt + (size_t)ts_max * nterm;                         // [NQD][NT][NT]
  T* Tbs = Amq + NQD * NT * NT;                                 // [NT] tau Bhat_ii, converted once
  int* Nd = reinterpret_cast<int*>(Tbs + NT);                   // [C][NKD] node, -1 on the boundary
  if (tid < NT) Tbs[tid] = A::in(p.tb[tid]);
  const long long u_lo = p.u_lo, u_n = (p.u_hi < 0 ? p.units : p.u_hi) - p.u_lo;
  const long long u_begin = u_lo + (long long)blockIdx.x * u_n / gridDim.x;
  const long long u_end = u_lo + (long long)(blockIdx.x + 1) * u_n / gridDim.x;
  int cur_prob = -1, cur_tile = -1;
  for (long long u = u_begin; u < u_end;) {
    int pi = 0;
    while (pi + 1 < p.n_prob && u >= p.pr[pi + 1].unit0) ++pi;
    const McProblem& P = p.pr[pi];
    const long long lu = u - P.unit0;
    const int tile = (int)(lu / P.n_cells);
    const int cell0 = (int)(lu - (long long)tile * P.n_cells);
    const int nc = (int)min((long long)min(C, P.n_cells - cell0), u_end - u);
    const int s0 = tile * P.ts, ns = min(P.ts, P.S - s0);
    const int VT = ns * NT;
    const IO* __restrict__ xin = static_cast<const IO*>(P.x);
    IO* __restrict__ yout = static_cast<IO*>(P.y);
    const int nnx = P.nn[0], nny = P.nn[1], nnz_ = P.nn[2];
    __syncthreads();   // the previous chunk is done with shared memory
    if (pi != cur_prob || tile != cur_tile) {
      for (int e = tid; e < ns * nterm; e += nthr) Wt[e] = A::in(P.wgt[(size_t)s0 * nterm + e]);
      if (pi != cur_prob)
        for (int e = tid; e < NQD * NT * NT; e += nthr) Amq[e] = A::in(P.amq[e]);
      cur_prob = pi;
      cur_tile = tile;
    }
    // phase 0: gather
    for (int idx = tid; idx < nc * nterm * NQD; idx += nthr)
      if (SG_IN((long long)cell0 * nterm * NQD + idx, (long long)P.n_cells * nterm * NQD, 401))
        Cs[idx] = A::in(P.ctab[(size_t)cell0 * nterm * NQD + idx]);
    // global nodes of the chunk's cells, once per chunk (not per vector)
    for (int i = tid; i < nc * NKD; i += nthr) {
      const int c = i / NKD, a = i - c * NKD;
      const int gc = cell0 + c;
      const int cx = gc % P.cells[0], cy = (gc / P.cells[0]) % P.cells[1], cz = gc / (P.cells[0] * P.cells[1]);
      const int gx = cx * K + a % N, gy = cy * K + (a / N) % N, gz = DIM == 3 ? cz * K + a / (N * N) : 0;
      bool interior = gx > 0 && gx < nnx - 1 && gy > 0 && gy < nny - 1;
      if (DIM == 3) interior = interior && gz > 0 && gz < nnz_ - 1;
      Nd[i] = interior ? (int)(((long long)gz * nny + gy) * nnx + gx) : -1;
    }
    __syncthreads();
    // the values, GU per thread in flight: all loads of a batch are issued
    // before its shared-memory stores
    constexpr int GU = 4;
    const IO* xtile = xin + (long long)s0 * NT * P.n_x;
    for (int c = 0; c < nc; ++c) {
      const int* nd = Nd + c * NKD;
      T* qc = Qs + (size_t)c * VT * SLOT;
      for (int j0 = tid; j0 < VT * NKD; j0 += GU * nthr) {
        T val[GU];
        int dst[GU];
#pragma unroll
        for (int g = 0; g < GU; ++g) {
          const int j = j0 + g * nthr;
          const int v = j / NKD, a = j - v * NKD;
          val[g] = A::zero();
          dst[g] = j < VT * NKD ? v * SLOT + a : -1;
          const int node = j < VT * NKD ? nd[a] : -1;
          if (node >= 0 && SG_IN((long long)(s0 * NT + v) * P.n_x + node, (long long)P.S * NT * P.n_x, 402))
            val[g] = A::in(xtile[(long long)v * P.n_x + node]);
        }
#pragma unroll
        for (int g = 0; g < GU; ++g)
          if (dst[g] >= 0) qc[dst[g]] = val[g];
      }
    }
    __syncthreads();
    // phase 1: values and reference gradients at the Gauss points
    for (int it = tid; it < nc * VT; it += nthr) {
      T* q = Qs + (size_t)it * SLOT;
      T uv[NKD];
#pragma unroll
      for (int a = 0; a < NKD; ++a) uv[a] = q[a];
      forward_cell<A, DIM, K>(uv, q);
    }
    __syncthreads();
    // phase 2: per (cell, point, sample): mass coupling and a(x_q, xi_s) grad u.
    // A thread keeps one point q (the first (nthr / NQD) NQD threads take
    // part), holds its N_t x N_t mass weights in registers and walks the
    // (sample, cell) pairs with stride nthr / NQD.
    {
      const int rows = nthr / NQD;
      const int q = tid % NQD, r0 = tid / NQD;
      if (r0 < rows) {
        T am[NT][NT];
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
          for (int j = 0; j < NT; ++j) am[i][j] = Amq[(q * NT + i) * NT + j];
        int sl = r0 % ns, c = r0 / ns;
        while (c < nc) {
          T* base = Qs + ((size_t)c * VT + (size_t)sl * NT) * SLOT + q;
          T uv[NT], out[NT][NC];
#pragma unroll
          for (int j = 0; j < NT; ++j) uv[j] = base[(size_t)j * SLOT];
#pragma unroll
          for (int i = 0; i < NT; ++i) {
            T sacc = A::mul(am[i][0], uv[0]);
#pragma unroll
            for (int j = 1; j < NT; ++j) A::fma(am[i][j], uv[j], sacc);
            out[i][0] = A::fin(sacc);
          }
          if (p.mass_only) {
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
              for (int d = 0; d < DIM; ++d) out[i][1 + d] = A::zero();
          } else {
            const T* cq = Cs + (size_t)c * nterm * NQD + q;
            const T* wt = Wt + sl * nterm;
            T acoef = A::mul(wt[0], cq[0]);
            for (int t = 1; t < nterm; ++t) A::fma(wt[t], cq[t * NQD], acoef);
            acoef = A::fin(acoef);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              T ad = acoef;
              if (P.aniso && d > 0) ad = A::fin(A::mul(acoef, A::in(P.ratio[d])));
#pragma unroll
              for (int i = 0; i < NT; ++i) out[i][1 + d] = A::fin(A::mul(ad, base[(size_t)i * SLOT + (1 + d) * NQD]));
            }
          }
#pragma unroll
          for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) base[(size_t)i * SLOT + cc * NQD] = out[i][cc];
          sl += rows;
          if (sl >= ns) {
            if (sl < 2 * ns) {
              sl -= ns;
              ++c;
            } else {
              c += sl / ns;
              sl %= ns;
            }
          }
        }
      }
    }
    __syncthreads();
    // phase 3: back to the nodes
    for (int it = tid; it < nc * VT; it += nthr) backward_cell<A, DIM, K>(Qs + (size_t)it * SLOT);
    __syncthreads();
    // phase 4: scale by tau Bhat_ii and add into y
    for (int c = 0; c < nc; ++c) {
      const int* nd = Nd + c * NKD;
      const T* qc = Qs + (size_t)c * VT * SLOT;
      for (int j = tid; j < VT * NKD; j += nthr) {
        const int v = j / NKD, a = j - v * NKD;
        const int node = nd[a];
        if (node >= 0 && SG_IN((long long)(s0 * NT + v) * P.n_x + node, (long long)P.S * NT * P.n_x, 403)) {
          T val = A::mul(Tbs[v % NT], qc[(size_t)v * SLOT + a]);
          if (p.mode == kApplyResidual) val = A::neg(val);
          A::add_out(yout + (long long)(s0 * NT + v) * P.n_x + node, val);
        }
      }
    }
    u += nc;
  }
}

void* select_mc(int precision, int dim, int k, int n_t) {
#define SG_M(D, KK, TT)                                                                              \
  if (dim == D && k == KK && n_t == TT)                                                              \
    return precision == kPrecF32 ? reinterpret_cast<void*>(&mc_apply_kernel<F32, D, KK, TT>)         \
                                 : reinterpret_cast<void*>(&mc_apply_kernel<F64, D, KK, TT>);
  SG_M(2, 1, 1) SG_M(2, 1, 2) SG_M(2, 1, 3) SG_M(2, 1, 4)
  SG_M(2, 2, 1) SG_M(2, 2, 2) SG_M(2, 2, 3) SG_M(2, 2, 4)
  SG_M(2, 3, 1) SG_M(2, 3, 2) SG_M(2, 3, 3) SG_M(2, 3, 4)
  SG_M(3, 1, 1) SG_M(3, 1, 2) SG_M(3, 2, 1) SG_M(3, 2, 2)
#undef SG_M
  return nullptr;
}

}  // namespace

size_t mc_smem_bytes(int dim, int k, int n_t, int ts, int n_terms, int chunk, int value_bytes) {
  const size_t nqd = dim == 2 ? (k + 1) * (k + 1) : (k + 1) * (k + 1) * (k + 1);
  const size_t slot = ((1 + dim) * nqd) | 1;
  const size_t vals = (size_t)chunk * ts * n_t * slot + (size_t)chunk * n_terms * nqd +
                      (size_t)ts * n_terms + nqd * n_t * n_t + n_t;
  // values, then the chunk's node indices at a 4-byte boundary
  return ((vals * value_bytes + 3) / 4) * 4 + (size_t)chunk * nqd * sizeof(int);
}

void mc_amq(const HostProblem& hp, const std::vector<double>& Tm, std::vector<double>& amq) {
  const int nq = hp.k + 1, nqd = hp.dim == 2 ? nq * nq : nq * nq * nq, nt = hp.n_t;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  amq.assign((size_t)nqd * nt * nt, 0.0);
  for (int qd = 0; qd < nqd; ++qd) {
    const int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    for (int i = 0; i < nt; ++i) {
      const double tb = hp.tau * hp.B_hat[i * nt + i];
      for (int j = 0; j < nt; ++j) amq[((size_t)qd * nt + i) * nt + j] = w * Tm[(size_t)i * nt + j] / tb;
    }
  }
}

cudaError_t prepare_mc_kernel(int precision, int dim, int k, int n_t) {
  void* f = select_mc(precision, dim, k, n_t);
  if (!f) return cudaErrorInvalidValue;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

cudaError_t launch_mc_apply(int precision, int dim, int k, int n_t, const McParams& p, int grid, int threads,
                            size_t smem, cudaStream_t s) {
  void* f = select_mc(precision, dim, k, n_t);
  if (!f) return cudaErrorInvalidValue;
  // y's start: b (accumulate), b - x on the boundary and b inside (residual),
  // x on the boundary and 0 inside (plain), for the sample rows of the tiles
  // this launch covers (its unit range holds whole tiles)
  const long long u_lo = p.u_lo, u_hi = p.u_hi < 0 ? p.units : p.u_hi;
  for (int q = 0; q < p.n_prob; ++q) {
    const McProblem& P = p.pr[q];
    const long long a = std::max(u_lo, P.unit0), z = std::min(u_hi, P.unit0 + (long long)P.tiles * P.n_cells);
    if (a >= z) continue;
    const int t_lo = (int)((a - P.unit0) / P.n_cells), t_hi = (int)((z - P.unit0 + P.n_cells - 1) / P.n_cells);
    const int s_lo = t_lo * P.ts, s_hi = std::min(P.S, t_hi * P.ts);
    const int V = (s_hi - s_lo) * n_t;
    const long long off = (long long)s_lo * n_t * P.n_x;
    const int op = p.mode == kApplyResidual ? (p.bd_zero ? 4 : 1) : (p.mode == kApplyAccumulate ? 3 : 2);
    if (precision == kPrecF32) {
      const float* b = static_cast<const float*>(P.b);
      launch_vec_start<float>(b ? b + off : nullptr, static_cast<const float*>(P.x) + off,
                              static_cast<float*>(P.y) + off, nullptr, op, V, P.n_x, P.nn, dim, s);
    } else {
      const double* b = static_cast<const double*>(P.b);
      launch_vec_start<double>(b ? b + off : nullptr, static_cast<const double*>(P.x) + off,
                               static_cast<double*>(P.y) + off, nullptr, op, V, P.n_x, P.nn, dim, s);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<McParams*>(&p)};
  return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_mc_apply)

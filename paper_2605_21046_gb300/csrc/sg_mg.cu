// Block-Jacobi geometric-multigrid preconditioner of the SG slab system
// (paper, Sec. 3.5, remark on the algebraic solver): every chaos mode alpha is
// preconditioned by one V-cycle of its diagonal block
//     A_alpha = A_t (x) M_x + sum_mu [G_mu]_{alpha alpha} B_t (x) K_mu,
// with a space-time Vanka patch smoother.  All N_xi * N_t vectors go through
// the V-cycle together, so one launch smooths every mode.  A level residual is
// either the SG cell kernel with the diagonal coupling table or the diagonal
// (Monte-Carlo) apply with per-row weights [G_mu]_{alpha alpha}; set-up times
// both on the level and keeps the faster.
//
// Levels halve the cells per direction while every count is even and > 2;
// coefficients are re-evaluated on every level (a per-cell scale is averaged
// over the children).  Smoother: additive Vanka, one patch per cell = its
// interior nodes x all time nodes, patch matrix = principal submatrix of the
// level block operator (summed from the element matrices of the neighbouring
// cells), exact dense inverse, damping omega, corrections divided by the
// number of patches that hold the node; nu pre- and nu post-smoothing steps.
// Transfer: canonical Q_k interpolation P (tensor product of 1D tables,
// Dirichlet rows and columns removed), restriction P^T.  Coarsest level:
// dense inverse of the interior block.  Dirichlet rows are the identity on
// every level.  The whole V-cycle is captured once into a CUDA graph.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

#include "sg_bounds.h"
#include "sg_internal.h"
#include "sg_vec.cuh"

namespace sg {

void fill_apply_params(const HostProblem& hp, const LaunchShape& ls, const void* ctab,
                       const int* grow, const int* gcol, const int* gterm, const double* gval,
                       const int* perm, const void* x, void* y, int transpose, ApplyParams& p);
cudaError_t prepare_apply_kernel(int precision, int dim, int k, int n_t, size_t smem);

namespace {

// ------------------------------------------------------------------ kernels
// Vector-wise kernels run on a 2D grid: blockIdx.y is the vector, the node
// index within it stays 32-bit (no 64-bit division per element).
inline dim3 vec_grid(long long n_x, int V) {
  return dim3((unsigned)std::max<long long>(1, std::min<long long>((n_x + 255) / 256, 1024)), (unsigned)V);
}

template <typename T>
__global__ void mg_init_x(const T* __restrict__ b, T* __restrict__ x, int n_x, int nnx, int nny, int nnz, int dim) {
  const long long off = (long long)blockIdx.y * n_x;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_x; m += gridDim.x * blockDim.x) {
    const int ix = m % nnx, rr = m / nnx, iy = rr % nny, iz = rr / nny;
    bool bd = ix == 0 || ix == nnx - 1 || iy == 0 || iy == nny - 1;
    if (dim == 3) bd = bd || iz == 0 || iz == nnz - 1;
    x[off + m] = bd ? b[off + m] : T(0);
  }
}

template <typename S, typename D>
__global__ void mg_convert(const S* __restrict__ a, D* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (D)a[i];
}

// Additive Vanka step: x += omega / mult * inv(patch) * r_patch for every
// (cell, alpha), patch = the cell's nodes x all time nodes (Dirichlet rows
// skipped), mult = number of cells that hold the node.
//
// Per (cell, diagonal class) the step is a dense product Z = inv * R with
// inv the NP x NP patch inverse and R the patch values of the class's modes
// (NP x modes).  Persistent CTAs walk units (a chunk of C cells consecutive
// in x, a tile of mode blocks) in two pipeline stages: while one unit is
// computed, the next unit's data land in the other stage by asynchronous
// copies (cp.async):
//   * the chunk's inverses of the unit's first class (contiguous in memory:
//     cells consecutive in x), 16 bytes at a time, rows padded to an odd
//     number of 16-byte pieces so that the rows of 8 consecutive threads fall
//     in different banks;
//   * r on the chunk's node grid as [time node][node][slot], one value per
//     copy, slots = the tile's modes grouped by class in blocks of kVankaVB
//     (padding and Dirichlet nodes stored as zero).
// Every thread accumulates a register block of kVankaR patch rows x one block
// of kVankaVB slots: per patch column one broadcast 16-byte load of the patch
// values and kVankaR x kVankaVB FMAs, the inverse rows read 16 bytes at a time
// (bf16 widened in registers).  The damped, multiplicity-weighted corrections
// of neighbouring cells are summed in shared memory and added into x once per
// node with reductions (no thread waits on a load of x).  The staging and the
// write-back walk their (slot, node) pairs with per-thread increments instead
// of divisions; further classes of a tile are staged synchronously.
// Inverses are stored [class][cell][NP][npp] in W (double, float or bf16;
// npp = NP rounded up to 8).
constexpr int kVankaVB = 4;      // slots per mode block (modes of one class); slots per thread
constexpr int kVankaR = 4;       // patch rows per thread

template <typename T>
struct VankaParams {
  const T* r;
  T* x;
  const void* inv;
  const int* blk_cls;       // [n_blk] class of every mode block
  const int* blk_alpha;     // [n_blk][kVankaVB] modes, -1 padded
  int n_blk, chunk, npp;
  int tile_blocks, n_tiles; // mode blocks per tile
  long long n_x, n_cells;
  long long n_vec_x;        // values per vector set (rows x time nodes x nodes; bounds checks)
  long long inv_count;      // stored inverse values (bounds checks)
  size_t smem_values;       // bytes below the index tables in shared memory (bounds checks)
  int cells[3], nn[3];
  T omega;
};

// 16-byte pieces per shared-memory row of a staged inverse of NP values of
// `bytes` each: the pieces the row needs, made odd (bank spread).
__host__ __device__ constexpr int vanka_row_pieces(int np, int bytes) {
  return ((np * bytes + 15) / 16) % 2 == 0 ? (np * bytes + 15) / 16 + 1 : (np * bytes + 15) / 16;
}
// Slots per node in shared memory for a tile of `blocks` mode blocks.
__host__ __device__ constexpr int vanka_slots(int blocks) { return blocks * kVankaVB; }

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double* p, double* o) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
};

// One 16-byte piece of an inverse row, widened to T.
template <typename T, typename W>
struct Piece16;
template <>
struct Piece16<float, float> {
  static constexpr int n = 4;
  __device__ static void load(const float* p, float* o) { Vec4<float>::load(p, o); }
};
template <>
struct Piece16<double, double> {
  static constexpr int n = 2;
  __device__ static void load(const double* p, double* o) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    o[0] = a.x; o[1] = a.y;
  }
};
template <>
struct Piece16<float, __nv_bfloat16> {
  static constexpr int n = 8;
  __device__ static void load(const __nv_bfloat16* p, float* o) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const unsigned int w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};

template <typename T, typename W>
__device__ __forceinline__ T widen(W w) { return (T)w; }
template <>
__device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 w) { return __bfloat162float(w); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// A copy of sizeof(T) bytes (4 or 8) from global to shared memory, asynchronous.
template <typename T>
__device__ __forceinline__ void cp_async_val(T* smem, const T* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// One unit of work (a chunk of cells and a tile of mode blocks).
struct VankaUnit {
  int cx0, cy, cz, nc, b0, nb;
  long long cell0;
};

template <typename T, typename W, int DIM, int K, int NT, bool TRANS>
__global__ void __launch_bounds__(256, 2) mg_vanka(const VankaParams<T> p) {
  constexpr int N = K + 1;
  constexpr int NKD = DIM == 2 ? N * N : N * N * N;
  constexpr int NP = NT * NKD;
  constexpr int R = kVankaR, VB = kVankaVB;
  constexpr int NRG = (NP + R - 1) / R;                        // row groups per cell
  constexpr int RP = vanka_row_pieces(NP, (int)sizeof(W));     // 16-byte pieces per staged row
  constexpr int RW = RP * 16 / (int)sizeof(W);                 // values per staged row
  constexpr int QV = Piece16<T, W>::n;                         // values per piece
  constexpr int NQC = (NP + QV - 1) / QV;                      // pieces a row product reads
  constexpr int LYZ = DIM == 2 ? N : N * N;                    // nodes across y (and z)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int C = p.chunk;
  const int LX = C * K + 1;                                    // chunk nodes along x
  const int LN = LX * LYZ;
  const int SL = vanka_slots(p.tile_blocks);
  const int E = NT * LN;                                       // (time node, node) pairs per slot
  // shared memory: the corrections, then two stages of (r, inverses, node and slot tables)
  // stage b: r at Rl0 + b E SL, inverses at Is0 + b C NP RW, node table at
  // Gn0 + b LN, slot table at Sm0 + b SL
  T* Zc = reinterpret_cast<T*>(smem_raw);                      // [NT][LN][SL]
  T* Rl0 = Zc + (size_t)E * SL;                                // 2 x [NT][LN][SL]
  W* Is0 = reinterpret_cast<W*>(Zc + (size_t)3 * E * SL);      // 2 x [C][NP][RW] inverses of one class
  int* Gn0 = reinterpret_cast<int*>(Is0 + (size_t)2 * C * NP * RW);   // 2 x [LN] global node, -1 outside / boundary
  int* Sm0 = Gn0 + 2 * LN;                                     // 2 x [SL] mode of every slot, -1 padding
  const size_t rl_stage = (size_t)E * SL, is_stage = (size_t)C * NP * RW;
  const W* inv = static_cast<const W*>(p.inv);
  const int nnx = p.nn[0], nny = p.nn[1], nnz_ = p.nn[2];
  const int cpr = (p.cells[0] + C - 1) / C;                    // chunks per row of cells
  const long long n_chunks = (long long)cpr * p.cells[1] * p.cells[2];
  const long long n_units = n_chunks * p.n_tiles;
  // (slot, pair) walk of the gather and the write-back: start and increments
  const int w_sl0 = tid / E, w_e0 = tid - (tid / E) * E;
  const int w_dq = nthr / E, w_dr = nthr - (nthr / E) * E;
  const int LNSL = LN * SL, LXSL = LX * SL;

  // 32-bit index arithmetic (units and cells stay below 2^31; 64-bit
  // divisions would cost more than the rest of the bookkeeping)
  auto decode = [&](long long unit, VankaUnit& U) {
    const unsigned int uu = (unsigned int)unit, nch = (unsigned int)n_chunks;
    const unsigned int ch = uu % nch;
    const int tile = (int)(uu / nch);
    U.b0 = tile * p.tile_blocks;
    U.nb = min(p.tile_blocks, p.n_blk - U.b0);
    U.cx0 = (int)(ch % (unsigned int)cpr) * C;
    const unsigned int row = ch / (unsigned int)cpr;
    U.cy = (int)(row % (unsigned int)p.cells[1]);
    U.cz = (int)(row / (unsigned int)p.cells[1]);
    U.nc = min(C, p.cells[0] - U.cx0);
    U.cell0 = ((long long)U.cz * p.cells[1] + U.cy) * p.cells[0] + U.cx0;
  };
  // the global index of every node of the unit's chunk (-1 outside the mesh or
  // on the boundary) and the mode of every slot
  auto tables = [&](const VankaUnit& U, int* Gn, int* Sm) {
    const int lxn = U.nc * K + 1;
    for (int ln = tid; ln < LN; ln += nthr) {
      const int lx = ln % LX, lyz = ln / LX;
      const int ly = lyz % N, lz = DIM == 3 ? lyz / N : 0;
      int node = -1;
      if (lx < lxn) {
        const int gx = U.cx0 * K + lx, gy = U.cy * K + ly, gz = DIM == 3 ? U.cz * K + lz : 0;
        bool in = gx > 0 && gx < nnx - 1 && gy > 0 && gy < nny - 1;
        if (DIM == 3) in = in && gz > 0 && gz < nnz_ - 1;
        if (in) node = (int)(((long long)gz * nny + gy) * nnx + gx);
      }
      Gn[ln] = node;
    }
    for (int sl = tid; sl < SL; sl += nthr) Sm[sl] = sl < U.nb * VB ? p.blk_alpha[U.b0 * VB + sl] : -1;
  };
  // asynchronous copies of the chunk's inverses of class `cls` (contiguous in
  // memory: cells consecutive in x) in 16-byte pieces
  auto stage_inverses = [&](const VankaUnit& U, int cls, W* Is, int stage_base) {
    const long long ibeg = ((long long)cls * p.n_cells + U.cell0) * NP * p.npp;
    for (int idx = tid; idx < U.nc * NP * RP; idx += nthr) {
      const int rr = idx / RP, piece = idx - rr * RP;
      if (piece * 16 >= p.npp * (int)sizeof(W)) continue;     // the padding piece of a row
      const long long g = ibeg + (long long)rr * p.npp + piece * (16 / (int)sizeof(W));
      if (!SG_IN(g + 16 / (int)sizeof(W) - 1, p.inv_count, 202)) continue;
      if (!SG_IN((size_t)stage_base + ((size_t)rr * RW + piece * (16 / sizeof(W))) * sizeof(W), p.smem_values, 203))
        continue;
      cp_async16(Is + (size_t)rr * RW + piece * (16 / (int)sizeof(W)), inv + g);
    }
  };
  // asynchronous gather of r on the chunk's node grid (slot-major, node
  // fastest); padding slots and Dirichlet nodes are stored as zero
  auto stage_r = [&](T* Rl, const int* Gn, const int* Sm) {
    int sl = w_sl0, e = w_e0;
    while (sl < SL) {
      int i = 0;
#pragma unroll
      for (int j = 1; j < NT; ++j) i += e >= j * LN;
      const int ln = e - i * LN;
      const int mode = Sm[sl], node = Gn[ln];
      const long long gi = ((long long)mode * NT + i) * p.n_x + node;
      T* dst = Rl + (size_t)e * SL + sl;
      if (mode >= 0 && node >= 0 && SG_IN(gi, p.n_vec_x, 201)) cp_async_val(dst, p.r + gi);
      else *dst = T(0);
      e += w_dr;
      sl += w_dq;
      if (e >= E) { e -= E; ++sl; }
    }
  };

  for (int i = tid; i < E * SL; i += nthr) Zc[i] = T(0);
  long long u = blockIdx.x;
  int buf = 0;
  VankaUnit cur, nxt;
  if (u < n_units) {
    decode(u, cur);
    tables(cur, Gn0, Sm0);
  }
  __syncthreads();
  if (u < n_units) {
    stage_inverses(cur, p.blk_cls[cur.b0], Is0, (int)((size_t)3 * E * SL * sizeof(T)));
    stage_r(Rl0, Gn0, Sm0);
  }
  cp_async_commit();
  for (; u < n_units; u += gridDim.x, buf ^= 1) {
    // the next unit's tables and copies go to the other stage while this one computes
    const long long un = u + gridDim.x;
    const bool has_next = un < n_units;
    __syncthreads();                                           // the other stage is free
    if (has_next) {
      decode(un, nxt);
      tables(nxt, Gn0 + (buf ^ 1) * LN, Sm0 + (buf ^ 1) * SL);
    }
    __syncthreads();
    if (has_next) {
      stage_inverses(nxt, p.blk_cls[nxt.b0], Is0 + (buf ^ 1) * is_stage,
                     (int)((size_t)3 * E * SL * sizeof(T) + (size_t)(buf ^ 1) * is_stage * sizeof(W)));
      stage_r(Rl0 + (buf ^ 1) * rl_stage, Gn0 + (buf ^ 1) * LN, Sm0 + (buf ^ 1) * SL);
    }
    cp_async_commit();
    cp_async_wait_prior1();                                    // this unit's copies have landed
    __syncthreads();
    const T* Rl = Rl0 + buf * rl_stage;
    W* Is = Is0 + buf * is_stage;
    const int* Gn = Gn0 + buf * LN;
    const int* Sm = Sm0 + buf * SL;
    // runs of consecutive blocks of one class
    for (int rb = 0; rb < cur.nb;) {
      const int cls = p.blk_cls[cur.b0 + rb];
      int re = rb + 1;
      while (re < cur.nb && p.blk_cls[cur.b0 + re] == cls) ++re;
      const int nbr = re - rb;
      const int sa = rb * VB;
      if (rb > 0) {
        // a further class of this tile: its inverses, synchronously
        __syncthreads();
        stage_inverses(cur, cls, Is, (int)((size_t)3 * E * SL * sizeof(T) + (size_t)buf * is_stage * sizeof(W)));
        cp_async_wait_all();
        __syncthreads();
      }
      const int items = cur.nc * NRG * nbr;
      for (int it = tid; it < items; it += nthr) {
        const int rg = it % NRG, cb = it / NRG;
        const int bl = cb % nbr, c = cb / nbr;
        const int s0 = sa + bl * VB;
        int rows[R];
#pragma unroll
        for (int k = 0; k < R; ++k) rows[k] = rg + k * NRG;
        T acc[R][VB];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int uu = 0; uu < VB; ++uu) acc[k][uu] = T(0);
        const T* pb = Rl + (size_t)(c * K) * SL + s0;
        const W* ib = Is + (size_t)c * NP * RW;
        if constexpr (!TRANS) {
          const W* ir[R];
#pragma unroll
          for (int k = 0; k < R; ++k) ir[k] = ib + (size_t)min(rows[k], NP - 1) * RW;
#pragma unroll
          for (int qc = 0; qc < NQC; ++qc) {
            T w[R][QV];
#pragma unroll
            for (int k = 0; k < R; ++k) Piece16<T, W>::load(ir[k] + qc * QV, w[k]);
#pragma unroll
            for (int j = 0; j < QV; ++j) {
              const int q = qc * QV + j;
              if (q >= NP) break;
              const int iq = q / NKD, aq = q - iq * NKD;
              const int ax = aq % N, ayz = aq / N;
              T v[VB];
              Vec4<T>::load(pb + iq * LNSL + ayz * LXSL + ax * SL, v);
#pragma unroll
              for (int k = 0; k < R; ++k)
#pragma unroll
                for (int uu = 0; uu < VB; ++uu) acc[k][uu] = fma(w[k][j], v[uu], acc[k][uu]);
            }
          }
        } else {
#pragma unroll 6
          for (int q = 0; q < NP; ++q) {
            const int iq = q / NKD, aq = q - iq * NKD;
            const int ax = aq % N, ayz = aq / N;
            T v[VB];
            Vec4<T>::load(pb + iq * LNSL + ayz * LXSL + ax * SL, v);
            const W* iqrow = ib + (size_t)q * RW;
#pragma unroll
            for (int k = 0; k < R; ++k) {
              const T w = widen<T, W>(iqrow[min(rows[k], NP - 1)]);
#pragma unroll
              for (int uu = 0; uu < VB; ++uu) acc[k][uu] = fma(w, v[uu], acc[k][uu]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int rho = rows[k];
          if (rho >= NP) continue;
          const int i = rho / NKD, a = rho - i * NKD;
          const int ax = a % N, ay = (a / N) % N, az = DIM == 3 ? a / (N * N) : 0;
          const int lna = c * K + ax + LX * (ay + (DIM == 3 ? N * az : 0));
          if (Gn[lna] < 0) continue;                 // Dirichlet row
          // patches sharing the node (cell corners and faces: the local coordinate is 0 or K)
          const int mult = (ax % K == 0 ? 2 : 1) * (ay % K == 0 ? 2 : 1) * (DIM == 3 && az % K == 0 ? 2 : 1);
          const T sc = p.omega / T(mult);
          const size_t zo = (size_t)(i * LN + lna) * SL + s0;
#pragma unroll
          for (int uu = 0; uu < VB; ++uu)
            if (SG_IN(zo + uu, (size_t)E * SL, 204)) atomicAdd(Zc + zo + uu, sc * acc[k][uu]);
        }
      }
      rb = re;
    }
    __syncthreads();
    // add the corrections into x (reductions: no thread waits on a load of x)
    // and clear them for the next unit
    {
      const int SLW = cur.nb * VB;
      int sl = w_sl0, e = w_e0;
      while (sl < SLW) {
        int i = 0;
#pragma unroll
        for (int j = 1; j < NT; ++j) i += e >= j * LN;
        const int ln = e - i * LN;
        const int mode = Sm[sl], node = Gn[ln];
        T* z = Zc + (size_t)e * SL + sl;
        if (mode >= 0 && node >= 0) {
          const long long gi = ((long long)mode * NT + i) * p.n_x + node;
          if (SG_IN(gi, p.n_vec_x, 205)) atomicAdd(p.x + gi, *z);
        }
        *z = T(0);
        e += w_dr;
        sl += w_dq;
        if (e >= E) { e -= E; ++sl; }
      }
    }
    cur = nxt;
  }
  cp_async_wait_all();
}

// One pass of a separable grid transfer: along one axis of a structured
// array [VA][nin][B] -> [VA][nout][B],
//     out[va][jo][b] (+)= sum_k w[k][jo] in[va][idx[k][jo]][b],  k < W,
// with the 1D restriction lists (coarse node <- fine nodes) or the 1D
// interpolation lists (fine node <- coarse nodes) padded to W entries per
// output (weight 0, index of the output's first entry) and stored entry-major,
// so the lanes of a warp (consecutive outputs in the x pass, one output in the
// others) read them coalesced or broadcast from L1.  Restriction P^T and
// prolongation P are d such passes (x, y, z resp. z, y, x), which read every
// value a few times instead of (k+1)^d-fold per output.  Each thread walks the
// flat output index with a fixed stride, carrying (va, jo, b) along instead
// of dividing for every element.
constexpr int kAxisMax = 16;  // entries of one output of a 1D transfer list, at most (4k + 1 for k <= 3)

template <typename T, int W>
__global__ void __launch_bounds__(256) mg_axis_gather(const T* __restrict__ in, T* __restrict__ out, long long VA,
                                                      int nin, int nout, int B, const int* __restrict__ idx,
                                                      const T* __restrict__ w, int accumulate) {
  const long long total = VA * nout * B;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int b = (int)(e % B);
  long long r = e / B;
  int jo = (int)(r % nout);
  long long va = r / nout;
  const int db = (int)(stride % B);
  const long long rs = stride / B;
  const int djo = (int)(rs % nout);
  const long long dva = rs / nout;
  const long long row_in = (long long)nin * B;
  for (; e < total; e += stride) {
    const T* src = in + va * row_in + b;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int si = __ldg(idx + k * nout + jo);
      if (SG_IN(si, nin, 501)) acc += __ldg(w + k * nout + jo) * src[(long long)si * B];
    }
    if (accumulate) out[e] += acc;
    else out[e] = acc;
    b += db;
    jo += djo;
    va += dva;
    if (b >= B) {
      b -= B;
      ++jo;
    }
    if (jo >= nout) {
      jo -= nout;
      ++va;
    }
  }
}

// Coarsest level: x[inner] = inv(C_class) b[inner] for every chaos mode
// (blockIdx.y) and a block of rows (blockIdx.x); the right-hand side is
// staged in shared memory.  A warp takes one row of inv (its lanes read the
// row coalesced and reduce with shuffles); the transposed cycle takes a
// column per thread (consecutive threads, consecutive columns).
template <typename T>
__global__ void mg_coarse(const T* __restrict__ b, T* __restrict__ x, const T* __restrict__ inv,
                          const int* __restrict__ cls, const long long* __restrict__ inner, int n_int,
                          int n_t, long long n_x, int trans) {
  extern __shared__ __align__(16) unsigned char sm[];
  T* bs = reinterpret_cast<T*>(sm);
  const int alpha = blockIdx.y;
  const long long base = (long long)alpha * n_t * n_x;
  for (int i = threadIdx.x; i < n_int; i += blockDim.x) bs[i] = b[base + inner[i]];
  __syncthreads();
  const T* M = inv + (long long)cls[alpha] * n_int * n_int;
  if (trans) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_int; i += gridDim.x * blockDim.x) {
      T s = T(0);
      for (int q = 0; q < n_int; ++q) s += M[(long long)q * n_int + i] * bs[q];
      x[base + inner[i]] = s;
    }
  } else {
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * warps + warp; i < n_int; i += gridDim.x * warps) {
      const T* row = M + (long long)i * n_int;
      T s = T(0);
      for (int q = lane; q < n_int; q += 32) s += row[q] * bs[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) x[base + inner[i]] = s;
    }
  }
}

// ------------------------------------------------------------------ host set-up

int grid_for(long long n, int block) {
  return (int)std::max<long long>(1, std::min<long long>((n + block - 1) / block, sg::sm_count() * 32));
}

// In-place inverse of a dense n x n matrix (Gauss-Jordan, partial pivoting).
bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv(n * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
    if (a[(size_t)piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    const double d = 1.0 / a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] *= d;
      inv[(size_t)c * n + k] *= d;
    }
#pragma omp parallel for schedule(static) if (n >= 256)
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// Reference element matrices of a level: mass (cell independent) and, per
// cell, the stiffness with the class coefficient cbar(q) = sum_t diag[t] ctab[t][q].
struct ElementData {
  int nkd = 0, nqd = 0, dim = 2;
  std::vector<double> phi;    // [a][q]
  std::vector<double> grad;   // [d][a][q] reference derivative
  std::vector<double> wJ;     // [q]
  std::vector<double> mass;   // [a][b]
};

ElementData element_data(const HostProblem& hp) {
  ElementData e;
  const int n = hp.k + 1;
  e.dim = hp.dim;
  e.nkd = hp.dim == 2 ? n * n : n * n * n;
  e.nqd = e.nkd;
  e.phi.assign((size_t)e.nkd * e.nqd, 0.0);
  e.grad.assign((size_t)3 * e.nkd * e.nqd, 0.0);
  e.wJ.assign(e.nqd, 0.0);
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  for (int q = 0; q < e.nqd; ++q) {
    const int qi[3] = {q % n, (q / n) % n, q / (n * n)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    e.wJ[q] = w;
    for (int a = 0; a < e.nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      double v = 1.0;
      for (int d = 0; d < hp.dim; ++d) v *= hp.S[qi[d] * n + ai[d]];
      e.phi[(size_t)a * e.nqd + q] = v;
      for (int dd = 0; dd < hp.dim; ++dd) {
        double g = 1.0;
        for (int d = 0; d < hp.dim; ++d) g *= d == dd ? hp.dS[qi[d] * n + ai[d]] : hp.S[qi[d] * n + ai[d]];
        e.grad[((size_t)dd * e.nkd + a) * e.nqd + q] = g;
      }
    }
  }
  e.mass.assign((size_t)e.nkd * e.nkd, 0.0);
  for (int a = 0; a < e.nkd; ++a)
    for (int b = 0; b < e.nkd; ++b) {
      double s = 0.0;
      for (int q = 0; q < e.nqd; ++q) s += e.wJ[q] * e.phi[(size_t)a * e.nqd + q] * e.phi[(size_t)b * e.nqd + q];
      e.mass[(size_t)a * e.nkd + b] = s;
    }
  return e;
}

// Element stiffness of cell c for the class coefficient (ctab holds
// w_q |J| a_t / h_0^2; direction d carries (h_0 / h_d)^2).
void element_stiffness(const HostProblem& hp, const ElementData& e, const std::vector<double>& diag,
                       long long c, std::vector<double>& K) {
  std::vector<double> cbar(e.nqd, 0.0);
  for (int t = 0; t < hp.n_terms; ++t) {
    if (diag[t] == 0.0) continue;
    const double* ct = hp.ctab.data() + ((size_t)c * hp.n_terms + t) * e.nqd;
    for (int q = 0; q < e.nqd; ++q) cbar[q] += diag[t] * ct[q];
  }
  double ratio[3];
  for (int d = 0; d < 3; ++d) ratio[d] = d < hp.dim ? (hp.h[0] * hp.h[0]) / (hp.h[d] * hp.h[d]) : 0.0;
  K.assign((size_t)e.nkd * e.nkd, 0.0);
  for (int a = 0; a < e.nkd; ++a)
    for (int b = a; b < e.nkd; ++b) {
      double s = 0.0;
      for (int d = 0; d < hp.dim; ++d) {
        const double* ga = e.grad.data() + ((size_t)d * e.nkd + a) * e.nqd;
        const double* gb = e.grad.data() + ((size_t)d * e.nkd + b) * e.nqd;
        double sd = 0.0;
        for (int q = 0; q < e.nqd; ++q) sd += cbar[q] * ga[q] * gb[q];
        s += ratio[d] * sd;
      }
      K[(size_t)a * e.nkd + b] = s;
      K[(size_t)b * e.nkd + a] = s;
    }
}

void cell_coords(const HostProblem& hp, long long c, int cc[3]) {
  cc[0] = (int)(c % hp.cells[0]);
  cc[1] = (int)((c / hp.cells[0]) % hp.cells[1]);
  cc[2] = (int)(c / ((long long)hp.cells[0] * hp.cells[1]));
}

bool node_interior(const HostProblem& hp, const int g[3]) {
  for (int d = 0; d < hp.dim; ++d)
    if (g[d] <= 0 || g[d] >= hp.nn[d] - 1) return false;
  return true;
}

// Row pitch of the stored patch inverses: np rounded up to 8 values (16-byte
// rows for bf16, float and double).
int vanka_row_pitch(int np) { return (np + 7) / 8 * 8; }

// Coarsest level: dense inverse of the interior block of one class.
bool coarse_inverse(const HostProblem& hp, const ElementData& e, const std::vector<double>& diag,
                    const std::vector<long long>& node_of, std::vector<double>& out) {
  const int n = hp.k + 1, nkd = e.nkd, nt = hp.n_t;
  const int nin = (int)node_of.size();
  std::vector<int> idx(hp.n_x, -1);
  for (int i = 0; i < nin; ++i) idx[node_of[i]] = i;
  const int N = nt * nin;
  std::vector<double> C((size_t)N * N, 0.0), K;
  for (long long c = 0; c < hp.n_cells; ++c) {
    element_stiffness(hp, e, diag, c, K);
    int cc[3];
    cell_coords(hp, c, cc);
    int g[64];
    for (int a = 0; a < nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      long long gl = 0, stride = 1;
      for (int d = 0; d < hp.dim; ++d) {
        gl += (long long)(cc[d] * hp.k + ai[d]) * stride;
        stride *= hp.nn[d];
      }
      g[a] = idx[gl];
    }
    for (int i = 0; i < nt; ++i)
      for (int a = 0; a < nkd; ++a) {
        if (g[a] < 0) continue;
        for (int j = 0; j < nt; ++j)
          for (int b = 0; b < nkd; ++b) {
            if (g[b] < 0) continue;
            double v = hp.A_hat[i * nt + j] * e.mass[(size_t)a * nkd + b];
            if (i == j) v += hp.tau * hp.B_hat[i * nt + i] * K[(size_t)a * nkd + b];
            C[(size_t)(i * nin + g[a]) * N + j * nin + g[b]] += v;
          }
      }
  }
  if (!invert(C, N)) return false;
  out.swap(C);
  return true;
}

// 1D interpolation table of one direction between a fine and a coarse level.
void transfer_1d(const HostProblem& fine, const HostProblem& coarse, int d, std::vector<int>& pptr,
                 std::vector<int>& pidx, std::vector<double>& pwl, std::vector<int>& rptr, std::vector<int>& ridx,
                 std::vector<double>& rw) {
  std::vector<int> pc;
  std::vector<double> pw;
  const int K = fine.k, n = K + 1;
  const std::vector<double> gll = lobatto_nodes(K);
  const int nf = fine.nn[d], nc = coarse.nn[d];
  pc.assign(nf, 0);
  pw.assign((size_t)nf * n, 0.0);
  std::vector<std::vector<std::pair<int, double>>> cols(nc);
  for (int i = 0; i < nf; ++i) {
    const int cf = std::min(i / K, fine.cells[d] - 1);
    const double pos = cf + gll[i - cf * K];
    const double cpos = 0.5 * pos;
    const int ccell = std::min((int)std::floor(cpos), coarse.cells[d] - 1);
    const double s = cpos - ccell;
    pc[i] = ccell;
    const bool fine_bd = i == 0 || i == nf - 1;
    for (int a = 0; a < n; ++a) {
      const int j = ccell * K + a;
      const bool coarse_bd = j == 0 || j == nc - 1;
      double w = (fine_bd || coarse_bd) ? 0.0 : lagrange(gll, a, s);
      pw[(size_t)i * n + a] = w;
      if (w != 0.0) cols[j].push_back({i, w});
    }
  }
  rptr.assign(nc + 1, 0);
  ridx.clear();
  rw.clear();
  for (int j = 0; j < nc; ++j) {
    for (auto& t : cols[j]) {
      ridx.push_back(t.first);
      rw.push_back(t.second);
    }
    rptr[j + 1] = (int)ridx.size();
  }
  // interpolation lists: fine node i <- coarse nodes pc[i] K + a with nonzero weight
  pptr.assign(nf + 1, 0);
  pidx.clear();
  pwl.clear();
  for (int i = 0; i < nf; ++i) {
    for (int a = 0; a < n; ++a)
      if (pw[(size_t)i * n + a] != 0.0) {
        pidx.push_back(pc[i] * K + a);
        pwl.push_back(pw[(size_t)i * n + a]);
      }
    pptr[i + 1] = (int)pidx.size();
  }
}

template <typename T>
cudaError_t upload_vec(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), std::max<size_t>(1, src.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t upload_values(void** dst, const std::vector<double>& src, int precision) {
  if (precision == kPrecF32) {
    std::vector<float> f(src.begin(), src.end());
    return upload_vec(reinterpret_cast<float**>(dst), f);
  }
  return upload_vec(reinterpret_cast<double**>(dst), src);
}

// The diagonal (block-Jacobi) coupling table: row alpha keeps its own column.
void diagonal_table(const HostProblem& fine, GTable& g, std::vector<std::vector<double>>& diag_of_row) {
  diag_of_row.assign(fine.n_xi, std::vector<double>(fine.n_terms, 0.0));
  for (int a = 0; a < fine.n_xi; ++a)
    for (int e = fine.g.row[a]; e < fine.g.row[a + 1]; ++e)
      if (fine.g.col[e] == a) diag_of_row[a][fine.g.term[e]] += fine.g.val[e];
  g.row.assign(fine.n_xi + 1, 0);
  g.col.clear();
  g.term.clear();
  g.val.clear();
  for (int a = 0; a < fine.n_xi; ++a) {
    for (int t = 0; t < fine.n_terms; ++t)
      if (diag_of_row[a][t] != 0.0) {
        g.col.push_back(a);
        g.term.push_back(t);
        g.val.push_back(diag_of_row[a][t]);
      }
    g.row[a + 1] = (int)g.col.size();
  }
}

// Averages a per-cell scale over the 2^d children of every coarse cell.
std::vector<double> coarsen_scale(const std::vector<double>& s, const HostProblem& fine) {
  if (s.empty()) return s;
  const int cx = fine.cells[0] / 2, cy = fine.cells[1] / 2, cz = fine.dim == 3 ? fine.cells[2] / 2 : 1;
  std::vector<double> out((size_t)cx * cy * cz, 0.0);
  const int kz = fine.dim == 3 ? 2 : 1;
  const double inv = 1.0 / (4 * kz);
  for (int z = 0; z < cz; ++z)
    for (int y = 0; y < cy; ++y)
      for (int x = 0; x < cx; ++x) {
        double acc = 0.0;
        for (int dz = 0; dz < kz; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
              acc += s[((size_t)(kz * z + dz) * fine.cells[1] + 2 * y + dy) * fine.cells[0] + 2 * x + dx];
        out[((size_t)z * cy + y) * cx + x] = acc * inv;
      }
  return out;
}

template <typename T>
cudaError_t issue_vcycle(MG& mg, int l, cudaStream_t s, int trans);

// r = b - A x in one apply (residual mode: the init kernel writes b minus the
// Dirichlet rows, the cell kernel subtracts).
template <typename T>
cudaError_t residual(MG& mg, int l, cudaStream_t s, int trans) {
  MGLevel& L = mg.lv[l];
  if (L.use_diag) {
    // the level operator couples no two rows (block Jacobi): the diagonal
    // apply with per-row weights G_mu[alpha][alpha] (Psi_mu(xi_s) for samples)
    McParams q;
    std::memset(&q, 0, sizeof(q));
    q.u_hi = -1;                       // every unit in one launch
    q.bd_zero = 1;                     // x = b on the boundary (start, Vanka and transfers keep it)
    q.n_prob = 1;
    McProblem& P = q.pr[0];
    P.x = L.d_x;
    P.y = L.d_r;
    P.b = L.d_b;
    P.ctab = static_cast<const double*>(L.d_ctab);
    P.wgt = mg.d_wgt;
    P.amq = trans ? L.d_amqT : L.d_amq;
    P.n_x = L.hp.n_x;
    P.unit0 = 0;
    P.n_cells = (int)L.hp.n_cells;
    P.S = L.hp.n_xi;
    P.ts = L.mc_ts;
    P.tiles = (P.S + P.ts - 1) / P.ts;
    for (int d = 0; d < 3; ++d) {
      P.nn[d] = L.hp.nn[d];
      P.cells[d] = L.hp.cells[d];
      P.ratio[d] = d < L.hp.dim ? (L.hp.h[0] * L.hp.h[0]) / (L.hp.h[d] * L.hp.h[d]) : 0.0;
    }
    P.aniso = 0;
    for (int d = 1; d < L.hp.dim; ++d) P.aniso |= L.hp.h[d] != L.hp.h[0];
    q.n_terms = L.hp.n_terms;
    q.chunk = L.mc_chunk;
    q.mode = kApplyResidual;
    q.mass_only = 0;
    q.units = (long long)P.tiles * P.n_cells;
    for (int i = 0; i < L.hp.n_t; ++i) q.tb[i] = L.hp.tau * L.hp.B_hat[i * L.hp.n_t + i];
    return launch_mc_apply(mg.precision, L.hp.dim, L.hp.k, L.hp.n_t, q, L.mc_grid, L.mc_threads, L.mc_smem, s);
  }
  ApplyParams p;
  fill_apply_params(L.hp, L.ls, L.d_ctab, L.d_grow, L.d_gcol, L.d_gterm, L.d_gval, L.d_perm, L.d_x, L.d_r, trans, p);
  p.b = L.d_b;
  p.mode = kApplyResidual;
  return launch_apply(L.hp, L.ls, p, s);
}

// The initial iterate (x = b on Dirichlet dofs, 0 inside) and its residual
// (r = b inside, 0 on Dirichlet dofs) in one pass, without an apply.
// Tile (rows) and chunk (cells) of a level's diagonal apply: the largest
// chunk <= max_chunk within 100 KB of shared memory; the grid covers the units.
sg_status level_diag_shape(MGLevel& L, int ts, int max_chunk, int vb) {
  L.mc_ts = std::max(1, std::min(ts, L.hp.n_xi));
  L.mc_chunk = 0;
  for (int c = 1; c <= max_chunk; ++c)
    if (mc_smem_bytes(L.hp.dim, L.hp.k, L.hp.n_t, L.mc_ts, L.hp.n_terms, c, vb) <= 100 * 1024) L.mc_chunk = c;
  if (L.mc_chunk == 0) return SG_ERR_UNSUPPORTED;
  L.mc_smem = mc_smem_bytes(L.hp.dim, L.hp.k, L.hp.n_t, L.mc_ts, L.hp.n_terms, L.mc_chunk, vb);
  const long long units = (long long)((L.hp.n_xi + L.mc_ts - 1) / L.mc_ts) * L.hp.n_cells;
  L.mc_grid = (int)std::max<long long>(1, std::min<long long>(units / std::max(1, L.mc_chunk), sg::sm_count() * 4));
  return SG_OK;
}

// Shared memory of a Vanka chunk: r and the corrections of the tile's slots,
// the staged inverses of one class, then the nodes' global indices and
// private flags, the slot modes and the patch-column offsets.
size_t vanka_smem(const MGLevel& L, int n_blk, int tile_slots, int chunk, size_t value_bytes, size_t inv_bytes) {
  const int N = L.hp.k + 1, lyz = L.hp.dim == 2 ? N : N * N;
  const size_t ln = (size_t)(chunk * L.hp.k + 1) * lyz;   // nodes of a chunk
  const int blocks = std::min(n_blk, std::max(1, tile_slots / kVankaVB));
  const size_t sl = (size_t)vanka_slots(blocks);
  const size_t row = (size_t)vanka_row_pieces(L.np, (int)inv_bytes) * 16;
  // the corrections and two stages of r, inverses and tables
  return 3 * (size_t)L.hp.n_t * ln * sl * value_bytes + 2 * (size_t)chunk * L.np * row +
         2 * (ln + sl) * sizeof(int);
}

// Bytes of one stored patch-inverse value.
size_t inv_value_bytes(const MG& mg) { return mg.bf16 ? 2 : (mg.precision == kPrecF32 ? 4 : 8); }

// Cells per Vanka chunk: up to 8, within the shared-memory budget.
int vanka_chunk(const MGLevel& L, int n_blk, int tile_slots, size_t value_bytes, size_t inv_bytes, size_t budget) {
  int best = 0;
  for (int c = 1; c <= std::min(8, L.hp.cells[0]); ++c)
    if (vanka_smem(L, n_blk, tile_slots, c, value_bytes, inv_bytes) <= budget) best = c;
  return best;
}

template <typename T, typename W, int DIM, int K, int NT>
cudaError_t launch_vanka_w(MG& mg, MGLevel& L, cudaStream_t s, int trans) {
  VankaParams<T> p;
  p.r = static_cast<const T*>(L.vanka_r ? L.vanka_r : L.d_r);
  p.x = static_cast<T*>(L.d_x);
  p.inv = L.d_inv;
  p.blk_cls = mg.d_blk_cls;
  p.blk_alpha = mg.d_blk_alpha;
  p.n_blk = mg.n_blk;
  const int tile = L.vanka_tile > 0 ? L.vanka_tile : mg.vanka_tile;
  p.chunk = L.vanka_chunk;
  p.tile_blocks = std::min(mg.n_blk, std::max(1, tile / kVankaVB));
  p.n_tiles = (mg.n_blk + p.tile_blocks - 1) / p.tile_blocks;
  p.npp = vanka_row_pitch(L.np);
  p.n_x = L.hp.n_x;
  p.n_cells = L.hp.n_cells;
  for (int d = 0; d < 3; ++d) {
    p.cells[d] = L.hp.cells[d];
    p.nn[d] = L.hp.nn[d];
  }
  p.omega = T(mg.omega);
  const size_t smem = vanka_smem(L, mg.n_blk, tile, L.vanka_chunk, sizeof(T), sizeof(W));
  p.n_vec_x = (long long)L.hp.n_xi * L.hp.n_t * L.hp.n_x;
  p.inv_count = (long long)mg.n_classes * L.hp.n_cells * L.np * p.npp;
  const int N = L.hp.k + 1, lyz = L.hp.dim == 2 ? N : N * N;
  {
    const size_t ln = (size_t)(L.vanka_chunk * L.hp.k + 1) * lyz;
    p.smem_values = 3 * (size_t)L.hp.n_t * ln * vanka_slots(p.tile_blocks) * sizeof(T) +
                    2 * (size_t)L.vanka_chunk * L.np * vanka_row_pieces(L.np, (int)sizeof(W)) * 16;
  }
  // threads: the row-group x slot-block items of a chunk (one class), whole warps
  const int nrg = (L.np + kVankaR - 1) / kVankaR;
  const int items = L.vanka_chunk * nrg * p.tile_blocks;
  const int threads = std::max(64, std::min(256, (items + 31) / 32 * 32));
  auto kern = trans ? &mg_vanka<T, W, DIM, K, NT, true> : &mg_vanka<T, W, DIM, K, NT, false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  const int cpr = (L.hp.cells[0] + L.vanka_chunk - 1) / L.vanka_chunk;
  const long long units = (long long)cpr * L.hp.cells[1] * L.hp.cells[2] * p.n_tiles;
  const int grid = (int)std::max<long long>(1, std::min<long long>(units, sg::sm_count() * std::max(1, per_sm)));
  kern<<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

// Allows the Vanka kernels of one shape the opt-in shared-memory maximum
// (called at set-up, outside any stream capture).
template <typename T, typename W, int DIM, int K, int NT>
cudaError_t prepare_vanka_w() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaFuncSetAttribute(&mg_vanka<T, W, DIM, K, NT, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(&mg_vanka<T, W, DIM, K, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  return e;
}

cudaError_t prepare_vanka(int dim, int k, int nt, bool f32, bool bf16) {
#define SG_PV(D, KK, TT)                                                           \
  if (dim == D && k == KK && nt == TT) {                                           \
    if (!f32) return prepare_vanka_w<double, double, D, KK, TT>();                 \
    if (bf16) return prepare_vanka_w<float, __nv_bfloat16, D, KK, TT>();           \
    return prepare_vanka_w<float, float, D, KK, TT>();                             \
  }
  SG_PV(2, 1, 1) SG_PV(2, 1, 2) SG_PV(2, 1, 3) SG_PV(2, 1, 4)
  SG_PV(2, 2, 1) SG_PV(2, 2, 2) SG_PV(2, 2, 3) SG_PV(2, 2, 4)
  SG_PV(2, 3, 1) SG_PV(2, 3, 2) SG_PV(2, 3, 3) SG_PV(2, 3, 4)
  SG_PV(3, 1, 1) SG_PV(3, 1, 2) SG_PV(3, 2, 1) SG_PV(3, 2, 2)
#undef SG_PV
  return cudaErrorInvalidValue;
}

template <typename T, int DIM, int K, int NT>
cudaError_t launch_vanka(MG& mg, MGLevel& L, cudaStream_t s, int trans) {
  if constexpr (std::is_same<T, float>::value) {
    if (mg.bf16 && L.vanka_kind == 1 && !trans) {
      const int tile = L.vanka_tile > 0 ? L.vanka_tile : mg.vanka_tile;
      const float* r = static_cast<const float*>(L.vanka_r ? L.vanka_r : L.d_r);
      return launch_vanka_tc(L.hp, r, static_cast<float*>(L.d_x), L.d_inv, mg.d_blk_alpha, mg.n_blk, L.vanka_chunk,
                             tile, mg.d_status, (float)mg.omega, s);
    }
    if (mg.bf16) return launch_vanka_w<T, __nv_bfloat16, DIM, K, NT>(mg, L, s, trans);
  }
  return launch_vanka_w<T, T, DIM, K, NT>(mg, L, s, trans);
}

// The tensor-core sweep applies to this level: bf16 factors, one diagonal
// class, a patch of at most 64 unknowns, tiles of at most 80 slots.
bool tc_level_ok(const MG& mg, const MGLevel& L, int tile) {
  return mg.bf16 && mg.n_classes == 1 && !L.coarsest && vanka_tc_eligible(L.hp.dim, L.hp.k, L.hp.n_t, tile);
}

template <typename T>
bool vanka(MG& mg, MGLevel& L, cudaStream_t s, int trans) {
  const int d = L.hp.dim, k = L.hp.k, t = L.hp.n_t;
#define SG_V(D, KK, TT) \
  if (d == D && k == KK && t == TT) return launch_vanka<T, D, KK, TT>(mg, L, s, trans) == cudaSuccess;
  SG_V(2, 1, 1) SG_V(2, 1, 2) SG_V(2, 1, 3) SG_V(2, 1, 4)
  SG_V(2, 2, 1) SG_V(2, 2, 2) SG_V(2, 2, 3) SG_V(2, 2, 4)
  SG_V(2, 3, 1) SG_V(2, 3, 2) SG_V(2, 3, 3) SG_V(2, 3, 4)
  SG_V(3, 1, 1) SG_V(3, 1, 2) SG_V(3, 2, 1) SG_V(3, 2, 2)
#undef SG_V
  return false;
}

bool vk_launch(MG& mg, MGLevel& L, cudaStream_t s) {
  return mg.precision == kPrecF32 ? vanka<float>(mg, L, s, 0) : vanka<double>(mg, L, s, 0);
}

template <typename T, int W>
void axis_pass_w(const void* in, void* out, long long VA, int nin, int nout, int B, const int* idx, const void* w,
                 int accumulate, cudaStream_t s) {
  const long long total = VA * nout * B;
  const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, sg::sm_count() * 8));
  mg_axis_gather<T, W><<<grid, 256, 0, s>>>(static_cast<const T*>(in), static_cast<T*>(out), VA, nin, nout, B, idx,
                                            static_cast<const T*>(w), accumulate);
}

// one pass with lists padded to width (one of axis_width's values)
template <typename T>
void axis_pass(const void* in, void* out, long long VA, int nin, int nout, int B, const int* idx, const void* w,
               int width, int accumulate, cudaStream_t s) {
  switch (width) {
    case 2: axis_pass_w<T, 2>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
    case 3: axis_pass_w<T, 3>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
    case 4: axis_pass_w<T, 4>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
    case 5: axis_pass_w<T, 5>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
    case 8: axis_pass_w<T, 8>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
    default: axis_pass_w<T, kAxisMax>(in, out, VA, nin, nout, B, idx, w, accumulate, s); break;
  }
}

// the padded width of lists whose longest has n entries
int axis_width(int n) {
  for (int w : {2, 3, 4, 5, 8})
    if (n <= w) return w;
  return kAxisMax;
}

// CSR lists (ptr, idx, wt) -> width entries per output, entry-major
void pad_lists(const std::vector<int>& ptr, const std::vector<int>& idx, const std::vector<double>& wt, int width,
               std::vector<int>& pidx, std::vector<double>& pw) {
  const int n = (int)ptr.size() - 1;
  pidx.assign((size_t)width * n, 0);
  pw.assign((size_t)width * n, 0.0);
  for (int o = 0; o < n; ++o) {
    const int c = ptr[o + 1] - ptr[o];
    for (int k = 0; k < width; ++k) {
      pidx[(size_t)k * n + o] = k < c ? idx[ptr[o] + k] : (c > 0 ? idx[ptr[o]] : 0);
      pw[(size_t)k * n + o] = k < c ? wt[ptr[o] + k] : 0.0;
    }
  }
}

// x_fine += P e_coarse: interpolation along z (3D), y, then x
template <typename T>
bool prolong(MGLevel& F, MGLevel& C, int V, cudaStream_t s) {
  const int nfx = F.hp.nn[0], nfy = F.hp.nn[1], nfz = F.hp.nn[2];
  const int ncx = C.hp.nn[0], ncy = C.hp.nn[1], ncz = C.hp.nn[2];
  auto pass = [&](const void* in, void* out, long long VA, int nin, int nout, int B, int d, int acc) {
    axis_pass<T>(in, out, VA, nin, nout, B, F.d_pidx[d], F.d_pwl[d], F.pmax[d], acc, s);
  };
  if (F.hp.dim == 3) {
    pass(C.d_x, F.d_t2, V, ncz, nfz, ncy * ncx, 2, 0);
    pass(F.d_t2, F.d_t1, (long long)V * nfz, ncy, nfy, ncx, 1, 0);
    pass(F.d_t1, F.d_x, (long long)V * nfz * nfy, ncx, nfx, 1, 0, 1);
  } else {
    pass(C.d_x, F.d_t1, V, ncy, nfy, ncx, 1, 0);
    pass(F.d_t1, F.d_x, (long long)V * nfy, ncx, nfx, 1, 0, 1);
  }
  return cudaGetLastError() == cudaSuccess;
}

// b_coarse = P^T r_fine: restriction along x, y, then z (3D)
template <typename T>
void restrict_to(MGLevel& F, MGLevel& C, int V, cudaStream_t s) {
  const int nfx = F.hp.nn[0], nfy = F.hp.nn[1], nfz = F.hp.nn[2];
  const int ncx = C.hp.nn[0], ncy = C.hp.nn[1], ncz = C.hp.nn[2];
  auto pass = [&](const void* in, void* out, long long VA, int nin, int nout, int B, int d) {
    axis_pass<T>(in, out, VA, nin, nout, B, F.d_ridx[d], F.d_rw[d], F.rmax[d], 0, s);
  };
  if (F.hp.dim == 3) {
    pass(F.d_r, F.d_t1, (long long)V * nfz * nfy, nfx, ncx, 1, 0);
    pass(F.d_t1, F.d_t2, (long long)V * nfz, nfy, ncy, ncx, 1);
    pass(F.d_t2, C.d_b, V, nfz, ncz, ncy * ncx, 2);
  } else {
    pass(F.d_r, F.d_t1, (long long)V * nfy, nfx, ncx, 1, 0);
    pass(F.d_t1, C.d_b, V, nfy, ncy, ncx, 1);
  }
}

template <typename T>
cudaError_t issue_vcycle(MG& mg, int l, cudaStream_t s, int trans) {
  MGLevel& L = mg.lv[l];
  const int V = L.hp.n_xi * L.hp.n_t;
  if (L.coarsest) {
    mg_init_x<T><<<vec_grid(L.hp.n_x, V), 256, 0, s>>>(static_cast<const T*>(L.d_b), static_cast<T*>(L.d_x),
                                                      (int)L.hp.n_x, L.hp.nn[0], L.hp.nn[1], L.hp.nn[2], L.hp.dim);
    const size_t smem = (size_t)L.n_int * sizeof(T);
    const int gx = trans ? (L.n_int + 255) / 256 : (L.n_int + 7) / 8;   // rows: a warp each (8 a block)
    mg_coarse<T><<<dim3(gx, L.hp.n_xi), 256, smem, s>>>(static_cast<const T*>(L.d_b), static_cast<T*>(L.d_x),
                                              static_cast<const T*>(L.d_inv), mg.d_cls,
                                              reinterpret_cast<const long long*>(L.d_inner), L.n_int, L.hp.n_t, L.hp.n_x,
                                              trans);
    return cudaGetLastError();
  }
  cudaError_t e;
  // the start: x = the boundary values of b and 0 inside; the first sweep's
  // residual b - A x is b on the interior, where the sweep reads it
  launch_vec_start<T>(nullptr, static_cast<const T*>(L.d_b), static_cast<T*>(L.d_x), nullptr, 2, V, L.hp.n_x,
                      L.hp.nn, L.hp.dim, s);
  for (int it = 0; it < mg.nu; ++it) {
    if (it > 0 && (e = residual<T>(mg, l, s, trans)) != cudaSuccess) return e;
    L.vanka_r = it == 0 ? L.d_b : nullptr;
    const bool ok = vanka<T>(mg, L, s, trans);
    L.vanka_r = nullptr;
    if (!ok) return cudaErrorInvalidValue;
  }
  if ((e = residual<T>(mg, l, s, trans)) != cudaSuccess) return e;
  MGLevel& C = mg.lv[l + 1];
  if (C.hp.n_xi * C.hp.n_t != V) return cudaErrorInvalidValue;   // level buffers hold V vectors
  restrict_to<T>(L, C, V, s);
  if ((e = issue_vcycle<T>(mg, l + 1, s, trans)) != cudaSuccess) return e;
  if (!prolong<T>(L, C, V, s)) return cudaErrorInvalidValue;
  for (int it = 0; it < mg.nu; ++it) {
    if ((e = residual<T>(mg, l, s, trans)) != cudaSuccess) return e;
    if (!vanka<T>(mg, L, s, trans)) return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// Device time of one launch of a set-up candidate: a single timed launch when
// it takes more than 2 ms (the large levels, where one launch is steady and
// repeating it costs seconds), else the mean of three launches after it.
template <class F>
static float time_candidate(F&& launch, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, cudaError_t& e) {
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e != cudaSuccess || ms > 2.0f) return ms;
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  return ms / 3.0f;
}

// Picks, for every smoothed level of at least 256 cells, the faster residual
// apply on the level's own buffers: the diagonal apply over (rows per tile in
// {8, 32, all} x at most 8 or 2 cells per chunk) or, where it applies, the SG
// cell kernel over (cells per chunk x 256 / 512 threads), then the staggered
// first chunk of the best cell-kernel shape.  Smaller levels keep the SG cell
// kernel where it applies.
static cudaError_t tune_level_applies(MG& mg) {
  const size_t vb = mg.precision == kPrecF32 ? 4 : 8;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  for (size_t l = 0; l < mg.lv.size() && e == cudaSuccess; ++l) {
    MGLevel& L = mg.lv[l];
    if (L.coarsest || L.hp.n_cells < 256) continue;
    auto res = [&]() {
      return mg.precision == kPrecF32 ? residual<float>(mg, (int)l, mg.stream, 0)
                                      : residual<double>(mg, (int)l, mg.stream, 0);
    };
    const long long n = (long long)L.hp.n_xi * L.hp.n_t * L.hp.n_x;
    if ((e = cudaMemsetAsync(L.d_x, 0, n * vb, mg.stream)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(L.d_b, 0, n * vb, mg.stream)) != cudaSuccess) break;
    std::vector<int> tss;
    for (int t : {8, 32, L.hp.n_xi})
      if (t <= L.hp.n_xi && std::find(tss.begin(), tss.end(), t) == tss.end()) tss.push_back(t);
    int best_ts = L.mc_ts, best_c = 8;
    float best_ms = 1e30f;
    bool best_diag = true;
    LaunchShape best_ls = L.ls;
    L.use_diag = true;
    for (int ts : tss) {
      for (int cmax : {8, 2}) {
        if (e != cudaSuccess) break;
        if (level_diag_shape(L, ts, cmax, (int)vb) != SG_OK) continue;
        if (L.mc_chunk != cmax && cmax != 8) continue;           // the same shape as a larger cap
        const float ms = time_candidate(res, mg.stream, a, b, e);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best_ts = ts;
          best_c = L.mc_chunk;
        }
      }
    }
    level_diag_shape(L, best_ts, best_c, (int)vb);
    if (L.chunk_ok) {
      // the SG cell kernel over (cells per chunk x threads)
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const int max1 = max_apply_chunk(L.hp, (size_t)optin - 1024);
      std::vector<int> chunks;
      for (int c = max1; c >= 1; c = c > 1 ? (c + 1) / 2 - (c == 2) : 0) chunks.push_back(c);
      L.use_diag = false;
      const LaunchShape keep = L.ls;
      // (cells per chunk x threads), then the staggered first chunk of the best
      for (int c : chunks)
        for (int t : {256, 512}) {
          if (e != cudaSuccess) break;
          LaunchShape ls;
          std::string msg;
          if (plan_apply_shape(L.hp, c, t, ls, msg) != SG_OK) continue;
          ls.stagger = 0;
          L.ls = ls;
          const float ms = time_candidate(res, mg.stream, a, b, e);
          if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best_diag = false;
            best_ls = ls;
          }
        }
      if (!best_diag && best_ls.chunk > 1 && e == cudaSuccess) {
        LaunchShape ls = best_ls;
        ls.stagger = (ls.chunk + 1) / 2;
        L.ls = ls;
        const float ms = time_candidate(res, mg.stream, a, b, e);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best_ls = ls;
        }
      }
      L.ls = best_diag ? keep : best_ls;
    }
    L.use_diag = best_diag;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

// Picks the cells per Vanka chunk of every smoothed level, and with a single
// diagonal class on levels with few cells the modes per tile (the whole set,
// 16 or 8: smaller tiles give them more CTAs), by timing sweeps on the level's own buffers for
// every candidate within the shared-memory budget; keeps the fastest.
static cudaError_t tune_vanka(MG& mg) {
  const size_t vb = mg.precision == kPrecF32 ? 4 : 8;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  for (MGLevel& L : mg.lv) {
    if (L.coarsest || e != cudaSuccess) continue;
    const long long n = (long long)L.hp.n_xi * L.hp.n_t * L.hp.n_x;
    if ((e = cudaMemsetAsync(L.d_r, 0, n * vb, mg.stream)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(L.d_x, 0, n * vb, mg.stream)) != cudaSuccess) break;
    std::vector<int> tiles = {mg.vanka_tile};
    // smaller tiles only where one-cell chunks of whole tiles leave the GPU short of CTAs
    const long long units1 = (long long)L.hp.n_cells * ((mg.n_blk * kVankaVB + mg.vanka_tile - 1) / mg.vanka_tile);
    if (units1 < sg::sm_count() * 16)
      for (int t : {16, 8})
        if (t < mg.vanka_tile && t % kVankaVB == 0) tiles.push_back(t);
    int best_c = L.vanka_chunk, best_t = 0;
    float best_ms = 1e30f;
    for (int tile : tiles) {
      const int max_c = vanka_chunk(L, mg.n_blk, tile, vb, inv_value_bytes(mg),
                                    tile == mg.vanka_tile
                                        ? std::max<size_t>(100 * 1024, vanka_smem(L, mg.n_blk, tile, L.vanka_chunk, vb,
                                                                                 inv_value_bytes(mg)))
                                        : 100 * 1024);
      if (max_c == 0) continue;
      std::vector<int> cand;
      for (int c = 1; c <= max_c; c *= 2) cand.push_back(c);
      if (cand.back() != max_c) cand.push_back(max_c);
      for (int c : cand) {
        if (e != cudaSuccess) break;
        L.vanka_chunk = c;
        L.vanka_tile = tile == mg.vanka_tile ? 0 : tile;
        const float ms = time_candidate(
            [&]() { return vk_launch(mg, L, mg.stream) ? cudaSuccess : cudaErrorInvalidValue; }, mg.stream, a, b, e);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best_c = c;
          best_t = L.vanka_tile;
        }
      }
    }
    L.vanka_chunk = L.ffma_chunk = best_c;
    L.vanka_tile = L.ffma_tile = best_t;
    L.vanka_kind = 0;
    // the tensor-core sweep over its chunk sizes, where it applies; kept if faster
    const int tile_all = mg.vanka_tile;
    if (e == cudaSuccess && tc_level_ok(mg, L, tile_all)) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      int tc_c = 0;
      float tc_ms = 1e30f;
      for (int c : {1, 2}) {                     // one or two staging buffers
        if (e != cudaSuccess) break;
        if (vanka_tc_smem(L.hp.dim, L.hp.k, L.hp.n_t, c, std::min(tile_all, mg.n_blk * kVankaVB)) >
            (size_t)optin - 1024)
          break;
        L.vanka_chunk = c;
        L.vanka_tile = 0;
        L.vanka_kind = 1;
        const float ms = time_candidate(
            [&]() { return vk_launch(mg, L, mg.stream) ? cudaSuccess : cudaErrorInvalidValue; }, mg.stream, a, b, e);
        if (e == cudaSuccess && ms < tc_ms) {
          tc_ms = ms;
          tc_c = c;
        }
      }
      if (tc_c > 0 && tc_ms < best_ms) {
        L.vanka_chunk = tc_c;
        L.vanka_tile = 0;
        L.vanka_kind = 1;
      } else {
        L.vanka_chunk = best_c;
        L.vanka_tile = best_t;
        L.vanka_kind = 0;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

void mg_free(MG& mg) {
  for (int t = 0; t < 2; ++t) {
    if (mg.exec_t[t]) cudaGraphExecDestroy(mg.exec_t[t]);
    if (mg.graph_t[t]) cudaGraphDestroy(mg.graph_t[t]);
    mg.exec_t[t] = nullptr;
    mg.graph_t[t] = nullptr;
  }
  if (mg.stream) cudaStreamDestroy(mg.stream);
  cudaFree(mg.d_cls);
  cudaFree(mg.d_blk_cls);
  cudaFree(mg.d_blk_alpha);
  cudaFree(mg.d_wgt);
  cudaFree(mg.d_status);
  mg.d_wgt = nullptr;
  mg.d_status = nullptr;
  mg.d_blk_cls = mg.d_blk_alpha = nullptr;
  for (MGLevel& L : mg.lv) {
    cudaFree(L.d_ctab); cudaFree(L.d_grow); cudaFree(L.d_gcol); cudaFree(L.d_gterm); cudaFree(L.d_gval);
    cudaFree(L.d_perm); cudaFree(L.d_inv); cudaFree(L.d_inner); cudaFree(L.d_amq); cudaFree(L.d_amqT);
    cudaFree(L.d_x); cudaFree(L.d_b); cudaFree(L.d_r); cudaFree(L.d_t1); cudaFree(L.d_t2);
    for (int d = 0; d < 3; ++d) {
      cudaFree(L.d_pidx[d]); cudaFree(L.d_pwl[d]);
      cudaFree(L.d_ridx[d]); cudaFree(L.d_rw[d]);
    }
  }
  mg.lv.clear();
  mg.stream = nullptr;
  mg.d_cls = nullptr;
}

sg_status mg_build(const HostProblem& fine, int precision, int nu, double omega, MG& mg, std::string& msg,
                   bool single_class) {
  const auto t0 = std::chrono::steady_clock::now();
  mg.requested = precision;
  mg.bf16 = precision == SG_PREC_BF16;
  if (mg.bf16) precision = kPrecF32;          // FP32 vectors, bf16-stored patch inverses
  mg.precision = precision;
  mg.nu = nu;
  mg.omega = omega;
  // diagonal classes of the chaos rows
  GTable gdiag;
  std::vector<std::vector<double>> drow;
  diagonal_table(fine, gdiag, drow);
  std::map<std::vector<double>, int> key;
  std::vector<std::vector<double>> class_diag;
  mg.cls.assign(fine.n_xi, 0);
  for (int a = 0; a < fine.n_xi; ++a) {
    auto it = key.find(drow[a]);
    if (it == key.end()) {
      key[drow[a]] = (int)class_diag.size();
      mg.cls[a] = (int)class_diag.size();
      class_diag.push_back(drow[a]);
    } else {
      mg.cls[a] = it->second;
    }
  }
  if (single_class) {
    // the mean block: coefficient term with the zero chaos index, weight 1
    std::vector<double> mean_diag(fine.n_terms, 0.0);
    for (int t = 0; t < fine.n_terms; ++t)
      if (std::all_of(fine.mus[t].begin(), fine.mus[t].end(), [](int v) { return v == 0; })) mean_diag[t] = 1.0;
    class_diag.assign(1, mean_diag);
    std::fill(mg.cls.begin(), mg.cls.end(), 0);
  }
  mg.n_classes = (int)class_diag.size();
  // Vanka mode blocks: the modes of one class, kVankaVB at a time
  std::vector<int> blk_cls, blk_alpha;
  for (int c = 0; c < mg.n_classes; ++c) {
    std::vector<int> modes;
    for (int a = 0; a < fine.n_xi; ++a)
      if (mg.cls[a] == c) modes.push_back(a);
    for (size_t i = 0; i < modes.size(); i += kVankaVB) {
      blk_cls.push_back(c);
      for (int u = 0; u < kVankaVB; ++u) blk_alpha.push_back(i + u < modes.size() ? modes[i + u] : -1);
    }
  }
  mg.n_blk = (int)blk_cls.size();
  // slots per Vanka tile: every block, or (Monte-Carlo batches) the requested
  // number of samples
  if (mg.vanka_tile <= 0 || !mg.mc || mg.vanka_tile > mg.n_blk * kVankaVB) mg.vanka_tile = mg.n_blk * kVankaVB;
  // level problems
  std::vector<HostProblem> hps;
  hps.push_back(fine);
  while (true) {
    const HostProblem& f = hps.back();
    bool ok = true;
    for (int d = 0; d < f.dim; ++d) ok = ok && f.cells[d] % 2 == 0 && f.cells[d] > 2;
    if (!ok) break;
    // a level small enough for the dense coarse solve ends the hierarchy
    long long inner = f.n_t;
    for (int d = 0; d < f.dim; ++d) inner *= std::max(0, f.nn[d] - 2);
    if (mg.coarse_dofs > 0 && inner <= mg.coarse_dofs) break;
    sg_mesh m;
    std::memset(&m, 0, sizeof(m));
    m.dim = f.dim;
    for (int d = 0; d < 3; ++d) {
      m.cells[d] = d < f.dim ? f.cells[d] / 2 : 1;
      m.lo[d] = f.lo[d];
      m.hi[d] = f.lo[d] + f.h[d] * f.cells[d];
    }
    std::vector<Piece> pieces = f.pieces;
    for (Piece& pc : pieces) pc.scale = coarsen_scale(pc.scale, f);
    HostProblem c;
    sg_status st = build_host_problem_pieces(&m, f.k, f.r, f.n_slabs, f.T, f.M, f.p, pieces, c, msg);
    if (st != SG_OK) return st;
    // every level carries the rows of the fine problem (chaos modes, or the
    // samples of a Monte-Carlo batch): same count, same coupling table
    c.n_xi = fine.n_xi;
    c.idx = fine.idx;
    hps.push_back(std::move(c));
  }
  for (const HostProblem& h : hps)
    if (h.n_xi != fine.n_xi || h.n_t != fine.n_t || h.n_terms != fine.n_terms) {
      msg = "multigrid levels disagree in rows, time nodes or coefficient terms";
      return SG_ERR_ARG;
    }
  mg.lv.resize(hps.size());
  cudaError_t e = cudaSuccess;
  for (size_t l = 0; l < hps.size(); ++l) {
    MGLevel& L = mg.lv[l];
    L.hp = std::move(hps[l]);
    L.hp.g = gdiag;
    L.hp.perm.resize(L.hp.n_xi);
    for (int a = 0; a < L.hp.n_xi; ++a) L.hp.perm[a] = a;
    L.hp.precision = precision;
    L.coarsest = l + 1 == mg.lv.size();
    {
      // the level residual is the diagonal apply: time-mass tables of A_t and A_t^T
      std::vector<double> amq, amqT, At((size_t)L.hp.n_t * L.hp.n_t);
      for (int i = 0; i < L.hp.n_t; ++i)
        for (int j = 0; j < L.hp.n_t; ++j) At[(size_t)i * L.hp.n_t + j] = L.hp.A_hat[(size_t)j * L.hp.n_t + i];
      mc_amq(L.hp, L.hp.A_hat, amq);
      mc_amq(L.hp, At, amqT);
      if ((e = upload_vec(&L.d_amq, amq)) != cudaSuccess) break;
      if ((e = upload_vec(&L.d_amqT, amqT)) != cudaSuccess) break;
      if ((e = prepare_mc_kernel(precision, L.hp.dim, L.hp.k, L.hp.n_t)) != cudaSuccess) break;
      if (level_diag_shape(L, mg.mc ? mg.mc_ts : std::min(L.hp.n_xi, 32), 8, precision == kPrecF32 ? 4 : 8) != SG_OK) {
        msg = "multigrid level tile does not fit in shared memory";
        return SG_ERR_UNSUPPORTED;
      }
      // the SG cell kernel with the diagonal coupling table, where it applies
      std::string m2;
      L.chunk_ok = !mg.mc && plan_apply(L.hp, L.ls, m2) == SG_OK;
      if (L.chunk_ok && (e = prepare_apply_kernel(precision, L.hp.dim, L.hp.k, L.hp.n_t, L.ls.smem)) != cudaSuccess) break;
      L.use_diag = !L.chunk_ok;
    }
    const int n = L.hp.k + 1;
    const int nkd = L.hp.dim == 2 ? n * n : n * n * n;
    L.np = L.hp.n_t * nkd;
    if (L.coarsest) {
      const ElementData ed = element_data(L.hp);
      std::vector<double> inv;
      std::vector<long long> node_of;
      for (long long m = 0; m < L.hp.n_x; ++m) {
        const int g[3] = {(int)(m % L.hp.nn[0]), (int)((m / L.hp.nn[0]) % L.hp.nn[1]),
                          (int)(m / ((long long)L.hp.nn[0] * L.hp.nn[1]))};
        if (node_interior(L.hp, g)) node_of.push_back(m);
      }
      L.n_int = L.hp.n_t * (int)node_of.size();
      if (L.n_int > 2048 || L.n_int * sizeof(double) > 48 * 1024) {
        msg = "coarsest multigrid level too large (mesh cannot be coarsened enough)";
        return SG_ERR_UNSUPPORTED;
      }
      std::vector<long long> inner_dofs;
      for (int i = 0; i < L.hp.n_t; ++i)
        for (long long m : node_of) inner_dofs.push_back((long long)i * L.hp.n_x + m);
      for (int c = 0; c < mg.n_classes; ++c) {
        std::vector<double> ci;
        if (!coarse_inverse(L.hp, ed, class_diag[c], node_of, ci)) { msg = "singular coarse operator"; return SG_ERR_ARG; }
        inv.insert(inv.end(), ci.begin(), ci.end());
      }
      if ((e = upload_vec(reinterpret_cast<long long**>(&L.d_inner), inner_dofs)) != cudaSuccess) break;
      if ((e = upload_values(&L.d_inv, inv, precision)) != cudaSuccess) break;
    }
    // level apply tables (coefficient stays double; vectors use the MG precision)
    if ((e = upload_vec(reinterpret_cast<double**>(&L.d_ctab), L.hp.ctab)) != cudaSuccess) break;
    if (!L.coarsest) {
      // Vanka patch inverses, assembled and factored on the device
      const int npp = vanka_row_pitch(L.np);
      const int kind = mg.bf16 ? 2 : precision == kPrecF32 ? 1 : 0;
      const size_t wb = kind == 2 ? sizeof(__nv_bfloat16) : kind == 1 ? sizeof(float) : sizeof(double);
      if ((e = cudaMalloc(&L.d_inv, (size_t)mg.n_classes * L.hp.n_cells * L.np * npp * wb)) != cudaSuccess) break;
      bool singular = false;
      const auto tf = std::chrono::steady_clock::now();
      if ((e = vanka_factor(L.hp, static_cast<const double*>(L.d_ctab), class_diag, kind, L.d_inv, npp, singular,
                            0)) != cudaSuccess)
        break;
      mg.factor_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf).count();
      if (singular) {
        msg = "singular Vanka patch";
        return SG_ERR_ARG;
      }
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const size_t vb = precision == kPrecF32 ? 4 : 8;
      L.vanka_chunk = vanka_chunk(L, mg.n_blk, mg.vanka_tile, vb, inv_value_bytes(mg), 100 * 1024);
      if (L.vanka_chunk == 0)
        L.vanka_chunk = vanka_chunk(L, mg.n_blk, mg.vanka_tile, vb, inv_value_bytes(mg), (size_t)optin - 1024);
      if (L.vanka_chunk == 0) {
        msg = "Vanka smoother: one cell with all rows does not fit in shared memory (fewer samples per batch)";
        return SG_ERR_UNSUPPORTED;
      }
      L.ffma_chunk = L.vanka_chunk;
      if ((e = prepare_vanka(L.hp.dim, L.hp.k, L.hp.n_t, precision == kPrecF32, mg.bf16)) != cudaSuccess) break;
      if (mg.bf16 && (e = prepare_vanka_tc(L.hp.dim, L.hp.k, L.hp.n_t)) != cudaSuccess) break;
    }
    if ((e = upload_vec(&L.d_grow, L.hp.g.row)) != cudaSuccess) break;
    if ((e = upload_vec(&L.d_gcol, L.hp.g.col)) != cudaSuccess) break;
    if ((e = upload_vec(&L.d_gterm, L.hp.g.term)) != cudaSuccess) break;
    if ((e = upload_vec(&L.d_gval, L.hp.g.val)) != cudaSuccess) break;
    if ((e = upload_vec(&L.d_perm, L.hp.perm)) != cudaSuccess) break;
    const size_t vb = precision == kPrecF32 ? 4 : 8;
    const size_t bytes = (size_t)L.hp.n_xi * L.hp.n_t * L.hp.n_x * vb;
    if ((e = cudaMalloc(&L.d_x, bytes)) != cudaSuccess) break;
    if ((e = cudaMalloc(&L.d_b, bytes)) != cudaSuccess) break;
    if ((e = cudaMalloc(&L.d_r, bytes)) != cudaSuccess) break;
    if (l > 0) {
      MGLevel& F = mg.lv[l - 1];
      for (int d = 0; d < F.hp.dim; ++d) {
        std::vector<int> pptr, pidx, rptr, ridx;
        std::vector<double> pwl, rw;
        transfer_1d(F.hp, L.hp, d, pptr, pidx, pwl, rptr, ridx, rw);
        int pm = 0, rm = 0;
        for (size_t i = 0; i + 1 < pptr.size(); ++i) pm = std::max(pm, pptr[i + 1] - pptr[i]);
        for (size_t j = 0; j + 1 < rptr.size(); ++j) rm = std::max(rm, rptr[j + 1] - rptr[j]);
        if (pm > kAxisMax || rm > kAxisMax) {
          e = cudaErrorInvalidValue;
          break;
        }
        F.pmax[d] = axis_width(pm);
        F.rmax[d] = axis_width(rm);
        std::vector<int> pi, ri;
        std::vector<double> pwv, rwv;
        pad_lists(pptr, pidx, pwl, F.pmax[d], pi, pwv);
        pad_lists(rptr, ridx, rw, F.rmax[d], ri, rwv);
        if ((e = upload_vec(&F.d_pidx[d], pi)) != cudaSuccess) break;
        if ((e = upload_values(&F.d_pwl[d], pwv, precision)) != cudaSuccess) break;
        if ((e = upload_vec(&F.d_ridx[d], ri)) != cudaSuccess) break;
        if ((e = upload_values(&F.d_rw[d], rwv, precision)) != cudaSuccess) break;
      }
      if (e != cudaSuccess) break;
      // intermediate arrays of the separable transfers between F and this level
      {
        const long long V = (long long)F.hp.n_xi * F.hp.n_t;
        const long long t1 = V * F.hp.nn[2] * F.hp.nn[1] * L.hp.nn[0];
        const long long t2 = F.hp.dim == 3 ? V * F.hp.nn[2] * L.hp.nn[1] * L.hp.nn[0] : 1;
        if ((e = cudaMalloc(&F.d_t1, t1 * vb)) != cudaSuccess) break;
        if ((e = cudaMalloc(&F.d_t2, t2 * vb)) != cudaSuccess) break;
      }
      if (e != cudaSuccess) break;
    }
  }
  if (e == cudaSuccess && !mg.d_wgt) {
    // per-row weights of the diagonal level apply: G_mu[alpha][alpha]
    std::vector<double> wgt((size_t)fine.n_xi * fine.n_terms);
    for (int a = 0; a < fine.n_xi; ++a)
      for (int t = 0; t < fine.n_terms; ++t) wgt[(size_t)a * fine.n_terms + t] = drow[a][t];
    e = upload_vec(&mg.d_wgt, wgt);
  }
  if (e == cudaSuccess) e = upload_vec(&mg.d_cls, mg.cls);
  if (e == cudaSuccess) e = upload_vec(&mg.d_blk_cls, blk_cls);
  if (e == cudaSuccess) e = upload_vec(&mg.d_blk_alpha, blk_alpha);
  if (e == cudaSuccess) e = cudaMalloc(&mg.d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(mg.d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mg.stream, cudaStreamNonBlocking);
  const auto tt = std::chrono::steady_clock::now();
  if (e == cudaSuccess) e = tune_level_applies(mg);
  if (e == cudaSuccess) e = tune_vanka(mg);
  mg.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tt).count();
  if (e == cudaSuccess) {
    int status = 0;
    e = cudaMemcpy(&status, mg.d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && status != 0) {
      msg = "multigrid set-up: a tensor-core Vanka sweep timed out waiting for its MMAs";
      return SG_ERR_TIMEOUT;
    }
  }
  if (e != cudaSuccess) {
    msg = std::string("multigrid set-up: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  mg.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return SG_OK;
}

sg_status mg_build_mc(const HostProblem& fine, int precision, int nu, double omega, const std::vector<double>& wgt,
                      int ts, MG& mg, std::string& msg) {
  if (ts < 1 || (size_t)fine.n_xi * fine.n_terms != wgt.size()) {
    msg = "Monte-Carlo weights or tile size inconsistent";
    return SG_ERR_ARG;
  }
  mg.mc = true;
  mg.mc_ts = std::min(ts, fine.n_xi);
  // Vanka tiles: a multiple of 8 samples whose patch data fit beside each other
  mg.vanka_tile = std::min(fine.n_xi, 64);
  if (mg.vanka_tile < fine.n_xi) mg.vanka_tile = 64;
  cudaError_t e = upload_vec(&mg.d_wgt, wgt);
  if (e != cudaSuccess) {
    msg = cudaGetErrorString(e);
    return SG_ERR_CUDA;
  }
  return mg_build(fine, precision, nu, omega, mg, msg, true);
}

sg_status mg_level_info(const MG& mg, int level, int info[10], std::string& msg) {
  if (level < 0 || level >= (int)mg.lv.size()) {
    msg = "level out of range";
    return SG_ERR_ARG;
  }
  const MGLevel& L = mg.lv[level];
  info[0] = (int)mg.lv.size();
  info[1] = (int)L.hp.n_cells;
  info[2] = L.coarsest ? 1 : 0;
  info[3] = L.coarsest ? -1 : (L.use_diag ? 1 : 0);
  info[4] = L.coarsest ? 0 : L.vanka_chunk;
  info[5] = L.coarsest ? 0 : (L.vanka_tile > 0 ? L.vanka_tile : mg.vanka_tile);
  info[6] = L.np;
  info[7] = mg.n_classes;
  info[8] = L.coarsest ? 0 : L.vanka_kind;
  info[9] = 0;
  return SG_OK;
}

sg_status mg_force_variant(MG& mg, int level, int residual_kind, int chunk, int tile, int kind, std::string& msg) {
  if (level < -1 || level >= (int)mg.lv.size()) {
    msg = "level out of range";
    return SG_ERR_ARG;
  }
  if (residual_kind < -1 || residual_kind > 1 || chunk < 0 || chunk > 8 || tile < -1 || kind < -1 || kind > 1) {
    msg = "variant out of range";
    return SG_ERR_ARG;
  }
  const size_t vb = mg.precision == kPrecF32 ? 4 : 8;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // check every level first, then change them
  for (int pass = 0; pass < 2; ++pass) {
    for (int l = 0; l < (int)mg.lv.size(); ++l) {
      if (level >= 0 && l != level) continue;
      MGLevel& L = mg.lv[l];
      if (L.coarsest) {
        if (level >= 0) {
          msg = "the coarsest level has no smoother";
          return SG_ERR_ARG;
        }
        continue;
      }
      if (residual_kind == 0 && !L.chunk_ok) {
        msg = "the SG cell kernel has no launch shape on this level";
        return SG_ERR_UNSUPPORTED;
      }
      const int kd = kind >= 0 ? kind : L.vanka_kind;
      // "keep" of a sweep that is not running: the FFMA sweep's last chunk and
      // tile, two staging buffers and all modes for the tensor-core sweep
      const int keep = kd == L.vanka_kind ? L.vanka_chunk : (kd == 0 ? L.ffma_chunk : 2);
      const int keep_tile = kd == L.vanka_kind ? L.vanka_tile : (kd == 0 ? L.ffma_tile : 0);
      const int t = tile < 0 ? (keep_tile > 0 ? keep_tile : mg.vanka_tile) : (tile == 0 ? mg.vanka_tile : tile);
      if (t != mg.vanka_tile && (t % kVankaVB != 0 || t > mg.vanka_tile)) {
        msg = "mode tiles are multiples of 4 slots, at most all of them";
        return SG_ERR_ARG;
      }
      int c = chunk > 0 ? std::min(chunk, L.hp.cells[0]) : keep;
      if (kd == 1) c = std::max(1, std::min(chunk > 0 ? chunk : c, 2));   // staging buffers of the tensor-core sweep
      if (c <= 0) c = 1;
      if (kd == 1) {
        if (!tc_level_ok(mg, L, t)) {
          msg = "the tensor-core Vanka sweep needs bf16 factors, one diagonal class, a patch of at most 64 and "
                "at most 80 slots per tile";
          return SG_ERR_UNSUPPORTED;
        }
        if (vanka_tc_smem(L.hp.dim, L.hp.k, L.hp.n_t, c, std::min(t, mg.n_blk * kVankaVB)) > (size_t)optin - 1024) {
          msg = "Vanka chunk does not fit in shared memory";
          return SG_ERR_UNSUPPORTED;
        }
      } else if (vanka_smem(L, mg.n_blk, t, c, vb, inv_value_bytes(mg)) > (size_t)optin - 1024) {
        msg = "Vanka chunk does not fit in shared memory";
        return SG_ERR_UNSUPPORTED;
      }
      if (pass == 1) {
        if (residual_kind >= 0) L.use_diag = residual_kind == 1;
        L.vanka_chunk = c;
        L.vanka_tile = t == mg.vanka_tile ? 0 : t;
        L.vanka_kind = kd;
        if (kd == 0) {
          L.ffma_chunk = c;
          L.ffma_tile = L.vanka_tile;
        }
      }
    }
  }
  // the captured V-cycles hold the old launches
  for (int t = 0; t < 2; ++t) {
    if (mg.exec_t[t]) cudaGraphExecDestroy(mg.exec_t[t]);
    if (mg.graph_t[t]) cudaGraphDestroy(mg.graph_t[t]);
    mg.exec_t[t] = nullptr;
    mg.graph_t[t] = nullptr;
  }
  return SG_OK;
}

sg_status mg_patch_inverse(const MG& mg, int level, int alpha, long long cell, double* out, std::string& msg) {
  if (level < 0 || level >= (int)mg.lv.size() || mg.lv[level].coarsest) {
    msg = "level out of range (or the coarsest level)";
    return SG_ERR_ARG;
  }
  const MGLevel& L = mg.lv[level];
  if (alpha < 0 || alpha >= (int)mg.cls.size() || cell < 0 || cell >= L.hp.n_cells) {
    msg = "mode or cell out of range";
    return SG_ERR_ARG;
  }
  const int np = L.np, npp = vanka_row_pitch(np);
  const size_t off = ((size_t)mg.cls[alpha] * L.hp.n_cells + (size_t)cell) * np * npp;
  const size_t cnt = (size_t)np * npp;
  std::vector<double> row(cnt);
  cudaError_t e;
  if (mg.bf16) {
    std::vector<__nv_bfloat16> v(cnt);
    e = cudaMemcpy(v.data(), static_cast<const __nv_bfloat16*>(L.d_inv) + off, cnt * sizeof(__nv_bfloat16),
                   cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < cnt; ++i) row[i] = (double)__bfloat162float(v[i]);
  } else if (mg.precision == kPrecF32) {
    std::vector<float> v(cnt);
    e = cudaMemcpy(v.data(), static_cast<const float*>(L.d_inv) + off, cnt * sizeof(float), cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < cnt; ++i) row[i] = v[i];
  } else {
    e = cudaMemcpy(row.data(), static_cast<const double*>(L.d_inv) + off, cnt * sizeof(double),
                   cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    msg = cudaGetErrorString(e);
    return SG_ERR_CUDA;
  }
  for (int r = 0; r < np; ++r)
    for (int c = 0; c < np; ++c) out[(size_t)r * np + c] = row[(size_t)r * npp + c];
  return SG_OK;
}

cudaError_t mg_issue(MG& mg, const double* r, double* z, cudaStream_t stream, int trans) {
  MGLevel& L0 = mg.lv[0];
  const long long n = (long long)L0.hp.n_xi * L0.hp.n_t * L0.hp.n_x;
  const bool f32 = mg.precision == kPrecF32;
  const int t = trans ? 1 : 0;
  cudaError_t e;
  if (f32)
    mg_convert<double, float><<<grid_for(n, 256), 256, 0, stream>>>(r, static_cast<float*>(L0.d_b), n);
  else
    mg_convert<double, double><<<grid_for(n, 256), 256, 0, stream>>>(r, static_cast<double*>(L0.d_b), n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = f32 ? issue_vcycle<float>(mg, 0, stream, t) : issue_vcycle<double>(mg, 0, stream, t)) != cudaSuccess)
    return e;
  if (f32)
    mg_convert<float, double><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const float*>(L0.d_x), z, n);
  else
    mg_convert<double, double><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const double*>(L0.d_x), z, n);
  return cudaGetLastError();
}

cudaError_t mg_apply(MG& mg, const double* r, double* z, cudaStream_t stream, int trans) {
  MGLevel& L0 = mg.lv[0];
  const long long n = (long long)L0.hp.n_xi * L0.hp.n_t * L0.hp.n_x;
  const bool f32 = mg.precision == kPrecF32;
  const int t = trans ? 1 : 0;
  cudaError_t e;
  if (!mg.exec_t[t]) {
    if ((e = cudaStreamBeginCapture(mg.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t ei = f32 ? issue_vcycle<float>(mg, 0, mg.stream, t) : issue_vcycle<double>(mg, 0, mg.stream, t);
    e = cudaStreamEndCapture(mg.stream, &mg.graph_t[t]);
    if (ei != cudaSuccess) return ei;
    if (e != cudaSuccess) return e;
    if ((e = cudaGraphInstantiate(&mg.exec_t[t], mg.graph_t[t], 0)) != cudaSuccess) return e;
  }
  if (f32)
    mg_convert<double, float><<<grid_for(n, 256), 256, 0, stream>>>(r, static_cast<float*>(L0.d_b), n);
  else
    mg_convert<double, double><<<grid_for(n, 256), 256, 0, stream>>>(r, static_cast<double*>(L0.d_b), n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaGraphLaunch(mg.exec_t[t], stream)) != cudaSuccess) return e;
  if (f32)
    mg_convert<float, double><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const float*>(L0.d_x), z, n);
  else
    mg_convert<double, double><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const double*>(L0.d_x), z, n);
  return cudaGetLastError();
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_mg)

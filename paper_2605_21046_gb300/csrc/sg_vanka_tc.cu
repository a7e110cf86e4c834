// Vanka sweep on the tensor cores (tcgen05) for bf16-stored patch inverses.
//
// The additive Vanka step of the multigrid levels (paper, Sec. 3.5 remark:
// local space-time patch problems) is, per cell, a dense product
//     Z = inv * R,   inv: NP x NP patch inverse (bf16),  R: NP x modes,
// followed by the damped, multiplicity-weighted sum of the cells' corrections.
// Here every cell's product is one chain of tcgen05.mma (kind::f16, FP32
// accumulation in tensor memory), issued by one thread:
//   * A = inv, M = 128 rows (NP <= 64 used, the rest zero), K = 64 (NP padded
//     with zeros), staged by asynchronous 16-byte copies straight from the
//     stored rows into the canonical no-swizzle K-major layout (8-row x 16-byte
//     core matrices);
//   * B = R split into three bf16 terms R = R1 + R2 + R3 (each the bf16
//     rounding of what the previous ones leave), side by side along N: the
//     bf16 x bf16 products are exact and accumulate in FP32, so the product
//     carries about the FP32 accuracy of the patch values;
//   * D (128 lanes x N columns of FP32 in tensor memory) is read back with
//     tcgen05.ld by the two warps whose lanes hold the patch rows, the three
//     split columns summed, and the corrections added into a shared-memory
//     accumulator.
// Two D / B buffers let cell c's MMAs run while cell c-1 is read back.  Units
// (a chunk of cells and a tile of modes) are double buffered as in the FFMA
// sweep: the next unit's inverses and r are copied in while one is computed.
// Waits on the MMA completion barrier are bounded; if one runs out the kernel
// records SG_ERR_TIMEOUT, stops issuing work, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sg_bounds.h"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;                  // MMA rows (patch rows; NP <= 64 are used)
constexpr int kTcK = 64;                   // patch columns, zero padded
constexpr int kTcACell = kTcM * kTcK * 2;  // bytes of one cell's A tile
constexpr int kTcLboA = (kTcM / 8) * 128;  // A: bytes between the 8-value K chunks
constexpr int kTcVB = 4;                   // slots per mode block
constexpr unsigned int kTcSpin = 1u << 22; // bound of a completion wait (polls)

struct TcParams {
  const float* r;
  float* x;
  const __nv_bfloat16* inv;
  const int* blk_alpha;     // [n_blk][kTcVB] modes, -1 padded
  int* status;              // SG_ERR_TIMEOUT is recorded here
  int n_blk, chunk, npp, tile_blocks, n_tiles, ncols, tmem_cols;
  long long n_x, n_cells, n_vec_x, inv_count;
  int cells[3], nn[3];
  float omega;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16_tc(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4_tc(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit_tc() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1_tc() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0_tc() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// shared-memory matrix descriptor: no swizzle, K-major; lbo = bytes between
// core matrices along K, sbo = bytes between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                  // descriptor version
  return d;                                // base offset 0, no swizzle
}
// instruction descriptor of kind::f16: FP32 D, bf16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

struct TcUnit {
  int cx0, cy, cz, nc, b0, nb;
  long long cell0;
};

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(kTcThreads, 2) mg_vanka_tc(const TcParams p) {
  constexpr int N = K + 1;
  constexpr int NKD = DIM == 2 ? N * N : N * N * N;
  constexpr int NP = NT * NKD;
  static_assert(NP <= kTcK, "patch larger than the MMA K extent");
  constexpr int LYZ = DIM == 2 ? N : N * N;
  constexpr int RPC = (NP * 2 + 15) / 16;        // 16-byte pieces of a stored row that hold values
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int C = p.chunk, LX = C * K + 1, LN = LX * LYZ, E = NT * LN;
  const int SL = p.tile_blocks * kTcVB;           // slots of a tile
  const int NCOL = p.ncols;                       // MMA N: 3 SL rounded up to 16
  const int BBYTES = NCOL * kTcK * 2;             // one B buffer
  const uint32_t LBO_B = (uint32_t)(NCOL / 8) * 128u;
  // shared memory: two stages of A tiles, two B buffers, corrections, two
  // stages of r, two stages of node / slot tables
  unsigned char* A0 = smem_raw;                                    // 2 x C x kTcACell
  unsigned char* Bb = A0 + (size_t)2 * C * kTcACell;               // 2 x BBYTES
  float* Zc = reinterpret_cast<float*>(Bb + (size_t)2 * BBYTES);   // [NT][LN][SL]
  float* Rl0 = Zc + (size_t)E * SL;                                // 2 x [NT][LN][SL]
  int* Gn0 = reinterpret_cast<int*>(Rl0 + (size_t)2 * E * SL);     // 2 x [LN]
  int* Sm0 = Gn0 + 2 * LN;                                         // 2 x [SL]
  const int nnx = p.nn[0], nny = p.nn[1], nnz_ = p.nn[2];
  const int cpr = (p.cells[0] + C - 1) / C;
  const unsigned int n_chunks = (unsigned int)(cpr * p.cells[1] * p.cells[2]);
  const unsigned int n_units = n_chunks * (unsigned int)p.n_tiles;
  const uint32_t idesc = idesc_bf16(kTcM, NCOL);

  // tensor memory (one warp), completion barriers, zeroed operands
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem_raw);
    const size_t n16 = ((size_t)2 * C * kTcACell + (size_t)2 * BBYTES) / 16;
    for (size_t i = tid; i < n16; i += kTcThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < E * SL; i += kTcThreads) Zc[i] = 0.0f;
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = s_tmem;
  uint32_t phase_bits = 0u;                       // parity of the next completion, per barrier

  auto decode = [&](unsigned int unit, TcUnit& U) {
    const unsigned int ch = unit % n_chunks;
    const int tile = (int)(unit / n_chunks);
    U.b0 = tile * p.tile_blocks;
    U.nb = min(p.tile_blocks, p.n_blk - U.b0);
    U.cx0 = (int)(ch % (unsigned int)cpr) * C;
    const unsigned int row = ch / (unsigned int)cpr;
    U.cy = (int)(row % (unsigned int)p.cells[1]);
    U.cz = (int)(row / (unsigned int)p.cells[1]);
    U.nc = min(C, p.cells[0] - U.cx0);
    U.cell0 = ((long long)U.cz * p.cells[1] + U.cy) * p.cells[0] + U.cx0;
  };
  auto tables = [&](const TcUnit& U, int* Gn, int* Sm) {
    const int lxn = U.nc * K + 1;
    for (int ln = tid; ln < LN; ln += kTcThreads) {
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
    for (int sl = tid; sl < SL; sl += kTcThreads) Sm[sl] = sl < U.nb * kTcVB ? p.blk_alpha[U.b0 * kTcVB + sl] : -1;
  };
  // the unit's inverses into the canonical A layout, r onto the node grid
  auto stage = [&](const TcUnit& U, unsigned char* A, float* Rl, const int* Gn, const int* Sm) {
    const long long ibeg = U.cell0 * NP * p.npp;
    for (int idx = tid; idx < U.nc * NP * RPC; idx += kTcThreads) {
      const int rr = idx / RPC, kc = idx - rr * RPC;
      const int c = rr / NP, row = rr - c * NP;
      const long long g = ibeg + (long long)rr * p.npp + kc * 8;
      if (!SG_IN(g + 7, p.inv_count, 601)) continue;
      cp_async16_tc(A + (size_t)c * kTcACell + (size_t)kc * kTcLboA + (row >> 3) * 128 + (row & 7) * 16, p.inv + g);
    }
    for (int idx = tid; idx < SL * E; idx += kTcThreads) {
      const int sl = idx / E, e = idx - sl * E;
      int i = 0;
#pragma unroll
      for (int j = 1; j < NT; ++j) i += e >= j * LN;
      const int ln = e - i * LN;
      const int mode = Sm[sl], node = Gn[ln];
      const long long gi = ((long long)mode * NT + i) * p.n_x + node;
      float* dst = Rl + (size_t)e * SL + sl;
      if (mode >= 0 && node >= 0 && SG_IN(gi, p.n_vec_x, 602)) cp_async4_tc(dst, p.r + gi);
      else *dst = 0.0f;
    }
  };
  // B of one cell: the three bf16 terms of its patch values, slot s of term
  // t in MMA column t SL + s, patch column q in K
  auto build_b = [&](const float* Rl, int c, unsigned char* B) {
    const int half = (NP + 1) / 2;
    for (int it = tid; it < half * SL; it += kTcThreads) {
      const int kp = it % half, s = it / half;
      const int q0 = 2 * kp;
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = q0 + h;
        v[h] = 0.0f;
        if (q < NP) {
          const int iq = q / NKD, aq = q - iq * NKD;
          const int ax = aq % N, ayz = aq / N;
          v[h] = Rl[(size_t)(iq * LN + c * K + ax + LX * ayz) * SL + s];
        }
      }
      const int kc = q0 >> 3, kw = q0 & 7;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        __nv_bfloat16 b[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          b[h] = __float2bfloat16_rn(v[h]);
          v[h] -= __bfloat162float(b[h]);
        }
        const int n = t * SL + s;
        __nv_bfloat162 pr;
        pr.x = b[0];
        pr.y = b[1];
        *reinterpret_cast<__nv_bfloat162*>(B + (size_t)kc * LBO_B + (n >> 3) * 128 + (n & 7) * 16 + kw * 2) = pr;
      }
    }
  };
  // wait (bounded) for the MMAs committed to barrier b
  auto wait_mma = [&](int b) {
    if (s_fail) return;
    unsigned int polls = 0;
    while (!mbar_test(&s_bar[b], (phase_bits >> b) & 1u)) {
      if (++polls > kTcSpin) {
        atomicExch(&s_fail, 1);
        atomicExch(p.status, (int)SG_ERR_TIMEOUT);
        break;
      }
    }
    phase_bits ^= 1u << b;
  };
  // D of one cell (buffer b) into the corrections
  auto read_back = [&](const TcUnit& U, const int* Gn, int c, int b) {
    wait_mma(b);
    tc_after_sync();
    // warp-uniform: tcgen05.ld is executed by all 32 lanes of a warp or none
    const int failed = __shfl_sync(0xffffffffu, s_fail, 0);
    if (warp < 2 && !failed) {
      const int rho = warp * 32 + lane;
      const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * NCOL);
      float d[16];
      const int i = rho / NKD, a = rho - i * NKD;
      const int ax = a % N, ay = (a / N) % N, az = DIM == 3 ? a / (N * N) : 0;
      const int lna = c * K + ax + LX * (ay + (DIM == 3 ? N * az : 0));
      const bool live = rho < NP && Gn[lna] >= 0 && c < U.nc;
      const int mult = (ax % K == 0 ? 2 : 1) * (ay % K == 0 ? 2 : 1) * (DIM == 3 && az % K == 0 ? 2 : 1);
      const float sc = p.omega / (float)mult;
      float* z = Zc + (size_t)(i * LN + lna) * SL;
      for (int c0 = 0; c0 < NCOL; c0 += 16) {
        tmem_ld16(base + (uint32_t)c0, d);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c0 + j;
          if (live && col < 3 * SL) {
            const int s = col % SL;
            if (SG_IN((size_t)(i * LN + lna) * SL + s, (size_t)E * SL, 603)) atomicAdd(z + s, sc * d[j]);
          }
        }
      }
    }
    tc_before_sync();
  };

  unsigned int u = blockIdx.x;
  int buf = 0;
  TcUnit cur, nxt;
  if (u < n_units) {
    decode(u, cur);
    tables(cur, Gn0, Sm0);
  }
  __syncthreads();
  if (u < n_units) stage(cur, A0, Rl0, Gn0, Sm0);
  cp_commit_tc();
  for (; u < n_units; u += gridDim.x, buf ^= 1) {
    const unsigned int un = u + gridDim.x;
    const bool has_next = un < n_units;
    __syncthreads();
    if (has_next) {
      decode(un, nxt);
      tables(nxt, Gn0 + (buf ^ 1) * LN, Sm0 + (buf ^ 1) * SL);
    }
    __syncthreads();
    if (has_next)
      stage(nxt, A0 + (size_t)(buf ^ 1) * C * kTcACell, Rl0 + (size_t)(buf ^ 1) * E * SL, Gn0 + (buf ^ 1) * LN,
            Sm0 + (buf ^ 1) * SL);
    cp_commit_tc();
    cp_wait1_tc();
    fence_async_smem();
    __syncthreads();
    const float* Rl = Rl0 + (size_t)buf * E * SL;
    const int* Gn = Gn0 + buf * LN;
    const unsigned char* A = A0 + (size_t)buf * C * kTcACell;
    for (int c = 0; c < cur.nc; ++c) {
      const int b = c & 1;
      unsigned char* B = Bb + (size_t)b * BBYTES;
      build_b(Rl, c, B);
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
      tc_after_sync();
      if (tid == 0 && !s_fail) {
        const uint32_t a_addr = smem_u32(A + (size_t)c * kTcACell), b_addr = smem_u32(B);
#pragma unroll
        for (int ks = 0; ks < kTcK / 16; ++ks) {
          const uint64_t ad = smem_desc(a_addr + (uint32_t)(ks * 2 * kTcLboA), (uint32_t)kTcLboA, 128u);
          const uint64_t bd = smem_desc(b_addr + (uint32_t)ks * 2u * LBO_B, LBO_B, 128u);
          mma_bf16(tmem + (uint32_t)(b * NCOL), ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&s_bar[b]);
      }
      if (c > 0) read_back(cur, Gn, c - 1, b ^ 1);
      __syncthreads();
    }
    if (cur.nc > 0) read_back(cur, Gn, cur.nc - 1, (cur.nc - 1) & 1);
    __syncthreads();
    // add the corrections into x and clear them
    for (int idx = tid; idx < cur.nb * kTcVB * E; idx += kTcThreads) {
      const int sl = idx / E, e = idx - sl * E;
      int i = 0;
#pragma unroll
      for (int j = 1; j < NT; ++j) i += e >= j * LN;
      const int ln = e - i * LN;
      const int mode = Sm0[buf * SL + sl], node = Gn[ln];
      float* z = Zc + (size_t)e * SL + sl;
      if (mode >= 0 && node >= 0) {
        const long long gi = ((long long)mode * NT + i) * p.n_x + node;
        if (SG_IN(gi, p.n_vec_x, 604)) atomicAdd(p.x + gi, *z);
      }
      *z = 0.0f;
    }
    cur = nxt;
  }
  cp_wait0_tc();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
}

}  // namespace

size_t vanka_tc_smem(int dim, int k, int nt, int chunk, int tile_slots) {
  const int n = k + 1, lyz = dim == 2 ? n : n * n;
  const size_t ln = (size_t)(chunk * k + 1) * lyz, e = (size_t)nt * ln;
  const int ncol = (3 * tile_slots + 15) / 16 * 16;
  return (size_t)2 * chunk * kTcACell + (size_t)2 * ncol * kTcK * 2 + 3 * e * tile_slots * sizeof(float) +
         2 * (ln + (size_t)tile_slots) * sizeof(int);
}

bool vanka_tc_eligible(int dim, int k, int nt, int tile_slots) {
  const int n = k + 1, np = nt * (dim == 2 ? n * n : n * n * n);
  return np <= kTcK && tile_slots >= kTcVB && 3 * tile_slots <= 128;
}

template <int DIM, int K, int NT>
static cudaError_t launch_tc(const TcParams& p, size_t smem, cudaStream_t s, int grid) {
  auto kern = &mg_vanka_tc<DIM, K, NT>;
  kern<<<grid, kTcThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t prepare_vanka_tc(int dim, int k, int nt) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the dynamic limit is the opt-in maximum less the kernel's static shared memory
#define SG_TP(D, KK, TT)                                                                                 \
  if (dim == D && k == KK && nt == TT) {                                                                 \
    cudaFuncAttributes fa;                                                                               \
    cudaError_t e = cudaFuncGetAttributes(&fa, &mg_vanka_tc<D, KK, TT>);                                 \
    if (e != cudaSuccess) return e;                                                                      \
    return cudaFuncSetAttribute(&mg_vanka_tc<D, KK, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                optin - (int)fa.sharedSizeBytes);                                        \
  }
  SG_TP(2, 1, 1) SG_TP(2, 1, 2) SG_TP(2, 1, 3) SG_TP(2, 1, 4)
  SG_TP(2, 2, 1) SG_TP(2, 2, 2) SG_TP(2, 2, 3) SG_TP(2, 2, 4)
  SG_TP(2, 3, 1) SG_TP(2, 3, 2) SG_TP(2, 3, 3) SG_TP(2, 3, 4)
  SG_TP(3, 1, 1) SG_TP(3, 1, 2) SG_TP(3, 2, 1) SG_TP(3, 2, 2)
#undef SG_TP
  return cudaErrorInvalidValue;
}

cudaError_t launch_vanka_tc(const HostProblem& hp, const float* r, float* x, const void* inv, const int* blk_alpha,
                            int n_blk, int chunk, int tile_slots, int* status, float omega, cudaStream_t s) {
  TcParams p{};
  p.r = r;
  p.x = x;
  p.inv = static_cast<const __nv_bfloat16*>(inv);
  p.blk_alpha = blk_alpha;
  p.status = status;
  p.n_blk = n_blk;
  p.chunk = chunk;
  const int n = hp.k + 1, np = hp.n_t * (hp.dim == 2 ? n * n : n * n * n);
  p.npp = (np + 7) / 8 * 8;
  p.tile_blocks = std::max(1, std::min(n_blk, tile_slots / kTcVB));
  p.n_tiles = (n_blk + p.tile_blocks - 1) / p.tile_blocks;
  const int sl = p.tile_blocks * kTcVB;
  p.ncols = (3 * sl + 15) / 16 * 16;
  p.tmem_cols = 32;
  while (p.tmem_cols < 2 * p.ncols) p.tmem_cols *= 2;
  p.n_x = hp.n_x;
  p.n_cells = hp.n_cells;
  p.n_vec_x = (long long)hp.n_xi * hp.n_t * hp.n_x;
  p.inv_count = hp.n_cells * (long long)np * p.npp;
  for (int d = 0; d < 3; ++d) {
    p.cells[d] = hp.cells[d];
    p.nn[d] = hp.nn[d];
  }
  p.omega = omega;
  const size_t smem = vanka_tc_smem(hp.dim, hp.k, hp.n_t, chunk, sl);
  const int cpr = (hp.cells[0] + chunk - 1) / chunk;
  const long long units = (long long)cpr * hp.cells[1] * hp.cells[2] * p.n_tiles;
  // at most two CTAs per SM: their tensor memory (2 x tmem_cols <= 512) never waits
  const int grid = (int)std::max<long long>(1, std::min<long long>(units, sm_count() * 2));
#define SG_TL(D, KK, TT) \
  if (hp.dim == D && hp.k == KK && hp.n_t == TT) return launch_tc<D, KK, TT>(p, smem, s, grid);
  SG_TL(2, 1, 1) SG_TL(2, 1, 2) SG_TL(2, 1, 3) SG_TL(2, 1, 4)
  SG_TL(2, 2, 1) SG_TL(2, 2, 2) SG_TL(2, 2, 3) SG_TL(2, 2, 4)
  SG_TL(2, 3, 1) SG_TL(2, 3, 2) SG_TL(2, 3, 3) SG_TL(2, 3, 4)
  SG_TL(3, 1, 1) SG_TL(3, 1, 2) SG_TL(3, 2, 1) SG_TL(3, 2, 2)
#undef SG_TL
  return cudaErrorInvalidValue;
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_vanka_tc)

// Vanka sweep on the tensor cores (tcgen05) for bf16-stored patch inverses.
//
// The additive Vanka step of the multigrid levels (paper, Sec. 3.5 remark:
// local space-time patch problems) is, per cell, a dense product
//     Z = inv * R,   inv: NP x NP patch inverse (bf16),  R: NP x modes,
// followed by the damped, multiplicity-weighted sum of the cells' corrections.
// The unit of work is a pair of neighbouring cells (along x) and a tile of
// chaos modes; the pair's two products are one chain of tcgen05.mma (kind::f16,
// FP32 accumulation in tensor memory) issued by one thread, as one
// block-diagonal product
//     [Z0]   [inv0   0 ] [R0]
//     [Z1] = [ 0   inv1] [R1]      M = 128 (64 rows per cell), K = 128,
// so the 128 lanes of the accumulator hold both cells' rows and all four
// warps read results back:
//   * A: each 8-value K chunk holds cell 0's NPR rows (NP rounded up to 8),
//     64 rows of zeros and cell 1's NPR rows; the K steps of cell 0 read 128
//     rows from the first, those of cell 1 from 64 rows before the second, so
//     the zero rows fill the off-diagonal blocks (rows of D past a cell's NP
//     are never read and may hold anything finite).  The stored inverse rows
//     (pitch npp, zero padded) are copied in by asynchronous 16-byte copies
//     into the canonical no-swizzle K-major layout (8-row x 16-byte core
//     matrices); K past npp stays zero.
//   * B: R split into two bf16 terms R = R1 + R2 (R1 the bf16 rounding of R,
//     R2 that of R - R1; |R - R1 - R2| <= 2^-18 |R|): the bf16 x bf16
//     products are exact and accumulate in FP32, so the product carries the
//     patch values to 2^-18, 2^9 times finer than the rounding of the stored
//     bf16 factors it multiplies.  Term t of slot s is MMA column
//     t SLP + s (SLP = the slots rounded up to 16), so one thread writes eight
//     K values of one column as a 16-byte store and consecutive slots fall in
//     consecutive core-matrix rows.  Cell 1's K chunks follow cell 0's
//     directly: where a K step of cell 0 reaches into them, A's columns are
//     zero.
//   * D (128 lanes x 2 SLP columns of FP32 in tensor memory) is read back with
//     tcgen05.ld (two loads of 16 columns give 16 slots' two terms, summed in
//     registers), damped, divided by the node's multiplicity and added into
//     x with one reduction per (patch row, slot).
// The next unit's r values and inverses are copied in while the current one
// computes: into a second buffer (two stages), or, with one buffer, r once B
// is built and the inverses once the MMAs are done.  Waits on the MMA
// completion barrier are bounded; if one runs out the kernel records
// SG_ERR_TIMEOUT, stops issuing work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sg_bounds.h"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcKC = 8;                       // 8-value K chunks per cell (K = 64 per cell)
// A: bytes between K chunks (cell 0's groups of 8 rows, 8 zero groups, cell
// 1's groups) and bytes of one buffer (8 chunks and the groups that the last
// K step of cell 1 reads past them)
__host__ __device__ constexpr int tc_lbo_a(int kc) { return (2 * kc + 8) * 128; }
__host__ __device__ constexpr int tc_a_stage(int kc) { return kTcKC * tc_lbo_a(kc) + (8 - kc) * 128; }
// B: K chunks of the pair (cell 1's follow cell 0's; one more when the last K
// step of cell 1 reads past them)
__host__ __device__ constexpr int tc_b_chunks(int kc) { return 2 * kc + (kc & 1); }
constexpr int kTcVB = 4;                       // slots per mode block
constexpr int kTcTerms = 2;                    // bf16 terms of a patch value
constexpr int kTcMaxSlots = 80;                // kTcTerms x 80 columns <= the MMA's N limit of 256
constexpr unsigned int kTcSpin = 1u << 20;     // bound of a completion wait (polls)

struct TcParams {
  const float* r;
  float* x;
  const __nv_bfloat16* inv;
  const int* blk_alpha;     // [n_blk][kTcVB] modes, -1 padded
  int* status;              // SG_ERR_TIMEOUT is recorded here
  int n_blk, npp, tile_blocks, n_tiles, slp, ncols, tmem_cols, stages;
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
// Waits for the phase of the given parity to complete, polling at most
// limit times; false if the limit ran out first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned int limit) {
  for (unsigned int polls = 0; polls < limit; ++polls)
    if (mbar_test(bar, parity)) return true;
  return false;
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
  int cx0, cy, cz, nc, b0, nb, tile;
  long long cell0;
};

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(kTcThreads, 4) mg_vanka_tc(const TcParams p) {
  constexpr int N = K + 1;
  constexpr int NKD = DIM == 2 ? N * N : N * N * N;
  constexpr int NP = NT * NKD;
  static_assert(NP <= 8 * kTcKC, "patch larger than 64 unknowns");
  constexpr int KC = (NP + 7) / 8;               // K chunks of a cell that hold values = row groups of a cell
  constexpr int LBO_A = tc_lbo_a(KC), A_STAGE = tc_a_stage(KC), B_CHUNKS = tc_b_chunks(KC);
  constexpr int RPC = (NP * 2 + 15) / 16;        // 16-byte pieces of a stored row that hold values
  constexpr int LX = 2 * K + 1;                  // nodes of the pair along x
  constexpr int LYZ = DIM == 2 ? N : N * N;
  constexpr int LN = LX * LYZ;                   // nodes of the pair
  constexpr int E = NT * LN;                     // (time node, node) entries of the pair
  constexpr int EP = E | 1;                      // odd pitch: slots of one entry fall in distinct banks
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_qoff[8 * kTcKC];              // patch column -> entry of cell 0
  __shared__ int s_ge[2][E];                     // offset of each entry in a mode's block of r (-1: none)
  __shared__ long long s_so[2][kTcMaxSlots];     // offset of each slot's mode block (-1: none)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int SL = p.tile_blocks * kTcVB;           // slots of a tile
  const int SLP = p.slp;                          // column pitch of a split term
  const int NCOL = p.ncols;                       // MMA N = kTcTerms SLP
  const bool two = p.stages == 2;
  const uint32_t LBO_B = (uint32_t)(NCOL / 8) * 128u;
  // shared memory: A buffers, B, r buffers
  unsigned char* A0 = smem_raw;                                         // stages x A_STAGE
  unsigned char* B = A0 + (size_t)p.stages * A_STAGE;                   // B_CHUNKS x LBO_B
  float* Rl0 = reinterpret_cast<float*>(B + (size_t)B_CHUNKS * LBO_B);  // stages x [SL][EP]
  const int nnx = p.nn[0], nny = p.nn[1], nnz_ = p.nn[2];
  const unsigned int ppr = (unsigned int)(p.cells[0] + 1) / 2u;
  const unsigned int n_pairs = ppr * (unsigned int)(p.cells[1] * p.cells[2]);
  const unsigned int n_units = n_pairs * (unsigned int)p.n_tiles;
  const uint32_t idesc = idesc_bf16(128, NCOL);

  // tensor memory (one warp), completion barrier, zeroed operands, column table
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem_raw);
    const int n16 = (p.stages * A_STAGE + B_CHUNKS * (int)LBO_B) / 16;
    for (int i = tid; i < n16; i += kTcThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int q = tid; q < 8 * kTcKC; q += kTcThreads) {
      int off = 0;
      if (q < NP) {
        const int iq = q / NKD, a = q - iq * NKD;
        const int ax = a % N, ay = (a / N) % N, az = DIM == 3 ? a / (N * N) : 0;
        off = iq * LN + ax + LX * (ay + N * az);
      }
      s_qoff[q] = off;
    }
  }

  // unit -> (mode tile, pair): unit = tile * n_pairs + (cz cells[1] + cy) ppr + cx0 / 2
  auto finish_unit = [&](TcUnit& U) {
    U.b0 = U.tile * p.tile_blocks;
    U.nb = min(p.tile_blocks, p.n_blk - U.b0);
    U.nc = min(2, p.cells[0] - U.cx0);
    U.cell0 = ((long long)U.cz * p.cells[1] + U.cy) * p.cells[0] + U.cx0;
  };
  auto decode = [&](unsigned int unit, TcUnit& U) {
    const unsigned int pr = unit % n_pairs;
    U.tile = (int)(unit / n_pairs);
    U.cx0 = (int)(pr % ppr) * 2;
    const unsigned int row = pr / ppr;
    U.cy = (int)(row % (unsigned int)p.cells[1]);
    U.cz = (int)(row / (unsigned int)p.cells[1]);
    finish_unit(U);
  };
  // the unit gridDim.x further on, by a mixed-radix addition of the grid's
  // stride (each digit carries at most once)
  const unsigned int g_pairs = gridDim.x % n_pairs, g_rows = g_pairs / ppr;
  const int st_tile = (int)(gridDim.x / n_pairs), st_px = (int)(g_pairs % ppr);
  const int st_cy = (int)(g_rows % (unsigned int)p.cells[1]), st_cz = (int)(g_rows / (unsigned int)p.cells[1]);
  auto advance = [&](const TcUnit& A, TcUnit& U) {
    int px = (A.cx0 >> 1) + st_px;
    const int c0 = px >= (int)ppr;
    px -= c0 * (int)ppr;
    int cy = A.cy + st_cy + c0;
    const int c1 = cy >= p.cells[1];
    cy -= c1 * p.cells[1];
    int cz = A.cz + st_cz + c1;
    const int c2 = cz >= p.cells[2];
    cz -= c2 * p.cells[2];
    U.tile = A.tile + st_tile + c2;
    U.cx0 = px * 2;
    U.cy = cy;
    U.cz = cz;
    finish_unit(U);
  };
  int so_tile0 = -1, so_tile1 = -1;               // mode tile whose slot offsets each buffer holds
  auto tables = [&](const TcUnit& U, int tb) {
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
#pragma unroll
      for (int i = 0; i < NT; ++i) s_ge[tb][i * LN + ln] = node >= 0 ? (int)(i * p.n_x + node) : -1;
    }
    // slot offsets depend on the mode tile only: rebuilt when the buffer
    // holds another tile's (the same for all threads)
    if ((tb ? so_tile1 : so_tile0) != U.b0) {
      for (int sl = tid; sl < SL; sl += kTcThreads) {
        const int mode = sl < U.nb * kTcVB ? p.blk_alpha[U.b0 * kTcVB + sl] : -1;
        s_so[tb][sl] = mode >= 0 ? (long long)mode * NT * p.n_x : -1;
      }
      if (tb) so_tile1 = U.b0;
      else so_tile0 = U.b0;
    }
  };
  // the unit's r values: slot-major, entries (time node, pair node)
  // contiguous; warp w takes slots w, w + 4, ..., its lanes the entries
  constexpr int EW = (E + 31) / 32;               // entries a lane takes
  auto stage_r = [&](int tb, float* Rl) {
    int ge[EW];
#pragma unroll
    for (int j = 0; j < EW; ++j) ge[j] = lane + 32 * j < E ? s_ge[tb][lane + 32 * j] : -1;
    for (int sl = warp; sl < SL; sl += kTcThreads / 32) {
      const long long so = s_so[tb][sl];
      float* row = Rl + sl * EP;
#pragma unroll
      for (int j = 0; j < EW; ++j) {
        const int e = lane + 32 * j;
        if (e < E) {
          if (so >= 0 && ge[j] >= 0 && SG_IN(so + ge[j], p.n_vec_x, 602)) cp_async4_tc(row + e, p.r + so + ge[j]);
          else row[e] = 0.0f;
        }
      }
    }
  };
  // the unit's inverses into A: row rho of cell c, K chunk kc; a thread's
  // (c, kc, rho) items are the same in every unit
  constexpr int A_ITEMS = 2 * RPC * NP, A_PER = (A_ITEMS + kTcThreads - 1) / kTcThreads;
  int a_src[A_PER], a_dst[A_PER];
#pragma unroll
  for (int j = 0; j < A_PER; ++j) {
    const int idx = tid + j * kTcThreads;
    const int rho = idx % NP, rest = idx / NP;
    const int kc = rest % RPC, c = rest / RPC;
    a_src[j] = idx < A_ITEMS ? (c * NP + rho) * p.npp + kc * 8 : -1;
    a_dst[j] = kc * LBO_A + (c * (KC + 8) + (rho >> 3)) * 128 + (rho & 7) * 16;
  }
  auto stage_a = [&](const TcUnit& U, unsigned char* A) {
    const long long base = U.cell0 * NP * (long long)p.npp;
    const int lim = U.nc * NP * p.npp;             // values of the unit's cells
#pragma unroll
    for (int j = 0; j < A_PER; ++j) {
      if (a_src[j] >= 0 && a_src[j] < lim && SG_IN(base + a_src[j] + 7, p.inv_count, 601))
        cp_async16_tc(A + a_dst[j], p.inv + base + a_src[j]);
    }
  };
  // B: eight K values (patch columns 8 kc ..) of slot s of cell c, kTcTerms terms
  // a thread's items (slot s, K chunk ck of either cell) step by kTcThreads:
  // (s, ck) advances by (kTcThreads % SL, kTcThreads / SL) with one carry
  const int bb_ds = kTcThreads % SL, bb_dck = kTcThreads / SL;
  const int bb_s0 = tid % SL, bb_ck0 = tid / SL;
  auto build_b = [&](const float* Rl) {
    for (int s = bb_s0, ck = bb_ck0; ck < 2 * KC;) {
      const int c = ck / KC, kc = ck - c * KC;
      const float* src = Rl + s * EP + c * K;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = kc * 8 + j;
        v[j] = q < NP ? src[s_qoff[q]] : 0.0f;
      }
      unsigned char* dst = B + (size_t)(KC * c + kc) * LBO_B;
#pragma unroll
      for (int t = 0; t < kTcTerms; ++t) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
          w[h] = *reinterpret_cast<const uint32_t*>(&b2);
          const float2 back = __bfloat1622float2(b2);
          v[2 * h] -= back.x;
          v[2 * h + 1] -= back.y;
        }
        const int n = t * SLP + s;
        *reinterpret_cast<uint4*>(dst + (n >> 3) * 128 + (n & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      s += bb_ds;
      ck += bb_dck;
      if (s >= SL) {
        s -= SL;
        ++ck;
      }
    }
  };
  // wait (bounded) for the MMAs committed to the barrier
  uint32_t phase = 0u;
  auto wait_mma = [&]() {
    if (!s_fail && !mbar_wait_bounded(&s_bar, phase, kTcSpin)) {
      atomicExch(&s_fail, 1);
      atomicExch(p.status, (int)SG_ERR_TIMEOUT);
    }
    phase ^= 1u;
  };
  // D into x: lane row = 64 c + patch row
  // this thread's accumulator row (lane row = 64 c + patch row): its entry
  // in the unit tables and its multiplicity weight, the same in every unit
  const int rb_c = (warp * 32 + lane) >> 6;
  int rb_entry = -1;
  float rb_sc = 0.0f;
  {
    const int rho = (warp * 32 + lane) & 63;
    if (rho < NP) {
      const int i = rho / NKD, a = rho - i * NKD;
      const int ax = a % N, ay = (a / N) % N, az = DIM == 3 ? a / (N * N) : 0;
      rb_entry = i * LN + rb_c * K + ax + LX * (ay + N * az);
      const int mult = (ax % K == 0 ? 2 : 1) * (ay % K == 0 ? 2 : 1) * (DIM == 3 && az % K == 0 ? 2 : 1);
      rb_sc = p.omega / (float)mult;
    }
  }
  auto read_back = [&](const TcUnit& U, int tb, uint32_t tmem) {
    const int failed = __shfl_sync(0xffffffffu, s_fail, 0);   // warp-uniform: tcgen05.ld is .sync.aligned
    if (failed) return;
    const int ge = rb_entry >= 0 ? s_ge[tb][rb_entry] : -1;
    const bool live = rb_c < U.nc && ge >= 0;
    const float sc = rb_sc;
    const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int s0 = 0; s0 < SL; s0 += 16) {
      float d0[16], d1[16];
      tmem_ld16(base + (uint32_t)s0, d0);
      tmem_ld16(base + (uint32_t)(SLP + s0), d1);
      tmem_ld_wait();
      static_assert(kTcTerms == 2, "the read-back sums two terms");
      if (live) {
        float* xrow = p.x + ge;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (s0 + j >= SL) break;
          const long long so = s_so[tb][s0 + j];
          if (so >= 0 && SG_IN(so + ge, p.n_vec_x, 604)) atomicAdd(xrow + so, sc * (d0[j] + d1[j]));
        }
      }
    }
  };

  unsigned int u = blockIdx.x;
  int tb = 0, ab = 0;
  TcUnit cur, nxt;
  if (u < n_units) {
    decode(u, cur);
    tables(cur, 0);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = s_tmem;
  if (u < n_units) {
    stage_r(0, Rl0);
    stage_a(cur, A0);
  }
  cp_commit_tc();
  for (; u < n_units; u += gridDim.x) {
    const unsigned int un = u + gridDim.x;
    const bool has_next = un < n_units;
    if (has_next) {
      advance(cur, nxt);
      tables(nxt, tb ^ 1);
    }
    cp_wait0_tc();
    fence_async_smem();
    __syncthreads();
    const int nb = two ? ab ^ 1 : ab;               // buffers of the next unit
    float* Rl = Rl0 + (size_t)ab * SL * EP;
    if (two && has_next) {
      stage_r(tb ^ 1, Rl0 + (size_t)nb * SL * EP);
      stage_a(nxt, A0 + (size_t)nb * A_STAGE);
      cp_commit_tc();
    }
    build_b(Rl);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && !s_fail) {
      const uint32_t a_addr = smem_u32(A0 + (size_t)ab * A_STAGE), b_addr = smem_u32(B);
      bool first = true;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const int kl = ks & 3;                      // K step within the cell
        if (2 * kl >= KC) continue;                 // only zeros there
        const uint32_t a_start = a_addr + (uint32_t)(2 * kl * LBO_A) + (ks >= 4 ? (uint32_t)KC * 128u : 0u);
        const uint64_t ad = smem_desc(a_start, (uint32_t)LBO_A, 128u);
        const uint32_t b_chunk = (uint32_t)((ks >= 4 ? KC : 0) + 2 * kl);
        const uint64_t bd = smem_desc(b_addr + b_chunk * LBO_B, LBO_B, 128u);
        mma_bf16(tmem, ad, bd, idesc, first ? 0u : 1u);
        first = false;
      }
      mma_commit(&s_bar);
    }
    if (!two && has_next) stage_r(tb ^ 1, Rl);      // B is built: r's buffer is free
    wait_mma();
    tc_after_sync();
    if (!two && has_next) stage_a(nxt, A0);         // the MMAs are done: A's buffer is free
    if (!two) cp_commit_tc();
    read_back(cur, tb, tmem);
    tc_before_sync();
    __syncthreads();
    cur = nxt;
    tb ^= 1;
    if (two) ab ^= 1;
  }
  cp_wait0_tc();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
}

// Self-test of the bounded wait: an mbarrier that nothing arrives on, waited
// for with the sweep's wait; the wait runs out and records SG_ERR_TIMEOUT.
__global__ void mbar_wait_probe(unsigned int limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0u, limit) && threadIdx.x == 0) atomicExch(status, (int)SG_ERR_TIMEOUT);
}

}  // namespace

cudaError_t vanka_tc_wait_probe(unsigned int polls, int* status_out) {
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) {
    mbar_wait_probe<<<1, 32>>>(polls, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(status_out, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e;
}

// slots of a tile rounded up to 16: the column pitch of one split term
static int tc_slot_pitch(int tile_slots) { return (tile_slots + 15) / 16 * 16; }

size_t vanka_tc_smem(int dim, int k, int nt, int stages, int tile_slots) {
  const int n = k + 1, lyz = dim == 2 ? n : n * n;
  const int e = nt * (2 * k + 1) * lyz, ep = e | 1;
  const int kc = (nt * (dim == 2 ? n * n : n * n * n) + 7) / 8;
  const int ncol = kTcTerms * tc_slot_pitch(tile_slots);
  return (size_t)stages * tc_a_stage(kc) + (size_t)tc_b_chunks(kc) * (ncol / 8) * 128 +
         (size_t)stages * tile_slots * ep * sizeof(float);
}

bool vanka_tc_eligible(int dim, int k, int nt, int tile_slots) {
  const int n = k + 1, np = nt * (dim == 2 ? n * n : n * n * n);
  return np <= 8 * kTcKC && tile_slots >= kTcVB && tile_slots % kTcVB == 0 && tile_slots <= kTcMaxSlots;
}

// static shared memory and registers of each instantiation (prepare_vanka_tc)
struct TcAttr {
  int static_smem = 0, regs = 0;
};
static TcAttr g_tc_attr[4][4][5];      // [dim][k][n_t]

// CTAs of one instantiation resident on an SM at once: shared memory (with the
// per-CTA reservation), registers, and tensor memory (512 columns an SM), so
// that no CTA of the persistent grid waits in its allocation.
static int tc_ctas_per_sm(const TcAttr& a, size_t smem, int tmem_cols) {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  const long long per_cta_smem = (long long)smem + a.static_smem + reserved;
  const int regs = (a.regs + 7) / 8 * 8;                      // allocated in steps of 8 a thread
  int n = 512 / tmem_cols;
  if (per_cta_smem > 0) n = std::min<long long>(n, smem_sm / per_cta_smem);
  if (regs > 0) n = std::min(n, regs_sm / (regs * kTcThreads));
  return std::max(1, n);
}

template <int DIM, int K, int NT>
static cudaError_t launch_tc(const TcParams& p, size_t smem, cudaStream_t s, long long units) {
  auto kern = &mg_vanka_tc<DIM, K, NT>;
  const int per_sm = tc_ctas_per_sm(g_tc_attr[DIM][K][NT], smem, p.tmem_cols);
  const int grid = (int)std::max<long long>(1, std::min<long long>(units, sm_count() * per_sm));
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
    g_tc_attr[D][KK][TT] = TcAttr{(int)fa.sharedSizeBytes, fa.numRegs};                                  \
    e = cudaFuncSetAttribute(&mg_vanka_tc<D, KK, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                             optin - (int)fa.sharedSizeBytes);                                           \
    if (e != cudaSuccess) return e;                                                                      \
    return cudaFuncSetAttribute(&mg_vanka_tc<D, KK, TT>, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                100);                                                                    \
  }
  SG_TP(2, 1, 1) SG_TP(2, 1, 2) SG_TP(2, 1, 3) SG_TP(2, 1, 4)
  SG_TP(2, 2, 1) SG_TP(2, 2, 2) SG_TP(2, 2, 3) SG_TP(2, 2, 4)
  SG_TP(2, 3, 1) SG_TP(2, 3, 2) SG_TP(2, 3, 3) SG_TP(2, 3, 4)
  SG_TP(3, 1, 1) SG_TP(3, 1, 2) SG_TP(3, 2, 1) SG_TP(3, 2, 2)
#undef SG_TP
  return cudaErrorInvalidValue;
}

cudaError_t launch_vanka_tc(const HostProblem& hp, const float* r, float* x, const void* inv, const int* blk_alpha,
                            int n_blk, int stages, int tile_slots, int* status, float omega, cudaStream_t s) {
  TcParams p{};
  p.r = r;
  p.x = x;
  p.inv = static_cast<const __nv_bfloat16*>(inv);
  p.blk_alpha = blk_alpha;
  p.status = status;
  p.n_blk = n_blk;
  p.stages = stages >= 2 ? 2 : 1;
  const int n = hp.k + 1, np = hp.n_t * (hp.dim == 2 ? n * n : n * n * n);
  p.npp = (np + 7) / 8 * 8;
  p.tile_blocks = std::max(1, std::min(n_blk, tile_slots / kTcVB));
  p.n_tiles = (n_blk + p.tile_blocks - 1) / p.tile_blocks;
  const int sl = p.tile_blocks * kTcVB;
  if (sl > kTcMaxSlots) return cudaErrorInvalidValue;
  p.slp = tc_slot_pitch(sl);
  p.ncols = kTcTerms * p.slp;             // a multiple of 16, at most 160
  p.tmem_cols = 32;
  while (p.tmem_cols < p.ncols) p.tmem_cols *= 2;
  p.n_x = hp.n_x;
  p.n_cells = hp.n_cells;
  p.n_vec_x = (long long)hp.n_xi * hp.n_t * hp.n_x;
  p.inv_count = hp.n_cells * (long long)np * p.npp;
  for (int d = 0; d < 3; ++d) {
    p.cells[d] = hp.cells[d];
    p.nn[d] = hp.nn[d];
  }
  p.omega = omega;
  const size_t smem = vanka_tc_smem(hp.dim, hp.k, hp.n_t, p.stages, sl);
  const long long units = (long long)((hp.cells[0] + 1) / 2) * hp.cells[1] * hp.cells[2] * p.n_tiles;
#define SG_TL(D, KK, TT) \
  if (hp.dim == D && hp.k == KK && hp.n_t == TT) return launch_tc<D, KK, TT>(p, smem, s, units);
  SG_TL(2, 1, 1) SG_TL(2, 1, 2) SG_TL(2, 1, 3) SG_TL(2, 1, 4)
  SG_TL(2, 2, 1) SG_TL(2, 2, 2) SG_TL(2, 2, 3) SG_TL(2, 2, 4)
  SG_TL(2, 3, 1) SG_TL(2, 3, 2) SG_TL(2, 3, 3) SG_TL(2, 3, 4)
  SG_TL(3, 1, 1) SG_TL(3, 1, 2) SG_TL(3, 2, 1) SG_TL(3, 2, 2)
#undef SG_TL
  return cudaErrorInvalidValue;
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_vanka_tc)

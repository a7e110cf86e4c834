// Vanka patch factorisation on the GPU (paper, Sec. 3.5 remark on the
// algebraic solver: the space-time Vanka smoother solves small local patch
// problems).  A patch is one cell's nodes x all N_t time nodes; its matrix is
// the principal submatrix of the level's block operator
//     A_c = A_t (x) M_x + sum_mu [G_mu]_{cc} B_t (x) K_mu      (class c)
// on those unknowns, with identity rows (and zero columns) for Dirichlet
// nodes.  Every patch is assembled and inverted in FP64 in shared memory by
// one CTA: the element mass and stiffness matrices of the 3^d cells around
// the patch cell are summed over the node pairs the patch holds, then
// Gauss-Jordan elimination with partial pivoting turns [P | I] into
// [I | P^-1].  The inverse is stored [class][cell][NP][pitch] as double,
// float or bf16 (rounded from FP64 through float), the layout the smoother
// reads.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "sg_bounds.h"
#include "sg_internal.h"

namespace sg {
namespace {

struct FactorParams {
  const double* ctab;      // [cell][term][nqd]  w_q |J| a_t(x_q) / h_0^2
  const double* diag;      // [class][term]      [G_t]_{alpha alpha} of the class
  const double* grad;      // [dim][nkd][nqd]    reference derivatives at the Gauss points
  const double* mass;      // [nkd][nkd]         element mass matrix (uniform mesh)
  void* out;
  int* status;             // set to 1 if a patch is singular
  int out_kind;            // 0 double, 1 float, 2 bf16
  int npp;                 // stored row pitch
  int n_terms, n_classes;
  long long n_cells;
  int cells[3], nn[3];
  double ratio[3];         // (h_0 / h_d)^2
  double at[kMaxNT * kMaxNT];   // A_hat
  double tb[kMaxNT];            // tau * Bhat_ii
};

template <int DIM, int K, int NT>
struct FactorShape {
  static constexpr int N = K + 1;
  static constexpr int NKD = DIM == 2 ? N * N : N * N * N;
  static constexpr int NQD = NKD;
  static constexpr int NP = NT * NKD;
  static constexpr int NP2 = 2 * NP;
  static constexpr int NOFF = DIM == 2 ? 9 : 27;
  static constexpr size_t doubles = (size_t)DIM * NKD * NQD + NKD * NKD + NOFF * NQD + 2 * NKD * NKD +
                                    (size_t)NP * NP2 + NP;
  static constexpr size_t smem = doubles * sizeof(double);
};

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(256) vanka_factor_kernel(const FactorParams p) {
  using S = FactorShape<DIM, K, NT>;
  constexpr int N = S::N, NKD = S::NKD, NQD = S::NQD, NP = S::NP, NP2 = S::NP2, NOFF = S::NOFF;
  extern __shared__ __align__(16) double fsm[];
  double* sg = fsm;                          // [DIM][NKD][NQD]
  double* smass = sg + DIM * NKD * NQD;      // [NKD][NKD]
  double* cb = smass + NKD * NKD;            // [NOFF][NQD] class coefficient of the neighbour cells
  double* Kg = cb + NOFF * NQD;              // [NKD][NKD] patch stiffness (summed over cells)
  double* Mg = Kg + NKD * NKD;               // [NKD][NKD] patch mass
  double* aug = Mg + NKD * NKD;              // [NP][NP2]  [P | I]
  double* fcol = aug + NP * NP2;             // [NP]       column being eliminated
  __shared__ int s_valid[NOFF];
  __shared__ int s_int[NKD];
  __shared__ int s_piv;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < DIM * NKD * NQD; i += nthr) sg[i] = p.grad[i];
  for (int i = tid; i < NKD * NKD; i += nthr) smass[i] = p.mass[i];
  const long long units = (long long)p.n_classes * p.n_cells;
  for (long long unit = blockIdx.x; unit < units; unit += gridDim.x) {
    const int cls = (int)(unit / p.n_cells);
    const long long cell = unit - (long long)cls * p.n_cells;
    const int cx = (int)(cell % p.cells[0]), cy = (int)((cell / p.cells[0]) % p.cells[1]);
    const int cz = DIM == 3 ? (int)(cell / ((long long)p.cells[0] * p.cells[1])) : 0;
    __syncthreads();
    // class coefficient at the Gauss points of the (up to) 3^d cells around the patch
    for (int i = tid; i < NOFF * NQD; i += nthr) {
      const int o = i / NQD, q = i - o * NQD;
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
      const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
      bool valid = nx >= 0 && nx < p.cells[0] && ny >= 0 && ny < p.cells[1];
      if (DIM == 3) valid = valid && nz >= 0 && nz < p.cells[2];
      double c = 0.0;
      if (valid) {
        const long long cn = ((long long)nz * p.cells[1] + ny) * p.cells[0] + nx;
        const double* ct = p.ctab + cn * p.n_terms * NQD + q;
        const double* dg = p.diag + (size_t)cls * p.n_terms;
        for (int t = 0; t < p.n_terms; ++t)
          if (SG_IN(cn * p.n_terms * NQD + q + (long long)t * NQD, p.n_cells * p.n_terms * NQD, 301))
            c += dg[t] * ct[(size_t)t * NQD];
      }
      cb[i] = c;
      if (q == 0) s_valid[o] = valid;
    }
    for (int a = tid; a < NKD; a += nthr) {
      const int g[3] = {cx * K + a % N, cy * K + (a / N) % N, DIM == 3 ? cz * K + a / (N * N) : 0};
      bool in = g[0] > 0 && g[0] < p.nn[0] - 1 && g[1] > 0 && g[1] < p.nn[1] - 1;
      if (DIM == 3) in = in && g[2] > 0 && g[2] < p.nn[2] - 1;
      s_int[a] = in;
    }
    __syncthreads();
    // patch mass and stiffness: sums over the cells that hold both nodes
    for (int pr = tid; pr < NKD * NKD; pr += nthr) {
      const int a = pr / NKD, b = pr - a * NKD;
      const int ai[3] = {a % N, (a / N) % N, DIM == 3 ? a / (N * N) : 0};
      const int bi[3] = {b % N, (b / N) % N, DIM == 3 ? b / (N * N) : 0};
      double ks = 0.0, ms = 0.0;
      for (int o = 0; o < NOFF; ++o) {
        if (!s_valid[o]) continue;
        const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, DIM == 3 ? o / 9 - 1 : 0};
        int la = 0, lb = 0, stride = 1;
        bool in = true;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const int xa = ai[d] - od[d] * K, xb = bi[d] - od[d] * K;
          in = in && xa >= 0 && xa <= K && xb >= 0 && xb <= K;
          la += xa * stride;
          lb += xb * stride;
          stride *= N;
        }
        if (!in) continue;
        ms += smass[la * NKD + lb];
        const double* c = cb + o * NQD;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const double* ga = sg + ((size_t)d * NKD + la) * NQD;
          const double* gb = sg + ((size_t)d * NKD + lb) * NQD;
          double s = 0.0;
#pragma unroll
          for (int q = 0; q < NQD; ++q) s += c[q] * ga[q] * gb[q];
          ks += p.ratio[d] * s;
        }
      }
      Kg[pr] = ks;
      Mg[pr] = ms;
    }
    __syncthreads();
    // [P | I]; row (i, a), column (j, b): A_hat_ij M_ab + delta_ij tau Bhat_ii K_ab
    for (int idx = tid; idx < NP * NP2; idx += nthr) {
      const int row = idx / NP2, col = idx - row * NP2;
      double v;
      if (col >= NP) {
        v = col - NP == row ? 1.0 : 0.0;
      } else {
        const int i = row / NKD, a = row - i * NKD, j = col / NKD, b = col - j * NKD;
        if (!s_int[a]) v = col == row ? 1.0 : 0.0;
        else if (!s_int[b]) v = 0.0;
        else {
          v = p.at[i * NT + j] * Mg[a * NKD + b];
          if (i == j) v += p.tb[i] * Kg[a * NKD + b];
        }
      }
      aug[idx] = v;
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting (the first row of largest magnitude)
    bool singular = false;
    for (int c = 0; c < NP; ++c) {
      if (tid < 32) {
        double best = -1.0;
        int bi = NP;
        for (int r = c + tid; r < NP; r += 32) {
          const double v = fabs(aug[r * NP2 + c]);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const double ov = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) s_piv = best > 0.0 ? bi : -1;
      }
      __syncthreads();
      const int piv = s_piv;
      if (piv < 0) { singular = true; break; }
      if (piv != c) {
        for (int k = tid; k < NP2; k += nthr) {
          const double t = aug[c * NP2 + k];
          aug[c * NP2 + k] = aug[piv * NP2 + k];
          aug[piv * NP2 + k] = t;
        }
        __syncthreads();
      }
      const double d = 1.0 / aug[c * NP2 + c];
      for (int r = tid; r < NP; r += nthr) fcol[r] = r == c ? 0.0 : aug[r * NP2 + c];
      __syncthreads();
      // the left block's columns before c hold zeros in row c: start at c
      for (int k = c + tid; k < NP2; k += nthr) aug[c * NP2 + k] *= d;
      __syncthreads();
      const int w = NP2 - c;
      for (int idx = tid; idx < NP * w; idx += nthr) {
        const int r = idx / w, k = c + (idx - r * w);
        const double f = fcol[r];
        if (f != 0.0) aug[r * NP2 + k] -= f * aug[c * NP2 + k];
      }
      __syncthreads();
    }
    if (singular) {
      if (tid == 0) atomicExch(p.status, 1);
      continue;
    }
    const long long base = ((long long)cls * p.n_cells + cell) * NP * p.npp;
    for (int idx = tid; idx < NP * p.npp; idx += nthr) {
      const int row = idx / p.npp, col = idx - row * p.npp;
      const double v = col < NP ? aug[row * NP2 + NP + col] : 0.0;
      if (!SG_IN(base + idx, units * NP * p.npp, 302)) continue;
      if (p.out_kind == 0) static_cast<double*>(p.out)[base + idx] = v;
      else if (p.out_kind == 1) static_cast<float*>(p.out)[base + idx] = (float)v;
      else static_cast<__nv_bfloat16*>(p.out)[base + idx] = __float2bfloat16_rn((float)v);
    }
  }
}

template <int DIM, int K, int NT>
cudaError_t launch_factor(const FactorParams& p, cudaStream_t s) {
  using S = FactorShape<DIM, K, NT>;
  auto kern = &vanka_factor_kernel<DIM, K, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, S::smem);
  if (e != cudaSuccess) return e;
  const long long units = (long long)p.n_classes * p.n_cells;
  const int grid = (int)std::max<long long>(1, std::min<long long>(units, sm_count() * std::max(1, per_sm)));
  kern<<<grid, 256, S::smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t vanka_factor(const HostProblem& hp, const double* d_ctab, const std::vector<std::vector<double>>& class_diag,
                         int out_kind, void* d_out, int npp, bool& singular, cudaStream_t s) {
  singular = false;
  const int n = hp.k + 1, nkd = hp.dim == 2 ? n * n : n * n * n, nqd = nkd;
  // reference derivatives [d][a][q] and the element mass matrix
  std::vector<double> grad((size_t)hp.dim * nkd * nqd), wJ(nqd), phi((size_t)nkd * nqd), mass((size_t)nkd * nkd);
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  for (int q = 0; q < nqd; ++q) {
    const int qi[3] = {q % n, (q / n) % n, q / (n * n)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    wJ[q] = w;
    for (int a = 0; a < nkd; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      double v = 1.0;
      for (int d = 0; d < hp.dim; ++d) v *= hp.S[qi[d] * n + ai[d]];
      phi[(size_t)a * nqd + q] = v;
      for (int dd = 0; dd < hp.dim; ++dd) {
        double g = 1.0;
        for (int d = 0; d < hp.dim; ++d) g *= d == dd ? hp.dS[qi[d] * n + ai[d]] : hp.S[qi[d] * n + ai[d]];
        grad[((size_t)dd * nkd + a) * nqd + q] = g;
      }
    }
  }
  for (int a = 0; a < nkd; ++a)
    for (int b = 0; b < nkd; ++b) {
      double m = 0.0;
      for (int q = 0; q < nqd; ++q) m += wJ[q] * phi[(size_t)a * nqd + q] * phi[(size_t)b * nqd + q];
      mass[(size_t)a * nkd + b] = m;
    }
  std::vector<double> diag;
  for (const auto& c : class_diag) diag.insert(diag.end(), c.begin(), c.end());
  double *d_diag = nullptr, *d_grad = nullptr, *d_mass = nullptr;
  int* d_status = nullptr;
  cudaError_t e = cudaMalloc(&d_diag, std::max<size_t>(1, diag.size()) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_grad, grad.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_mass, mass.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_diag, diag.data(), diag.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_grad, grad.data(), grad.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mass, mass.data(), mass.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    FactorParams p{};
    p.ctab = d_ctab;
    p.diag = d_diag;
    p.grad = d_grad;
    p.mass = d_mass;
    p.out = d_out;
    p.status = d_status;
    p.out_kind = out_kind;
    p.npp = npp;
    p.n_terms = hp.n_terms;
    p.n_classes = (int)class_diag.size();
    p.n_cells = hp.n_cells;
    for (int d = 0; d < 3; ++d) {
      p.cells[d] = hp.cells[d];
      p.nn[d] = hp.nn[d];
      p.ratio[d] = d < hp.dim ? (hp.h[0] * hp.h[0]) / (hp.h[d] * hp.h[d]) : 0.0;
    }
    for (int i = 0; i < hp.n_t; ++i) {
      for (int j = 0; j < hp.n_t; ++j) p.at[i * hp.n_t + j] = hp.A_hat[(size_t)i * hp.n_t + j];
      p.tb[i] = hp.tau * hp.B_hat[(size_t)i * hp.n_t + i];
    }
    e = cudaErrorInvalidValue;
#define SG_F(D, KK, TT) \
    if (hp.dim == D && hp.k == KK && hp.n_t == TT) e = launch_factor<D, KK, TT>(p, s);
    SG_F(2, 1, 1) SG_F(2, 1, 2) SG_F(2, 1, 3) SG_F(2, 1, 4)
    SG_F(2, 2, 1) SG_F(2, 2, 2) SG_F(2, 2, 3) SG_F(2, 2, 4)
    SG_F(2, 3, 1) SG_F(2, 3, 2) SG_F(2, 3, 3) SG_F(2, 3, 4)
    SG_F(3, 1, 1) SG_F(3, 1, 2) SG_F(3, 2, 1) SG_F(3, 2, 2)
#undef SG_F
  }
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  singular = status != 0;
  cudaFree(d_diag);
  cudaFree(d_grad);
  cudaFree(d_mass);
  cudaFree(d_status);
  return e;
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_factor)

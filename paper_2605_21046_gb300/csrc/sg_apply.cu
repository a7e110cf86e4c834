// sg_apply: y = A^(n) x for the stochastic-Galerkin slab operator
//     A^(n) = I (x) A_t (x) M_x + sum_mu G_mu (x) B_t (x) K_mu
// (eq. local_rhs_tensor), matrix-free, on a uniform Cartesian Q_k mesh.
//
// One CTA owns a tile of TX x TY (x TZ) cells and ALL N_xi * N_t vectors of
// that tile, because the quadrature-point work couples every chaos mode
// (through G_mu) and every time node (through A_t):
//   phase 0  gather the tile's nodal values of every vector into shared
//            memory (Dirichlet nodes read as 0) plus the tile's coefficient
//            values and the sparse G table;
//   phase 1  per (cell, vector): sum-factorised interpolation to the
//            (k+1)^d Gauss points and collocation gradients;
//   phase 2  per (cell, Gauss point, alpha): the time-node mass coupling
//            sum_j A_t[i][j] u[alpha,j] and the sparse chaos contraction
//            sum_(beta,mu) G_mu[alpha][beta] a_mu(x_q) grad u[beta,i];
//   phase 3  per (cell, vector): the transposed sum factorisation back to
//            the cell's nodes;
//   phase 4  per (tile node, vector): deterministic sum over the tile's cells
//            that share the node, scaling by tau*Bhat_ii, and the store:
//            nodes inside the tile are written, nodes on the tile border are
//            added atomically (the init kernel zeroed them beforehand).
// The time mass matrix of the right Radau basis is diagonal (the (r+1)-point
// Radau rule is exact to degree 2r), so B_t = tau diag(Bhat) and the
// stiffness part never mixes time nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "sg_internal.h"

namespace sg {

template <int DIM, int K>
struct Shape {
  static constexpr int NK = K + 1;                      // nodes per direction per cell
  static constexpr int NQ = K + 1;                      // Gauss points per direction
  static constexpr int NKD = DIM == 2 ? NK * NK : NK * NK * NK;
  static constexpr int NQD = DIM == 2 ? NQ * NQ : NQ * NQ * NQ;
  static constexpr int NC = 1 + DIM;                    // value + gradient per point
};

// y = (x on Dirichlet nodes, 0 elsewhere): every node the tile kernel adds
// into atomically starts from zero, boundary rows are the identity.
__global__ void sg_init_y_kernel(const double* __restrict__ x, double* __restrict__ y,
                                 long long n_total, long long n_x, int nnx, int nny, int nnz,
                                 int dim) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n_total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long m = idx % n_x;
    int ix = (int)(m % nnx);
    int iy = (int)((m / nnx) % nny);
    int iz = (int)(m / ((long long)nnx * nny));
    bool bd = ix == 0 || ix == nnx - 1 || iy == 0 || iy == nny - 1;
    if (dim == 3) bd = bd || iz == 0 || iz == nnz - 1;
    y[idx] = bd ? x[idx] : 0.0;
  }
}

// --------------------------------------------------------------- phase 1
// Nodal values u (lexicographic, x fastest) -> values and gradients at the
// tensor Gauss points, written to q[comp * NQD + point].
template <int DIM, int K>
__device__ __forceinline__ void forward_cell(const ApplyParams& p, const double* u, double* q) {
  using Sh = Shape<DIM, K>;
  constexpr int N = Sh::NK;
  if constexpr (DIM == 2) {
    double t[N][N];   // [ny][qx]
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double s = p.S[qx][0] * u[ny * N];
#pragma unroll
        for (int nx = 1; nx < N; ++nx) s = fma(p.S[qx][nx], u[ny * N + nx], s);
        t[ny][qx] = s;
      }
    double v[N][N];   // [qy][qx]
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double s = p.S[qy][0] * t[0][qx];
#pragma unroll
        for (int ny = 1; ny < N; ++ny) s = fma(p.S[qy][ny], t[ny][qx], s);
        v[qy][qx] = s;
        q[qy * N + qx] = s;
      }
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double gx = p.D[0][qx][0] * v[qy][0];
        double gy = p.D[1][qy][0] * v[0][qx];
#pragma unroll
        for (int r = 1; r < N; ++r) {
          gx = fma(p.D[0][qx][r], v[qy][r], gx);
          gy = fma(p.D[1][qy][r], v[r][qx], gy);
        }
        q[Sh::NQD + qy * N + qx] = gx;
        q[2 * Sh::NQD + qy * N + qx] = gy;
      }
  } else {
    double t1[N][N][N];  // [nz][ny][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          const double* row = u + (nz * N + ny) * N;
          double s = p.S[qx][0] * row[0];
#pragma unroll
          for (int nx = 1; nx < N; ++nx) s = fma(p.S[qx][nx], row[nx], s);
          t1[nz][ny][qx] = s;
        }
    double t2[N][N][N];  // [nz][qy][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double s = p.S[qy][0] * t1[nz][0][qx];
#pragma unroll
          for (int ny = 1; ny < N; ++ny) s = fma(p.S[qy][ny], t1[nz][ny][qx], s);
          t2[nz][qy][qx] = s;
        }
    double v[N][N][N];   // [qz][qy][qx]
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double s = p.S[qz][0] * t2[0][qy][qx];
#pragma unroll
          for (int nz = 1; nz < N; ++nz) s = fma(p.S[qz][nz], t2[nz][qy][qx], s);
          v[qz][qy][qx] = s;
          q[(qz * N + qy) * N + qx] = s;
        }
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double gx = p.D[0][qx][0] * v[qz][qy][0];
          double gy = p.D[1][qy][0] * v[qz][0][qx];
          double gz = p.D[2][qz][0] * v[0][qy][qx];
#pragma unroll
          for (int r = 1; r < N; ++r) {
            gx = fma(p.D[0][qx][r], v[qz][qy][r], gx);
            gy = fma(p.D[1][qy][r], v[qz][r][qx], gy);
            gz = fma(p.D[2][qz][r], v[r][qy][qx], gz);
          }
          const int o = (qz * N + qy) * N + qx;
          q[Sh::NQD + o] = gx;
          q[2 * Sh::NQD + o] = gy;
          q[3 * Sh::NQD + o] = gz;
        }
  }
}

// --------------------------------------------------------------- phase 3
// Point values (q[0..NQD)) and point gradient coefficients (q[NQD*(1+d)...])
// -> nodal contributions, written over q[0..NKD).  All reads of q happen
// before the first write.
template <int DIM, int K>
__device__ __forceinline__ void backward_cell(const ApplyParams& p, double* q) {
  using Sh = Shape<DIM, K>;
  constexpr int N = Sh::NK;
  if constexpr (DIM == 2) {
    double r[N][N];   // [qy][qx] combined point residual
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double s = q[qy * N + qx];
#pragma unroll
        for (int m = 0; m < N; ++m) {
          s = fma(p.D[0][m][qx], q[Sh::NQD + qy * N + m], s);
          s = fma(p.D[1][m][qy], q[2 * Sh::NQD + m * N + qx], s);
        }
        r[qy][qx] = s;
      }
    double t[N][N];   // [ny][qx]
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double s = p.S[0][ny] * r[0][qx];
#pragma unroll
        for (int qy = 1; qy < N; ++qy) s = fma(p.S[qy][ny], r[qy][qx], s);
        t[ny][qx] = s;
      }
#pragma unroll
    for (int ny = 0; ny < N; ++ny)
#pragma unroll
      for (int nx = 0; nx < N; ++nx) {
        double s = p.S[0][nx] * t[ny][0];
#pragma unroll
        for (int qx = 1; qx < N; ++qx) s = fma(p.S[qx][nx], t[ny][qx], s);
        q[ny * N + nx] = s;
      }
  } else {
    double r[N][N][N];
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double s = q[(qz * N + qy) * N + qx];
#pragma unroll
          for (int m = 0; m < N; ++m) {
            s = fma(p.D[0][m][qx], q[Sh::NQD + (qz * N + qy) * N + m], s);
            s = fma(p.D[1][m][qy], q[2 * Sh::NQD + (qz * N + m) * N + qx], s);
            s = fma(p.D[2][m][qz], q[3 * Sh::NQD + (m * N + qy) * N + qx], s);
          }
          r[qz][qy][qx] = s;
        }
    double t1[N][N][N];  // [nz][qy][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double s = p.S[0][nz] * r[0][qy][qx];
#pragma unroll
          for (int qz = 1; qz < N; ++qz) s = fma(p.S[qz][nz], r[qz][qy][qx], s);
          t1[nz][qy][qx] = s;
        }
    double t2[N][N][N];  // [nz][ny][qx]
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          double s = p.S[0][ny] * t1[nz][0][qx];
#pragma unroll
          for (int qy = 1; qy < N; ++qy) s = fma(p.S[qy][ny], t1[nz][qy][qx], s);
          t2[nz][ny][qx] = s;
        }
#pragma unroll
    for (int nz = 0; nz < N; ++nz)
#pragma unroll
      for (int ny = 0; ny < N; ++ny)
#pragma unroll
        for (int nx = 0; nx < N; ++nx) {
          double s = p.S[0][nx] * t2[nz][ny][0];
#pragma unroll
          for (int qx = 1; qx < N; ++qx) s = fma(p.S[qx][nx], t2[nz][ny][qx], s);
          q[(nz * N + ny) * N + nx] = s;
        }
  }
}

size_t apply_smem_bytes(int dim, int k, int n_t, int n_xi, int n_terms, int nnz,
                        const int tile[3]) {
  const int tz = dim == 3 ? tile[2] : 1;
  const size_t ncell = (size_t)tile[0] * tile[1] * tz;
  const size_t nnode = (size_t)(k * tile[0] + 1) * (k * tile[1] + 1) * (dim == 3 ? k * tz + 1 : 1);
  const size_t nqd = dim == 2 ? (k + 1) * (k + 1) : (k + 1) * (k + 1) * (k + 1);
  const size_t V = (size_t)n_xi * n_t;
  size_t doubles = V * nnode + ncell * V * (1 + dim) * nqd + ncell * n_terms * nqd + nnz;
  size_t ints = (n_xi + 1) + 2 * (size_t)nnz;
  return doubles * sizeof(double) + ints * sizeof(int);
}

template <int DIM, int K, int NT>
__global__ void __launch_bounds__(512) sg_apply_tile_kernel(const ApplyParams p) {
  using Sh = Shape<DIM, K>;
  constexpr int NQD = Sh::NQD, NKD = Sh::NKD, NC = Sh::NC, N = Sh::NK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int n_xi = p.n_xi, V = n_xi * NT;

  int b = blockIdx.x;
  const int tcx = b % p.ntiles[0];
  b /= p.ntiles[0];
  const int tcy = b % p.ntiles[1];
  const int tcz = DIM == 3 ? b / p.ntiles[1] : 0;
  const int TX = p.tile[0], TY = p.tile[1], TZ = DIM == 3 ? p.tile[2] : 1;
  const int ncell = TX * TY * TZ;
  const int NNX = K * TX + 1, NNY = K * TY + 1, NNZ = DIM == 3 ? K * TZ + 1 : 1;
  const int nnode = NNX * NNY * NNZ;
  const int c0x = tcx * TX, c0y = tcy * TY, c0z = tcz * TZ;

  double* Xs = reinterpret_cast<double*>(smem_raw);            // [V][nnode]
  double* Qs = Xs + (size_t)V * nnode;                          // [cell][V][NC][NQD]
  double* Cs = Qs + (size_t)ncell * V * NC * NQD;               // [cell][term][NQD]
  double* Gv = Cs + (size_t)ncell * p.n_terms * NQD;            // [nnz]
  int* Gr = reinterpret_cast<int*>(Gv + p.nnz);                 // [n_xi+1]
  int* Gc = Gr + n_xi + 1;                                      // [nnz]
  int* Gt = Gc + p.nnz;                                         // [nnz]

  // ------------------------------------------------------------ phase 0
  for (int e = tid; e < p.nnz; e += nthr) {
    Gv[e] = p.g_val[e];
    Gc[e] = p.g_col[e];
    Gt[e] = p.g_term[e];
  }
  for (int e = tid; e <= n_xi; e += nthr) Gr[e] = p.g_row[e];
  {
    const int per_cell = p.n_terms * NQD;
    for (int idx = tid; idx < ncell * per_cell; idx += nthr) {
      const int c = idx / per_cell, rem = idx - c * per_cell;
      const int cx = c0x + c % TX, cy = c0y + (c / TX) % TY, cz = c0z + c / (TX * TY);
      double v = 0.0;
      if (cx < p.cells[0] && cy < p.cells[1] && cz < p.cells[2]) {
        const long long gc = ((long long)cz * p.cells[1] + cy) * p.cells[0] + cx;
        v = p.ctab[gc * per_cell + rem];
      }
      Cs[idx] = v;
    }
  }
  for (int idx = tid; idx < V * nnode; idx += nthr) {
    const int v = idx / nnode, ln = idx - v * nnode;
    const int gx = c0x * K + ln % NNX;
    const int gy = c0y * K + (ln / NNX) % NNY;
    const int gz = c0z * K + ln / (NNX * NNY);
    bool ok = gx < p.nn[0] && gy < p.nn[1] && gz < p.nn[2];
    ok = ok && gx > 0 && gx < p.nn[0] - 1 && gy > 0 && gy < p.nn[1] - 1;
    if (DIM == 3) ok = ok && gz > 0 && gz < p.nn[2] - 1;
    double val = 0.0;
    if (ok) val = p.x[(long long)v * p.n_x + ((long long)gz * p.nn[1] + gy) * p.nn[0] + gx];
    Xs[idx] = val;
  }
  __syncthreads();

  // ------------------------------------------------------------ phase 1
  for (int it = tid; it < ncell * V; it += nthr) {
    const int c = it / V, v = it - c * V;
    const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    if (c0x + lx >= p.cells[0] || c0y + ly >= p.cells[1] || c0z + lz >= p.cells[2]) continue;
    double u[NKD];
    const double* xv = Xs + (size_t)v * nnode;
#pragma unroll
    for (int a = 0; a < NKD; ++a) {
      const int ax = a % N, ay = (a / N) % N, az = a / (N * N);
      u[a] = xv[((lz * K + az) * NNY + ly * K + ay) * NNX + lx * K + ax];
    }
    forward_cell<DIM, K>(p, u, Qs + ((size_t)c * V + v) * NC * NQD);
  }
  __syncthreads();

  // ------------------------------------------------------------ phase 2
  {
    const int gpr = nthr / n_xi;                 // (cell, point) groups per round
    const int gl = tid / n_xi, a = tid - gl * n_xi;
    const int ngroups = ncell * NQD;
    for (int g0 = 0; g0 < ngroups; g0 += gpr) {
      const int g = g0 + gl;
      bool act = gl < gpr && g < ngroups;
      int c = 0, q = 0;
      if (act) {
        c = g / NQD;
        q = g - c * NQD;
        const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
        act = c0x + lx < p.cells[0] && c0y + ly < p.cells[1] && c0z + lz < p.cells[2];
      }
      double out[NT][NC];
      if (act) {
        const double* base = Qs + (size_t)c * V * NC * NQD + q;
        double uv[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) uv[j] = base[(size_t)((a * NT + j) * NC) * NQD];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
          double s = p.Am[i][0] * uv[0];
#pragma unroll
          for (int j = 1; j < NT; ++j) s = fma(p.Am[i][j], uv[j], s);
          out[i][0] = p.wJ[q] * s;
#pragma unroll
          for (int d = 0; d < DIM; ++d) out[i][1 + d] = 0.0;
        }
        const double* cq = Cs + (size_t)c * p.n_terms * NQD + q;
        for (int e = Gr[a]; e < Gr[a + 1]; ++e) {
          const double w = Gv[e] * cq[Gt[e] * NQD];
          const double* gb = base + (size_t)(Gc[e] * NT) * NC * NQD;
#pragma unroll
          for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int d = 0; d < DIM; ++d)
              out[i][1 + d] = fma(w, gb[(size_t)(i * NC + 1 + d) * NQD], out[i][1 + d]);
        }
      }
      __syncthreads();
      if (act) {
        double* base = Qs + (size_t)c * V * NC * NQD + q;
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) base[(size_t)((a * NT + i) * NC + cc) * NQD] = out[i][cc];
      }
      __syncthreads();
    }
  }

  // ------------------------------------------------------------ phase 3
  for (int it = tid; it < ncell * V; it += nthr) {
    const int c = it / V, v = it - c * V;
    const int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    if (c0x + lx >= p.cells[0] || c0y + ly >= p.cells[1] || c0z + lz >= p.cells[2]) continue;
    backward_cell<DIM, K>(p, Qs + ((size_t)c * V + v) * NC * NQD);
  }
  __syncthreads();

  // ------------------------------------------------------------ phase 4
  for (int idx = tid; idx < V * nnode; idx += nthr) {
    const int v = idx / nnode, ln = idx - v * nnode;
    const int lx = ln % NNX, ly = (ln / NNX) % NNY, lz = ln / (NNX * NNY);
    const int gx = c0x * K + lx, gy = c0y * K + ly, gz = c0z * K + lz;
    bool ok = gx > 0 && gx < p.nn[0] - 1 && gy > 0 && gy < p.nn[1] - 1;
    if (DIM == 3) ok = ok && gz > 0 && gz < p.nn[2] - 1;
    if (!ok) continue;
    // cells of the tile containing the node, per direction: one or two
    int cxs[2], cys[2], czs[2], nxc = 0, nyc = 0, nzc = 0;
    if (lx % K == 0) {
      if (lx / K - 1 >= 0) cxs[nxc++] = lx / K - 1;
      if (lx / K < TX) cxs[nxc++] = lx / K;
    } else {
      cxs[nxc++] = lx / K;
    }
    if (ly % K == 0) {
      if (ly / K - 1 >= 0) cys[nyc++] = ly / K - 1;
      if (ly / K < TY) cys[nyc++] = ly / K;
    } else {
      cys[nyc++] = ly / K;
    }
    if (DIM == 3) {
      if (lz % K == 0) {
        if (lz / K - 1 >= 0) czs[nzc++] = lz / K - 1;
        if (lz / K < TZ) czs[nzc++] = lz / K;
      } else {
        czs[nzc++] = lz / K;
      }
    } else {
      czs[nzc++] = 0;
    }
    double s = 0.0;
    for (int iz = 0; iz < nzc; ++iz)
      for (int iy = 0; iy < nyc; ++iy)
        for (int ix = 0; ix < nxc; ++ix) {
          const int cx = cxs[ix], cy = cys[iy], cz = czs[iz];
          if (c0x + cx >= p.cells[0] || c0y + cy >= p.cells[1] || c0z + cz >= p.cells[2]) continue;
          const int c = (cz * TY + cy) * TX + cx;
          const int a = ((lz - cz * K) * N + (ly - cy * K)) * N + (lx - cx * K);
          s += Qs[((size_t)c * V + v) * NC * NQD + a];
        }
    s *= p.tb[v % NT];
    const long long gidx = (long long)v * p.n_x + ((long long)gz * p.nn[1] + gy) * p.nn[0] + gx;
    const bool inner = lx > 0 && lx < NNX - 1 && ly > 0 && ly < NNY - 1 &&
                       (DIM == 2 || (lz > 0 && lz < NNZ - 1));
    if (inner) p.y[gidx] = s;
    else atomicAdd(p.y + gidx, s);
  }
}

template <int DIM, int K, int NT>
static void* kernel_ptr() {
  return reinterpret_cast<void*>(&sg_apply_tile_kernel<DIM, K, NT>);
}

static void* select_kernel(int dim, int k, int n_t) {
#define SG_CASE(D, KK, T) \
  if (dim == D && k == KK && n_t == T) return kernel_ptr<D, KK, T>();
  SG_CASE(2, 1, 1) SG_CASE(2, 1, 2) SG_CASE(2, 1, 3) SG_CASE(2, 1, 4)
  SG_CASE(2, 2, 1) SG_CASE(2, 2, 2) SG_CASE(2, 2, 3) SG_CASE(2, 2, 4)
  SG_CASE(2, 3, 1) SG_CASE(2, 3, 2) SG_CASE(2, 3, 3) SG_CASE(2, 3, 4)
  SG_CASE(3, 1, 1) SG_CASE(3, 1, 2) SG_CASE(3, 2, 1) SG_CASE(3, 2, 2)
#undef SG_CASE
  return nullptr;
}

cudaError_t prepare_apply_kernel(int dim, int k, int n_t, size_t smem) {
  void* f = select_kernel(dim, k, n_t);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

sg_status plan_apply(const HostProblem& hp, LaunchShape& ls, std::string& msg) {
  if (!select_kernel(hp.dim, hp.k, hp.n_t)) {
    msg = "no apply kernel built for this (dim, degree, time nodes)";
    return SG_ERR_UNSUPPORTED;
  }
  int dev = 0, smem_optin = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (smem_optin <= 0) smem_optin = 227 * 1024;
  if (n_sm <= 0) n_sm = 1;
  const int nnz = (int)hp.g.col.size();
  // Two CTAs per SM when possible; the largest tile that fits the budget,
  // but never so large that the grid leaves SMs idle.
  const size_t budget2 = (size_t)smem_optin / 2 - 1024;
  const size_t budget1 = (size_t)smem_optin - 1024;
  int best[3] = {1, 1, 1};
  long best_score = -1;
  const int maxt = 16;
  for (int tz = 1; tz <= (hp.dim == 3 ? maxt : 1); ++tz)
    for (int ty = 1; ty <= maxt; ++ty)
      for (int tx = 1; tx <= maxt; ++tx) {
        int t[3] = {tx, ty, tz};
        if (tx > hp.cells[0] || ty > hp.cells[1] || tz > hp.cells[2]) continue;
        size_t sm = apply_smem_bytes(hp.dim, hp.k, hp.n_t, hp.n_xi, hp.n_terms, nnz, t);
        if (sm > budget1) continue;
        long ncell = (long)tx * ty * tz;
        long tiles = (long)((hp.cells[0] + tx - 1) / tx) * ((hp.cells[1] + ty - 1) / ty) *
                     ((hp.cells[2] + tz - 1) / tz);
        if (tiles < n_sm && ncell > 1) continue;  // keep every SM busy
        long score = ncell * 4 + (sm <= budget2 ? 1000 : 0) - std::abs(tx - ty) - (hp.dim == 3 ? std::abs(ty - tz) : 0);
        if (score > best_score) { best_score = score; best[0] = tx; best[1] = ty; best[2] = tz; }
      }
  if (best_score < 0) {
    int t1[3] = {1, 1, 1};
    if (apply_smem_bytes(hp.dim, hp.k, hp.n_t, hp.n_xi, hp.n_terms, nnz, t1) > budget1) {
      msg = "one cell with all chaos modes does not fit in shared memory";
      return SG_ERR_UNSUPPORTED;
    }
  }
  for (int d = 0; d < 3; ++d) ls.tile[d] = best[d];
  ls.smem = apply_smem_bytes(hp.dim, hp.k, hp.n_t, hp.n_xi, hp.n_terms, nnz, ls.tile);
  // threads: phase 2 runs whole (cell, point) groups of n_xi threads
  const int V = hp.n_xi * hp.n_t;
  int thr = 256;
  if (hp.n_xi > thr) thr = ((hp.n_xi + 31) / 32) * 32;
  int groups = std::max(1, thr / hp.n_xi);
  thr = std::max(V < 64 ? 64 : 128, ((groups * hp.n_xi + 31) / 32) * 32);
  if (thr > 512) thr = 512;
  if (hp.n_xi > 512) { msg = "more than 512 chaos modes"; return SG_ERR_UNSUPPORTED; }
  ls.threads = thr;
  long long tiles = 1;
  for (int d = 0; d < 3; ++d) tiles *= (hp.cells[d] + ls.tile[d] - 1) / ls.tile[d];
  if (tiles > 0x7fffffffLL) { msg = "too many tiles"; return SG_ERR_UNSUPPORTED; }
  ls.grid = (int)tiles;
  return SG_OK;
}

cudaError_t launch_apply(const HostProblem& hp, const LaunchShape& ls, const ApplyParams& prm,
                         cudaStream_t stream) {
  const long long n_total = (long long)hp.n_xi * hp.n_t * hp.n_x;
  int ib = 256;
  long long ig = std::min<long long>((n_total + ib - 1) / ib, 152LL * 16);
  sg_init_y_kernel<<<(int)ig, ib, 0, stream>>>(prm.x, prm.y, n_total, hp.n_x, hp.nn[0], hp.nn[1],
                                              hp.nn[2], hp.dim);
  void* f = select_kernel(hp.dim, hp.k, hp.n_t);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<ApplyParams*>(&prm)};
  cudaError_t e = cudaLaunchKernel(f, dim3(ls.grid), dim3(ls.threads), args, ls.smem, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sg

// Internal declarations of libsg: the context, the host-side discretisation
// tables and the kernel parameter block.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sg.h"

namespace sg {

constexpr int kMaxK = 3;          // largest spatial degree built
constexpr int kMaxNQ = kMaxK + 1; // Gauss points per direction
constexpr int kMaxNT = 4;         // largest number of time nodes (dG(3))
constexpr int kMaxQD = 64;        // largest tensor Gauss rule per cell (4^3)
constexpr int kMaxAmq = 256;      // largest (points x time nodes^2) coupling table

// ---------------------------------------------------------------- host maths
// One-dimensional rules and bases on the reference interval [0, 1].
struct Rule1D {
  std::vector<double> x, w;
};
Rule1D gauss_legendre(int n);                       // n-point Gauss rule
std::vector<double> lobatto_nodes(int k);           // k+1 Gauss-Lobatto points
std::vector<double> radau_right_nodes(int r);       // r+1 right Radau points
double lagrange(const std::vector<double>& nodes, int i, double t);
double lagrange_deriv(const std::vector<double>& nodes, int i, double t);

// dG(r) reference time matrices on [0, 1]: A_hat (eq. At), B_hat (eq. Bt / tau).
void time_matrices(int r, std::vector<double>& A, std::vector<double>& B);

// Chaos index set (graded order) and 1D Hermite triple products.
std::vector<int> chaos_indices(int M, int p);       // n_xi x M
double hermite_triple(int a, int b, int c);         // E[psi_a psi_b psi_c]

// Sparse pattern of the stochastic coupling: for each row alpha the entries
// (beta, term, value) of G_mu[alpha][beta] over all active terms mu.
struct GTable {
  std::vector<int> row, col, term;
  std::vector<double> val;
};

struct HostProblem {
  int precision = SG_PREC_FP64;
  int dim = 2, k = 1, r = 1, M = 1, p = 0, n_slabs = 1;
  double T = 1.0, tau = 1.0;
  int cells[3] = {1, 1, 1}, nn[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  int64_t n_x = 0, n_cells = 0;
  int n_xi = 0, n_t = 0, n_terms = 0;
  std::vector<int> idx;                 // chaos indices
  std::vector<std::vector<int>> mus;    // active coefficient terms
  GTable g;
  std::vector<double> A_hat, B_hat;     // (r+1)^2 each
  std::vector<double> S, Dhat;          // [q][n] interpolation, [q][p] collocation derivative
  std::vector<double> wq;               // 1D Gauss weights
  std::vector<double> ctab;             // [cell][term][qd]: w_q |J| a_mu(x_q) / h_0^2
  std::vector<int> perm;                // chaos rows sorted by their number of G entries
};

// Builds every host table of a problem.  Returns SG_OK or an error with msg.
sg_status build_host_problem(const sg_mesh* mesh, int k, int r, int n_slabs, double T,
                             int M, int p, const sg_coeff* coef, HostProblem& hp,
                             std::string& msg);

// ---------------------------------------------------------------- kernels
struct ApplyParams {
  const double* x;
  double* y;
  const double* ctab;     // [n_cells][n_terms][NQD], w_q |J| a_mu(x_q) / h_0^2
  const int* g_row;       // [n_xi + 1]
  const int* g_col;       // [nnz]
  const int* g_term;      // [nnz]
  const double* g_val;    // [nnz]
  const int* perm;        // [n_xi] chaos rows sorted by row length
  long long n_x;
  long long n_cells;
  int nn[3];              // nodes per direction
  int cells[3];
  int chunk;              // cells per shared-memory chunk
  int n_xi, n_terms, nnz;
  int aniso;              // 1 if the cell is not a cube / square
  double ratio[3];        // (h_0 / h_d)^2
  double amq[kMaxAmq];    // [q][i][j] w_q |J| A_t[i][j] / (tau Bhat_ii) (A_t^T for the transpose)
  double tb[kMaxNT];      // tau Bhat_ii
};

struct LaunchShape {
  int chunk;              // cells per chunk
  int threads;
  size_t smem;
  int grid;               // persistent CTAs
};

// Chooses a tile shape and thread count for the apply kernel of a problem.
sg_status plan_apply(const HostProblem& hp, LaunchShape& ls, std::string& msg);
// Size of the dynamic shared memory the apply kernel needs for a chunk of cells.
size_t apply_smem_bytes(int dim, int k, int n_t, int n_xi, int n_terms, int nnz, int chunk);
// Launches y = A x (init kernel + tile kernel) on a stream.
cudaError_t launch_apply(const HostProblem& hp, const LaunchShape& ls, const ApplyParams& prm,
                         cudaStream_t stream);
// Kernel attribute set-up (max dynamic shared memory).
cudaError_t prepare_apply_kernel(int precision, int dim, int k, int n_t, size_t smem);

}  // namespace sg

struct sg_ctx {
  sg::HostProblem hp;
  sg::LaunchShape ls;
  int device = 0;
  double* d_ctab = nullptr;
  int* d_grow = nullptr;
  int* d_gcol = nullptr;
  int* d_gterm = nullptr;
  double* d_gval = nullptr;
  int* d_perm = nullptr;
  double* d_xbuf = nullptr;   // workspaces of sg_apply_host (lazy)
  double* d_ybuf = nullptr;
  cudaStream_t host_stream = nullptr;
};

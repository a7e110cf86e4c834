// Internal declarations of libsg: the context, the host-side discretisation
// tables and the kernel parameter block.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <functional>
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
constexpr int kMaxPairs = 32;     // largest number of distinct (term, G value) pairs pre-multiplied

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

// One separable coefficient piece (see sg_coeff), kept so that coarse
// multigrid levels can re-evaluate the coefficient on their own meshes.
struct Piece {
  std::vector<int> mu;
  double amp = 0.0;
  int kind[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  std::vector<double> scale;           // per cell, empty = 1
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
  std::vector<double> dS;               // [q][n] derivative of the nodal basis at the Gauss points
  std::vector<Piece> pieces;            // the coefficient as given
  std::vector<int> piece_term;          // active term of every piece
  std::vector<double> wq;               // 1D Gauss weights
  std::vector<double> ctab;             // [cell][term][qd]: w_q |J| a_mu(x_q) / h_0^2
  std::vector<int> perm;                // chaos rows sorted by their number of G entries
};

// Builds every host table of a problem.  Returns SG_OK or an error with msg.
sg_status build_host_problem(const sg_mesh* mesh, int k, int r, int n_slabs, double T,
                             int M, int p, const sg_coeff* coef, HostProblem& hp,
                             std::string& msg);
// The same from stored pieces (used for the coarse multigrid levels).
sg_status build_host_problem_pieces(const sg_mesh* mesh, int k, int r, int n_slabs, double T,
                                    int M, int p, const std::vector<Piece>& pieces,
                                    HostProblem& hp, std::string& msg);

// Coefficient pieces of an sg_coeff (M-long indices, n_cells scales).
sg_status parse_pieces(const sg_coeff* coef, int M, int64_t n_cells, std::vector<Piece>& pieces, std::string& msg);
// hp.ctab from hp.pieces / hp.piece_term (mesh, degree and terms already set).
sg_status fill_ctab(HostProblem& hp, std::string& msg);

// ---------------------------------------------------------------- kernels
struct ApplyParams {
  const void* x;          // double (FP64, DW) or float (F32) vectors
  void* y;
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
  const void* b;          // right-hand side of the residual / accumulate modes
  int mode;               // kApplyPlain: y = A x; kApplyResidual: y = b - A x;
                          // kApplyAccumulate: y = b + A x without the Dirichlet identity rows
  // Distinct (term, G value) pairs of the coupling table.  With premul set the
  // kernel stages G value x a_term(x_q) per pair and cell once per chunk, so a
  // coupling entry costs no multiply at the Gauss points; without it (more
  // than kMaxPairs pairs) every entry multiplies G by a_term(x_q).
  int premul;
  int stagger;            // cells in the first chunk of CTAs blockIdx >= grid / 2 (0: a full chunk)
  int n_pairs;
  int pair_term[kMaxPairs];
  double pair_val[kMaxPairs];
};
constexpr int kApplyPlain = 0, kApplyResidual = 1, kApplyAccumulate = 2;

struct LaunchShape {
  int chunk;              // cells per chunk
  int threads;
  size_t smem;
  int grid;               // persistent CTAs
  int stagger;            // first-chunk cells of the upper half of the CTAs (0: none)
};

// Chooses a chunk size and thread count for the apply kernel of a problem.
sg_status plan_apply(const HostProblem& hp, LaunchShape& ls, std::string& msg);
// The same for a given chunk / thread count (0 = default); used by the autotuner.
sg_status plan_apply_shape(const HostProblem& hp, int chunk, int threads, LaunchShape& ls, std::string& msg);
// Largest chunk whose shared memory fits the budget.
int max_apply_chunk(const HostProblem& hp, size_t budget);
// Size of the dynamic shared memory the apply kernel needs for a chunk of cells
// (value_bytes = 8 for FP64 / DW, 4 for FP32; coef_rows = coefficient rows
// staged per cell: the pairs with premul, else the terms).
size_t apply_smem_bytes(int dim, int k, int n_t, int n_xi, int coef_rows, int nnz, int chunk,
                        int value_bytes, bool premul);
// Distinct (term, G value) pairs of the coupling table in order of first
// appearance; returns their number, or -1 if there are more than kMaxPairs.
int coupling_pairs(const HostProblem& hp, int* term, double* val);
// Fills the kernel parameter block of an apply (device table pointers given).
void fill_apply_params(const HostProblem& hp, const LaunchShape& ls, const void* ctab,
                       const int* grow, const int* gcol, const int* gterm, const double* gval,
                       const int* perm, const void* x, void* y, int transpose, ApplyParams& p);
// Launches y = A x (init kernel + chunk kernel) on a stream.
cudaError_t launch_apply(const HostProblem& hp, const LaunchShape& ls, const ApplyParams& prm,
                         cudaStream_t stream);
// Kernel attribute set-up (max dynamic shared memory).
cudaError_t prepare_apply_kernel(int precision, int dim, int k, int n_t, size_t smem);

// ---------------------------------------------------------------- Monte-Carlo apply
// One pathwise problem family of a Monte-Carlo apply launch: S samples of the
// deterministic slab operator A_t (x) M + B_t (x) K[a(., xi_s)] on one mesh.
constexpr int kMcMaxProb = 4;
struct McProblem {
  const void* x;             // S x N_t x n_x input (IO type of the arithmetic)
  void* y;                   // output
  const void* b;             // right-hand side of the residual / accumulate modes
  const double* ctab;        // [cell][term][NQD]: w_q |J| a_t(x_q) / h_0^2
  const double* wgt;         // [S][n_terms]: Psi_t(xi_s)
  const double* amq;         // [NQD][N_t][N_t]: w_q |J| T[i][j] / (tau Bhat_ii)
  long long n_x;
  long long unit0;           // first work unit (cell x sample tile) of this problem
  int n_cells, S, ts, tiles;
  int nn[3], cells[3];
  int aniso;
  double ratio[3];
};
// Bytes of y rows one Monte-Carlo apply launch covers (whole sample tiles):
// preset and then reduced into while they stay in L2.
constexpr double kMcWaveBytes = 64.0 * 1024 * 1024;

struct McParams {
  McProblem pr[kMcMaxProb];
  int n_prob, n_terms, chunk, mode, mass_only;
  long long units;
  long long u_lo = 0, u_hi = -1;   // units of this launch (whole sample tiles); u_hi < 0: all of them
  int bd_zero = 0;                  // residual whose x equals b on the boundary: its Dirichlet rows are 0
  double tb[kMaxNT];
};
// Shared memory of the Monte-Carlo apply for a chunk of cells and a sample tile.
size_t mc_smem_bytes(int dim, int k, int n_t, int ts, int n_terms, int chunk, int value_bytes);
// w_q |J| T[i][j] / (tau Bhat_ii) for one mesh (T = A_hat, its transpose, or C_t).
void mc_amq(const HostProblem& hp, const std::vector<double>& T, std::vector<double>& amq);
// Launches the init kernels of every problem and one Monte-Carlo apply.
cudaError_t launch_mc_apply(int precision, int dim, int k, int n_t, const McParams& p, int grid, int threads,
                            size_t smem, cudaStream_t s);
// Kernel attribute set-up for the Monte-Carlo apply of one shape.
cudaError_t prepare_mc_kernel(int precision, int dim, int k, int n_t);

// Precision of the apply kernels used inside the multigrid preconditioner.
constexpr int kPrecF32 = SG_PREC_FP32;

// ---------------------------------------------------------------- multigrid
struct MGLevel {
  HostProblem hp;            // level discretisation; hp.g holds the diagonal (block-Jacobi) coupling
  LaunchShape ls;
  bool coarsest = false;
  int np = 0;                // padded patch size N_t * (k+1)^d
  int n_int = 0;             // coarsest level: interior dofs per vector (N_t * interior nodes)
  void* d_ctab = nullptr;    // device tables of the level apply (value type of the MG precision
  int* d_grow = nullptr;     //  only for the vectors; tables stay double)
  int* d_gcol = nullptr;
  int* d_gterm = nullptr;
  double* d_gval = nullptr;
  int* d_perm = nullptr;
  double* d_amq = nullptr;   // time-mass tables of the level's diagonal apply (A_t and A_t^T)
  double* d_amqT = nullptr;
  int mc_ts = 0;             // rows per tile of the level's diagonal apply
  bool use_diag = true;      // residual by the diagonal apply (else the SG cell kernel, ls)
  bool chunk_ok = false;     // the SG cell kernel has a launch shape for this level
  int mc_chunk = 0, mc_grid = 0, mc_threads = 256;
  size_t mc_smem = 0;
  void* d_inv = nullptr;     // [class][cell][np][pitch] patch inverses (pitch = np rounded up to 8;
                             //  bf16 when MG::bf16), or coarsest [class][n_int][n_int]
  int vanka_chunk = 0;       // cells per Vanka chunk
  int vanka_tile = 0;        // modes per Vanka tile on this level (0: the multigrid's tile)
  int vanka_kind = 0;        // Vanka sweep: 0 FFMA kernel, 1 tensor-core kernel (bf16 factors)
  int ffma_chunk = 0, ffma_tile = 0;   // the FFMA sweep's timed choice (kept while the other sweep runs)
  const void* vanka_r = nullptr;       // residual the next sweep reads when not d_r (the first sweep reads b)
  int* d_inner = nullptr;    // coarsest: dof offset (i * n_x + node) of every interior dof
  void* d_x = nullptr;       // level vectors (N_xi * N_t * n_x values of the MG precision)
  void* d_b = nullptr;
  void* d_r = nullptr;
  // transfer to and from the next coarser level, per direction d: the
  // interpolation lists (fine node <- coarse nodes) and the restriction lists
  // (coarse node <- fine nodes), padded to pmax / rmax entries per output
  // (weight 0) and stored entry-major, [entry][output]; weights in the MG
  // precision;
  // d_t1 / d_t2 hold the intermediate arrays of the separable passes
  int* d_pidx[3] = {nullptr, nullptr, nullptr};
  void* d_pwl[3] = {nullptr, nullptr, nullptr};
  int* d_ridx[3] = {nullptr, nullptr, nullptr};
  void* d_rw[3] = {nullptr, nullptr, nullptr};
  int pmax[3] = {0, 0, 0};    // entries per output of the padded lists
  int rmax[3] = {0, 0, 0};
  void* d_t1 = nullptr;
  void* d_t2 = nullptr;
};

// Coarsening stops at the first level with at most this many interior
// space-time unknowns per chaos row (its dense solve); 0: at two cells per
// direction.
constexpr int kCoarseDofsDefault = 1024;

struct MG {
  int coarse_dofs = kCoarseDofsDefault;   // see kCoarseDofsDefault
  int precision = SG_PREC_FP64;   // vector precision: SG_PREC_FP64 or kPrecF32
  int requested = SG_PREC_FP64;   // as passed to mg_build (SG_PREC_BF16 included)
  bool bf16 = false;              // patch inverses stored in bf16 (FP32 vectors)
  int n_blk = 0;                  // Vanka mode blocks (modes of one class)
  int vanka_tile = 0;             // modes per Vanka tile (all of them unless Monte-Carlo)
  bool mc = false;                // rows are Monte-Carlo samples: residuals by the MC apply
  int mc_ts = 0;                  // samples per tile of the MC apply
  double* d_wgt = nullptr;        // [S][n_terms] Psi_t(xi_s)
  int* d_blk_cls = nullptr;
  int* d_blk_alpha = nullptr;
  int nu = 2;
  double omega = 0.7;
  int n_classes = 0;
  std::vector<int> cls;           // diagonal class of every chaos row
  int* d_cls = nullptr;
  std::vector<MGLevel> lv;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph_t[2] = {nullptr, nullptr};       // V-cycle of A (0) and of A^T (1)
  cudaGraphExec_t exec_t[2] = {nullptr, nullptr};
  double setup_ms = 0.0;
  double factor_ms = 0.0;         // Vanka patch factorisation (device, all levels)
  int* d_status = nullptr;        // kernel status word (SG_ERR_TIMEOUT from a bounded wait)
  double tune_ms = 0.0;           // timing of the level residual and Vanka variants
};

// single_class: precondition every row with the block of the mean coefficient
// term (used for Monte-Carlo sample batches, whose rows all differ).
sg_status mg_build(const HostProblem& fine, int precision, int nu, double omega, MG& mg, std::string& msg,
                   bool single_class = false);
// The mean-operator V-cycle of a Monte-Carlo system whose rows are samples
// (weights [S][n_terms]): level residuals use the Monte-Carlo apply with ts
// samples per tile, the Vanka smoother works in tiles of vanka_tile samples.
sg_status mg_build_mc(const HostProblem& fine, int precision, int nu, double omega, const std::vector<double>& wgt,
                      int ts, MG& mg, std::string& msg);
size_t krylov_bytes(long long N, int m);
void mg_free(MG& mg);
// Per-level choices of a built multigrid: info = {levels, cells, coarsest,
// residual (0 SG cell kernel, 1 diagonal apply, -1 none), Vanka cells per
// chunk, Vanka modes per tile, patch size, diagonal classes, Vanka kernel
// (0 FFMA, 1 tensor cores), 0}.
sg_status mg_level_info(const MG& mg, int level, int info[10], std::string& msg);
// Forces the level residual kind (-1 keep, 0 cell kernel, 1 diagonal apply),
// the Vanka cells per chunk (0 keep), modes per tile (-1 keep, 0 all) and
// Vanka kernel (-1 keep, 0 FFMA, 1 tensor cores) on one smoothed level (or
// every one with level = -1); drops the captured graphs.
sg_status mg_force_variant(MG& mg, int level, int residual_kind, int chunk, int tile, int kind, std::string& msg);
// The stored inverse of the Vanka patch of (mode alpha's class, cell) on a
// smoothed level, as np x np doubles (host).
sg_status mg_patch_inverse(const MG& mg, int level, int alpha, long long cell, double* out, std::string& msg);
// The tensor-core Vanka sweep (bf16 patch inverses, FP32 vectors, one diagonal
// class): whether a level shape and tile can take it, its shared memory per
// CTA, the kernel attributes, and one forward sweep.
bool vanka_tc_eligible(int dim, int k, int nt, int tile_slots);
size_t vanka_tc_smem(int dim, int k, int nt, int stages, int tile_slots);
cudaError_t prepare_vanka_tc(int dim, int k, int nt);
// Runs the sweep's bounded completion wait on an mbarrier that nothing
// arrives on (polls polls at most); status_out gets SG_ERR_TIMEOUT.
cudaError_t vanka_tc_wait_probe(unsigned int polls, int* status_out);
cudaError_t launch_vanka_tc(const HostProblem& hp, const float* r, float* x, const void* inv, const int* blk_alpha,
                            int n_blk, int stages, int tile_slots, int* status, float omega, cudaStream_t s);
// Vanka patch inverses of one multigrid level, assembled and inverted in FP64
// on the device (Gauss-Jordan, partial pivoting) for every class and cell:
// out[class][cell][np][npp] as double (out_kind 0), float (1) or bf16 (2).
// Synchronous on stream s; singular is set if any patch has no inverse.
cudaError_t vanka_factor(const HostProblem& hp, const double* d_ctab, const std::vector<std::vector<double>>& class_diag,
                         int out_kind, void* d_out, int npp, bool& singular, cudaStream_t s);
// z = P^{-1} r for one slab vector (double in, double out) on a stream; with
// trans != 0 the V-cycle of the transposed blocks A_alpha^T.
cudaError_t mg_apply(MG& mg, const double* r, double* z, cudaStream_t stream, int trans = 0);
// The same V-cycle launched kernel by kernel on `stream` (no graph launch), so
// that it can be recorded into an enclosing graph.
cudaError_t mg_issue(MG& mg, const double* r, double* z, cudaStream_t stream, int trans = 0);

}  // namespace sg

namespace sg {
sg_status make_ctx(HostProblem&& hp, int precision, sg_ctx** out, std::string& msg);
void destroy_ctx(sg_ctx* c);
// y = A x with the context's own tables (FP64 / DW vectors).
cudaError_t apply_device_ctx(sg_ctx* c, const double* x, double* y, cudaStream_t s);
// A manufactured finite-chaos solution and the slab-independent parts of its
// load vector (see sg_manufactured.cu).
struct ExactData {
  int q = 0;
  std::vector<int> idx_q;            // Lambda_q, graded order
  std::vector<double> c;             // per alpha in Lambda_q
  std::vector<int> freq;             // per alpha: 3 integer frequencies
  std::vector<double> t_coef;
  std::vector<int> p_in_q;           // position in Lambda_q of every row of the context, or -1
  double* d_P = nullptr;             // [n_xi][n_x]
  double* d_K = nullptr;             // [n_xi][n_x]
  double* d_tpk = nullptr;           // 2 * kMaxNT slab scalars
  int* d_zero_rows = nullptr;        // empty coupling table of the transfer apply
};
sg_status mc_solve_meshes(const std::vector<sg_ctx*>& parents, const std::vector<int>& n_samples,
                          const std::vector<const double*>& xis, int tile, int mg_precision, double rtol, int max_it,
                          const std::vector<double*>& mean_T, const std::vector<double*>& var_T,
                          const std::vector<double*>& u_T, sg_mc_stats* st, cudaStream_t stream, std::string& msg);
sg_status mc_solve(sg_ctx* parent, int n_samples, const double* xi, int batch, int mg_precision, double rtol,
                   int max_it, double* mean_T, double* var_T, double* u_T, sg_mc_stats* st, cudaStream_t stream,
                   std::string& msg);
sg_status exact_build(const HostProblem& hp, int q, const double* c, const int* freq, int t_degree,
                      const double* t_coef, ExactData*& out, std::string& msg);
void exact_free(ExactData* e);
cudaError_t exact_rhs(const HostProblem& hp, const LaunchShape& ls, ExactData& E, const void* ctab, const int* gcol,
                      const int* gterm, const double* gval, const int* perm, int slab, const double* u_prev,
                      double* rhs, cudaStream_t s);
// rhs += (I (x) C_t (x) M_x) u_prev (nothing on the first slab or without u_prev).
cudaError_t exact_transfer(const HostProblem& hp, const LaunchShape& ls, ExactData& E, const void* ctab,
                           const int* gcol, const int* gterm, const double* gval, const int* perm, int slab,
                           const double* u_prev, double* rhs, cudaStream_t s);
cudaError_t moments(const HostProblem& hp, const double* u, int node, double* mean, double* var, cudaStream_t s);
sg_status exact_errors(const HostProblem& hp, const ExactData& E, const double* u_dev, int slab, double err[3],
                       std::string& msg);
sg_status stat_errors(const HostProblem& hp, const ExactData& E, const double* mean_dev, const double* var_dev,
                      double t, double err[2], std::string& msg);
// Records the message sg_last_error() returns on this thread.
void set_last_error(const std::string& msg);
// Streaming multiprocessors of the current device (read once per device;
// grid caps of the grid-stride kernels are multiples of it).
long long sm_count();
sg_status fgmres(sg_ctx* ctx, const double* b, double* x, double rtol, int max_it, int m, sg_solve_stats* st,
                 cudaStream_t s, std::string& msg,
                 cudaError_t (*apply)(sg_ctx*, const double*, double*, cudaStream_t), int trans = 0);
cudaError_t apply_device_ctx_t(sg_ctx* c, const double* x, double* y, cudaStream_t s);
// A stream-ordered operation on N-vectors that launches kernels only (no host
// synchronisation, no graph launch), so that it can be captured.
using IssueFn = std::function<cudaError_t(const double*, double*, cudaStream_t)>;
// One FGMRES solve recorded as a CUDA graph (fgmres_graph) and what it was
// recorded for.
struct KrylovGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr, bs = nullptr, is = nullptr;   // capture streams
  double* host = nullptr;                                  // page-locked state mirror
  double* ws = nullptr;
  long long N = 0;
  int m = 0;
  unsigned long long key = 0;
};
void krylov_graph_free(KrylovGraph& G);
// Restarted right-preconditioned FGMRES(m) on N unknowns with caller-given
// apply and preconditioner, the whole solve (start, every Arnoldi step, the
// restarts) in one CUDA graph with device-side convergence tests; the graph
// works on workspace copies of b and x, is recorded on the first call for
// (N, m, workspace, key) and replayed afterwards.  apply and prec are
// captured into it.
sg_status fgmres_graph(long long N, const double* b, double* x, double rtol, int max_it, int m, sg_solve_stats* st,
                       cudaStream_t s, std::string& msg, const IssueFn& apply, const IssueFn& prec, double* workspace,
                       KrylovGraph& G, unsigned long long key);
// rhs = F^(n) (+ B_0 on slab 0) for hp.n_xi rows of E's load tables (no transfer term).
cudaError_t exact_rhs_load(const HostProblem& hp, ExactData& E, int slab, double* rhs, cudaStream_t s);
// Value of a coefficient factor (SG_F_ONE / SIN / POW) at one coordinate.
double factor_value(int kind, int k, double s);
// y = y + (I (x) Tm (x) M_x) x on interior rows (y unchanged on Dirichlet rows);
// Tm an N_t x N_t row-major time matrix.
cudaError_t time_mass_apply(const HostProblem& hp, const LaunchShape& ls, const void* ctab, const int* zero_rows,
                            const int* gcol, const int* gterm, const double* gval, const int* perm,
                            const double* Tm, const double* x, double* y, cudaStream_t s);
sg_status adjoint_gradient(sg_ctx* ctx, double rtol, int max_it, int K, int cell_piece, double* J_out,
                           double* g_amp, double* g_cell, sg_adjoint_stats* st, cudaStream_t s, std::string& msg);
}

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
  // pipelined host-buffer apply (sg_apply_host_async, lazy): copies in, applies
  // and copies out on three streams, through two device staging slots
  struct HostPipe {
    cudaStream_t in = nullptr, cmp = nullptr, out = nullptr;
    double* dx[2] = {nullptr, nullptr};
    double* dy[2] = {nullptr, nullptr};
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    int slot = 0;
    bool ready = false;
  } pipe;
  sg::MG* mg = nullptr;       // multigrid preconditioner (sg_mg_setup)
  int mg_coarse_dofs = sg::kCoarseDofsDefault;   // coarsest-level size of the next sg_mg_setup
  sg::ExactData* exact = nullptr;  // manufactured solution (sg_set_exact)
  double* d_krylov = nullptr; // FGMRES workspace (lazy): V, Z, w, r and partial sums
  size_t krylov_bytes = 0;
  int krylov_restart = 0;
  // recorded FGMRES solves (A and A^T) and the set-up generation they were
  // recorded in: anything that changes a launch (preconditioner, launch
  // shape, coefficient) increments gen and so forces a new recording
  sg::KrylovGraph kgraph[2];
  unsigned long long gen = 1;
};

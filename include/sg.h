/*
 * sg.h - C ABI of the GB300 stochastic-Galerkin slab-operator library (libsg).
 *
 * The library applies the coupled stochastic-Galerkin (SG) space-time slab
 * operator of the random heat equation (Problem "tensor-product slab system",
 * eq. local_rhs_tensor of the paper):
 *
 *     A^(n) = M_xi (x) A_t (x) M_x  +  sum_{mu in M_a} G_mu (x) B_t (x) K_mu
 *
 * with Q_k finite elements in space (Sec. 3.1), dG(r) in time with the right
 * Gauss-Radau nodal basis (Sec. 3.2, eqs. At, Bt), a total-degree Hermite chaos
 * Lambda_p in M standard Gaussian variables (Sec. 3.3), M_xi = I and the
 * triple-product matrices G_mu (eq. triple_stoch), and a coefficient given as
 * a finite chaos expansion a = sum_mu a_mu(x) Psi_mu(xi) (eq. coeff_expansion).
 * The operator is never assembled (the matrix-free remark after eq.
 * local_rhs_tensor): only its action is computed, by sum-factorised CUDA
 * kernels for sm_103a.
 *
 * Conventions shared by every call
 * --------------------------------
 * Vector layout.  A slab vector holds N = N_xi * N_t * N_x doubles with index
 *     (alpha * N_t + i) * N_x + m,
 * alpha the chaos index in the order returned by sg_get_multi_indices
 * (ascending total degree; inside a degree alpha_1 descending, then alpha_2,
 * ...), i = 0..r the time node (right Radau nodes ascending), m the spatial
 * node, lexicographic with x fastest over all (k*cells_d + 1) nodes per
 * direction, boundary nodes included.
 *
 * Dirichlet rows.  V_h is a subspace of H^1_0 (Sec. 3.1).  Boundary nodes are
 * stored; every product reads them as 0 and the operator's boundary rows are
 * the identity: y_b = x_b.
 *
 * Ownership.  The caller owns every vector it passes (device or host memory
 * as stated per call); the library never frees them and keeps no pointer to
 * them after a call returns.  The context owns all tables and workspaces it
 * allocates; sg_destroy releases them.
 *
 * Streams and errors.  Device calls are stream ordered and asynchronous: the
 * status reports argument validation and launch errors only.  A returned
 * error leaves the context usable.  sg_last_error() gives a one-line message
 * for the most recent failing call on the calling thread.
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque context: one discretised problem resident on the current device. */
typedef struct sg_ctx sg_ctx;

/* A cudaStream_t (the same type); NULL means the legacy default stream. */
typedef struct CUstream_st* sg_stream;

typedef enum {
  SG_OK = 0,
  SG_ERR_ARG = 1,          /* invalid argument (null, size, alias, range)   */
  SG_ERR_CUDA = 2,         /* a CUDA runtime call failed                    */
  SG_ERR_OOM = 3,          /* device or host allocation failed              */
  SG_ERR_UNSUPPORTED = 4,  /* valid but not built (degree, dimension, size) */
  SG_ERR_NOT_CONVERGED = 5,
  SG_ERR_NONFINITE = 6,
  SG_ERR_TIMEOUT = 7
} sg_status;

/* Spatial factor kinds of a separable coefficient piece (see sg_coeff). */
enum { SG_F_ONE = 0, SG_F_SIN = 1, SG_F_POW = 2 };

/* Arithmetic of the operator kernels.
 *   SG_PREC_FP64  native IEEE double (the FP64 pipe).
 *   SG_PREC_DW    double-word arithmetic: every value is an unevaluated sum of
 *                 two floats, computed on the FP32 pipe with error-free
 *                 transformations (exact FMA product errors, TwoSum); about 48
 *                 significant bits.  Inputs and outputs stay double.  Inputs
 *                 with magnitude below 2^-74 keep only 24 significant bits.
 *                 Meets the 1e-12 relative apply tolerance of the FP64 path.
 *   SG_PREC_FP32  native single precision; accepted by sg_mg_setup and
 *                 mc_solve_batch only (the multigrid preconditioner inside the
 *                 FP64 outer FGMRES).
 *   SG_PREC_BF16  as SG_PREC_FP32, with the Vanka patch inverses stored in
 *                 bfloat16 (rounded to nearest from FP32) and applied in FP32:
 *                 half the factor bytes of the FP32 V-cycle. */
enum { SG_PREC_FP64 = 0, SG_PREC_DW = 1, SG_PREC_FP32 = 2, SG_PREC_BF16 = 3 };

/* Uniform Cartesian mesh of [lo, hi] (dim = 2 or 3; entries beyond dim are
 * ignored).  cells[d] >= 1 cells in direction d. */
typedef struct {
  int dim;
  int cells[3];
  double lo[3];
  double hi[3];
} sg_mesh;

/* Coefficient expansion a(x, xi) = sum_mu a_mu(x) Psi_mu(xi)
 * (eq. coeff_expansion) given as n_pieces separable pieces; piece p adds
 *     amp[p] * s_p(cell) * prod_d f(kind[p][d], k[p][d], x_d)
 * to a_{mu_p}(x), with f(SG_F_ONE) = 1, f(SG_F_SIN, k, s) = sin(k pi s),
 * f(SG_F_POW, k, s) = s^k of the physical coordinate s, and s_p(cell) = 1
 * unless cell_scale[p] is given (one value per cell, cells lexicographic with
 * x fastest).  The distinct mu form the active set M_a, in order of first
 * appearance.  All arrays are host memory, read during sg_setup only.
 *   mu           n_pieces x M chaos multi-indices (row major)
 *   amp          n_pieces amplitudes
 *   factor_kind  n_pieces x 3 kinds (entries beyond dim ignored)
 *   factor_k     n_pieces x 3 integer parameters
 *   cell_scale   NULL, or n_pieces pointers each NULL or n_cells doubles */
typedef struct {
  int n_pieces;
  const int* mu;
  const double* amp;
  const int* factor_kind;
  const int* factor_k;
  const double* const* cell_scale;
} sg_coeff;

/* Sizes of a set-up problem. */
typedef struct {
  int dim, fe_degree, time_degree, M, chaos_order;
  int precision;   /* SG_PREC_*                         */
  int n_xi;        /* N_xi = binom(M + p, p)            */
  int n_t;         /* N_t = r + 1                       */
  int n_terms;     /* |M_a|                             */
  int g_nnz;       /* nonzeros of sum_mu |G_mu| pattern */
  int n_slabs;
  int64_t n_x;     /* spatial nodes, boundary included  */
  int64_t n_cells;
  int64_t n_unknowns; /* N_xi * N_t * N_x per slab      */
  double tau;      /* slab length T / n_slabs           */
  int chunk;       /* cells per shared-memory chunk of sg_apply */
  int grid;        /* persistent CTAs of sg_apply       */
  int threads;     /* threads per CTA of sg_apply       */
  int smem_bytes;  /* dynamic shared memory per CTA     */
  int stagger;     /* cells in the first chunk of the upper half of the CTAs (0: a full chunk) */
} sg_info;

/* Statistics of one sg_solve_slab call (host struct out). */
typedef struct {
  int iterations;       /* FGMRES iterations (Arnoldi steps)                 */
  int restarts;         /* completed FGMRES cycles                           */
  int vmult_calls;      /* applications of A^(n)                             */
  int prec_calls;       /* V-cycles                                          */
  int converged;        /* 1 if rel_residual <= rtol                          */
  double rel_residual;  /* ||rhs - A x|| / ||rhs|| of the returned x, FP64     */
  double solve_ms;      /* wall time of the call                              */
  double mg_setup_ms;   /* wall time of the last sg_mg_setup                  */
} sg_solve_stats;

/* Statistics of one mc_solve_batch call (host struct out). */
typedef struct {
  int n_samples;
  int batches;
  int total_iterations;    /* FGMRES iterations over all batches and slabs   */
  int max_slab_iterations; /* largest per-slab iteration count               */
  double max_rel_residual; /* largest final relative residual of a slab      */
  double solve_ms;         /* wall time of the call                          */
  int tile;                /* samples per tile of the apply (autotuned)      */
  int chunk;               /* cells per chunk of the apply (autotuned)       */
} sg_mc_stats;

/* Statistics of one sg_adjoint_gradient call (host struct out). */
typedef struct {
  int forward_solves;   /* slab solves of the forward sweep and the recomputed segments */
  int adjoint_solves;   /* transposed slab solves (one per slab)                        */
  int max_iterations;   /* largest FGMRES iteration count of any of them                */
  int checkpoints;      /* slab states kept between the sweeps                          */
  double J;             /* the quantity of interest (as returned in *J)                 */
  double solve_ms;      /* wall time of the call                                        */
} sg_adjoint_stats;

/* sg_setup - discretise one problem and make it resident on the current
 * CUDA device (Sec. 3: Q_k in space, dG(r) in time, Lambda_p chaos; Sec. 3.5:
 * time matrices eqs. At/Bt/Ct, G_mu eq. triple_stoch and its factorisation
 * remark, coefficient modes eq. coeff_expansion).
 *   mesh         uniform Cartesian mesh (host)
 *   fe_degree    k = 1, 2 or 3 (3D: 1 or 2)
 *   time_degree  r = 0..3 (N_t = r + 1)
 *   n_slabs, T   uniform slabs of length tau = T / n_slabs (tau > 0)
 *   M, chaos_order  M >= 1 Gaussian variables, total degree p >= 0
 *   coef         coefficient expansion (host), see sg_coeff
 *   precision    SG_PREC_FP64 or SG_PREC_DW
 *   out          receives the new context; untouched on error
 * Errors: SG_ERR_ARG for invalid sizes or pointers, SG_ERR_UNSUPPORTED for
 * degrees or sizes no kernel is built for, SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_setup(const sg_mesh* mesh, int fe_degree, int time_degree, int n_slabs,
                   double T, int M, int chaos_order, const sg_coeff* coef, int precision,
                   sg_ctx** out);

/* sg_apply - y = A^(n) x on slab n (eq. local_rhs_tensor), or y = A^(n)^T x
 * when transpose != 0 (A_t replaced by A_t^T; G_mu, B_t, K_mu are symmetric).
 * The slab operator is the same on every slab of a uniform partition; slab is
 * validated (0 <= slab < n_slabs).
 *   x, y    DEVICE pointers to n_unknowns doubles in the layout above,
 *           8-byte aligned, not overlapping (x == y is SG_ERR_ARG)
 *   stream  stream the kernels are launched on
 * Asynchronous: y is complete when the stream reaches this point. */
sg_status sg_apply(sg_ctx* ctx, int slab, const double* x, double* y, int transpose,
                   sg_stream stream);

/* sg_apply_host - as sg_apply with HOST vectors: copies x to a device
 * workspace owned by the context (allocated on the first call), applies, and
 * copies y back.  Synchronous: returns when y_host is written.  Pinned host
 * memory gives full copy bandwidth; pageable memory works. */
sg_status sg_apply_host(sg_ctx* ctx, int slab, const double* x_host, double* y_host,
                        int transpose);

/* sg_apply_host_async - y_host = A^(n) x_host (eq. local_rhs_tensor; A^(n)^T
 * when transpose != 0) for PAGE-LOCKED host vectors of n_unknowns doubles in
 * the layout above, pipelined.  The call enqueues the copy of x_host into one of two
 * device staging slots owned by the context (allocated on the first call),
 * the apply and the copy back to y_host on three internal streams, makes
 * `stream` wait for the copy back, and returns without waiting.  The copy in
 * starts as soon as its slot is free, NOT after the prior work of `stream`:
 * x_host must hold its values when the call is made.  Consecutive calls
 * alternate slots, so one call's copies overlap the neighbouring calls'
 * applies.  The caller must not write x_host or read y_host until `stream`
 * has been synchronized (or has passed the call).  Errors: SG_ERR_ARG for
 * null, overlapping or pageable vectors (use sg_apply_host for those) and a
 * slab out of range, before anything is enqueued. */
sg_status sg_apply_host_async(sg_ctx* ctx, int slab, const double* x_host, double* y_host,
                              int transpose, sg_stream stream);

/* sg_mg_setup - build the block-Jacobi geometric-multigrid preconditioner
 * (the matrix-free remark after eq. local_rhs_tensor: every chaos mode alpha
 * is preconditioned by one V-cycle of its diagonal block
 * A_alpha = A_t (x) M_x + sum_mu [G_mu]_{alpha alpha} B_t (x) K_mu with a
 * space-time Vanka smoother).  Levels halve the cells per direction while all
 * counts are even and > 2; the coarsest block is inverted densely (at most
 * 2048 interior unknowns per mode, else SG_ERR_UNSUPPORTED).  Vanka patches
 * are one cell's interior nodes x all time nodes, inverted exactly.
 *   mg_precision  SG_PREC_FP64, SG_PREC_FP32 (vectors, patch inverses,
 *                 transfers and coarse solve; the outer solver stays FP64) or
 *                 SG_PREC_BF16 (FP32 with bfloat16-stored patch inverses)
 *   nu            smoothing steps before and after the coarse correction (>= 1)
 *   omega         Vanka damping (0 < omega <= 1)
 * Allocates device memory owned by the context (replaces an earlier set-up).
 * Synchronous. */
sg_status sg_mg_setup(sg_ctx* ctx, int mg_precision, int nu, double omega);

/* sg_mg_set_coarse_dofs - size of the coarsest multigrid level for the next
 * sg_mg_setup (and the mean-operator V-cycles of mc_solve_batch /
 * mc_solve_meshes on this context).  Coarsening (halving the cells per
 * direction while every count is even and above 2) stops at the first level
 * with at most max_dofs interior space-time unknowns per chaos row, N_t times
 * the interior nodes, which is solved exactly by its dense inverse; 0 coarsens
 * down to two cells per direction.  Default 1024 (64x64 Q2 dG(1): levels 64^2,
 * 32^2, 16^2 and the 8^2 coarse solve with 450 unknowns per row; 32^3 Q2:
 * 32^3, 16^3, 8^3 and 4^3 with 686).  max_dofs 0..2048, else SG_ERR_ARG.  The
 * paper defers the hierarchy (Sec. 3.5 remark). */
sg_status sg_mg_set_coarse_dofs(sg_ctx* ctx, int max_dofs);

/* sg_mg_level_info - the choices of a built preconditioner on one level
 * (0 = finest).  info: HOST int[10] out = {number of levels, cells, 1 if the
 * coarsest (dense) level, level residual (0 the SG cell kernel with the
 * diagonal coupling table, 1 the diagonal apply, -1 none on the coarsest),
 * Vanka cells per shared-memory chunk (tensor-core sweep: staging buffers),
 * Vanka chaos modes per tile, patch size
 * N_t (k+1)^d, diagonal classes, Vanka kernel (0 FFMA, 1 tensor cores),
 * reserved 0}.  SG_ERR_ARG without sg_mg_setup or for a level out of range. */
sg_status sg_mg_level_info(sg_ctx* ctx, int level, int* info);

/* sg_mg_setup_times - wall times (HOST doubles out, ms) of the last
 * sg_mg_setup: the whole set-up, the device factorisation of the Vanka
 * patches (every level) and the timing of the level variants (the launch
 * shapes set-up picks).  SG_ERR_ARG without sg_mg_setup. */
sg_status sg_mg_setup_times(sg_ctx* ctx, double* total_ms, double* factor_ms, double* tune_ms);

/* sg_mg_set_level_variant - replace set-up's timed choices on one smoothed
 * level (level >= 0) or on all of them (level = -1): residual_kind -1 keeps,
 * 0 forces the SG cell kernel, 1 the diagonal apply; vanka_chunk 0 keeps, else
 * 1..8 cells per chunk (the tensor-core sweep works on pairs of cells and
 * reads it as 1 or 2 staging buffers, larger values as 2); vanka_tile -1
 * keeps, 0 all modes, else a multiple of 4 modes; vanka_kind -1 keeps, 0 the
 * FFMA sweep, 1 the tensor-core sweep (SG_PREC_BF16 factors, one diagonal
 * class, patches of at most 64 unknowns, at most 80 modes per tile; the
 * transposed V-cycle keeps the FFMA sweep).
 * The results stay the same up to rounding (the variants compute the same
 * V-cycle).  The next sg_vcycle records a new graph.  SG_ERR_ARG /
 * SG_ERR_UNSUPPORTED (nothing changed) when a level cannot take the variant.
 * Synchronous. */
sg_status sg_mg_set_level_variant(sg_ctx* ctx, int level, int residual_kind, int vanka_chunk, int vanka_tile,
                                  int vanka_kind);

/* sg_mg_patch_inverse - copy the stored inverse of one Vanka patch (the
 * class of chaos mode alpha, one cell of a smoothed level) to HOST memory as
 * np x np doubles, np = N_t (k+1)^d, rows and columns ordered (time node,
 * local node with x fastest); Dirichlet rows and columns are those of the
 * identity.  Values are the stored ones (FP64, FP32 or bf16, widened).
 * Synchronous. */
sg_status sg_mg_patch_inverse(sg_ctx* ctx, int level, int alpha, long long cell, double* out_host);

/* sg_vcycle - z = P^{-1} r: one V-cycle per chaos mode, all modes and time
 * nodes at once (block-Jacobi in alpha).  r, z: DEVICE slab vectors (layout
 * above), not overlapping.  Needs sg_mg_setup.  Stream ordered, async.  The
 * first call records the V-cycle into a CUDA graph (make it outside any
 * stream capture of the caller). */
sg_status sg_vcycle(sg_ctx* ctx, const double* r, double* z, sg_stream stream);

/* sg_solve_slab - solve A^(n) x = rhs (eq. local_tensor_system with the
 * right-hand side already formed) by restarted flexible GMRES(restart) in
 * FP64, right-preconditioned by sg_vcycle; Arnoldi by classical Gram-Schmidt
 * with one reorthogonalisation.
 *   rhs     DEVICE slab vector
 *   x       DEVICE slab vector: initial guess in, solution out
 *   rtol    stop when ||rhs - A x|| / ||rhs|| <= rtol (true residual, FP64)
 *   max_it  iteration limit (SG_ERR_NOT_CONVERGED when reached; x holds the
 *           last iterate and st the statistics)
 *   restart Krylov basis size (1..200)
 *   st      statistics out (may be NULL)
 * Needs sg_mg_setup.  Allocates a Krylov workspace of (2 restart + 3) slab
 * vectors on first use (kept by the context).  Synchronous: returns when x is
 * written; launches go to `stream`.  SG_ERR_NONFINITE if a residual norm is
 * not finite. */
sg_status sg_solve_slab(sg_ctx* ctx, int slab, const double* rhs, double* x, double rtol, int max_it,
                        int restart, sg_solve_stats* st, sg_stream stream);

/* sg_set_coefficient - replace the coefficient of a context (Sec. 2,
 * eq. coeff_expansion: the fields a_mu(x)) by pieces with the same count and
 * the same chaos index mu per piece (amplitudes, factors and cell scales may
 * change), keeping the mesh, the coupling tables and the manufactured load
 * vector of sg_set_exact (which stays the one of the old coefficient).  The
 * paper has no counterpart; an optimisation loop over the coefficient uses it.
 * Rebuilds the multigrid preconditioner when there is one.  Synchronous. */
sg_status sg_set_coefficient(sg_ctx* ctx, const sg_coeff* coef);

/* sg_solve_slab_adjoint - solve the transposed slab system A^T x = rhs
 * (A of eq. local_tensor_system) with FGMRES preconditioned by the V-cycle of
 * the transposed blocks A_alpha^T.  The paper solves only A; the transposed
 * system is the adjoint equation of sg_adjoint_gradient.  A^T here keeps the
 * Dirichlet rows as identity rows (transpose of the interior block).
 * Arguments, layout, workspace and errors as sg_solve_slab. */
sg_status sg_solve_slab_adjoint(sg_ctx* ctx, int slab, const double* rhs, double* x, double rtol,
                                int max_it, int restart, sg_solve_stats* st, sg_stream stream);

/* sg_adjoint_gradient - march the manufactured problem of sg_set_exact over
 * all slabs (eq. local_tensor_system with the load vector of eq. load_vector
 * held fixed as data) and return the quantity of interest
 *     J = sum_alpha U_alpha(T)^T M_x U_alpha(T) = E[ ||u_h(., T)||^2_{L2(D)} ]
 * (the variance identity eq. qoi-variance-chaos summed with the mean) and its
 * gradient with respect to the coefficient: the amplitude of every piece
 * (sg_coeff.amp) and the per-cell scale of one piece.  The paper has no
 * gradient; this is the discrete adjoint of its marching: transposed slab
 * solves (sg_solve_slab_adjoint) backwards in time with the adjoint transfer
 * (I (x) C_t^T (x) M_x) (eq. Ct transposed), then
 *     dJ/dp = - sum_n lambda_n^T (G_mu (x) B_t (x) dK/dp) U_n.
 * Forward states are kept every `checkpoint_every` slabs and each segment is
 * recomputed before its backward pass (memory (N / checkpoint_every +
 * checkpoint_every + 4) slab vectors).
 *   rtol, max_it      FGMRES(30) tolerance and limit of every slab solve
 *   cell_piece        index of the piece whose per-cell scale gets a gradient
 *                     (-1: none)
 *   J                 HOST double out (may be NULL)
 *   grad_amp          HOST n_pieces doubles out (may be NULL)
 *   grad_cell         HOST n_cells doubles out (NULL allowed; ignored if
 *                     cell_piece < 0).  With grad_amp and grad_cell both
 *                     NULL only the forward sweep runs (J alone).
 *   st                statistics out (may be NULL)
 * Needs sg_set_exact and sg_mg_setup; the Dirichlet data of the manufactured
 * solution are zero, so J covers all nodes.  At most 16 coefficient terms.
 * Allocates and frees its device workspaces.  Synchronous. */
sg_status sg_adjoint_gradient(sg_ctx* ctx, double rtol, int max_it, int checkpoint_every, int cell_piece,
                              double* J, double* grad_amp, double* grad_cell, sg_adjoint_stats* st,
                              sg_stream stream);

/* sg_apply_host_static - sg_apply_host for callers that cannot let a library
 * allocate device memory when they call it: applications whose memory pool
 * owns the whole device, code paths that must not stall or fail on an
 * allocation after start-up, or phases in which cudaMalloc / cudaFree are not
 * allowed.  The paper has no counterpart; this is a deployment variant of the
 * host-buffer apply.  x and y are staged in a fixed 32 MiB array compiled into
 * the library (reserved on every device that loads the library, held until the
 * process exits): at most 2,097,152 unknowns, larger problems get SG_ERR_ARG.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again when
 * the device's CUDA context has been replaced since (after cudaDeviceReset,
 * for instance).  The context's device must be current.  Every call uses the same array, which
 * keeps the last call's contents (each call overwrites what it reads); calls
 * that overlap on the GPU, from several threads or contexts, race on it.
 * Synchronous: it copies with cudaMemcpy and launches on the legacy default
 * stream, and returns once y is on the host. */
sg_status sg_apply_host_static(sg_ctx* ctx, int slab, const double* x_host, double* y_host,
                               int transpose);

/* sg_debug_bounds - the device bounds records of the debug build.  The
 * library built with -DSG_DEBUG_BOUNDS (libsg_debug.so) tests the index of
 * every instrumented global and shared-memory access of the apply, Monte-Carlo
 * apply, Vanka, patch-factorisation and grid-transfer kernels against the
 * extent of its array; an index outside it is skipped (never accessed), the
 * first one is recorded and all are counted.  Nothing traps.  Out (HOST):
 * enabled = 1 in that build (0 in the release build, where everything else
 * is 0 and no device call is made), count = violations since the last call,
 * site / index / limit of the first one.  Reading clears the records.
 * Synchronizes the device (debug build).  The paper has no counterpart. */
sg_status sg_debug_bounds(int* enabled, unsigned int* count, int* site, long long* index, long long* limit);

/* sg_debug_bounds_probe - self-test of the record path: one thread writes
 * element `index` of a 16-element device array if the bounds check against
 * `limit` (1..16) lets it through.  The debug build records an index outside
 * [0, limit) as site 901 and skips the write; the release build, which has
 * no device check, refuses such an index with SG_ERR_ARG before any launch.
 * Synchronous. */
sg_status sg_debug_bounds_probe(long long index, long long limit);

/* sg_debug_wait_probe - self-test of the bounded completion wait of the
 * tensor-core Vanka sweep: one CTA waits, polling at most `polls` (1..2^20)
 * times, on an mbarrier that nothing arrives on.  The wait runs out and the
 * kernel writes SG_ERR_TIMEOUT to *status (HOST int out); the kernel returns
 * normally and the context stays usable.  Synchronous.  The paper has no
 * counterpart. */
sg_status sg_debug_wait_probe(unsigned int polls, int* status);

/* sg_autotune - time the apply kernel of this context over candidate launch
 * shapes (cells per shared-memory chunk x threads per CTA x whether the upper
 * half of the CTAs starts with a half chunk, so that CTAs sharing an SM reach
 * their memory phases at different times) on the current device and keep the
 * fastest for every later sg_apply / sg_solve_slab; each
 * candidate runs 2 + reps applies on a synthetic vector.  Allocates and frees
 * two temporary device vectors.  Synchronous.  Results are unchanged up to
 * the order of the atomic additions. */
sg_status sg_autotune(sg_ctx* ctx, int reps);

/* sg_set_apply_shape - fix the launch shape of this context's apply (the
 * operator of eq. local_rhs_tensor, as sg_apply) instead of the default or
 * tuned one: `chunk` cells per shared-memory chunk, `threads`
 * per CTA (a multiple of 32 within the kernel's launch bound, with
 * threads * items_per_thread >= N_xi), and `stagger` cells in the first chunk
 * of the upper half of the CTAs (0: a full chunk; at most `chunk`).  For
 * reproducible launch shapes and tests; sg_get_info reports the shape.
 * Returns SG_ERR_ARG, leaving the shape unchanged, when it does not fit the
 * kernel or the device.  Results are unchanged up to the order of the atomic
 * additions. */
sg_status sg_set_apply_shape(sg_ctx* ctx, int chunk, int threads, int stagger);

/* sg_set_exact - attach a manufactured finite-chaos solution (Sec. 4.3,
 * eqs. finite-exact-separated .. finite-chaos-coefficients)
 *     u(x, t, xi) = T(t) sum_{alpha in Lambda_q} c_alpha Phi_alpha(x) Psi_alpha(xi),
 *     Phi_alpha(x) = prod_d sin(pi freq[alpha][d] (x_d - lo_d) / (hi_d - lo_d)),
 *     T(t) = sum_{j <= t_degree} t_coef[j] t^j,
 * (zero on the boundary of the box) and precompute the slab-independent parts
 * of its load vector (eq. load_vector with f = d_t u - div(a grad u), eq.
 * manufactured_rhs_benchmark).  q may differ from the context's chaos order:
 * modes outside Lambda_p enter through the coupling G_mu[beta][alpha].
 *   c       N_xi(q) coefficients in the order of Lambda_q (graded, as
 *           sg_get_multi_indices orders Lambda_p)          (host)
 *   freq    N_xi(q) x 3 integer frequencies (entries beyond dim ignored) (host)
 * Integrals use (k+4)^d Gauss points per cell.  Synchronous; allocates two
 * slab-mode arrays on the device (kept by the context). */
sg_status sg_set_exact(sg_ctx* ctx, int q, const double* c, const int* freq, int t_degree,
                       const double* t_coef);

/* sg_rhs - right-hand side of slab n (eq. local_tensor_system):
 *   rhs = F^(n) + J u_prev  with J = I (x) C_t (x) M_x (eq. local_rhs_tensor),
 *   rhs = F^(1) + B_0^(1)   on the first slab (eq. initial_vector, with the L2
 *                           projection of u(0); u_prev ignored, may be NULL).
 * u_prev: DEVICE solution of the previous slab (layout above); rhs: DEVICE
 * output; Dirichlet entries are 0.  Needs sg_set_exact.  Stream ordered. */
sg_status sg_rhs(sg_ctx* ctx, int slab, const double* u_prev, double* rhs, sg_stream stream);

/* sg_moments - pointwise mean and variance of a slab solution at one time
 * node (eqs. qoi-mean-chaos and qoi-variance-chaos): mean[m] = u[0, i, m],
 * var[m] = sum_{alpha != 0} u[alpha, i, m]^2.  u, mean, var: DEVICE (mean or
 * var may be NULL; n_x doubles each).  Stream ordered. */
sg_status sg_moments(sg_ctx* ctx, const double* u, int time_node, double* mean, double* var,
                     sg_stream stream);

/* sg_qoi_errors - L2(D) errors at the end time t_n of slab n of the mean, the
 * variance and the full stochastic solution against the manufactured solution
 * (Definition "error norms and quantities" at one time; the full error by the
 * modal identity eq. modal-sum-L2, truncated modes included).  u: DEVICE slab
 * solution; err: HOST array of 3 doubles (mean, variance, full).  Needs
 * sg_set_exact.  Synchronous (evaluated on the host, post-processing). */
sg_status sg_qoi_errors(sg_ctx* ctx, const double* u, int slab, double* err);

/* sg_stat_errors - L2(D) errors of a nodal mean field and a nodal variance
 * field (Q_k functions on the context's mesh, e.g. the output of sg_moments or
 * of mc_solve_batch) against the exact mean and variance of the manufactured
 * solution at time t (eqs. qoi-mean-chaos / qoi-variance-chaos applied to the
 * exact chaos coefficients).  mean, var: DEVICE n_x doubles; err: HOST array
 * of 2 doubles (mean, variance).  (k+4)^d Gauss points per cell.  Needs
 * sg_set_exact.  Synchronous (host post-processing). */
sg_status sg_stat_errors(sg_ctx* ctx, const double* mean, const double* var, double t, double* err);

/* mc_solve_batch - Monte-Carlo estimate of the mean and variance at t = T
 * (Sec. 5: the pathwise problem and its slab system eq. mc-slab-system, the
 * sample mean eq. mc-mean-estimator and the unbiased variance eq.
 * mc-variance-estimator-unbiased; Algorithm 1).  For every sample xi_s the
 * deterministic heat equation with a(x, xi_s) = sum_mu a_mu(x) Psi_mu(xi_s) and
 * the manufactured forcing f(x, t, xi_s) of sg_set_exact is marched over all
 * slabs of the context (same mesh, Q_k and dG(r)).  All samples form one
 * block-diagonal system per slab: one Monte-Carlo apply launch covers every
 * sample (in tiles of `batch` samples), FGMRES(10) iterates on the whole
 * system to rtol with a graph-captured mean-operator V-cycle as
 * preconditioner.  Samples are split into groups solved one after another
 * only when the device memory cannot hold them at once.
 *   xi        HOST n_samples x M standard-normal samples
 *   batch     samples per tile of the apply launch, 1..512 (reduced to fit
 *             shared memory)
 *   mg_precision  SG_PREC_FP64, SG_PREC_FP32 or SG_PREC_BF16 V-cycle
 *   mean_T, var_T  DEVICE n_x doubles out: nodal sample mean and unbiased
 *             sample variance of u(x, T)
 *   u_T       DEVICE n_samples x N_t x n_x doubles out (last slab of every
 *             sample), or NULL
 *   st        statistics out (may be NULL; batches = sample groups)
 * Needs sg_set_exact.  Allocates and frees its device workspaces.
 * Synchronous. */
sg_status mc_solve_batch(sg_ctx* ctx, int n_samples, const double* xi, int batch, int mg_precision,
                         double rtol, int max_it, double* mean_T, double* var_T, double* u_T,
                         sg_mc_stats* st, sg_stream stream);

/* mc_solve_meshes - mc_solve_batch for samples on several meshes at once
 * (up to 4 contexts of the same dimension, degrees, slabs, T and coefficient
 * terms; mesh sizes may differ): the samples of every mesh join ONE system
 * per slab, ONE apply launch covers every (mesh, sample tile, cell) unit, and
 * each mesh keeps its own mean-operator V-cycle.  Per mesh p: ctxs[p],
 * n_samples[p], xi[p] (HOST n_samples[p] x M), mean_T[p], var_T[p] (DEVICE
 * n_x[p] doubles out), u_T[p] (DEVICE or NULL; u_T itself may be NULL).
 * Other arguments and behaviour as mc_solve_batch.  Synchronous. */
sg_status mc_solve_meshes(int n_meshes, sg_ctx* const* ctxs, const int* n_samples, const double* const* xi,
                          int tile, int mg_precision, double rtol, int max_it, double* const* mean_T,
                          double* const* var_T, double* const* u_T, sg_mc_stats* st, sg_stream stream);

/* sg_get_info - sizes and launch shape of a context (host struct out). */
sg_status sg_get_info(const sg_ctx* ctx, sg_info* out);

/* sg_get_multi_indices - the chaos index set Lambda_p (Sec. 3.3) in the
 * library's order: out receives n_xi x M ints (host, row major). */
sg_status sg_get_multi_indices(const sg_ctx* ctx, int* out);

/* sg_destroy - release a context and everything it owns (NULL is a no-op).
 * Synchronises the device work of the context first. */
void sg_destroy(sg_ctx* ctx);

/* Static strings, never freed by the caller. */
const char* sg_status_string(sg_status s);
const char* sg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */

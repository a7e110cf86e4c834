// The extern "C" entry points of libsg declared in include/sg.h.
#include <cuda_runtime.h>

#include <atomic>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace {

thread_local std::string g_last_error;

sg_status fail(sg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

sg_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void free_ctx_device(sg_ctx* c) {
  cudaFree(c->d_ctab);
  cudaFree(c->d_grow);
  cudaFree(c->d_gcol);
  cudaFree(c->d_gterm);
  cudaFree(c->d_gval);
  cudaFree(c->d_perm);
  cudaFree(c->d_xbuf);
  cudaFree(c->d_ybuf);
  cudaFree(c->d_krylov);
  for (sg::KrylovGraph& g : c->kgraph) sg::krylov_graph_free(g);
  if (c->host_stream) cudaStreamDestroy(c->host_stream);
  {
    sg_ctx::HostPipe& p = c->pipe;
    for (cudaStream_t st : {p.in, p.cmp, p.out})
      if (st) cudaStreamSynchronize(st);
    for (int i = 0; i < 2; ++i) {
      cudaFree(p.dx[i]);
      cudaFree(p.dy[i]);
      for (cudaEvent_t ev : {p.ev_in[i], p.ev_done[i], p.ev_out[i]})
        if (ev) cudaEventDestroy(ev);
    }
    for (cudaStream_t st : {p.in, p.cmp, p.out})
      if (st) cudaStreamDestroy(st);
    p = sg_ctx::HostPipe();
  }
  if (c->mg) {
    sg::mg_free(*c->mg);
    delete c->mg;
    c->mg = nullptr;
  }
  sg::exact_free(c->exact);
  c->exact = nullptr;
}

cudaError_t apply_device(sg_ctx* c, const double* x, double* y, cudaStream_t s) {
  return sg::apply_device_ctx(c, x, y, s);
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void fill_params(const sg_ctx* c, const void* x, void* y, int transpose, sg::ApplyParams& p) {
  sg::fill_apply_params(c->hp, c->ls, c->d_ctab, c->d_grow, c->d_gcol, c->d_gterm, c->d_gval, c->d_perm, x, y,
                        transpose, p);
}

}  // namespace

namespace sg {
void set_last_error(const std::string& msg) { g_last_error = msg; }

long long sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cached[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev >= kMaxDev) dev = kMaxDev - 1;
  int n = cached[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cached[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}
}  // namespace sg

namespace sg {
cudaError_t apply_device_ctx(sg_ctx* c, const double* x, double* y, cudaStream_t s) {
  ApplyParams p;
  fill_apply_params(c->hp, c->ls, c->d_ctab, c->d_grow, c->d_gcol, c->d_gterm, c->d_gval, c->d_perm, x, y, 0, p);
  return launch_apply(c->hp, c->ls, p, s);
}

cudaError_t apply_device_ctx_t(sg_ctx* c, const double* x, double* y, cudaStream_t s) {
  ApplyParams p;
  fill_apply_params(c->hp, c->ls, c->d_ctab, c->d_grow, c->d_gcol, c->d_gterm, c->d_gval, c->d_perm, x, y, 1, p);
  return launch_apply(c->hp, c->ls, p, s);
}

// Plans the apply kernel and uploads the tables of a host problem into a new
// context (used by sg_setup and by the Monte-Carlo sample batches).
sg_status make_ctx(HostProblem&& hp, int precision, sg_ctx** out, std::string& msg) {
  sg_ctx* c = new (std::nothrow) sg_ctx();
  if (!c) { msg = "host allocation failed"; return SG_ERR_OOM; }
  c->hp = std::move(hp);
  c->hp.precision = precision;
  cudaGetDevice(&c->device);
  sg_status st = sg::plan_apply(c->hp, c->ls, msg);
  if (st != SG_OK) { delete c; return st; }
  cudaError_t e = sg::prepare_apply_kernel(precision, c->hp.dim, c->hp.k, c->hp.n_t, c->ls.smem);
  if (e != cudaSuccess) { delete c; msg = cudaGetErrorString(e); return SG_ERR_CUDA; }
  if ((e = upload(&c->d_ctab, c->hp.ctab)) != cudaSuccess ||
      (e = upload(&c->d_grow, c->hp.g.row)) != cudaSuccess ||
      (e = upload(&c->d_gcol, c->hp.g.col)) != cudaSuccess ||
      (e = upload(&c->d_gterm, c->hp.g.term)) != cudaSuccess ||
      (e = upload(&c->d_gval, c->hp.g.val)) != cudaSuccess ||
      (e = upload(&c->d_perm, c->hp.perm)) != cudaSuccess) {
    free_ctx_device(c);
    delete c;
    msg = std::string("upload of tables: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
  }
  *out = c;
  return SG_OK;
}

void destroy_ctx(sg_ctx* c) {
  if (!c) return;
  free_ctx_device(c);
  delete c;
}
}  // namespace sg

extern "C" {

const char* sg_status_string(sg_status s) {
  switch (s) {
    case SG_OK: return "ok";
    case SG_ERR_ARG: return "invalid argument";
    case SG_ERR_CUDA: return "CUDA error";
    case SG_ERR_OOM: return "out of memory";
    case SG_ERR_UNSUPPORTED: return "unsupported configuration";
    case SG_ERR_NOT_CONVERGED: return "not converged";
    case SG_ERR_NONFINITE: return "non-finite value";
    case SG_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

const char* sg_last_error(void) { return g_last_error.c_str(); }


sg_status sg_setup(const sg_mesh* mesh, int fe_degree, int time_degree, int n_slabs, double T,
                   int M, int chaos_order, const sg_coeff* coef, int precision, sg_ctx** out) {
  if (!out) return fail(SG_ERR_ARG, "sg_setup: out is NULL");
  if (precision != SG_PREC_FP64 && precision != SG_PREC_DW)
    return fail(SG_ERR_UNSUPPORTED, "sg_setup: precision not built");
  std::string msg;
  sg::HostProblem hp;
  sg_status st = sg::build_host_problem(mesh, fe_degree, time_degree, n_slabs, T, M, chaos_order, coef, hp, msg);
  if (st != SG_OK) return fail(st, "sg_setup: " + msg);
  st = sg::make_ctx(std::move(hp), precision, out, msg);
  if (st != SG_OK) return fail(st, "sg_setup: " + msg);
  return SG_OK;
}

sg_status sg_apply(sg_ctx* ctx, int slab, const double* x, double* y, int transpose,
                   sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_apply: ctx is NULL");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_apply: slab out of range");
  if (!x || !y) return fail(SG_ERR_ARG, "sg_apply: null vector");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 7)
    return fail(SG_ERR_ARG, "sg_apply: vectors must be 8-byte aligned");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (x < y + n && y < x + n) return fail(SG_ERR_ARG, "sg_apply: x and y overlap");
  // A host pointer handed to a kernel would fault the device: accept only
  // device or managed memory.
  for (const void* ptr : {static_cast<const void*>(x), static_cast<const void*>(y)}) {
    cudaPointerAttributes at;
    cudaError_t pe = cudaPointerGetAttributes(&at, ptr);
    if (pe != cudaSuccess) {
      cudaGetLastError();
      return fail(SG_ERR_ARG, "sg_apply: vector is not CUDA memory");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return fail(SG_ERR_ARG, "sg_apply: vector is not device memory");
  }
  sg::ApplyParams p;
  fill_params(ctx, x, y, transpose, p);
  cudaError_t e = sg::launch_apply(ctx->hp, ctx->ls, p, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "sg_apply: launch");
  return SG_OK;
}

sg_status sg_apply_host(sg_ctx* ctx, int slab, const double* x_host, double* y_host,
                        int transpose) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_apply_host: ctx is NULL");
  if (!x_host || !y_host) return fail(SG_ERR_ARG, "sg_apply_host: null vector");
  const size_t n = (size_t)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (x_host < y_host + n && y_host < x_host + n) return fail(SG_ERR_ARG, "sg_apply_host: x and y overlap");
  cudaError_t e;
  if (!ctx->host_stream) {
    e = cudaStreamCreateWithFlags(&ctx->host_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ctx->host_stream = nullptr; return cuda_fail(e, "sg_apply_host: stream"); }
  }
  if (!ctx->d_xbuf) {
    e = cudaMalloc(&ctx->d_xbuf, n * sizeof(double));
    if (e != cudaSuccess) { ctx->d_xbuf = nullptr; return cuda_fail(e, "sg_apply_host: workspace"); }
    e = cudaMalloc(&ctx->d_ybuf, n * sizeof(double));
    if (e != cudaSuccess) {
      cudaFree(ctx->d_xbuf);
      ctx->d_xbuf = ctx->d_ybuf = nullptr;
      return cuda_fail(e, "sg_apply_host: workspace");
    }
  }
  e = cudaMemcpyAsync(ctx->d_xbuf, x_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->host_stream);
  if (e != cudaSuccess) return cuda_fail(e, "sg_apply_host: copy in");
  sg_status st = sg_apply(ctx, slab, ctx->d_xbuf, ctx->d_ybuf, transpose,
                          reinterpret_cast<sg_stream>(ctx->host_stream));
  if (st != SG_OK) return st;
  e = cudaMemcpyAsync(y_host, ctx->d_ybuf, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->host_stream);
  if (e != cudaSuccess) return cuda_fail(e, "sg_apply_host: copy out");
  e = cudaStreamSynchronize(ctx->host_stream);
  if (e != cudaSuccess) return cuda_fail(e, "sg_apply_host: synchronize");
  return SG_OK;
}

static bool is_page_locked(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

sg_status sg_apply_host_async(sg_ctx* ctx, int slab, const double* x_host, double* y_host, int transpose,
                              sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_apply_host_async: ctx is NULL");
  if (!x_host || !y_host) return fail(SG_ERR_ARG, "sg_apply_host_async: null vector");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_apply_host_async: slab out of range");
  const size_t n = (size_t)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (x_host < y_host + n && y_host < x_host + n) return fail(SG_ERR_ARG, "sg_apply_host_async: x and y overlap");
  if (!is_page_locked(x_host) || !is_page_locked(y_host))
    return fail(SG_ERR_ARG, "sg_apply_host_async: vectors must be page-locked host memory");
  sg_ctx::HostPipe& p = ctx->pipe;
  cudaError_t e = cudaSuccess;
  if (!p.ready) {
    for (cudaStream_t* st : {&p.in, &p.cmp, &p.out})
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      for (cudaEvent_t* ev : {&p.ev_in[i], &p.ev_done[i], &p.ev_out[i]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaMalloc(&p.dx[i], n * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&p.dy[i], n * sizeof(double));
    }
    if (e != cudaSuccess) return cuda_fail(e, "sg_apply_host_async: workspace");
    p.ready = true;
  }
  const int s = p.slot;
  cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
  // copy in once the apply that last read this slot is done (not after the
  // caller's stream, which waits for every earlier call's copy back)
  if (p.used[s]) e = cudaStreamWaitEvent(p.in, p.ev_done[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.dx[s], x_host, n * sizeof(double), cudaMemcpyHostToDevice, p.in);
  if (e == cudaSuccess) e = cudaEventRecord(p.ev_in[s], p.in);
  // apply after the copy in and after the copy out that last read this slot's y
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p.cmp, p.ev_in[s], 0);
  if (e == cudaSuccess && p.used[s]) e = cudaStreamWaitEvent(p.cmp, p.ev_out[s], 0);
  if (e == cudaSuccess) {
    sg::ApplyParams prm;
    fill_params(ctx, p.dx[s], p.dy[s], transpose, prm);
    e = sg::launch_apply(ctx->hp, ctx->ls, prm, p.cmp);
  }
  if (e == cudaSuccess) e = cudaEventRecord(p.ev_done[s], p.cmp);
  // copy out, and make the caller's stream wait for it
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p.out, p.ev_done[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y_host, p.dy[s], n * sizeof(double), cudaMemcpyDeviceToHost, p.out);
  if (e == cudaSuccess) e = cudaEventRecord(p.ev_out[s], p.out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(us, p.ev_out[s], 0);
  if (e != cudaSuccess) return cuda_fail(e, "sg_apply_host_async");
  p.used[s] = true;
  p.slot = s ^ 1;
  return SG_OK;
}

sg_status sg_mg_setup(sg_ctx* ctx, int mg_precision, int nu, double omega) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_mg_setup: ctx is NULL");
  if (mg_precision != SG_PREC_FP64 && mg_precision != SG_PREC_FP32 && mg_precision != SG_PREC_BF16)
    return fail(SG_ERR_UNSUPPORTED, "sg_mg_setup: precision must be SG_PREC_FP64, SG_PREC_FP32 or SG_PREC_BF16");
  if (nu < 1 || nu > 16 || !(omega > 0.0 && omega <= 1.0)) return fail(SG_ERR_ARG, "sg_mg_setup: nu or omega out of range");
  cudaDeviceSynchronize();
  if (ctx->mg) {
    sg::mg_free(*ctx->mg);
    delete ctx->mg;
    ctx->mg = nullptr;
  }
  sg::MG* mg = new (std::nothrow) sg::MG();
  if (!mg) return fail(SG_ERR_OOM, "sg_mg_setup: host allocation failed");
  std::string msg;
  mg->coarse_dofs = ctx->mg_coarse_dofs;
  sg_status st = sg::mg_build(ctx->hp, mg_precision, nu, omega, *mg, msg);
  if (st != SG_OK) {
    sg::mg_free(*mg);
    delete mg;
    return fail(st, "sg_mg_setup: " + msg);
  }
  ctx->mg = mg;
  ++ctx->gen;
  return SG_OK;
}

sg_status sg_mg_set_coarse_dofs(sg_ctx* ctx, int max_dofs) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_mg_set_coarse_dofs: ctx is NULL");
  if (max_dofs < 0 || max_dofs > 2048) return fail(SG_ERR_ARG, "sg_mg_set_coarse_dofs: max_dofs must be 0..2048");
  ctx->mg_coarse_dofs = max_dofs;
  return SG_OK;
}

sg_status sg_set_coefficient(sg_ctx* ctx, const sg_coeff* coef) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_set_coefficient: ctx is NULL");
  sg::HostProblem& hp = ctx->hp;
  std::vector<sg::Piece> pieces;
  std::string msg;
  sg_status st = sg::parse_pieces(coef, hp.M, hp.n_cells, pieces, msg);
  if (st != SG_OK) return fail(st, "sg_set_coefficient: " + msg);
  if (pieces.size() != hp.pieces.size()) return fail(SG_ERR_ARG, "sg_set_coefficient: number of pieces differs");
  for (size_t i = 0; i < pieces.size(); ++i) {
    if (pieces[i].mu != hp.pieces[i].mu) return fail(SG_ERR_ARG, "sg_set_coefficient: chaos index of a piece differs");
    for (int d = 0; d < hp.dim; ++d) {
      const int kd = pieces[i].kind[d];
      if (kd != SG_F_ONE && kd != SG_F_SIN && kd != SG_F_POW) return fail(SG_ERR_ARG, "sg_set_coefficient: unknown factor kind");
      if (kd == SG_F_POW && pieces[i].k[d] < 0) return fail(SG_ERR_ARG, "sg_set_coefficient: negative power");
    }
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sg_set_coefficient: synchronize");
  std::vector<sg::Piece> old = std::move(hp.pieces);
  hp.pieces = std::move(pieces);
  st = sg::fill_ctab(hp, msg);
  if (st != SG_OK) {
    hp.pieces = std::move(old);
    sg::fill_ctab(hp, msg);
    return fail(st, "sg_set_coefficient: " + msg);
  }
  e = cudaMemcpy(ctx->d_ctab, hp.ctab.data(), hp.ctab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "sg_set_coefficient: upload");
  if (ctx->mg) {
    const int prec = ctx->mg->requested, nu = ctx->mg->nu;
    const double omega = ctx->mg->omega;
    return sg_mg_setup(ctx, prec, nu, omega);
  }
  return SG_OK;
}

sg_status sg_mg_level_info(sg_ctx* ctx, int level, int* info) {
  if (!ctx || !info) return fail(SG_ERR_ARG, "sg_mg_level_info: null argument");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_mg_level_info: call sg_mg_setup first");
  std::string msg;
  const sg_status st = sg::mg_level_info(*ctx->mg, level, info, msg);
  return st == SG_OK ? SG_OK : fail(st, "sg_mg_level_info: " + msg);
}

sg_status sg_mg_setup_times(sg_ctx* ctx, double* total_ms, double* factor_ms, double* tune_ms) {
  if (!ctx || !total_ms || !factor_ms || !tune_ms) return fail(SG_ERR_ARG, "sg_mg_setup_times: null argument");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_mg_setup_times: call sg_mg_setup first");
  *total_ms = ctx->mg->setup_ms;
  *factor_ms = ctx->mg->factor_ms;
  *tune_ms = ctx->mg->tune_ms;
  return SG_OK;
}

sg_status sg_mg_set_level_variant(sg_ctx* ctx, int level, int residual_kind, int vanka_chunk, int vanka_tile,
                                  int vanka_kind) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_mg_set_level_variant: ctx is NULL");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_mg_set_level_variant: call sg_mg_setup first");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sg_mg_set_level_variant: synchronize");
  std::string msg;
  const sg_status st =
      sg::mg_force_variant(*ctx->mg, level, residual_kind, vanka_chunk, vanka_tile, vanka_kind, msg);
  ++ctx->gen;
  return st == SG_OK ? SG_OK : fail(st, "sg_mg_set_level_variant: " + msg);
}

sg_status sg_mg_patch_inverse(sg_ctx* ctx, int level, int alpha, long long cell, double* out_host) {
  if (!ctx || !out_host) return fail(SG_ERR_ARG, "sg_mg_patch_inverse: null argument");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_mg_patch_inverse: call sg_mg_setup first");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sg_mg_patch_inverse: synchronize");
  std::string msg;
  const sg_status st = sg::mg_patch_inverse(*ctx->mg, level, alpha, cell, out_host, msg);
  return st == SG_OK ? SG_OK : fail(st, "sg_mg_patch_inverse: " + msg);
}

sg_status sg_vcycle(sg_ctx* ctx, const double* r, double* z, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_vcycle: ctx is NULL");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_vcycle: call sg_mg_setup first");
  if (!r || !z) return fail(SG_ERR_ARG, "sg_vcycle: null vector");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (r < z + n && z < r + n) return fail(SG_ERR_ARG, "sg_vcycle: r and z overlap");
  if (!is_device_ptr(r) || !is_device_ptr(z)) return fail(SG_ERR_ARG, "sg_vcycle: vectors must be device memory");
  cudaError_t e = sg::mg_apply(*ctx->mg, r, z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "sg_vcycle");
  return SG_OK;
}

sg_status sg_solve_slab(sg_ctx* ctx, int slab, const double* rhs, double* x, double rtol, int max_it,
                        int restart, sg_solve_stats* st, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_solve_slab: ctx is NULL");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_solve_slab: call sg_mg_setup first");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_solve_slab: slab out of range");
  if (!rhs || !x) return fail(SG_ERR_ARG, "sg_solve_slab: null vector");
  if (!(rtol > 0.0) || max_it < 1 || restart < 1 || restart > 200) return fail(SG_ERR_ARG, "sg_solve_slab: rtol, max_it or restart out of range");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (rhs < x + n && x < rhs + n) return fail(SG_ERR_ARG, "sg_solve_slab: rhs and x overlap");
  if (!is_device_ptr(rhs) || !is_device_ptr(x)) return fail(SG_ERR_ARG, "sg_solve_slab: vectors must be device memory");
  std::string msg;
  sg_status s = sg::fgmres(ctx, rhs, x, rtol, max_it, restart, st, reinterpret_cast<cudaStream_t>(stream), msg,
                           &apply_device);
  if (s != SG_OK) return fail(s, "sg_solve_slab: " + msg);
  return SG_OK;
}

sg_status sg_solve_slab_adjoint(sg_ctx* ctx, int slab, const double* rhs, double* x, double rtol, int max_it,
                                int restart, sg_solve_stats* st, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: ctx is NULL");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: call sg_mg_setup first");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: slab out of range");
  if (!rhs || !x) return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: null vector");
  if (!(rtol > 0.0) || max_it < 1 || restart < 1 || restart > 200)
    return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: rtol, max_it or restart out of range");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (rhs < x + n && x < rhs + n) return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: rhs and x overlap");
  if (!is_device_ptr(rhs) || !is_device_ptr(x))
    return fail(SG_ERR_ARG, "sg_solve_slab_adjoint: vectors must be device memory");
  std::string msg;
  sg_status s = sg::fgmres(ctx, rhs, x, rtol, max_it, restart, st, reinterpret_cast<cudaStream_t>(stream), msg,
                           &sg::apply_device_ctx_t, 1);
  if (s != SG_OK) return fail(s, "sg_solve_slab_adjoint: " + msg);
  return SG_OK;
}

sg_status sg_adjoint_gradient(sg_ctx* ctx, double rtol, int max_it, int checkpoint_every, int cell_piece,
                              double* J, double* grad_amp, double* grad_cell, sg_adjoint_stats* st,
                              sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_adjoint_gradient: ctx is NULL");
  if (!ctx->exact) return fail(SG_ERR_ARG, "sg_adjoint_gradient: call sg_set_exact first");
  if (!ctx->mg) return fail(SG_ERR_ARG, "sg_adjoint_gradient: call sg_mg_setup first");
  if (!(rtol > 0.0) || max_it < 1) return fail(SG_ERR_ARG, "sg_adjoint_gradient: rtol or max_it out of range");
  if (checkpoint_every < 1) return fail(SG_ERR_ARG, "sg_adjoint_gradient: checkpoint_every must be >= 1");
  if (cell_piece < -1 || cell_piece >= (int)ctx->hp.pieces.size())
    return fail(SG_ERR_ARG, "sg_adjoint_gradient: cell_piece out of range");
  std::string msg;
  sg_status s = sg::adjoint_gradient(ctx, rtol, max_it, checkpoint_every, cell_piece, J, grad_amp, grad_cell, st,
                                     reinterpret_cast<cudaStream_t>(stream), msg);
  if (s != SG_OK) return fail(s, "sg_adjoint_gradient: " + msg);
  return SG_OK;
}

__global__ void autotune_fill(double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = (double)((i * 2654435761LL) % 2001) / 1000.0 - 1.0;
}

sg_status sg_autotune(sg_ctx* ctx, int reps) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_autotune: ctx is NULL");
  if (reps < 1 || reps > 1000) return fail(SG_ERR_ARG, "sg_autotune: reps out of range");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  double *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&y, n * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(x);
    return cuda_fail(e, "sg_autotune: workspace");
  }
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    autotune_fill<<<256, 256, 0, s>>>(x, n);
    e = cudaGetLastError();
  }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const sg::LaunchShape orig = ctx->ls;
  sg::LaunchShape best = ctx->ls;
  float best_ms = 1e30f;
  const int max1 = sg::max_apply_chunk(ctx->hp, (size_t)optin - 1024);
  // every chunk size: the cells a CTA takes (cells / CTAs) split into whole
  // chunks for some sizes only, and a ragged last chunk costs a chunk's time
  std::vector<int> chunks;
  for (int c = std::min(max1, 16); c >= 1; --c) chunks.push_back(c);
  const int thread_opts[] = {128, 256, 384, 512};
  for (int c : chunks) {
    if (e != cudaSuccess) break;
    for (int t : thread_opts)
      for (int staggered = 0; staggered < (c > 1 ? 2 : 1); ++staggered) {
        sg::LaunchShape ls;
        std::string msg;
        if (sg::plan_apply_shape(ctx->hp, c, t, ls, msg) != SG_OK) continue;
        ls.stagger = staggered ? (c + 1) / 2 : 0;
        ctx->ls = ls;
  ++ctx->gen;
        sg::ApplyParams p;
        fill_params(ctx, x, y, 0, p);
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = sg::launch_apply(ctx->hp, ls, p, s);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = sg::launch_apply(ctx->hp, ls, p, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = ls;
        }
      }
  }
  ctx->ls = e == cudaSuccess ? best : orig;
  ++ctx->gen;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  cudaFree(x);
  cudaFree(y);
  if (e != cudaSuccess) return cuda_fail(e, "sg_autotune");
  return SG_OK;
}

sg_status sg_set_apply_shape(sg_ctx* ctx, int chunk, int threads, int stagger) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_set_apply_shape: ctx is NULL");
  if (chunk < 1 || threads < 1 || stagger < 0 || stagger > chunk)
    return fail(SG_ERR_ARG, "sg_set_apply_shape: chunk, threads or stagger out of range");
  sg::LaunchShape ls;
  std::string msg;
  const sg_status st = sg::plan_apply_shape(ctx->hp, chunk, threads, ls, msg);
  if (st != SG_OK) return fail(SG_ERR_ARG, "sg_set_apply_shape: " + msg);
  ls.stagger = stagger;
  ctx->ls = ls;
  ++ctx->gen;
  return SG_OK;
}

sg_status sg_set_exact(sg_ctx* ctx, int q, const double* c, const int* freq, int t_degree, const double* t_coef) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_set_exact: ctx is NULL");
  std::string msg;
  sg::ExactData* e = nullptr;
  sg_status st = sg::exact_build(ctx->hp, q, c, freq, t_degree, t_coef, e, msg);
  if (st != SG_OK) return fail(st, "sg_set_exact: " + msg);
  sg::exact_free(ctx->exact);
  ctx->exact = e;
  return SG_OK;
}

sg_status sg_rhs(sg_ctx* ctx, int slab, const double* u_prev, double* rhs, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_rhs: ctx is NULL");
  if (!ctx->exact) return fail(SG_ERR_ARG, "sg_rhs: call sg_set_exact first");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_rhs: slab out of range");
  if (!rhs || !is_device_ptr(rhs)) return fail(SG_ERR_ARG, "sg_rhs: rhs must be device memory");
  const long long n = (long long)ctx->hp.n_xi * ctx->hp.n_t * ctx->hp.n_x;
  if (u_prev) {
    if (!is_device_ptr(u_prev)) return fail(SG_ERR_ARG, "sg_rhs: u_prev must be device memory");
    if (u_prev < rhs + n && rhs < u_prev + n) return fail(SG_ERR_ARG, "sg_rhs: u_prev and rhs overlap");
  } else if (slab > 0) {
    return fail(SG_ERR_ARG, "sg_rhs: u_prev is required after the first slab");
  }
  cudaError_t e = sg::exact_rhs(ctx->hp, ctx->ls, *ctx->exact, ctx->d_ctab, ctx->d_gcol, ctx->d_gterm, ctx->d_gval,
                                ctx->d_perm, slab, u_prev, rhs, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "sg_rhs");
  return SG_OK;
}

sg_status sg_moments(sg_ctx* ctx, const double* u, int time_node, double* mean, double* var, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_moments: ctx is NULL");
  if (!u || !is_device_ptr(u)) return fail(SG_ERR_ARG, "sg_moments: u must be device memory");
  if (time_node < 0 || time_node >= ctx->hp.n_t) return fail(SG_ERR_ARG, "sg_moments: time node out of range");
  if ((mean && !is_device_ptr(mean)) || (var && !is_device_ptr(var)))
    return fail(SG_ERR_ARG, "sg_moments: outputs must be device memory");
  cudaError_t e = sg::moments(ctx->hp, u, time_node, mean, var, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "sg_moments");
  return SG_OK;
}

sg_status sg_qoi_errors(sg_ctx* ctx, const double* u, int slab, double* err) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_qoi_errors: ctx is NULL");
  if (!ctx->exact) return fail(SG_ERR_ARG, "sg_qoi_errors: call sg_set_exact first");
  if (!u || !is_device_ptr(u) || !err) return fail(SG_ERR_ARG, "sg_qoi_errors: bad pointer");
  if (slab < 0 || slab >= ctx->hp.n_slabs) return fail(SG_ERR_ARG, "sg_qoi_errors: slab out of range");
  cudaDeviceSynchronize();
  std::string msg;
  sg_status st = sg::exact_errors(ctx->hp, *ctx->exact, u, slab, err, msg);
  if (st != SG_OK) return fail(st, "sg_qoi_errors: " + msg);
  return SG_OK;
}

sg_status sg_stat_errors(sg_ctx* ctx, const double* mean, const double* var, double t, double* err) {
  if (!ctx) return fail(SG_ERR_ARG, "sg_stat_errors: ctx is NULL");
  if (!ctx->exact) return fail(SG_ERR_ARG, "sg_stat_errors: call sg_set_exact first");
  if (!mean || !var || !is_device_ptr(mean) || !is_device_ptr(var) || !err)
    return fail(SG_ERR_ARG, "sg_stat_errors: bad pointer");
  if (!(t >= 0.0) || !std::isfinite(t)) return fail(SG_ERR_ARG, "sg_stat_errors: t out of range");
  cudaDeviceSynchronize();
  std::string msg;
  sg_status st = sg::stat_errors(ctx->hp, *ctx->exact, mean, var, t, err, msg);
  if (st != SG_OK) return fail(st, "sg_stat_errors: " + msg);
  return SG_OK;
}

sg_status mc_solve_batch(sg_ctx* ctx, int n_samples, const double* xi, int batch, int mg_precision, double rtol,
                         int max_it, double* mean_T, double* var_T, double* u_T, sg_mc_stats* st, sg_stream stream) {
  if (!ctx) return fail(SG_ERR_ARG, "mc_solve_batch: ctx is NULL");
  if (!ctx->exact) return fail(SG_ERR_ARG, "mc_solve_batch: call sg_set_exact first");
  if (n_samples < 1 || !xi) return fail(SG_ERR_ARG, "mc_solve_batch: no samples");
  if (batch < 1 || batch > 512) return fail(SG_ERR_ARG, "mc_solve_batch: batch must be 1..512");
  if (mg_precision != SG_PREC_FP64 && mg_precision != SG_PREC_FP32 && mg_precision != SG_PREC_BF16)
    return fail(SG_ERR_ARG, "mc_solve_batch: mg_precision must be SG_PREC_FP64, SG_PREC_FP32 or SG_PREC_BF16");
  if (!(rtol > 0.0) || max_it < 1) return fail(SG_ERR_ARG, "mc_solve_batch: rtol or max_it out of range");
  if (!mean_T || !var_T || !is_device_ptr(mean_T) || !is_device_ptr(var_T) || mean_T == var_T)
    return fail(SG_ERR_ARG, "mc_solve_batch: mean_T and var_T must be distinct device vectors");
  if (u_T && !is_device_ptr(u_T)) return fail(SG_ERR_ARG, "mc_solve_batch: u_T must be device memory");
  std::string msg;
  sg_status s = sg::mc_solve(ctx, n_samples, xi, batch, mg_precision, rtol, max_it, mean_T, var_T, u_T, st,
                             reinterpret_cast<cudaStream_t>(stream), msg);
  if (s != SG_OK) return fail(s, "mc_solve_batch: " + msg);
  return SG_OK;
}

sg_status mc_solve_meshes(int n_meshes, sg_ctx* const* ctxs, const int* n_samples, const double* const* xi, int tile,
                          int mg_precision, double rtol, int max_it, double* const* mean_T, double* const* var_T,
                          double* const* u_T, sg_mc_stats* st, sg_stream stream) {
  if (n_meshes < 1 || n_meshes > sg::kMcMaxProb || !ctxs || !n_samples || !xi || !mean_T || !var_T)
    return fail(SG_ERR_ARG, "mc_solve_meshes: 1 to 4 meshes with their samples and outputs");
  if (tile < 1 || tile > 512) return fail(SG_ERR_ARG, "mc_solve_meshes: tile must be 1..512");
  if (mg_precision != SG_PREC_FP64 && mg_precision != SG_PREC_FP32 && mg_precision != SG_PREC_BF16)
    return fail(SG_ERR_ARG, "mc_solve_meshes: mg_precision must be SG_PREC_FP64, SG_PREC_FP32 or SG_PREC_BF16");
  if (!(rtol > 0.0) || max_it < 1) return fail(SG_ERR_ARG, "mc_solve_meshes: rtol or max_it out of range");
  std::vector<sg_ctx*> cs;
  std::vector<int> ns;
  std::vector<const double*> xs;
  std::vector<double*> mean, var, ut;
  for (int p = 0; p < n_meshes; ++p) {
    if (!ctxs[p] || !ctxs[p]->exact) return fail(SG_ERR_ARG, "mc_solve_meshes: every context needs sg_set_exact");
    if (n_samples[p] < 1 || !xi[p]) return fail(SG_ERR_ARG, "mc_solve_meshes: no samples for a mesh");
    if (!mean_T[p] || !var_T[p] || !is_device_ptr(mean_T[p]) || !is_device_ptr(var_T[p]) || mean_T[p] == var_T[p])
      return fail(SG_ERR_ARG, "mc_solve_meshes: mean_T and var_T must be distinct device vectors");
    if (u_T && u_T[p] && !is_device_ptr(u_T[p])) return fail(SG_ERR_ARG, "mc_solve_meshes: u_T must be device memory");
    cs.push_back(ctxs[p]);
    ns.push_back(n_samples[p]);
    xs.push_back(xi[p]);
    mean.push_back(mean_T[p]);
    var.push_back(var_T[p]);
    ut.push_back(u_T ? u_T[p] : nullptr);
  }
  std::string msg;
  sg_status s = sg::mc_solve_meshes(cs, ns, xs, tile, mg_precision, rtol, max_it, mean, var, ut, st,
                                    reinterpret_cast<cudaStream_t>(stream), msg);
  if (s != SG_OK) return fail(s, "mc_solve_meshes: " + msg);
  return SG_OK;
}

sg_status sg_get_info(const sg_ctx* ctx, sg_info* out) {
  if (!ctx || !out) return fail(SG_ERR_ARG, "sg_get_info: null argument");
  const sg::HostProblem& hp = ctx->hp;
  std::memset(out, 0, sizeof(*out));
  out->dim = hp.dim;
  out->fe_degree = hp.k;
  out->time_degree = hp.r;
  out->M = hp.M;
  out->chaos_order = hp.p;
  out->precision = hp.precision;
  out->n_xi = hp.n_xi;
  out->n_t = hp.n_t;
  out->n_terms = hp.n_terms;
  out->g_nnz = (int)hp.g.col.size();
  out->n_slabs = hp.n_slabs;
  out->n_x = hp.n_x;
  out->n_cells = hp.n_cells;
  out->n_unknowns = (int64_t)hp.n_xi * hp.n_t * hp.n_x;
  out->tau = hp.tau;
  out->chunk = ctx->ls.chunk;
  out->grid = ctx->ls.grid;
  out->threads = ctx->ls.threads;
  out->smem_bytes = (int)ctx->ls.smem;
  out->stagger = ctx->ls.stagger;
  return SG_OK;
}

sg_status sg_get_multi_indices(const sg_ctx* ctx, int* out) {
  if (!ctx || !out) return fail(SG_ERR_ARG, "sg_get_multi_indices: null argument");
  std::memcpy(out, ctx->hp.idx.data(), ctx->hp.idx.size() * sizeof(int));
  return SG_OK;
}

void sg_destroy(sg_ctx* ctx) {
  if (!ctx) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  free_ctx_device(ctx);
  cudaSetDevice(cur);
  delete ctx;
}

}  // extern "C"

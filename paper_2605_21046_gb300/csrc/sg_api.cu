// The extern "C" entry points of libsg declared in include/sg.h.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

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
  if (c->host_stream) cudaStreamDestroy(c->host_stream);
}

void fill_params(const sg_ctx* c, const double* x, double* y, int transpose, sg::ApplyParams& p) {
  const sg::HostProblem& hp = c->hp;
  std::memset(&p, 0, sizeof(p));
  p.x = x;
  p.y = y;
  p.ctab = c->d_ctab;
  p.g_row = c->d_grow;
  p.g_col = c->d_gcol;
  p.g_term = c->d_gterm;
  p.g_val = c->d_gval;
  p.perm = c->d_perm;
  p.n_x = hp.n_x;
  p.n_cells = hp.n_cells;
  for (int d = 0; d < 3; ++d) {
    p.nn[d] = hp.nn[d];
    p.cells[d] = hp.cells[d];
    p.ratio[d] = d < hp.dim ? (hp.h[0] * hp.h[0]) / (hp.h[d] * hp.h[d]) : 1.0;
    if (d < hp.dim && p.ratio[d] != 1.0) p.aniso = 1;
  }
  p.chunk = c->ls.chunk;
  p.n_xi = hp.n_xi;
  p.n_terms = hp.n_terms;
  p.nnz = (int)hp.g.col.size();
  const int nq = hp.k + 1;
  const int nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  double wJ[sg::kMaxQD];
  for (int qd = 0; qd < nqd; ++qd) {
    int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
    double w = detJ;
    for (int d = 0; d < hp.dim; ++d) w *= hp.wq[qi[d]];
    wJ[qd] = w;
  }
  const int nt = hp.n_t;
  for (int i = 0; i < nt; ++i) {
    const double tb = hp.tau * hp.B_hat[i * nt + i];
    p.tb[i] = tb;
    for (int j = 0; j < nt; ++j) {
      const double a = transpose ? hp.A_hat[j * nt + i] : hp.A_hat[i * nt + j];
      for (int qd = 0; qd < nqd; ++qd) p.amq[(qd * nt + i) * nt + j] = wJ[qd] * (a / tb);
    }
  }
}

}  // namespace

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
  sg_ctx* c = new (std::nothrow) sg_ctx();
  if (!c) return fail(SG_ERR_OOM, "sg_setup: host allocation failed");
  std::string msg;
  sg_status st = sg::build_host_problem(mesh, fe_degree, time_degree, n_slabs, T, M, chaos_order,
                                        coef, c->hp, msg);
  if (st != SG_OK) { delete c; return fail(st, "sg_setup: " + msg); }
  c->hp.precision = precision;
  cudaGetDevice(&c->device);
  st = sg::plan_apply(c->hp, c->ls, msg);
  if (st != SG_OK) { delete c; return fail(st, "sg_setup: " + msg); }
  cudaError_t e = sg::prepare_apply_kernel(precision, c->hp.dim, c->hp.k, c->hp.n_t, c->ls.smem);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "sg_setup: kernel attributes"); }
  if ((e = upload(&c->d_ctab, c->hp.ctab)) != cudaSuccess ||
      (e = upload(&c->d_grow, c->hp.g.row)) != cudaSuccess ||
      (e = upload(&c->d_gcol, c->hp.g.col)) != cudaSuccess ||
      (e = upload(&c->d_gterm, c->hp.g.term)) != cudaSuccess ||
      (e = upload(&c->d_gval, c->hp.g.val)) != cudaSuccess ||
      (e = upload(&c->d_perm, c->hp.perm)) != cudaSuccess) {
    free_ctx_device(c);
    delete c;
    return cuda_fail(e, "sg_setup: upload of tables");
  }
  *out = c;
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

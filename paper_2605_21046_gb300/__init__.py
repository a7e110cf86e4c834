"""GB300-native stochastic-Galerkin slab operator for the random heat equation.

Python binding of the C-ABI library libsg (include/sg.h).  The functions keep
the C names; they only marshal arguments (torch CUDA tensors for device
vectors, numpy arrays for host vectors) and raise ``SGError`` on a non-zero
status.  Every step of the operator runs in the library's CUDA kernels; there
is no CPU fallback: without libsg.so every call raises.

    ctx = sg_setup(mesh, fe_degree, time_degree, n_slabs, T, M, chaos_order, coef)
    sg_apply(ctx, slab, x, y)            # y = A^(n) x on the current stream
    sg_destroy(ctx)
"""
import ctypes as C

import numpy as np

from . import _abi, coefficients

SG_PREC_FP64, SG_PREC_DW, SG_PREC_FP32, SG_PREC_BF16 = (_abi.SG_PREC_FP64, _abi.SG_PREC_DW, _abi.SG_PREC_FP32,
                                                      _abi.SG_PREC_BF16)

__all__ = ["SG_PREC_FP64", "SG_PREC_DW", "SG_PREC_FP32", "SG_PREC_BF16", "sg_mg_setup", "sg_mg_level_info", "sg_mg_set_level_variant", "sg_mg_patch_inverse", "sg_vcycle", "sg_solve_slab", "sg_autotune", "sg_set_apply_shape", "sg_set_exact", "sg_rhs", "sg_moments", "sg_qoi_errors", "mc_solve_batch", "SGError", "SGContext", "sg_setup", "sg_setup_spec", "sg_apply", "sg_apply_host", "sg_apply_host_async", "sg_get_info",
           "sg_get_multi_indices", "sg_destroy", "sg_status_string", "mesh_spec"]

_KIND = {"one": _abi.SG_F_ONE, "sin": _abi.SG_F_SIN, "pow": _abi.SG_F_POW}


class SGError(RuntimeError):
    def __init__(self, status, where):
        lib = _abi.load()
        super().__init__(f"{where}: {lib.sg_status_string(status).decode()} "
                         f"({lib.sg_last_error().decode()})")
        self.status = status


def _check(status, where):
    if status != _abi.SG_OK:
        raise SGError(status, where)


class SGContext:
    """Owns one sg_ctx; ``info`` holds its sizes."""

    def __init__(self, handle, n_pieces=None):
        self._h = C.c_void_p(handle)
        self.info = sg_get_info(self)
        self.n_pieces = n_pieces

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("context destroyed")
        return self._h

    @property
    def shape(self):
        return (self.info["n_xi"], self.info["n_t"], self.info["n_x"])

    def apply(self, x, y=None, slab=0, transpose=False, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        sg_apply(self, slab, x, y, transpose, stream)
        return y

    def destroy(self):
        if self._h:
            _abi.load().sg_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mesh_spec(dim, cells, lo, hi):
    m = _abi.sg_mesh()
    m.dim = dim
    for d in range(3):
        m.cells[d] = int(cells[d]) if d < dim else 1
        m.lo[d] = float(lo[d]) if d < dim else 0.0
        m.hi[d] = float(hi[d]) if d < dim else 1.0
    return m


def _coeff_struct(pieces, M, dim):
    pieces = coefficients.pieces(pieces, M)
    n = len(pieces)
    mu = np.zeros((n, M), dtype=np.int32)
    amp = np.zeros(n, dtype=np.float64)
    kind = np.zeros((n, 3), dtype=np.int32)
    kk = np.zeros((n, 3), dtype=np.int32)
    scales = (C.POINTER(C.c_double) * n)()
    keep = [mu, amp, kind, kk, scales]
    any_scale = False
    for i, p in enumerate(pieces):
        mu[i] = np.asarray(p["mu"], dtype=np.int32)
        amp[i] = float(p["amp"])
        for d in range(min(dim, 3, len(p["factors"]))):
            kd, kv = p["factors"][d]
            kind[i, d] = _KIND[kd]
            kk[i, d] = int(kv)
        cs = p.get("cell_scale")
        if cs is not None:
            arr = np.ascontiguousarray(cs, dtype=np.float64)
            keep.append(arr)
            scales[i] = arr.ctypes.data_as(C.POINTER(C.c_double))
            any_scale = True
    s = _abi.sg_coeff()
    s.n_pieces = n
    s.mu = mu.ctypes.data_as(C.POINTER(C.c_int))
    s.amp = amp.ctypes.data_as(C.POINTER(C.c_double))
    s.factor_kind = kind.ctypes.data_as(C.POINTER(C.c_int))
    s.factor_k = kk.ctypes.data_as(C.POINTER(C.c_int))
    s.cell_scale = C.cast(scales, C.POINTER(C.POINTER(C.c_double))) if any_scale else None
    return s, keep


def sg_setup(mesh, fe_degree, time_degree, n_slabs, T, M, chaos_order, coef, precision=0):
    """sg_setup of include/sg.h.  ``mesh`` is an sg_mesh or a dict with
    dim/cells/lo/hi; ``coef`` a list of separable pieces
    {"mu", "amp", "factors": [(kind, k) per direction], "cell_scale"} or a
    ``square_of_linear`` description (``coefficients``)."""
    lib = _abi.load()
    if isinstance(mesh, dict):
        mesh = mesh_spec(mesh["dim"], mesh["cells"], mesh["lo"], mesh["hi"])
    cs, keep = _coeff_struct(coef, M, mesh.dim)
    h = C.c_void_p()
    _check(lib.sg_setup(C.byref(mesh), fe_degree, time_degree, n_slabs, float(T), M, chaos_order,
                        C.byref(cs), precision, C.byref(h)), "sg_setup")
    del keep
    return SGContext(h.value, cs.n_pieces)


def sg_setup_spec(spec, precision=0):
    """sg_setup from a problem spec dict (the format of ``inputs``)."""
    return sg_setup(dict(dim=spec["dim"], cells=spec["cells"], lo=spec["lo"], hi=spec["hi"]),
                    spec["k"], spec["r"], spec["n_slabs"], spec["T"], spec["M"], spec["P"],
                    spec["coef"], precision)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sg_apply(ctx, slab, x, y, transpose=False, stream=None):
    """y = A^(n) x (or A^T x) for torch float64 CUDA tensors of n_unknowns
    elements, launched on ``stream`` (default: torch's current stream)."""
    lib = _abi.load()
    n = ctx.info["n_unknowns"]
    for t in (x, y):
        if not (t.is_cuda and t.dtype.itemsize == 8 and str(t.dtype) == "torch.float64"):
            raise TypeError("sg_apply wants float64 CUDA tensors")
        if t.numel() != n or not t.is_contiguous():
            raise ValueError(f"sg_apply wants contiguous tensors of {n} elements")
    _check(lib.sg_apply(ctx.handle, int(slab), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                        int(bool(transpose)), C.c_void_p(_stream_handle(stream))), "sg_apply")
    return y


def sg_apply_host(ctx, slab, x, y=None, transpose=False):
    """Host-buffer variant: numpy float64 (or pinned torch CPU tensors) in,
    result written to ``y`` (allocated if None); synchronous."""
    lib = _abi.load()
    n = ctx.info["n_unknowns"]

    def ptr(a):
        if hasattr(a, "data_ptr"):
            if a.numel() != n or not a.is_contiguous() or a.is_cuda:
                raise ValueError("host tensor of n_unknowns contiguous elements expected")
            return a.data_ptr()
        if a.dtype != np.float64 or a.size != n or not a.flags.c_contiguous:
            raise ValueError("float64 contiguous host array of n_unknowns elements expected")
        return a.ctypes.data
    if y is None:
        y = np.empty(n, dtype=np.float64)
    _check(lib.sg_apply_host(ctx.handle, int(slab), C.c_void_p(ptr(x)), C.c_void_p(ptr(y)),
                             int(bool(transpose))), "sg_apply_host")
    return y


def sg_apply_host_async(ctx, slab, x, y, transpose=False, stream=None):
    """Pipelined host-buffer apply (sg_apply_host_async): page-locked torch CPU
    float64 tensors ``x`` (read) and ``y`` (written); returns without waiting,
    ``y`` is valid once ``stream`` (default: the current CUDA stream) is
    synchronized."""
    n = ctx.info["n_unknowns"]
    for t in (x, y):
        if (not hasattr(t, "is_pinned") or t.is_cuda or not t.is_pinned() or t.numel() != n
                or not t.is_contiguous() or str(t.dtype) != "torch.float64"):
            raise ValueError("page-locked contiguous float64 CPU tensors of n_unknowns elements expected")
    _check(_abi.load().sg_apply_host_async(ctx.handle, int(slab), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                           int(bool(transpose)), C.c_void_p(_stream_handle(stream))),
           "sg_apply_host_async")
    return y


def _check_vec(ctx, *ts):
    n = ctx.info["n_unknowns"]
    for t in ts:
        if not (t.is_cuda and str(t.dtype) == "torch.float64"):
            raise TypeError("float64 CUDA tensors expected")
        if t.numel() != n or not t.is_contiguous():
            raise ValueError(f"contiguous tensors of {n} elements expected")


def sg_mg_setup(ctx, mg_precision=SG_PREC_FP64, nu=2, omega=0.7):
    """Build the block-Jacobi multigrid preconditioner (sg_mg_setup)."""
    _check(_abi.load().sg_mg_setup(ctx.handle, int(mg_precision), int(nu), float(omega)), "sg_mg_setup")


def sg_debug_bounds():
    """The device bounds records of the debug build (sg_debug_bounds): a dict
    with enabled, count and the first violation's site, index and limit."""
    en, cnt, site, idx, lim = C.c_int(), C.c_uint(), C.c_int(), C.c_longlong(), C.c_longlong()
    _check(_abi.load().sg_debug_bounds(C.byref(en), C.byref(cnt), C.byref(site), C.byref(idx), C.byref(lim)),
           "sg_debug_bounds")
    return {"enabled": en.value, "count": cnt.value, "site": site.value, "index": idx.value, "limit": lim.value}


def sg_debug_bounds_probe(index, limit):
    """Self-test of the bounds record path (sg_debug_bounds_probe)."""
    _check(_abi.load().sg_debug_bounds_probe(int(index), int(limit)), "sg_debug_bounds_probe")


def sg_mg_set_coarse_dofs(ctx, max_dofs):
    """Coarsest-level size of the next sg_mg_setup (sg_mg_set_coarse_dofs):
    coarsening stops at the first level with at most max_dofs interior
    space-time unknowns per chaos row; 0 coarsens to two cells per direction."""
    _check(_abi.load().sg_mg_set_coarse_dofs(ctx.handle, int(max_dofs)), "sg_mg_set_coarse_dofs")


def sg_debug_wait_probe(polls=1000):
    """Self-test of the bounded completion wait (sg_debug_wait_probe): the
    status the waiting kernel recorded (SG_ERR_TIMEOUT when the wait ran out)."""
    st = C.c_int(0)
    _check(_abi.load().sg_debug_wait_probe(int(polls), C.byref(st)), "sg_debug_wait_probe")
    return st.value


def sg_mg_level_info(ctx, level):
    """The choices of the preconditioner on one level (sg_mg_level_info)."""
    info = (C.c_int * 10)()
    _check(_abi.load().sg_mg_level_info(ctx.handle, int(level), info), "sg_mg_level_info")
    keys = ("levels", "cells", "coarsest", "residual", "vanka_chunk", "vanka_tile", "np", "classes", "vanka_kind")
    return dict(zip(keys, list(info)))


def sg_mg_setup_times(ctx):
    """Wall times of the last sg_mg_setup in ms: total, patch factorisation and
    variant timing (sg_mg_setup_times)."""
    t, f, u = C.c_double(), C.c_double(), C.c_double()
    _check(_abi.load().sg_mg_setup_times(ctx.handle, C.byref(t), C.byref(f), C.byref(u)), "sg_mg_setup_times")
    return {"total_ms": t.value, "factor_ms": f.value, "tune_ms": u.value}


def sg_mg_set_level_variant(ctx, level=-1, residual_kind=-1, vanka_chunk=0, vanka_tile=-1, vanka_kind=-1):
    """Force the residual kind / Vanka chunk / Vanka tile / Vanka kernel of one
    smoothed level or of all of them (sg_mg_set_level_variant)."""
    _check(_abi.load().sg_mg_set_level_variant(ctx.handle, int(level), int(residual_kind), int(vanka_chunk),
                                               int(vanka_tile), int(vanka_kind)), "sg_mg_set_level_variant")


def sg_mg_patch_inverse(ctx, level, alpha, cell):
    """The stored inverse of one Vanka patch as an (np, np) numpy array."""
    info = sg_mg_level_info(ctx, level)
    out = np.zeros((info["np"], info["np"]), dtype=np.float64)
    _check(_abi.load().sg_mg_patch_inverse(ctx.handle, int(level), int(alpha), int(cell),
                                           out.ctypes.data_as(C.POINTER(C.c_double))), "sg_mg_patch_inverse")
    return out


def sg_vcycle(ctx, r, z, stream=None):
    """z = P^{-1} r (one V-cycle per chaos mode) on ``stream``."""
    _check_vec(ctx, r, z)
    _check(_abi.load().sg_vcycle(ctx.handle, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()),
                                 C.c_void_p(_stream_handle(stream))), "sg_vcycle")
    return z


def sg_solve_slab(ctx, slab, rhs, x, rtol=1e-8, max_it=500, restart=30, stream=None, check=True):
    """FGMRES solve of A^(n) x = rhs; x holds the initial guess.  Returns the
    statistics dict; raises SGError on failure when ``check``."""
    _check_vec(ctx, rhs, x)
    st = _abi.sg_solve_stats()
    status = _abi.load().sg_solve_slab(ctx.handle, int(slab), C.c_void_p(rhs.data_ptr()),
                                       C.c_void_p(x.data_ptr()), float(rtol), int(max_it), int(restart),
                                       C.byref(st), C.c_void_p(_stream_handle(stream)))
    out = {name: getattr(st, name) for name, _ in _abi.sg_solve_stats._fields_}
    out["status"] = status
    if check:
        _check(status, "sg_solve_slab")
    return out


def sg_solve_slab_adjoint(ctx, slab, rhs, x, rtol=1e-8, max_it=500, restart=30, stream=None, check=True):
    """FGMRES solve of the transposed slab system A^T x = rhs (the adjoint
    equation); x holds the initial guess.  Returns the statistics dict."""
    _check_vec(ctx, rhs, x)
    st = _abi.sg_solve_stats()
    status = _abi.load().sg_solve_slab_adjoint(ctx.handle, int(slab), C.c_void_p(rhs.data_ptr()),
                                               C.c_void_p(x.data_ptr()), float(rtol), int(max_it), int(restart),
                                               C.byref(st), C.c_void_p(_stream_handle(stream)))
    out = {name: getattr(st, name) for name, _ in _abi.sg_solve_stats._fields_}
    out["status"] = status
    if check:
        _check(status, "sg_solve_slab_adjoint")
    return out


def sg_adjoint_gradient(ctx, rtol=1e-10, max_it=500, checkpoint_every=10, cell_piece=-1, stream=None,
                        gradient=True):
    """J = E ||u_h(T)||^2 of the marched manufactured problem and its gradient
    with respect to every piece amplitude and (cell_piece >= 0) the per-cell
    scale of one piece.  Returns (J, grad_amp, grad_cell or None, stats);
    ``gradient=False`` runs the forward sweep only (grads None)."""
    n_pieces = ctx.n_pieces
    g_amp = np.zeros(max(n_pieces, 1), dtype=np.float64) if gradient else None
    g_cell = np.zeros(ctx.info["n_cells"], dtype=np.float64) if (cell_piece >= 0 and gradient) else None
    J = C.c_double(0.0)
    st = _abi.sg_adjoint_stats()
    _check(_abi.load().sg_adjoint_gradient(
        ctx.handle, float(rtol), int(max_it), int(checkpoint_every), int(cell_piece), C.byref(J),
        g_amp.ctypes.data_as(C.POINTER(C.c_double)) if g_amp is not None else None,
        g_cell.ctypes.data_as(C.POINTER(C.c_double)) if g_cell is not None else None,
        C.byref(st), C.c_void_p(_stream_handle(stream))), "sg_adjoint_gradient")
    stats = {name: getattr(st, name) for name, _ in _abi.sg_adjoint_stats._fields_}
    return J.value, (g_amp[:n_pieces] if g_amp is not None else None), g_cell, stats


def sg_set_coefficient(ctx, coef):
    """Replace the coefficient pieces (same count, same mu per piece) keeping
    the mesh, tables and manufactured load vector (sg_set_coefficient)."""
    cs, keep = _coeff_struct(coef, ctx.info["M"], ctx.info["dim"])
    _check(_abi.load().sg_set_coefficient(ctx.handle, C.byref(cs)), "sg_set_coefficient")
    del keep


def _pieces_with(spec, amp, cell_piece=-1, cell_scale=None):
    coef = [dict(p) for p in spec["coef"]]
    for i, p in enumerate(coef):
        p["amp"] = float(amp[i])
    if cell_piece >= 0 and cell_scale is not None:
        coef[cell_piece]["cell_scale"] = np.asarray(cell_scale, dtype=np.float64)
    return coef


def _make_energy_function():
    import torch

    class EnergyAtT(torch.autograd.Function):
        """J(amp, cell_scale) = E ||u_h(T)||^2 of the marched manufactured
        problem; backward is the discrete adjoint (sg_adjoint_gradient)."""

        @staticmethod
        def forward(fctx, amp, cell_scale, spec, exact, cell_piece, mg_precision, rtol, checkpoint_every):
            a = amp.detach().cpu().numpy()
            cs = cell_scale.detach().cpu().numpy() if cell_scale is not None else None
            ctx = sg_setup_spec(spec)
            try:
                sg_set_exact(ctx, exact)   # load vector of the nominal coefficient, held fixed
                sg_set_coefficient(ctx, _pieces_with(spec, a, cell_piece, cs))
                sg_mg_setup(ctx, mg_precision)
                J, g_amp, g_cell, _ = sg_adjoint_gradient(ctx, rtol=rtol, checkpoint_every=checkpoint_every,
                                                          cell_piece=cell_piece if cs is not None else -1)
            finally:
                ctx.destroy()
            fctx.has_cell = g_cell is not None
            fctx.save_for_backward(torch.from_numpy(g_amp.copy()).to(amp),
                                   torch.from_numpy(g_cell.copy()).to(cell_scale) if fctx.has_cell
                                   else amp.new_zeros(0))
            return amp.new_tensor(J)

        @staticmethod
        def backward(fctx, gJ):
            g_amp, g_cell = fctx.saved_tensors
            return (gJ * g_amp, gJ * g_cell if fctx.has_cell else None, None, None, None, None, None, None)

    return EnergyAtT


_ENERGY = None


def energy_at_T(spec, exact, amp, cell_scale=None, cell_piece=-1, mg_precision=0, rtol=1e-10,
                checkpoint_every=10):
    """J = E ||u_h(T)||^2 as a differentiable torch function of the piece
    amplitudes (1-D float64 CPU tensor) and, with cell_piece >= 0, of the
    per-cell scale of that piece.  The operator uses (amp, cell_scale); the
    load vector is the one of ``spec``'s own coefficient, held fixed; the
    gradient comes from the discrete adjoint on the GPU."""
    global _ENERGY
    if _ENERGY is None:
        _ENERGY = _make_energy_function()
    return _ENERGY.apply(amp, cell_scale, spec, exact, cell_piece, mg_precision, rtol, checkpoint_every)


def sg_set_exact(ctx, exact):
    """Attach a manufactured solution {"q", "c", "freq" (per mode, per
    direction), "T" (polynomial coefficients)} (sg_set_exact)."""
    c = np.ascontiguousarray(exact["c"], dtype=np.float64)
    freq = np.zeros((c.size, 3), dtype=np.int32)
    for a, f in enumerate(exact["freq"]):
        freq[a, :len(f)] = f
    tc = np.ascontiguousarray(exact["T"], dtype=np.float64)
    _check(_abi.load().sg_set_exact(ctx.handle, int(exact["q"]), c.ctypes.data_as(C.POINTER(C.c_double)),
                                    freq.ctypes.data_as(C.POINTER(C.c_int)), tc.size - 1,
                                    tc.ctypes.data_as(C.POINTER(C.c_double))), "sg_set_exact")


def sg_rhs(ctx, slab, u_prev, rhs, stream=None):
    """rhs = F^(n) + J u_prev (first slab: F^(1) + B_0) on ``stream``."""
    _check_vec(ctx, rhs)
    if u_prev is not None:
        _check_vec(ctx, u_prev)
    _check(_abi.load().sg_rhs(ctx.handle, int(slab), C.c_void_p(u_prev.data_ptr() if u_prev is not None else None),
                              C.c_void_p(rhs.data_ptr()), C.c_void_p(_stream_handle(stream))), "sg_rhs")
    return rhs


def sg_moments(ctx, u, time_node, mean=None, var=None, stream=None):
    """Pointwise mean and variance at one time node (device tensors of n_x)."""
    import torch
    _check_vec(ctx, u)
    n_x = ctx.info["n_x"]
    mean = torch.empty(n_x, dtype=torch.float64, device=u.device) if mean is None else mean
    var = torch.empty(n_x, dtype=torch.float64, device=u.device) if var is None else var
    _check(_abi.load().sg_moments(ctx.handle, C.c_void_p(u.data_ptr()), int(time_node), C.c_void_p(mean.data_ptr()),
                                  C.c_void_p(var.data_ptr()), C.c_void_p(_stream_handle(stream))), "sg_moments")
    return mean, var


def sg_qoi_errors(ctx, u, slab):
    """(mean, variance, full) L2 errors at the end of slab ``slab``."""
    _check_vec(ctx, u)
    err = (C.c_double * 3)()
    _check(_abi.load().sg_qoi_errors(ctx.handle, C.c_void_p(u.data_ptr()), int(slab), err), "sg_qoi_errors")
    return {"mean": err[0], "var": err[1], "full": err[2]}


def sg_stat_errors(ctx, mean, var, t):
    """L2(D) errors (mean, variance) of nodal fields against the manufactured
    solution's exact statistics at time t."""
    _check_vec_n(ctx, mean, var)
    err = (C.c_double * 2)()
    _check(_abi.load().sg_stat_errors(ctx.handle, C.c_void_p(mean.data_ptr()), C.c_void_p(var.data_ptr()),
                                      float(t), err), "sg_stat_errors")
    return {"mean": err[0], "var": err[1]}


def _check_vec_n(ctx, *ts):
    n = ctx.info["n_x"]
    for t in ts:
        if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.numel() == n and t.is_contiguous()):
            raise ValueError(f"wants contiguous float64 CUDA tensors of {n} elements")


def mc_solve_batch(ctx, xi, batch=256, mg_precision=SG_PREC_FP32, rtol=1e-8, max_it=500, keep_paths=False,
                   stream=None):
    """Monte-Carlo mean and unbiased variance at t = T over the samples ``xi``
    (numpy array n_samples x M); returns (mean, var, u_T or None, stats)."""
    import torch
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    n_s = xi.shape[0]
    n_x, n_t = ctx.info["n_x"], ctx.info["n_t"]
    dev = torch.device("cuda", torch.cuda.current_device())
    mean = torch.empty(n_x, dtype=torch.float64, device=dev)
    var = torch.empty(n_x, dtype=torch.float64, device=dev)
    u_T = torch.empty(n_s * n_t * n_x, dtype=torch.float64, device=dev) if keep_paths else None
    st = _abi.sg_mc_stats()
    _check(_abi.load().mc_solve_batch(ctx.handle, n_s, xi.ctypes.data_as(C.POINTER(C.c_double)), int(batch),
                                      int(mg_precision), float(rtol), int(max_it), C.c_void_p(mean.data_ptr()),
                                      C.c_void_p(var.data_ptr()), C.c_void_p(u_T.data_ptr() if u_T is not None else None),
                                      C.byref(st), C.c_void_p(_stream_handle(stream))), "mc_solve_batch")
    return mean, var, u_T, {name: getattr(st, name) for name, _ in _abi.sg_mc_stats._fields_}


def mc_solve_meshes(ctxs, xis, tile=64, mg_precision=SG_PREC_FP32, rtol=1e-8, max_it=500, keep_paths=False,
                    stream=None):
    """Monte-Carlo on several meshes in one system per slab: ``ctxs`` and
    ``xis`` (numpy n_samples_p x M arrays) per mesh.  Returns
    (means, vars, paths or None per mesh, stats)."""
    import torch
    P = len(ctxs)
    dev = torch.device("cuda", torch.cuda.current_device())
    xs = [np.ascontiguousarray(x, dtype=np.float64) for x in xis]
    means = [torch.empty(c.info["n_x"], dtype=torch.float64, device=dev) for c in ctxs]
    vars_ = [torch.empty(c.info["n_x"], dtype=torch.float64, device=dev) for c in ctxs]
    paths = [torch.empty(x.shape[0] * c.info["n_t"] * c.info["n_x"], dtype=torch.float64, device=dev)
             for c, x in zip(ctxs, xs)] if keep_paths else None
    vp = C.c_void_p
    h = (vp * P)(*[c.handle.value for c in ctxs])
    ns = (C.c_int * P)(*[x.shape[0] for x in xs])
    xp = (C.POINTER(C.c_double) * P)(*[x.ctypes.data_as(C.POINTER(C.c_double)) for x in xs])
    mp = (vp * P)(*[t.data_ptr() for t in means])
    vv = (vp * P)(*[t.data_ptr() for t in vars_])
    up = (vp * P)(*[t.data_ptr() for t in paths]) if paths is not None else None
    st = _abi.sg_mc_stats()
    _check(_abi.load().mc_solve_meshes(P, h, ns, xp, int(tile), int(mg_precision), float(rtol), int(max_it), mp, vv,
                                       up, C.byref(st), C.c_void_p(_stream_handle(stream))), "mc_solve_meshes")
    return means, vars_, paths, {name: getattr(st, name) for name, _ in _abi.sg_mc_stats._fields_}


def sg_autotune(ctx, reps=10):
    """Pick the fastest apply launch shape for this context (sg_autotune)."""
    _check(_abi.load().sg_autotune(ctx.handle, int(reps)), "sg_autotune")
    ctx.info = sg_get_info(ctx)
    return ctx.info


def sg_set_apply_shape(ctx, chunk, threads, stagger=0):
    """Fix the apply launch shape (sg_set_apply_shape): cells per chunk,
    threads per CTA, first-chunk cells of the upper half of the CTAs."""
    _check(_abi.load().sg_set_apply_shape(ctx.handle, int(chunk), int(threads), int(stagger)),
           "sg_set_apply_shape")
    ctx.info = sg_get_info(ctx)
    return ctx.info


def sg_get_info(ctx):
    lib = _abi.load()
    info = _abi.sg_info()
    _check(lib.sg_get_info(ctx.handle, C.byref(info)), "sg_get_info")
    return {name: getattr(info, name) for name, _ in _abi.sg_info._fields_}


def sg_get_multi_indices(ctx):
    lib = _abi.load()
    n, M = ctx.info["n_xi"], ctx.info["M"]
    out = np.zeros((n, M), dtype=np.int32)
    _check(lib.sg_get_multi_indices(ctx.handle, out.ctypes.data_as(C.POINTER(C.c_int))),
           "sg_get_multi_indices")
    return out


def sg_destroy(ctx):
    ctx.destroy()


def sg_status_string(status):
    return _abi.load().sg_status_string(status).decode()

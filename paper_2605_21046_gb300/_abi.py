"""ctypes declarations of the C ABI in include/sg.h (argument marshalling only)."""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsg.so")
# the build with device bounds checks (loaded instead when SG_DEBUG_BOUNDS=1)
LIB_DEBUG_PATH = os.path.join(PKG, "libsg_debug.so")

SG_OK, SG_ERR_ARG, SG_ERR_CUDA, SG_ERR_OOM, SG_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
SG_ERR_NOT_CONVERGED, SG_ERR_NONFINITE, SG_ERR_TIMEOUT = 5, 6, 7
SG_F_ONE, SG_F_SIN, SG_F_POW = 0, 1, 2
SG_PREC_FP64, SG_PREC_DW, SG_PREC_FP32, SG_PREC_BF16 = 0, 1, 2, 3

# every symbol include/sg.h declares
EXPORTED = sorted(["sg_setup", "sg_apply", "sg_apply_host", "sg_get_info", "sg_get_multi_indices",
                   "sg_destroy", "sg_status_string", "sg_last_error", "sg_mg_setup", "sg_vcycle",
                   "sg_solve_slab", "sg_apply_host_static", "sg_autotune", "sg_set_exact",
                   "sg_rhs", "sg_moments", "sg_qoi_errors", "mc_solve_batch",
                   "sg_solve_slab_adjoint", "sg_adjoint_gradient", "sg_set_coefficient",
                   "sg_stat_errors", "mc_solve_meshes", "sg_set_apply_shape",
                   "sg_apply_host_async", "sg_mg_level_info", "sg_mg_set_level_variant",
                   "sg_mg_patch_inverse", "sg_debug_bounds", "sg_debug_bounds_probe", "sg_mg_setup_times",
                   "sg_debug_wait_probe", "sg_mg_set_coarse_dofs"])


class sg_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("cells", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3)]


class sg_coeff(C.Structure):
    _fields_ = [("n_pieces", C.c_int), ("mu", C.POINTER(C.c_int)), ("amp", C.POINTER(C.c_double)),
                ("factor_kind", C.POINTER(C.c_int)), ("factor_k", C.POINTER(C.c_int)),
                ("cell_scale", C.POINTER(C.POINTER(C.c_double)))]


class sg_info(C.Structure):
    _fields_ = [("dim", C.c_int), ("fe_degree", C.c_int), ("time_degree", C.c_int), ("M", C.c_int),
                ("chaos_order", C.c_int), ("precision", C.c_int), ("n_xi", C.c_int), ("n_t", C.c_int), ("n_terms", C.c_int),
                ("g_nnz", C.c_int), ("n_slabs", C.c_int), ("n_x", C.c_int64), ("n_cells", C.c_int64),
                ("n_unknowns", C.c_int64), ("tau", C.c_double), ("chunk", C.c_int),
                ("grid", C.c_int), ("threads", C.c_int), ("smem_bytes", C.c_int),
                ("stagger", C.c_int)]


class sg_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("vmult_calls", C.c_int),
                ("prec_calls", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("mg_setup_ms", C.c_double)]


class sg_adjoint_stats(C.Structure):
    _fields_ = [("forward_solves", C.c_int), ("adjoint_solves", C.c_int), ("max_iterations", C.c_int),
                ("checkpoints", C.c_int), ("J", C.c_double), ("solve_ms", C.c_double)]


class sg_mc_stats(C.Structure):
    _fields_ = [("n_samples", C.c_int), ("batches", C.c_int), ("total_iterations", C.c_int),
                ("max_slab_iterations", C.c_int), ("max_rel_residual", C.c_double), ("solve_ms", C.c_double),
                ("tile", C.c_int), ("chunk", C.c_int)]


_lib = None


def load():
    """Load libsg.so once; raises if it has not been built (there is no
    fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB_DEBUG_PATH if os.environ.get("SG_DEBUG_BOUNDS") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run paper_2605_21046_gb300.build.build()")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.sg_setup.argtypes = [C.POINTER(sg_mesh), C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                             C.POINTER(sg_coeff), C.c_int, C.POINTER(vp)]
    lib.sg_setup.restype = C.c_int
    lib.sg_apply.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp]
    lib.sg_apply.restype = C.c_int
    lib.sg_apply_host.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    lib.sg_apply_host.restype = C.c_int
    lib.sg_get_info.argtypes = [vp, C.POINTER(sg_info)]
    lib.sg_get_info.restype = C.c_int
    lib.sg_get_multi_indices.argtypes = [vp, C.POINTER(C.c_int)]
    lib.sg_get_multi_indices.restype = C.c_int
    lib.sg_mg_setup.argtypes = [vp, C.c_int, C.c_int, C.c_double]
    lib.sg_mg_setup.restype = C.c_int
    lib.sg_vcycle.argtypes = [vp, vp, vp, vp]
    lib.sg_vcycle.restype = C.c_int
    lib.sg_debug_bounds.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_uint), C.POINTER(C.c_int),
                                    C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.sg_debug_bounds.restype = C.c_int
    lib.sg_debug_bounds_probe.argtypes = [C.c_longlong, C.c_longlong]
    lib.sg_debug_bounds_probe.restype = C.c_int
    lib.sg_mg_set_coarse_dofs.argtypes = [vp, C.c_int]
    lib.sg_mg_set_coarse_dofs.restype = C.c_int
    lib.sg_debug_wait_probe.argtypes = [C.c_uint, C.POINTER(C.c_int)]
    lib.sg_debug_wait_probe.restype = C.c_int
    lib.sg_mg_setup_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.sg_mg_setup_times.restype = C.c_int
    lib.sg_mg_level_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    lib.sg_mg_level_info.restype = C.c_int
    lib.sg_mg_set_level_variant.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.sg_mg_set_level_variant.restype = C.c_int
    lib.sg_mg_patch_inverse.argtypes = [vp, C.c_int, C.c_int, C.c_longlong, C.POINTER(C.c_double)]
    lib.sg_mg_patch_inverse.restype = C.c_int
    lib.sg_solve_slab.argtypes = [vp, C.c_int, vp, vp, C.c_double, C.c_int, C.c_int,
                                  C.POINTER(sg_solve_stats), vp]
    lib.sg_solve_slab.restype = C.c_int
    lib.sg_set_exact.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int,
                                 C.POINTER(C.c_double)]
    lib.sg_set_exact.restype = C.c_int
    lib.sg_rhs.argtypes = [vp, C.c_int, vp, vp, vp]
    lib.sg_rhs.restype = C.c_int
    lib.sg_moments.argtypes = [vp, vp, C.c_int, vp, vp, vp]
    lib.sg_moments.restype = C.c_int
    lib.sg_qoi_errors.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_double)]
    lib.sg_qoi_errors.restype = C.c_int
    lib.mc_solve_batch.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double, C.c_int,
                                   vp, vp, vp, C.POINTER(sg_mc_stats), vp]
    lib.mc_solve_batch.restype = C.c_int
    lib.sg_solve_slab_adjoint.argtypes = [vp, C.c_int, vp, vp, C.c_double, C.c_int, C.c_int,
                                          C.POINTER(sg_solve_stats), vp]
    lib.sg_solve_slab_adjoint.restype = C.c_int
    lib.sg_adjoint_gradient.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(sg_adjoint_stats),
                                        vp]
    lib.sg_adjoint_gradient.restype = C.c_int
    lib.sg_set_coefficient.argtypes = [vp, C.POINTER(sg_coeff)]
    lib.sg_set_coefficient.restype = C.c_int
    lib.mc_solve_meshes.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(C.POINTER(C.c_double)),
                                    C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(vp), C.POINTER(vp),
                                    C.POINTER(vp), C.POINTER(sg_mc_stats), vp]
    lib.mc_solve_meshes.restype = C.c_int
    lib.sg_stat_errors.argtypes = [vp, vp, vp, C.c_double, C.POINTER(C.c_double)]
    lib.sg_stat_errors.restype = C.c_int
    lib.sg_autotune.argtypes = [vp, C.c_int]
    lib.sg_autotune.restype = C.c_int
    lib.sg_set_apply_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    lib.sg_set_apply_shape.restype = C.c_int
    lib.sg_apply_host_async.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp]
    lib.sg_apply_host_async.restype = C.c_int
    lib.sg_apply_host_static.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    lib.sg_apply_host_static.restype = C.c_int
    lib.sg_destroy.argtypes = [vp]
    lib.sg_destroy.restype = None
    lib.sg_status_string.argtypes = [C.c_int]
    lib.sg_status_string.restype = C.c_char_p
    lib.sg_last_error.argtypes = []
    lib.sg_last_error.restype = C.c_char_p
    _lib = lib
    return lib

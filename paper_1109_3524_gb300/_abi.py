"""ctypes declarations of the C ABI in include/ibm.h (argument marshalling only)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibm.so")

IBM_OK = 0
IBM_ERR_ARG = 1
IBM_ERR_CUDA = 2
IBM_ERR_NO_MEM = 3
IBM_ERR_NOT_CONVERGED = 4
IBM_ERR_BREAKDOWN = 5
IBM_ERR_UNIMPLEMENTED = 6
IBM_ERR_STATE = 7
STATUS_NAMES = {0: "ok", 1: "bad argument", 2: "cuda error", 3: "workspace too small",
                4: "not converged", 5: "breakdown", 6: "unimplemented", 7: "bad state"}

IBM_BC_FREESTREAM = 0
IBM_BC_WALLS = 1
IBM_PRECOND_NONE = 0
IBM_PRECOND_JACOBI = 1
IBM_PRECOND_AMG = 2
IBM_PRECOND_SCHUR = 3
IBM_PREC_FP64 = 0
IBM_PREC_MIXED = 1
IBM_WARM_ZERO = 0
IBM_WARM_PREV = 1
IBM_WARM_EXTRAP = 2
IBM_WARM_CNN = 3
IBM_WARM_PROJ = 4


class ibm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nu", C.c_double), ("dt", C.c_double),
                ("uinf", C.c_double), ("vinf", C.c_double), ("bc", C.c_int32), ("bn_order", C.c_int32),
                ("h", C.c_double), ("tol1", C.c_double), ("tol2", C.c_double),
                ("max_iter1", C.c_int32), ("max_iter2", C.c_int32), ("poisson_precond", C.c_int32),
                ("precision", C.c_int32), ("warm", C.c_int32), ("pin_i", C.c_int32), ("pin_j", C.c_int32),
                ("amg_theta", C.c_double), ("amg_omega", C.c_double), ("amg_pre", C.c_int32),
                ("amg_post", C.c_int32), ("amg_max_coarse", C.c_int32), ("amg_max_levels", C.c_int32),
                ("amg_rebuild_every", C.c_int32), ("moving", C.c_int32), ("amg_trunc", C.c_double),
                ("amg_tail_rows", C.c_int32), ("amg_sweeps0", C.c_int32),
                ("schur_cache", C.c_int32), ("reserved_", C.c_int32)]


class ibm_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("rel_res", C.c_double), ("rel_res0", C.c_double)]


class ibm_step_stats(C.Structure):
    _fields_ = [("t", C.c_double), ("solve1", ibm_solve_stats), ("solve2", ibm_solve_stats),
                ("fx", C.c_double), ("fy", C.c_double), ("cd", C.c_double), ("cl", C.c_double),
                ("div_max", C.c_double), ("slip_max", C.c_double),
                ("poisson_ms", C.c_double), ("poisson_bytes", C.c_double),
                ("amg_rebuilt", C.c_int32), ("pad_", C.c_int32)]


P = C.c_void_p
DP = C.POINTER(C.c_double)
I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
CTX = C.c_void_p

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "ibm_config_defaults": (None, [C.POINTER(ibm_config)]),
    "ibm_create": (C.c_int, [C.POINTER(ibm_config), DP, DP, C.c_int32, DP, DP, C.POINTER(CTX)]),
    "ibm_workspace_bytes": (C.c_int, [CTX, C.POINTER(C.c_size_t)]),
    "ibm_bind_workspace": (C.c_int, [CTX, P, C.c_size_t, P]),
    "ibm_setup": (C.c_int, [C.POINTER(ibm_config), DP, DP, C.c_int32, DP, DP, P, C.c_size_t, P,
                            C.POINTER(CTX)]),
    "ibm_destroy": (None, [CTX]),
    "ibm_last_error": (C.c_char_p, [CTX]),
    "ibm_sizes": (C.c_int, [CTX, I64P, I64P, I32P]),
    "ibm_set_body": (C.c_int, [CTX, DP, DP, DP, DP]),
    "ibm_step": (C.c_int, [CTX, C.c_int32, C.POINTER(ibm_step_stats)]),
    "ibm_solve_poisson": (C.c_int, [CTX, P, P, P, C.POINTER(ibm_solve_stats)]),
    "ibm_forces": (C.c_int, [CTX, DP, DP, DP, DP]),
    "ibm_get_state": (C.c_int, [CTX, DP, DP, DP, DP, DP, DP, I64P]),
    "ibm_set_state": (C.c_int, [CTX, DP, DP, DP, DP, DP, C.c_double, C.c_int64]),
    "ibm_layout": (C.c_int, [CTX, I64P]),
    "ibm_apply_poisson": (C.c_int, [CTX, P, P]),
    "ibm_vcycle": (C.c_int, [CTX, P, P]),
    "ibm_poisson_residual_norms_noalloc": (C.c_int, [CTX, P, P, DP]),
    "ibm_amg_levels": (C.c_int, [CTX, I32P]),
    "ibm_amg_matrix": (C.c_int, [CTX, C.c_int32, C.c_int32, I64P, I64P, I64P, I64P, I32P, DP]),
    "ibm_amg_level_info": (C.c_int, [CTX, C.c_int32, I64P, DP]),
    "ibm_cnn_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.POINTER(CTX)]),
    "ibm_cnn_destroy": (None, [CTX]),
    "ibm_cnn_last_error": (C.c_char_p, [CTX]),
    "ibm_cnn_param_count": (C.c_int, [CTX, I64P]),
    "ibm_cnn_workspace_bytes": (C.c_int, [CTX, C.POINTER(C.c_size_t)]),
    "ibm_cnn_bind": (C.c_int, [CTX, P, C.c_size_t, P]),
    "ibm_cnn_set_params": (C.c_int, [CTX, DP, C.c_int64]),
    "ibm_cnn_get_params": (C.c_int, [CTX, DP, C.c_int64]),
    "ibm_cnn_forward": (C.c_int, [CTX, C.c_int32, C.c_int32, C.c_int32, P, P]),
    "ibm_cnn_loss_grad": (C.c_int, [CTX, C.c_int32, C.c_int32, C.c_int32, P, P, DP, DP]),
    "ibm_cnn_adam_step": (C.c_int, [CTX, C.c_double, C.c_double, C.c_double, C.c_double]),
    "ibm_cnn_time_forward": (C.c_int, [CTX, C.c_int32, C.c_int32, C.c_int32, C.c_int32, DP, C.c_int32]),
    "ibm_cnn_layer_info": (C.c_int, [CTX, C.c_int32, I32P, I32P, I32P, I32P, I32P]),
    "ibm_cnn_prepare": (C.c_int, [CTX, C.c_int32, C.c_int32, P, P, P, P, C.c_int32, I32P, C.c_int32,
                                  C.c_int32, P, P]),
    "ibm_cnn_set_window": (C.c_int, [CTX, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "ibm_attach_cnn": (C.c_int, [CTX, CTX]),
    "ibm_snapshot": (C.c_int, [CTX, P, P, P, P]),
    "ibm_profile_enable": (C.c_int, [CTX, C.c_int32]),
    "ibm_profile_reset": (C.c_int, [CTX]),
    "ibm_profile_count": (C.c_int, [CTX, I32P]),
    "ibm_profile_get": (C.c_int, [CTX, C.c_int32, C.POINTER(C.c_char_p), I64P, DP, DP]),
    "ibm_profile_graph_class": (C.c_int, [CTX, C.c_int32, C.c_int32, I64P, DP, DP]),
    "ibm_transfer_bytes": (C.c_int, [CTX, I64P, I64P]),
    "ibm_launch_count": (C.c_int, [CTX, I64P]),
}

_lib = None


def load():
    """Loads libibm.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

"""ctypes binding of the C ABI in include/rchfsi.h (argument marshalling only).

Every computation runs inside librchfsi.so; this module only converts Python / NumPy / torch
arguments into the C structs and pointers the ABI takes.  The library must have been built
(`paper_2503_22652_gb300.build.build()`); loading fails with an exception otherwise.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librchfsi.so")

OK = 0
PENDING = 1
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_NOT_CONVERGED = -3
ERR_STAGNATED = -4
ERR_ILL_CONDITIONED = -5
ERR_NUMERIC = -6
ERR_TIMEOUT = -7
ERR_CUDA = -8
ERR_NO_OPERATOR = -9
ERR_UNSUPPORTED = -10

# RCHFSI_STATIC_SCRATCH_FLOATS of include/rchfsi.h
STATIC_SCRATCH_FLOATS = 4 * 1024 * 1024

FP64, FP32, TF32, BF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}
METHOD_RCHFSI, METHOD_CHFSI = 0, 1
REAL, COMPLEX = 0, 1
OP_DENSE, OP_FE_CELL = 0, 1
KERNEL_CLASSES = {"filter_tc": 0, "splitk_reduce": 1, "filter_simt": 2, "gemm_f64": 3, "fe_cell": 4,
                  "fe_cell_f64": 5, "gemm_f64_emu": 6, "small_dense": 7, "eig": 8, "rr_aux": 9}
RR_MODES = {"fp64": 0, "emulated": 1}
EIG_MODES = {"syevd": 0, "jacobi": 1, "tridiag": 2}

dptr = C.POINTER(C.c_double)


class rchfsi_params(C.Structure):
    _fields_ = [("m", C.c_int64), ("nev", C.c_int32), ("block", C.c_int32), ("degree", C.c_int32),
                ("precision", C.c_int32), ("method", C.c_int32), ("field", C.c_int32),
                ("max_iter", C.c_int32), ("min_iter", C.c_int32), ("lanczos_steps", C.c_int32),
                ("stall_iters", C.c_int32), ("fixed_bounds", C.c_int32), ("tol", C.c_double),
                ("lmin", C.c_double), ("lT", C.c_double), ("lmax", C.c_double),
                ("hbm_budget_bytes", C.c_uint64), ("rr_mode", C.c_int32), ("eig_mode", C.c_int32)]


class rchfsi_operator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("field", C.c_int32), ("m", C.c_int64), ("A", C.c_void_p),
                ("B", C.c_void_p), ("A_filter", C.c_void_p), ("Dinv", C.c_void_p),
                ("Dinv_dense", C.c_void_p), ("n_cells", C.c_int64), ("n_c", C.c_int32),
                ("B_cells_shared", C.c_int32), ("cell_dofs", C.c_void_p), ("A_cells", C.c_void_p),
                ("B_cells", C.c_void_p)]


class rchfsi_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("max_rel_residual", C.c_double),
                ("max_abs_residual", C.c_double), ("lmax", C.c_double), ("normA", C.c_double),
                ("t_total_ms", C.c_double), ("t_filter_ms", C.c_double), ("t_rr_ms", C.c_double),
                ("filter_flops", C.c_double), ("operator_applies", C.c_int64), ("history", C.c_void_p),
                ("cholqr_retries", C.c_int32)]


class rchfsi_request(C.Structure):
    _fields_ = [("op", rchfsi_operator), ("params", rchfsi_params), ("X0", C.c_void_p),
                ("warm_key", C.c_uint64)]


class rchfsi_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("max_rel_residual", C.c_double),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double), ("evals", C.c_void_p),
                ("X", C.c_void_p), ("error", C.c_char * 160)]


# name -> (restype, argtypes); the exported symbols of include/rchfsi.h
SIGNATURES = {
    "rchfsi_params_default": (C.c_int, [C.POINTER(rchfsi_params)]),
    "rchfsi_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(rchfsi_params), C.c_void_p]),
    "rchfsi_destroy": (C.c_int, [C.c_void_p]),
    "rchfsi_set_params": (C.c_int, [C.c_void_p, C.POINTER(rchfsi_params)]),
    "rchfsi_set_operator": (C.c_int, [C.c_void_p, C.POINTER(rchfsi_operator)]),
    "rchfsi_filter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_void_p]),
    "rchfsi_chfsi_filter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int,
                                      C.c_void_p]),
    "rchfsi_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rchfsi_rayleigh_ritz": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rchfsi_lanczos_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, dptr, dptr]),
    "rchfsi_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(rchfsi_stats)]),
    "rchfsi_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.POINTER(rchfsi_stats)]),
    "rchfsi_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_uint64]),
    "rchfsi_server_destroy": (C.c_int, [C.c_void_p]),
    "rchfsi_submit": (C.c_int, [C.c_void_p, C.POINTER(rchfsi_request), C.POINTER(C.c_uint64)]),
    "rchfsi_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(rchfsi_result)]),
    "rchfsi_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "rchfsi_profile_read": (C.c_int, [C.c_void_p, C.c_int, dptr, C.POINTER(C.c_int64), dptr, dptr]),
    "rchfsi_filter_step_tf32_static": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                                 C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_int64,
                                                 C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
    "rchfsi_strerror": (C.c_char_p, [C.c_int]),
    "rchfsi_last_error": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t]),
}

_lib = None


def load(path=LIB_PATH):
    """Load librchfsi.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("librchfsi.so not found at %s: run paper_2503_22652_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib

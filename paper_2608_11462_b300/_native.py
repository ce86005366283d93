"""ctypes binding of libphs_b300.so (include/phs.h).  Argument marshalling only:
every computation runs in the CUDA library.  Importing this module fails loudly
when the library has not been built; there is no CPU fallback."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphs_b300.so")

STATUS = {0: "PHS_OK", 1: "PHS_ERR_INVALID_ARG", 2: "PHS_ERR_DUPLICATE_POINTS", 3: "PHS_ERR_OOM",
          4: "PHS_ERR_CUDA", 5: "PHS_ERR_NOT_CONVERGED", 6: "PHS_ERR_CHOLESKY", 7: "PHS_ERR_TIMEOUT"}


class PhsOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("atol", ctypes.c_double),
                ("maxiter", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("ordering", ctypes.c_int),
                ("nu", ctypes.c_double), ("alpha", ctypes.c_double), ("domain_halfwidth", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("fmm_eps", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("m2l_tensor", ctypes.c_int),
                ("precond_lowrank", ctypes.c_int)]


class PhsServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("max_active", ctypes.c_int), ("setup_threads", ctypes.c_int)]


class PhsFitInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("jittered", ctypes.c_int), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("ms_plan", ctypes.c_float), ("ms_fit", ctypes.c_float),
                ("ms_matvec_avg", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "phs_options_default", "phs_last_error", "phs_kernel_launches", "phs_plan_create", "phs_matvec", "phs_fit", "phs_eval",
    "phs_fit_predict_host", "phs_plan_destroy", "phs_plan_frame", "phs_plan_vecchia", "phs_plan_vecchia_factor",
    "phs_plan_precond", "phs_plan_work", "phs_plan_kernel_work", "phs_plan_memory", "phs_plan_set_wait_limit", "phs_plan_set_timing",
    "phs_plan_timing", "phs_dense_matvec",
    "phs_dense_matvec_noalloc",
    "phs_random_order", "phs_maxmin_order", "phs_hmaxmin_order", "phs_amaxmin_order", "phs_knn_prev",
    "phs_vecchia_factor", "phs_gmres", "phs_tune_alpha", "phs_server_create", "phs_server_submit",
    "phs_server_wait", "phs_server_stats", "phs_server_destroy",
]

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2608_11462_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32, d, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    st = ctypes.c_int
    sig = {
        "phs_options_default": (None, [ctypes.POINTER(PhsOptions), i32]),
        "phs_last_error": (ctypes.c_char_p, []),
        "phs_kernel_launches": (i64, []),
        "phs_plan_create": (st, [P, i64, i32, i32, i32, i32, ctypes.POINTER(PhsOptions), P, ctypes.POINTER(P)]),
        "phs_matvec": (st, [P, P, P, i32, P]),
        "phs_fit": (st, [P, P, P, P, ctypes.POINTER(PhsFitInfo), P]),
        "phs_eval": (st, [P, P, P, P, i64, P, P]),
        "phs_fit_predict_host": (st, [P, P, i64, P, i64, i32, i32, i32, i32, ctypes.POINTER(PhsOptions), P, P, P,
                                      ctypes.POINTER(PhsFitInfo), P]),
        "phs_plan_destroy": (st, [P]),
        "phs_plan_frame": (st, [P, P, P]),
        "phs_plan_vecchia": (st, [P, P, P]),
        "phs_plan_vecchia_factor": (st, [P, P, P]),
        "phs_plan_precond": (st, [P, P, P, P]),
        "phs_plan_work": (st, [P, P]),
        "phs_plan_kernel_work": (st, [P, P]),
        "phs_plan_memory": (st, [P, P]),
        "phs_plan_set_wait_limit": (st, [P, i64, i32]),
        "phs_plan_set_timing": (st, [P, i32]),
        "phs_plan_timing": (st, [P, P, P]),
        "phs_dense_matvec": (st, [P, i64, i32, P, P, P]),
        "phs_dense_matvec_noalloc": (st, [P, i64, i32, P, P, P]),
        "phs_random_order": (st, [i64, u64, P, P]),
        "phs_maxmin_order": (st, [P, i64, P, P]),
        "phs_hmaxmin_order": (st, [P, i64, ctypes.c_uint64, P, P]),
        "phs_amaxmin_order": (st, [P, i64, P, P]),
        "phs_knn_prev": (st, [P, i64, P, i32, P, P]),
        "phs_vecchia_factor": (st, [P, i64, P, P, i32, d, d, P, P, P, P]),
        "phs_gmres": (st, [P, P, P, i32, i32, ctypes.POINTER(PhsFitInfo), P]),
        "phs_tune_alpha": (st, [P, P, i64, i32, i32, i32, i32, ctypes.POINTER(PhsOptions), i64,
                                ctypes.POINTER(d), ctypes.POINTER(i32), P]),
        "phs_server_create": (st, [ctypes.POINTER(PhsServerConfig), ctypes.POINTER(P)]),
        "phs_server_submit": (st, [P, P, P, i64, P, i64, i32, i32, i32, i32, ctypes.POINTER(PhsOptions),
                                   ctypes.POINTER(i64)]),
        "phs_server_wait": (st, [P, i64, P, P, P, ctypes.POINTER(PhsFitInfo), P]),
        "phs_server_stats": (st, [P, P]),
        "phs_server_destroy": (st, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class PhsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def check(code, allow=()):
    if code != 0 and code not in allow:
        raise PhsError(code, lib().phs_last_error().decode())
    return code

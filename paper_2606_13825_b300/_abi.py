"""ctypes declarations of the C ABI in ``include/cosmo_du.h``.

Argument marshalling only: every computation happens in ``libcosmo_du.so``.
Loading fails loudly if the library is missing; there is no fallback path.
"""
import ctypes
import os
from ctypes import c_size_t, POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcosmo_du.so")
HEADER_PATH = os.path.join(os.path.dirname(HERE), "include", "cosmo_du.h")

COSMO_OK, COSMO_E_INVAL, COSMO_E_NOMEM, COSMO_E_CUDA = 0, 1, 2, 3
COSMO_E_NOTCONV, COSMO_E_NONFINITE, COSMO_E_TIMEOUT, COSMO_E_STATE, COSMO_E_NODEVICE = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_NOTCONV",
                5: "E_NONFINITE", 6: "E_TIMEOUT", 7: "E_STATE", 8: "E_NODEVICE"}
PREC_MIXED, PREC_FP64 = 0, 1
VAL_F32, VAL_BF16 = 0, 1
FLAG_CG_CAP, FLAG_ADJ_CG_CAP, FLAG_EIG_CAP, FLAG_NONFINITE, FLAG_BAD_PARAM, FLAG_TIMEOUT = 1, 2, 4, 8, 16, 32


class CosmoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Cone(ctypes.Structure):
    _fields_ = [("type", c_int32), ("dim", c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("ninst", c_int32),
                ("col_off", POINTER(c_int64)), ("row_off", POINTER(c_int64)),
                ("P_rowptr", POINTER(c_int64)), ("P_col", POINTER(c_int32)),
                ("P_val", POINTER(c_double)),
                ("A_rowptr", POINTER(c_int64)), ("A_col", POINTER(c_int32)),
                ("A_val", POINTER(c_double)),
                ("q", POINTER(c_double)), ("b", POINTER(c_double)),
                ("box_l", POINTER(c_double)), ("box_u", POINTER(c_double)),
                ("cone_count", POINTER(c_int32)), ("cones", POINTER(Cone))]


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("value_type", c_int32), ("cg_tol", c_double),
                ("cg_max_iter", c_int32), ("checkpoint_every", c_int32),
                ("dk_gap_tau", c_double), ("eig_jacobi_max_p", c_int32),
                ("eig_max_sweeps", c_int32), ("eig_tol", c_double), ("use_graph", c_int32),
                ("device", c_int32), ("eig_warm_start", c_int32), ("dk_tensor_cores", c_int32),
                ("cg_cluster", c_int32), ("loss_kind", c_int32), ("eig_variant", c_int32),
                ("eig_threads", c_int32), ("autotune", c_int32),
                ("fwd_persistent", c_int32)]


MAX_PSD_CLASSES = 8


class Tuning(ctypes.Structure):
    _fields_ = [("n_classes", c_int32), ("class_maxp", c_int32 * MAX_PSD_CLASSES),
                ("class_count", c_int32 * MAX_PSD_CLASSES), ("class_method", c_int32 * MAX_PSD_CLASSES),
                ("class_threads", c_int32 * MAX_PSD_CLASSES), ("cg_kernel", c_int32), ("tuned", c_int32),
                ("tune_ms", c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("ninst", c_int32), ("precision", c_int32), ("n_total", c_int64),
                ("m_total", c_int64), ("nnzA", c_int64), ("nnzP", c_int64),
                ("n_soc", c_int32), ("n_psd", c_int32), ("max_psd_p", c_int32),
                ("psd_u_entries", c_int64), ("device_bytes", c_int64), ("last_K", c_int32),
                ("tape_valid", c_int32), ("kernels_launched", c_int64),
                ("eig_sweeps", c_int64), ("eig_blocks", c_int64), ("cg_iters", c_int64),
                ("cg_solves", c_int64), ("adj_cg_iters", c_int64), ("adj_cg_solves", c_int64),
                ("fwd_persistent", c_int32)]


PCG_PHASES = ("R stage", "R stream (warp 0)", "R stream rest + cluster barrier", "R epilogue",
              "R->C grid barrier", "C stage", "C stream (warp 0)", "C stream rest + cluster barrier",
              "update", "C->R grid barrier")


class SolveParams(ctypes.Structure):
    _fields_ = [("sigma", c_double), ("alpha", c_double), ("rho0", c_double), ("rho_eq_scale", c_double),
                ("eps", c_double), ("rebalance_tol", c_double), ("rho_min", c_double), ("rho_max", c_double),
                ("max_iter", c_int32), ("check_every", c_int32), ("rebalance_every", c_int32),
                ("pad", c_int32)]


class PcgPlanInfo(ctypes.Structure):
    _fields_ = [("nseg_a", c_int32), ("nseg_at", c_int32), ("grid", c_int32), ("threads", c_int32),
                ("cluster", c_int32), ("ring_slots", c_int32),
                ("layout_bytes", c_int64), ("smem_bytes", c_int64), ("quads_a", c_int64),
                ("quads_at", c_int64)]


_SIGS = {
    "cosmo_version": (c_char_p, []),
    "cosmo_kernel_launch_count": (c_int64, []),
    "cosmo_last_error": (c_char_p, []),
    "cosmo_options_default": (c_int32, [POINTER(Options), c_int32]),
    "cosmo_problem_validate": (c_int32, [POINTER(Problem)]),
    "cosmo_batch_create": (c_int32, [POINTER(Problem), POINTER(Options), POINTER(c_void_p)]),
    "cosmo_batch_destroy": (c_int32, [c_void_p]),
    "cosmo_batch_get_info": (c_int32, [c_void_p, POINTER(BatchInfo)]),
    "cosmo_batch_get_tuning": (c_int32, [c_void_p, POINTER(Tuning)]),
    "cosmo_batch_set_tuning": (c_int32, [c_void_p, POINTER(Tuning)]),
    "cosmo_forward": (c_int32, [c_void_p, c_int32, POINTER(c_double), c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_int32, c_void_p]),
    "cosmo_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "cosmo_residuals": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p]),
    "cosmo_rho_from_log": (c_int32, [c_void_p, c_int32, c_void_p, c_double, c_void_p, c_void_p]),
    "cosmo_rho_from_log_backward": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                              c_void_p]),
    "cosmo_alpha_broadcast": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "cosmo_alpha_reduce": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "cosmo_step_host": (c_int32, [c_void_p, c_int32, c_double, c_double, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p]),
    "cosmo_status_sync": (c_int32, [c_void_p, POINTER(c_int32)]),
    "cosmo_tape_eigen": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "cosmo_workspace_bytes": (c_int32, [c_void_p, c_int32, POINTER(c_size_t)]),
    "cosmo_batch_set_workspace": (c_int32, [c_void_p, c_int32, c_void_p, c_size_t]),
    "cosmo_profile_enable": (c_int32, [c_void_p, c_char_p]),
    "cosmo_profile_read": (c_int32, [c_void_p, c_char_p, POINTER(c_double), POINTER(c_int64),
                                     c_int32]),
    "cosmo_pcg_solve": (c_int32, [c_int32, c_int32, c_int64, c_int64] + [c_void_p] * 11 +
                        [c_double, c_void_p, c_void_p, c_void_p, c_int32, c_double, c_int32,
                         c_void_p, c_void_p]),
    "cosmo_pcg_solve_noalloc": (c_int32, [c_int32, c_int32, c_int64, c_int64] + [c_void_p] * 11 +
                                [c_double, c_void_p, c_void_p, c_void_p, c_int32, c_double,
                                 c_int32, c_void_p, c_void_p]),
    "cosmo_solve_params_default": (c_int32, [POINTER(SolveParams)]),
    "cosmo_solve": (c_int32, [c_void_p, POINTER(SolveParams), c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_void_p]),
    "cosmo_policy_sizes": (c_int32, [POINTER(c_int32), POINTER(c_int32)]),
    "cosmo_policy_forward": (c_int32, [c_void_p, c_int32, POINTER(c_double)] + [c_void_p] * 10 + [c_int32, c_void_p]),
    "cosmo_policy_backward": (c_int32, [c_void_p] * 12),
    "cosmo_policy_schedule": (c_int32, [c_void_p] * 4),
    "cosmo_ws_sizes": (c_int32, [POINTER(c_int32), POINTER(c_int32)]),
    "cosmo_ws_forward": (c_int32, [c_void_p] * 7),
    "cosmo_ws_backward": (c_int32, [c_void_p] * 9),
    "cosmo_pcg_plan_create": (c_int32, [c_int32, c_int32, c_int64, c_int64] + [c_void_p] * 11 +
                              [POINTER(c_void_p), c_void_p]),
    "cosmo_pcg_plan_solve": (c_int32, [c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_double,
                                       c_int32, c_void_p, c_void_p]),
    "cosmo_pcg_plan_get_info": (c_int32, [c_void_p, POINTER(PcgPlanInfo)]),
    "cosmo_pcg_plan_destroy": (c_int32, [c_void_p]),
    "cosmo_pcg_plan_set_timing": (c_int32, [c_void_p, c_int32]),
    "cosmo_pcg_plan_get_timing": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "cosmo_psd_project": (c_int32, [c_int32, c_int32, POINTER(c_int32), POINTER(c_int64),
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "cosmo_psd_dk_backward": (c_int32, [c_int32, c_int32, POINTER(c_int32), POINTER(c_int64),
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_double,
                                        c_void_p]),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2606_13825_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != COSMO_OK:
        msg = lib().cosmo_last_error().decode(errors="replace")
        raise CosmoError(status, msg)
    return status


def header_functions():
    """Names of the functions declared in include/cosmo_du.h."""
    import re
    txt = open(HEADER_PATH).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cosmo_[a-z0-9_]+)\s*\(", txt)))

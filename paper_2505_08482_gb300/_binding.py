"""ctypes binding of ``libpat.so`` (argument marshalling only).

Every entry point of ``include/pat.h`` is declared here under its C name.
There is no fallback: if the library cannot be loaded the import of the
product API fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_size_t, c_void_p

from ._build import LIB, LIB_DEBUG

PAT_OK = 0
PAT_EINVAL = -1
PAT_ENOMEM = -2
PAT_ECUDA = -3
PAT_ENONFINITE = -4
PAT_ETIMEOUT = -5
PAT_ELINESEARCH = -6
PAT_K_ROW_RHO = 1
PAT_K_ROW_U = 2
PAT_K_COL_GRAD = 3
PAT_K_COL_PAIR = 4
PAT_K_COL_SUM = 5
PAT_K_ROW_ADJ_RHO = 6
PAT_K_ROW_ADJ_U = 7
KERNEL_CLASSES = {1: "k_row_rho", 2: "k_row_u", 3: "k_col(grad)", 4: "k_col(pair)", 5: "k_col(sum)",
                  6: "k_row_adj_rho", 7: "k_row_adj_u"}
PAT_WS_FORWARD = 0
PAT_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024
PAT_WS_GRADIENT = 1
PAT_STATUS_NONFINITE = 1
PAT_STATUS_WAIT = 2
PAT_STATUS_QUEUE = 4
PAT_STATUS_TC05 = 8
PAT_STATUS_BOUNDS = 16


class PatGrid(ctypes.Structure):
    _fields_ = [("n", c_int), ("pml", c_int), ("dx", c_double), ("dt", c_double), ("nt", c_int),
                ("c_ref", c_double), ("rho0", c_double), ("pml_alpha", c_double), ("c_bg", c_double)]


class PatReconCfg(ctypes.Structure):
    _fields_ = [("nlevels", c_int), ("levels", POINTER(c_int)), ("L", c_double), ("dt_data", c_double),
                ("nt_data", c_int), ("m", c_int), ("h_sensor_xy", POINTER(c_double)), ("K", c_int),
                ("cfl", c_double), ("c_lo", c_double), ("c_hi", c_double), ("p0_lo", c_double),
                ("c_bg", c_double), ("rho0", c_double), ("pml_alpha", c_double), ("min_pml", c_int),
                ("mem", c_int), ("iters", c_int), ("max_halvings", c_int), ("ckpt_every", c_int),
                ("rtol", c_double), ("alpha0", c_double), ("c1", c_double), ("sigma_p0", c_double),
                ("autotune", c_int), ("prior_tau", c_double), ("prior_eta_c", c_double), ("prior_sigma_c", c_double),
                ("prior_eta_p0", c_double), ("prior_sigma_p0", c_double), ("persistent", c_int)]


class PatInstance(ctypes.Structure):
    pass


class PatIterReport(ctypes.Structure):
    _fields_ = [("level", c_int), ("iter", c_int), ("J", c_double), ("gnorm", c_double), ("alpha", c_double),
                ("trials", c_int), ("J_new", c_double), ("ms", c_double), ("Ec", c_double), ("Ep0", c_double)]


class PatReport(ctypes.Structure):
    _fields_ = [("capacity", c_int), ("count", c_int), ("iters", POINTER(PatIterReport)), ("status", c_int),
                ("total_ms", c_double)]


PatInstance._fields_ = [("d_y_meas", c_void_p), ("d_w", c_void_p), ("d_c_io", c_void_p), ("d_p0_io", c_void_p),
                        ("K", c_int), ("report", POINTER(PatReport)), ("d_c_true", c_void_p),
                        ("ec_target", c_double), ("d_p0_true", c_void_p), ("ep0_target", c_double)]

# name -> (restype, argtypes)
SIGNATURES = {
    "pat_plan_create": (c_int, [POINTER(c_void_p), POINTER(PatGrid), c_int, POINTER(c_double), c_int, c_int]),
    "pat_plan_create_batched": (c_int, [POINTER(c_void_p), POINTER(PatGrid), c_int, POINTER(c_double), c_int,
                                        POINTER(c_int), c_int]),
    "pat_plan_destroy": (None, [c_void_p]),
    "pat_plan_shape": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "pat_plan_ng": (c_int, [c_void_p]),
    "pat_plan_variants": (c_int, [c_void_p]),
    "pat_plan_set_variant": (c_int, [c_void_p, c_int]),
    "pat_plan_variant": (c_int, [c_void_p]),
    "pat_pml_auto": (c_int, [c_int, c_int]),
    "pat_workspace_bytes": (c_size_t, [c_void_p, c_int]),
    "pat_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pat_forward_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pat_forward_noalloc_status": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "pat_adjoint_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_size_t, c_void_p]),
    "pat_vjp": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pat_status": (c_int, [c_void_p, c_void_p, POINTER(c_int), c_void_p]),
    "pat_selftest_wait": (c_int, [c_void_p, ctypes.c_uint, c_void_p]),
    "pat_selftest_queue": (c_int, [c_void_p, c_void_p, ctypes.c_uint, c_void_p]),
    "pat_debug_bounds": (c_int, []),
    "pat_selftest_bounds": (c_int, [c_void_p, c_void_p]),
    "pat_plan_set_persistent": (c_int, [c_void_p, c_int]),
    "pat_plan_persistent": (c_int, [c_void_p]),
    "pat_plan_set_cluster": (c_int, [c_void_p, c_int]),
    "pat_plan_cluster": (c_int, [c_void_p]),
    "pat_plan_cluster_capacity": (c_int, [c_void_p]),
    "pat_prior_create": (c_int, [c_int, c_double, c_double, c_int, POINTER(c_void_p)]),
    "pat_prior_destroy": (c_int, [c_void_p]),
    "pat_prior_xi": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "pat_prior_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_int, POINTER(c_int),
                                c_void_p]),
    "pat_prior_eval": (c_int, [c_void_p, c_void_p, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double),
                               c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, POINTER(c_int), c_void_p]),
    "pat_reconstruct": (c_int, [POINTER(PatReconCfg), c_void_p, c_void_p, c_void_p, c_void_p, POINTER(PatReport),
                                c_void_p]),
    "pat_reconstruct_batched": (c_int, [POINTER(PatReconCfg), c_int, POINTER(PatInstance), c_void_p]),
    "pat_prolong": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "pat_time_interp": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_double, c_double, c_void_p]),
    "pat_plan_set_graphs": (c_int, [c_void_p, c_int]),
    "pat_plan_autotune": (c_int, [c_void_p, c_void_p, c_size_t, POINTER(c_double), c_void_p]),
    "pat_kernel_launches": (ctypes.c_ulonglong, []),
    "pat_timing_enable": (c_int, [c_int, c_int, c_int]),
    "pat_timing_read": (c_int, [POINTER(c_double), POINTER(ctypes.c_longlong)]),
    "pat_unet_create": (c_int, [POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int, c_int]),
    "pat_unet_destroy": (None, [c_void_p]),
    "pat_unet_param_count": (c_size_t, [c_void_p]),
    "pat_unet_param_layout": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "pat_unet_set_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pat_unet_get_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pat_unet_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "pat_unet_grads": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "pat_unet_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p, c_void_p]),
    "pat_unet_set_gemm_path": (c_int, [c_void_p, c_int]),
    "pat_unet_status": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "pat_gemm_bf16": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_int, c_void_p,
                              c_void_p]),
    "pat_last_error": (c_char_p, []),
}

_lib = None


def lib_path() -> str:
    """libpat.so, or libpat_debug.so (the bounds-checked build) when PAT_DEBUG_BOUNDS=1."""
    return LIB_DEBUG if os.environ.get("PAT_DEBUG_BOUNDS") == "1" else LIB


def lib() -> ctypes.CDLL:
    """Load libpat.so (built in-tree by ``build()``; libpat_debug.so from ``build(debug=True)`` when the
    environment has PAT_DEBUG_BOUNDS=1); raises if it is missing."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not found at {path}: run "
                               f"paper_2505_08482_gb300.build({'debug=True' if path == LIB_DEBUG else ''}) first")
        try:
            import torch  # noqa: F401  (loads the CUDA runtime first)
        except ImportError:
            pass
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(SIGNATURES)


class PatError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().pat_last_error()
        super().__init__(f"{where} failed with code {code}: {msg.decode() if msg else ''}")
        self.code = code


def check(code: int, where: str):
    if code != PAT_OK:
        raise PatError(code, where)

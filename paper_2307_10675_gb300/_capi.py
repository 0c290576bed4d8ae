"""ctypes declarations of the C ABI in ``include/ifci.h`` (no logic here)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_LIB = None

c_int, c_double, c_size_t, c_ll, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_longlong, ctypes.c_void_p
c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)

IFCI_OK = 0
IFCI_ERR_INVALID_ARG = 1
IFCI_ERR_OOM = 2
IFCI_ERR_CUDA = 3
IFCI_ERR_NOT_CONVERGED = 4
IFCI_ERR_TIMEOUT = 5
IFCI_ERR_UNSUPPORTED = 6
IFCI_SCREENED = 7

IFCI_FP64, IFCI_FP32, IFCI_TF32, IFCI_BF16, IFCI_FP64E = 0, 1, 2, 3, 4
IFCI_SIGMA_SPIN_SYMMETRIC = 0x100

EXPORTS = [
    "ifci_handle_create", "ifci_handle_destroy", "ifci_last_error_string", "ifci_workspace_bytes",
    "ifci_kernel_launches", "ifci_string_counts", "ifci_build_strings", "ifci_sigma", "ifci_hdiag",
    "ifci_frozen_core", "ifci_davidson_default_opts", "ifci_davidson_batched", "ifci_num_subsets",
    "ifci_increments", "ifci_rdm_backward", "ifci_profile_enable", "ifci_profile_read",
    "ifci_sigma_noalloc", "ifci_sigma_noalloc_max_bytes", "ifci_h_elements", "ifci_wait_selftest",
    "ifci_hbci_batched",
]
PROFILE_KINDS = {"gather": 0, "contract": 1, "scatter": 2, "vector": 3, "other": 4, "contract_hi": 5, "setup": 6, "pspace": 7}


class Strings(ctypes.Structure):
    _fields_ = [("norb", c_int), ("nelec_spin", c_int), ("nstr", c_int), ("nexc", c_int),
                ("strings", c_void_p), ("exc", c_void_p)]


class System(ctypes.Structure):
    _fields_ = [("nbody", c_int), ("body_offset", c_int_p), ("norb", c_int), ("h", c_void_p),
                ("eri", c_void_p), ("on_host", c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("norb", c_int), ("nelec_spin", c_int), ("h1", c_void_p), ("eri", c_void_p),
                ("e_core", c_double), ("c_out", c_void_p)]


class DavidsonOpts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("max_iter", c_int), ("max_space", c_int), ("e_tol", c_double),
                ("r_tol", c_double), ("refine", c_int), ("hi_precision", c_int), ("det_budget", c_ll),
                ("graph_iters", c_int), ("sector_passes", c_int), ("decouple_tol", c_double),
                ("cnb_threshold", c_double), ("hbci_max_rounds", c_int), ("hbci_eps1", c_double),
                ("hbci_eps2", c_double)]


class HbciOpts(ctypes.Structure):
    _fields_ = [("eps1", c_double), ("eps2", c_double), ("max_rounds", c_int)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libifci.so (building it when missing).  Raises if it cannot be had."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library missing: {_build.LIB}")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    H = c_void_p
    L.ifci_handle_create.argtypes = [ctypes.POINTER(H), c_size_t, c_int]
    L.ifci_handle_destroy.argtypes = [H]
    L.ifci_last_error_string.argtypes = [H]
    L.ifci_last_error_string.restype = ctypes.c_char_p
    L.ifci_workspace_bytes.argtypes = [H]
    L.ifci_workspace_bytes.restype = c_size_t
    L.ifci_kernel_launches.argtypes = [H]
    L.ifci_kernel_launches.restype = c_ll
    L.ifci_string_counts.argtypes = [c_int, c_int, c_int_p, c_int_p]
    L.ifci_build_strings.argtypes = [H, c_int, c_int, c_void_p, c_void_p, c_void_p]
    L.ifci_sigma.argtypes = [H, ctypes.POINTER(Strings), c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]
    L.ifci_hdiag.argtypes = [H, ctypes.POINTER(Strings), c_void_p, c_void_p, c_void_p, c_void_p]
    L.ifci_wait_selftest.argtypes = [H, ctypes.c_longlong, c_void_p]
    L.ifci_h_elements.argtypes = [H, ctypes.POINTER(Strings), c_void_p, c_void_p, ctypes.c_longlong, c_void_p,
                                  c_void_p, c_void_p, c_void_p]
    L.ifci_frozen_core.argtypes = [H, ctypes.POINTER(System), c_int, c_int_p, c_void_p, c_void_p, c_double_p,
                                   c_void_p]
    L.ifci_davidson_default_opts.argtypes = [ctypes.POINTER(DavidsonOpts)]
    L.ifci_davidson_default_opts.restype = None
    L.ifci_davidson_batched.argtypes = [H, c_int, ctypes.POINTER(Problem), ctypes.POINTER(DavidsonOpts),
                                        c_double_p, c_int_p, c_int_p, c_void_p]
    L.ifci_hbci_batched.argtypes = [H, c_int, ctypes.POINTER(Problem), ctypes.POINTER(c_ll),
                                    ctypes.POINTER(DavidsonOpts), ctypes.POINTER(HbciOpts), c_double_p, c_double_p,
                                    ctypes.POINTER(c_ll), c_int_p, c_int_p, c_void_p]
    L.ifci_num_subsets.argtypes = [c_int, c_int, ctypes.POINTER(c_ll)]
    L.ifci_increments.argtypes = [H, ctypes.POINTER(System), c_int, ctypes.POINTER(DavidsonOpts), c_double_p,
                                  c_double_p, c_double_p, c_double_p, c_int_p, c_int_p, c_void_p]
    L.ifci_rdm_backward.argtypes = [H, ctypes.POINTER(System), c_int, ctypes.POINTER(DavidsonOpts), c_double,
                                    c_void_p, c_void_p, c_int, c_void_p]
    L.ifci_sigma_noalloc.argtypes = [ctypes.POINTER(Strings), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.ifci_sigma_noalloc_max_bytes.argtypes = []
    L.ifci_sigma_noalloc_max_bytes.restype = c_size_t
    L.ifci_profile_enable.argtypes = [H, c_int]
    L.ifci_profile_read.argtypes = [H, c_int, c_double_p, ctypes.POINTER(c_ll)]
    _LIB = L
    return L

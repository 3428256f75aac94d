"""ctypes declarations of the libtd C ABI (include/td.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtd.so")

TD_OK, TD_ERR_INVALID, TD_ERR_NONLOCAL, TD_ERR_OOM, TD_ERR_CUDA, TD_ERR_TIMEOUT, TD_ERR_NUMERIC, \
    TD_ERR_UNSUPPORTED = range(8)
TD_FP64, TD_FP32, TD_TC = 0, 1, 2
STATUS_NAMES = {0: "TD_OK", 1: "TD_ERR_INVALID", 2: "TD_ERR_NONLOCAL", 3: "TD_ERR_OOM", 4: "TD_ERR_CUDA",
                5: "TD_ERR_TIMEOUT", 6: "TD_ERR_NUMERIC", 7: "TD_ERR_UNSUPPORTED"}

EXPORTS = ["td_default_options", "td_build_network", "td_coset_logprob", "td_decode",
           "td_coset_logprob_host", "td_grad_logprob", "td_grad_logprob_forced", "td_network_set_schedule",
           "td_network_tune", "td_network_get_info", "td_debug_sweep",
           "td_network_profile", "td_network_get_work", "td_coset_logprob_static", "td_free_network",
           "td_network_check", "td_measure_fma_peak", "td_build_gen_network", "td_gen_coset_logprob",
           "td_gen_decode", "td_coset_logprob_stats", "td_gen_rows_host", "td_last_error"]


class td_dem(C.Structure):
    _fields_ = [("n_det", C.c_int32), ("n_mech", C.c_int32), ("n_obs", C.c_int32),
                ("H_indptr", C.POINTER(C.c_int32)), ("H_indices", C.POINTER(C.c_int32)),
                ("L_indptr", C.POINTER(C.c_int32)), ("L_indices", C.POINTER(C.c_int32)),
                ("p", C.POINTER(C.c_double))]


class td_gen(C.Structure):
    _fields_ = [("n_gen", C.c_int32), ("n_qubits", C.c_int32), ("n_checks", C.c_int32),
                ("qubit_gens", C.POINTER(C.c_int32)), ("p", C.POINTER(C.c_double)),
                ("gen_xyt", C.POINTER(C.c_int32)), ("check_indptr", C.POINTER(C.c_int32)),
                ("check_indices", C.POINTER(C.c_int32)), ("n_xbar", C.c_int32), ("xbar", C.POINTER(C.c_int32)),
                ("n_zbar", C.c_int32), ("zbar", C.POINTER(C.c_int32))]


class td_layout(C.Structure):
    _fields_ = [("det_xyt", C.POINTER(C.c_int32))]


class td_options(C.Structure):
    _fields_ = [("chi", C.c_int32), ("chi_mps", C.c_int32), ("precision", C.c_int32),
                ("ckpt_stride", C.c_int32), ("svd_cutoff", C.c_double), ("multiplet_rtol", C.c_double),
                ("gram_cutoff", C.c_double), ("mem_budget", C.c_size_t), ("max_wave", C.c_int32)]


class td_network_info(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("n_layers", C.c_int32), ("n_bonds", C.c_int32),
                ("n_gates", C.c_int32), ("n_counter_sites", C.c_int32), ("nx", C.c_int32),
                ("ny", C.c_int32), ("wave", C.c_int32), ("chi", C.c_int32), ("chi_mps", C.c_int32),
                ("precision", C.c_int32), ("offset_all", C.c_int32), ("generator", C.c_int32),
                ("workspace_bytes", C.c_size_t),
                ("launches_per_wave", C.c_int64)]


KERNEL_CLASSES = ["init", "local", "gram", "pre", "core", "update", "final", "finalize"]

_lib = None


def load(path: str | None = None):
    """Load libtd.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libtd.so not found at {path}; build it with "
                           "`python -m paper_2310_10722_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.td_default_options.argtypes = [C.POINTER(td_options)]
    lib.td_default_options.restype = None
    lib.td_build_network.argtypes = [C.POINTER(td_dem), C.POINTER(td_layout), C.POINTER(td_options),
                                     C.POINTER(vp)]
    lib.td_build_network.restype = C.c_int
    lib.td_coset_logprob.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.td_coset_logprob.restype = C.c_int
    lib.td_gen_rows_host.argtypes = [C.POINTER(td_gen), vp, C.c_int64, vp, vp, vp]
    lib.td_gen_rows_host.restype = C.c_int
    lib.td_coset_logprob_stats.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.td_coset_logprob_stats.restype = C.c_int
    lib.td_decode.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.td_decode.restype = C.c_int
    lib.td_coset_logprob_host.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.td_coset_logprob_host.restype = C.c_int
    lib.td_grad_logprob.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp]
    lib.td_grad_logprob.restype = C.c_int
    lib.td_grad_logprob_forced.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp]
    lib.td_grad_logprob_forced.restype = C.c_int
    lib.td_network_set_schedule.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
    lib.td_network_set_schedule.restype = C.c_int
    lib.td_network_tune.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, vp]
    lib.td_network_tune.restype = C.c_int
    lib.td_network_get_info.argtypes = [vp, C.POINTER(td_network_info)]
    lib.td_network_get_info.restype = C.c_int
    lib.td_debug_sweep.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, vp, C.POINTER(C.c_int32), vp]
    lib.td_debug_sweep.restype = C.c_int
    lib.td_network_profile.argtypes = [vp, C.c_int32, vp, vp]
    lib.td_network_profile.restype = C.c_int
    lib.td_network_get_work.argtypes = [vp, vp, vp, vp]
    lib.td_network_get_work.restype = C.c_int
    lib.td_coset_logprob_static.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.td_coset_logprob_static.restype = C.c_int
    lib.td_network_check.argtypes = [vp, vp]
    lib.td_network_check.restype = C.c_int
    lib.td_measure_fma_peak.argtypes = [C.c_int32, C.c_int32, vp, vp]
    lib.td_measure_fma_peak.restype = C.c_int
    lib.td_build_gen_network.argtypes = [C.POINTER(td_gen), C.POINTER(td_options), C.POINTER(vp)]
    lib.td_build_gen_network.restype = C.c_int
    lib.td_gen_coset_logprob.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.td_gen_coset_logprob.restype = C.c_int
    lib.td_gen_decode.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.td_gen_decode.restype = C.c_int
    lib.td_free_network.argtypes = [vp]
    lib.td_free_network.restype = None
    lib.td_last_error.argtypes = []
    lib.td_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class TDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != TD_OK:
        raise TDError(status, load().td_last_error().decode())

"""ctypes declarations of libmuffin.so (mirrors include/muffin.h)."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmuffin.so")

c_int32 = ctypes.c_int32
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
c_size_t = ctypes.c_size_t


class Params(ctypes.Structure):
    _fields_ = [("n", c_int32), ("nbands", c_int32), ("n_wavelets", c_int32),
                ("levels", c_int32), ("sigma", c_double), ("step_rule", c_int32),
                ("tau_safety", c_double), ("positivity", c_int32), ("sure", c_int32),
                ("batch", c_int32), ("dictionary", c_int32), ("precision", c_int32),
                ("tau", c_double)]


class Info(ctypes.Structure):
    _fields_ = [("iters_done", c_int32), ("tau", c_double), ("sigma", c_double),
                ("lipschitz", c_double), ("mu", c_double), ("gamma", c_double),
                ("records", c_int32), ("checks", c_int32), ("stopped_early", c_int32),
                ("rel_change", c_double), ("objective", c_double)]


class MonitorParams(ctypes.Structure):
    _fields_ = [("every", c_int32), ("objective", c_int32), ("rel_tol", c_double)]


class MonitorRecord(ctypes.Structure):
    _fields_ = [("k", c_int32), ("cube", c_int32), ("rel_change", c_double),
                ("objective", c_double), ("nonfinite", ctypes.c_int64)]


class SureParams(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("window", c_int32), ("eta_mu", c_double),
                ("eta_gamma", c_double), ("theta_min", c_double),
                ("reset_each_window", c_int32), ("eps", c_double)]


class SureRecord(ctypes.Structure):
    _fields_ = [("k", c_int32), ("mu", c_double), ("gamma", c_double),
                ("sugar_mu", c_double), ("sugar_gamma", c_double),
                ("psure", c_double), ("tau", c_double)]


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_size_t), ("max_batch", c_int32),
                ("n_wavelets", c_int32), ("levels", c_int32), ("sigma", c_double),
                ("step_rule", c_int32), ("tau_safety", c_double), ("chunk", c_int32),
                ("max_active_voxels", c_size_t)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("syn_packed", c_int32), ("dct_ctas_per_sm", c_int32),
                ("spectral_tcgen05", c_int32),
                ("from_cache", c_int32), ("candidates", c_int32),
                ("ms_default", c_double), ("ms_best", c_double), ("grad_chunk", c_int32),
                ("fft_radix", c_int32), ("group_order", c_int32), ("ana_ring", c_int32),
                ("ana_pipe", c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("syn_packed", c_int32), ("dct_ctas_per_sm", c_int32),
                ("spectral_tcgen05", c_int32), ("grad_chunk", c_int32),
                ("fft_radix", c_int32), ("group_order", c_int32), ("ana_ring", c_int32),
                ("ana_pipe", c_int32)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", c_double), ("bytes_per_launch", c_double),
                ("flops_per_launch", c_double)]


STATUS = {0: "MUFFIN_OK", 1: "MUFFIN_EINVAL", 2: "MUFFIN_ENOMEM", 3: "MUFFIN_ECUDA",
          4: "MUFFIN_ETIMEOUT", 5: "MUFFIN_ENUMERIC", 6: "MUFFIN_ESTATE"}
MUFFIN_WARM = 1

# name -> (restype, argtypes)
SIGNATURES = {
    "muffin_params_default": (None, [ctypes.POINTER(Params), c_int32, c_int32]),
    "muffin_plan_create": (c_int32, [ctypes.POINTER(Params), c_void_p, c_void_p,
                                     c_void_p, c_void_p, ctypes.POINTER(c_void_p)]),
    "muffin_plan_destroy": (None, [c_void_p]),
    "muffin_plan_device_bytes": (c_size_t, [c_void_p]),
    "muffin_plan_lipschitz": (c_int32, [c_void_p, ctypes.POINTER(c_double)]),
    "muffin_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double,
                               c_double, c_int32, ctypes.POINTER(Info)]),
    "muffin_solve_batch": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32,
                                     ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                     c_int32, ctypes.POINTER(Info)]),
    "muffin_plan_graphs": (c_int32, [c_void_p, c_int32]),
    "muffin_plan_autotune": (c_int32, [c_void_p, ctypes.c_char_p, ctypes.POINTER(TuneInfo)]),
    "muffin_plan_set_tuning": (c_int32, [c_void_p, c_int32, c_int32]),
    "muffin_plan_set_spectral_kernel": (c_int32, [c_void_p, c_int32]),
    "muffin_plan_get_schedule": (c_int32, [c_void_p, ctypes.POINTER(Schedule)]),
    "muffin_plan_set_schedule": (c_int32, [c_void_p, ctypes.POINTER(Schedule)]),
    "muffin_plan_inject_timeout": (c_int32, [c_void_p, c_int32]),
    "muffin_sure_params_default": (None, [ctypes.POINTER(SureParams)]),
    "muffin_sure_tune": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p,
                                   ctypes.POINTER(SureParams), c_void_p,
                                   ctypes.POINTER(c_double), ctypes.POINTER(SureRecord),
                                   c_int32, ctypes.POINTER(Info)]),
    "muffin_sure_global": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                     c_void_p, ctypes.POINTER(c_double),
                                     ctypes.POINTER(SureRecord), ctypes.POINTER(Info)]),
    "muffin_sure_global_auto": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_int32, c_int32, c_double, c_void_p,
                                          ctypes.POINTER(c_double), ctypes.POINTER(SureRecord),
                                          ctypes.POINTER(Info)]),
    "muffin_plan_set_monitor": (c_int32, [c_void_p, ctypes.POINTER(MonitorParams)]),
    "muffin_plan_monitor_read": (c_int32, [c_void_p, ctypes.POINTER(MonitorRecord), c_int32,
                                           ctypes.POINTER(c_int32)]),
    "muffin_objective": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "muffin_plan_set_weights": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "muffin_plan_weights_from_x0": (c_int32, [c_void_p, c_void_p, c_double, c_double,
                                              c_void_p, c_void_p]),
    "muffin_noise_mad": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "muffin_shard_spatial": (c_int32, [c_void_p, c_void_p, c_void_p, c_double, c_double,
                                       c_double]),
    "muffin_shard_spectral": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p,
                                        ctypes.c_int64, ctypes.c_int64, c_double]),
    "muffin_state_size": (c_int32, [c_void_p, ctypes.POINTER(c_size_t)]),
    "muffin_state_export": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "muffin_state_import": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "muffin_op_gradient": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "muffin_op_analysis": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "muffin_op_synthesis": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "muffin_op_dct": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "muffin_plan_estimate_bytes": (c_int32, [ctypes.POINTER(Params), ctypes.POINTER(c_size_t)]),
    "muffin_plan_load_psf": (c_int32, [c_void_p, c_int32, c_int32, c_void_p]),
    "muffin_plan_load_visibilities": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "muffin_server_params_default": (None, [ctypes.POINTER(ServerParams)]),
    "muffin_server_create": (c_int32, [ctypes.POINTER(ServerParams), c_void_p,
                                       ctypes.POINTER(c_void_p)]),
    "muffin_server_destroy": (None, [c_void_p]),
    "muffin_serve_submit": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                      c_double, c_double, c_int32,
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "muffin_serve_step": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "muffin_serve_poll": (c_int32, [c_void_p, ctypes.c_uint64, ctypes.POINTER(c_int32),
                                    c_void_p]),
    "muffin_server_stats": (c_int32, [c_void_p, ctypes.POINTER(c_size_t),
                                      ctypes.POINTER(c_int32)]),
    "muffin_op_analysis_noalloc": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32,
                                             c_int32, c_void_p]),
    "muffin_profile_enable": (c_int32, [c_void_p, c_int32]),
    "muffin_profile_read": (c_int32, [c_void_p, ctypes.POINTER(KernelStat), c_int32,
                                      ctypes.POINTER(c_int32)]),
    "muffin_filter_taps": (c_int32, [c_int32, ctypes.POINTER(c_double)]),
    "muffin_dct_table": (c_int32, [c_int32, ctypes.POINTER(c_double)]),
    "muffin_last_error": (ctypes.c_char_p, []),
    "muffin_version": (ctypes.c_char_p, []),
}

_lib = None


class MuffinError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load the in-tree libmuffin.so; fails loudly when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != 0:
        raise MuffinError(status, load().muffin_last_error().decode())

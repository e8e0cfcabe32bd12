"""ctypes declarations of the C ABI in include/wct_sim.h (argument marshalling only).

Every function keeps its C name; the structures mirror the header field by field.  Loading
fails loudly if the CUDA library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_i32, c_i64, c_u64, c_dbl, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
c_vp = ctypes.c_void_p

WCT_OK, WCT_EINVAL, WCT_ENOMEM, WCT_ECUDA, WCT_ETIMEOUT, WCT_EBUSY, WCT_EDEVICE = range(7)
STATUS_NAMES = {0: "WCT_OK", 1: "WCT_EINVAL", 2: "WCT_ENOMEM", 3: "WCT_ECUDA", 4: "WCT_ETIMEOUT",
                5: "WCT_EBUSY", 6: "WCT_EDEVICE"}
WCT_MAX_WINDOW_TICKS = 128
WCT_MAX_WINDOW_IMPACTS = 512
WCT_MAX_RESPONSE_WIRES = 21


class wct_plane_t(ctypes.Structure):
    _fields_ = [("n_wires", c_i32), ("n_impact_per_pitch", c_i32), ("n_ticks", c_i32),
                ("pitch_mm", c_dbl), ("pitch_origin_mm", c_dbl), ("wire_angle_rad", c_dbl),
                ("tick_us", c_dbl), ("t_window0_us", c_dbl)]


class wct_response_t(ctypes.Structure):
    _fields_ = [("n_wires_resp", c_i32), ("n_ticks_resp", c_i32), ("host_data", ctypes.POINTER(ctypes.c_float))]


class wct_diffusion_t(ctypes.Structure):
    _fields_ = [("DL_cm2_s", c_dbl), ("DT_cm2_s", c_dbl), ("v_drift_mm_us", c_dbl), ("nsigma", c_dbl),
                ("fluctuate", c_i32), ("seed", c_u64)]


class wct_opts_t(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_sz), ("schedule_id", c_i32), ("deterministic", c_i32)]


class wct_depos_t(ctypes.Structure):
    _fields_ = [("t0_us", c_vp), ("x_mm", c_vp), ("y_mm", c_vp), ("z_mm", c_vp), ("q_e", c_vp),
                ("n", c_i64), ("event_id", c_u64)]


class wct_adc_t(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_double), ("baseline", ctypes.c_double), ("noise_rms", ctypes.c_double),
                ("bits", c_i32), ("add_noise", c_i32)]


class wct_field_response_t(ctypes.Structure):
    _fields_ = [("n_paths", c_i32), ("n_samples", c_i32), ("period_us", c_dbl), ("path_pos_mm", c_vp),
                ("current", c_vp)]


class wct_host_depos_t(ctypes.Structure):
    _fields_ = [("t0_us", c_vp), ("x_mm", c_vp), ("y_mm", c_vp), ("z_mm", c_vp), ("q_e", c_vp),
                ("n", c_i64), ("event_id", c_u64)]


EXPORTS = {
    "wct_sim_create": ([ctypes.POINTER(wct_plane_t), ctypes.c_int, ctypes.POINTER(wct_response_t),
                        ctypes.POINTER(wct_diffusion_t), ctypes.POINTER(wct_opts_t), ctypes.POINTER(c_vp)],
                       ctypes.c_int),
    "wct_sim_destroy": ([c_vp], ctypes.c_int),
    "wct_sim_rasterize": ([c_vp, ctypes.c_int, ctypes.POINTER(wct_depos_t), c_vp, c_i64, c_vp,
                           ctypes.POINTER(c_i64), c_vp], ctypes.c_int),
    "wct_sim_rasterize_fixed": ([c_vp, ctypes.c_int, ctypes.POINTER(wct_depos_t), c_vp, c_i64, c_vp, c_vp],
                                ctypes.c_int),
    "wct_sim_patch_slot_bins": ([c_vp, ctypes.c_int, c_dbl, ctypes.POINTER(c_i64)], ctypes.c_int),
    "wct_sim_scatter": ([c_vp, ctypes.c_int, ctypes.POINTER(wct_depos_t), c_vp, c_vp, c_vp, c_vp], ctypes.c_int),
    "wct_sim_convolve": ([c_vp, ctypes.c_int, c_vp, c_vp, c_vp], ctypes.c_int),
    "wct_sim_run_event": ([c_vp, ctypes.POINTER(wct_depos_t), ctypes.POINTER(c_vp), c_vp], ctypes.c_int),
    "wct_sim_run_batch": ([c_vp, ctypes.POINTER(wct_depos_t), ctypes.c_int, ctypes.POINTER(c_vp), c_vp],
                          ctypes.c_int),
    "wct_sim_set_impact_responses": ([c_vp, ctypes.c_int, ctypes.POINTER(wct_response_t), ctypes.c_int], ctypes.c_int),
    "wct_sim_convolve_impact": ([c_vp, ctypes.c_int, c_vp, c_vp, c_vp], ctypes.c_int),
    "wct_sim_run_host": ([c_vp, ctypes.POINTER(wct_host_depos_t), ctypes.c_int, ctypes.POINTER(c_vp)], ctypes.c_int),
    "wct_sim_digitize": ([c_vp, ctypes.c_int, c_vp, c_vp, ctypes.POINTER(wct_adc_t), c_u64, c_vp], ctypes.c_int),
    "wct_sim_set_noise_spectrum": ([c_vp, ctypes.c_int, c_vp, ctypes.c_int], ctypes.c_int),
    "wct_sim_set_lifetime": ([c_vp, ctypes.c_double, c_i32], ctypes.c_int),
    "wct_sim_sync": ([c_vp, c_vp], ctypes.c_int),
    "wct_sim_plane_info": ([c_vp, ctypes.c_int, ctypes.POINTER(c_i64)], ctypes.c_int),
    "wct_sim_set_timing": ([c_vp, ctypes.c_int], ctypes.c_int),
    "wct_sim_stage_times": ([c_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int], ctypes.c_int),
    "wct_sim_counters": ([c_vp, ctypes.POINTER(c_i64), ctypes.c_int], ctypes.c_int),
    "wct_sim_selftest_wait": ([c_vp, c_i64, c_vp], ctypes.c_int),
    "wct_sim_last_error": ([c_vp], ctypes.c_char_p),
    "wct_philox4x32_10": ([c_vp, c_u64, c_i64, c_vp, c_vp], ctypes.c_int),
    "wct_debug_fail_alloc": ([c_i64], ctypes.c_int),
    "wct_debug_bounds": ([c_vp, ctypes.POINTER(c_i64)], ctypes.c_int),
    "wct_convolve_static": ([c_vp, c_i32, c_i32, c_vp, c_i32, c_i32, c_vp, c_vp], ctypes.c_int),
    "wct_convolve_static_status": ([c_vp], ctypes.c_int),
    "wct_convolve_static_selftest_wait": ([c_i64, c_vp], ctypes.c_int),
    "wct_response_from_field": ([ctypes.POINTER(wct_field_response_t), c_vp, c_i32, c_dbl, c_i32, c_dbl, c_i32,
                                 c_i32, c_vp, c_vp], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (building it first only if asked).  $WCT_LIB names another build
    of the same sources instead (e.g. the bounds-checked one, build.build(bounds_check=True))."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("WCT_LIB") or _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build() first")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


class WctError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code

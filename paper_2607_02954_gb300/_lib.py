"""ctypes binding of libmc (include/mc.h): argument marshalling only.

Every computation runs in the CUDA library.  Loading fails loudly when the
library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmc.so")

MC_OK = 0
MC_MEM_HOST = 0
MC_MEM_DEVICE = 1
STATUS_NAMES = {0: "MC_OK", 1: "MC_ERR_INVALID_ARG", 2: "MC_ERR_OOM", 3: "MC_ERR_CUDA",
                4: "MC_ERR_TIMEOUT", 5: "MC_ERR_UNSTABLE", 6: "MC_ERR_BUSY", 7: "MC_ERR_NOT_FOUND",
                8: "MC_ERR_CANCELLED"}

FIELDS = {"fel": 0, "fs": 1, "ubead": 2, "rho_s": 3, "rho_bar": 4, "force": 5, "u": 6,
          "cell": 7, "bin": 8, "bin_off": 9, "bin_beads": 10, "ebead": 11}


class MCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mc_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("nu", "dt", "Lambda", "kappa", "k_bend", "k_stretch", "k_shear", "k_rep", "sigma", "orient")] + \
               [("n_pbd", ctypes.c_int), ("pbd_order", ctypes.c_int), ("layers", ctypes.c_int),
                ("layer_half", ctypes.c_float), ("ib", ctypes.c_int), ("mdf_iters", ctypes.c_int)]


_fp = ctypes.POINTER(ctypes.c_float)


class mc_world_desc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("n_fil", ctypes.c_int),
                ("fil_off", ctypes.POINTER(ctypes.c_int)),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("L_rest", ctypes.c_void_p), ("theta0", ctypes.c_void_p), ("drive_amp", ctypes.c_void_p),
                ("drive_freq", ctypes.c_void_p), ("drive_phase", ctypes.c_void_p), ("f0", ctypes.c_void_p),
                ("t0", ctypes.c_int64), ("p", mc_params), ("mem_kind", ctypes.c_int),
                ("len_amp", ctypes.c_void_p), ("len_freq", ctypes.c_void_p), ("len_phase", ctypes.c_void_p),
                ("energy", ctypes.c_void_p), ("observe", ctypes.c_int)]


class mc_world_info(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("n_fil", ctypes.c_int), ("N", ctypes.c_int),
                ("E", ctypes.c_int), ("J", ctypes.c_int), ("bin_edge", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("t", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


class mc_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("steps_per_tick", ctypes.c_int), ("max_pending", ctypes.c_int)]


class mc_result(ctypes.Structure):
    _fields_ = [("com_disp", ctypes.c_double * 2), ("e_bend", ctypes.c_double), ("e_pos", ctypes.c_double),
                ("energy", ctypes.c_double), ("status", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class mc_launch_config(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int), ("pbd_warps", ctypes.c_int), ("scan_kernels", ctypes.c_int),
                ("force_kernel", ctypes.c_int)]


class mc_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "steps_run", "ticks", "pending")]


# name -> (restype, argtypes): every entry point declared in include/mc.h
_vp, _i, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "mc_params_default": (_i, [ctypes.POINTER(mc_params)]),
    "mc_world_create": (_i, [ctypes.POINTER(mc_world_desc), _vp, ctypes.POINTER(_vp)]),
    "mc_world_destroy": (_i, [_vp]),
    "mc_world_save_size": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "mc_world_save": (_i, [_vp, _vp, ctypes.c_size_t, _vp]),
    "mc_world_load": (_i, [_vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "mc_world_info_get": (_i, [_vp, ctypes.POINTER(mc_world_info)]),
    "mc_step": (_i, [_vp, _i, _vp]),
    "mc_step_batched": (_i, [ctypes.POINTER(_vp), _i, _i, _vp]),
    "mc_step_stage": (_i, [_vp, _i, _vp]),
    "mc_autotune": (_i, [ctypes.POINTER(_vp), _i, _vp, ctypes.POINTER(mc_launch_config)]),
    "mc_launch_config_get": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(mc_launch_config)]),
    "mc_launch_config_set": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(mc_launch_config)]),
    "mc_autotune_mode": (_i, [_i]),
    "mc_debug_barrier_test": (_i, [ctypes.c_uint, ctypes.c_int64]),
    "mc_world_get_state": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "mc_world_get_positions_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "mc_world_get_field": (_i, [_vp, _i, _vp, _i, _vp]),
    "mc_world_check": (_i, [_vp, _vp]),
    "mc_world_clear_flags": (_i, [_vp, _vp]),
    "mc_world_get_observables": (_i, [_vp, _vp, _vp]),
    "mc_rollout_forward": (_i, [_vp, _i, _i, _vp]),
    "mc_rollout_backward": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "mc_rollout_forward_stored": (_i, [_vp, _i, _vp]),
    "mc_rollout_rewind": (_i, [_vp, _vp]),
    "mc_world_set_rest": (_i, [_vp, _vp, _vp, _i, _vp]),
    "mc_rollout_backward_params": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mc_loss_polyline": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "mc_loss_splat": (_i, [_vp, _vp, _i, ctypes.c_float, _vp, _vp, _vp, _vp]),
    "mc_server_create": (_i, [ctypes.POINTER(mc_server_cfg), ctypes.POINTER(_vp)]),
    "mc_serve_submit": (_i, [_vp, ctypes.POINTER(mc_world_desc), _i, ctypes.POINTER(ctypes.c_uint64)]),
    "mc_serve_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(mc_result)]),
    "mc_serve_wait": (_i, [_vp, ctypes.c_uint64, _i, ctypes.POINTER(mc_result)]),
    "mc_server_stats_get": (_i, [_vp, ctypes.POINTER(mc_server_stats)]),
    "mc_server_destroy": (_i, [_vp]),
    "mc_serve_cancel": (_i, [_vp, ctypes.c_uint64]),
    "mc_inject_world_alloc_failure": (_i, [_i]),
    "mc_last_error": (ctypes.c_char_p, []),
    "mc_abi_version": (_i, []),
}

_lib = None


ABI_VERSION = 7   # MC_ABI_VERSION of include/mc.h that these structures mirror


def load():
    """Loads libmc.so once; raises if it is missing (build it with build())
    or was built from another version of the C ABI."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmc.so is not built ({LIB_PATH}); run paper_2607_02954_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if lib.mc_abi_version() != ABI_VERSION:
            raise RuntimeError(f"libmc.so has C ABI version {lib.mc_abi_version()}, this binding expects "
                               f"{ABI_VERSION}: rebuild it with paper_2607_02954_gb300.build.build()")
        _lib = lib
    return _lib


def check(status: int):
    if status != MC_OK:
        raise MCError(status, load().mc_last_error().decode())


def __getattr__(name):
    if name.startswith("mc_"):
        return getattr(load(), name)
    raise AttributeError(name)

"""CPU checks of the C ABI library: it loads, exports every entry point that
include/mc.h declares, and its host-side validation rejects bad worlds before
touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2607_02954_gb300 import _lib as L
from paper_2607_02954_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**(mc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("mc_world_create", "mc_world_destroy", "mc_step", "mc_step_batched", "mc_world_get_state"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/mc.h but not exported"
    assert set(names) == set(L.SIGNATURES), "binding signatures out of sync with include/mc.h"


def test_defaults_match_the_frozen_constants():
    p = L.mc_params()
    assert L.load().mc_params_default(ctypes.byref(p)) == 0
    ref = synth.Params()
    for name, _ in L.mc_params._fields_:
        assert abs(getattr(p, name) - getattr(ref, name)) < 1e-7, name


def _desc(spec, **over):
    from paper_2607_02954_gb300.world import params_struct
    d = L.mc_world_desc()
    d.H, d.W, d.n_fil = over.get("H", spec.H), over.get("W", spec.W), spec.n_fil
    fo = np.ascontiguousarray(over.get("fil_off", spec.fil_off), np.int32)
    keep = [fo]
    d.fil_off = fo.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    for name in ("x", "y", "theta", "L_rest", "theta0", "drive_amp", "drive_freq", "drive_phase"):
        a = np.ascontiguousarray(over.get(name, getattr(spec, name)), np.float32)
        keep.append(a)
        setattr(d, name, ctypes.c_void_p(a.ctypes.data if a.size else 0))
    d.t0 = over.get("t0", 0)
    d.p = params_struct(over.get("params", spec.params))
    d.mem_kind = L.MC_MEM_HOST
    return d, keep


@pytest.mark.parametrize("case", ["H_not_mult8", "W_small", "short_filament", "nan_x", "bad_nu",
                                  "bad_sigma", "neg_L", "bad_t0", "bad_npbd", "bad_pbd_order",
                                  "bad_layers", "bad_layer_half", "bad_ib", "ib_two_layers", "bad_mdf_iters"])
def test_create_rejects_invalid_worlds_on_host(case):
    spec = synth.tiny_world(0, side=16, lengths=(5, 4))
    over = {}
    if case == "H_not_mult8":
        over["H"] = 20
    elif case == "W_small":
        over["W"] = 0
    elif case == "short_filament":
        over["fil_off"] = np.array([0, 1, 9], np.int32)
    elif case == "nan_x":
        x = spec.x.copy()
        x[2] = np.nan
        over["x"] = x
    elif case == "bad_nu":
        over["params"] = synth.Params(nu=0.0)
    elif case == "bad_sigma":
        over["params"] = synth.Params(sigma=3.0)
    elif case == "neg_L":
        over["L_rest"] = -spec.L_rest
    elif case == "bad_t0":
        over["t0"] = 1 << 24
    elif case == "bad_npbd":
        over["params"] = synth.Params(n_pbd=65)
    elif case == "bad_pbd_order":
        over["params"] = synth.Params(pbd_order=2)
    elif case == "bad_layers":
        over["params"] = synth.Params(layers=3)
    elif case == "bad_layer_half":
        over["params"] = synth.Params(layers=2, layer_half=0.0)
    elif case == "bad_ib":
        over["params"] = synth.Params(ib=2)
    elif case == "ib_two_layers":
        over["params"] = synth.Params(ib=1, mdf_iters=2, layers=2)
    elif case == "bad_mdf_iters":
        over["params"] = synth.Params(ib=1, mdf_iters=65)
    d, keep = _desc(spec, **over)
    h = ctypes.c_void_p()
    lib = L.load()
    status = lib.mc_world_create(ctypes.byref(d), None, ctypes.byref(h))
    assert status == 1, (case, status, lib.mc_last_error())
    assert h.value is None
    assert lib.mc_last_error()


def test_step_rejects_null_world():
    lib = L.load()
    assert lib.mc_step(None, 1, None) == 1
    assert lib.mc_step_batched(None, 1, 1, None) == 1
    assert lib.mc_rollout_forward(None, 4, 2, None) == 1
    assert lib.mc_rollout_forward_stored(None, 4, None) == 1


def test_fault_injection_and_cancel_validate_arguments():
    lib = L.load()
    assert lib.mc_inject_world_alloc_failure(-1) == 1
    assert lib.mc_inject_world_alloc_failure(0) == 0
    assert lib.mc_serve_cancel(None, 1) == 1


def test_launch_config_calls_validate_arguments():
    lib = L.load()
    c = L.mc_launch_config(persistent=0, pbd_warps=8, scan_kernels=0)
    assert lib.mc_launch_config_set(None, 0, ctypes.byref(c)) == 1
    assert lib.mc_launch_config_get(None, 1, ctypes.byref(c)) == 1
    assert lib.mc_autotune(None, 1, None, None) == 1
    assert lib.mc_autotune_mode(2) == 1
    assert lib.mc_autotune_mode(1) == 0
    assert lib.mc_debug_barrier_test(2, 1000) == 1
    assert lib.mc_debug_barrier_test(0, 10) == 1


def test_world_load_rejects_corrupt_images_on_host():
    lib = L.load()
    h = ctypes.c_void_p()
    junk = ctypes.create_string_buffer(b"not a world image at all" * 8)
    assert lib.mc_world_load(junk, len(junk), None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.mc_world_load(junk, 4, None, ctypes.byref(h)) == 1
    n = ctypes.c_size_t()
    assert lib.mc_world_save_size(None, ctypes.byref(n)) == 1

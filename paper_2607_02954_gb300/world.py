"""User-facing Python API over the C ABI: World, step_batched.

Argument marshalling only: inputs go to mc_world_create as host (numpy) or
device (torch CUDA tensor) pointers, every step runs in libmc's kernels, and
outputs come back through mc_world_get_state / mc_world_get_field.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional, Sequence

import numpy as np

from . import _lib as L
from .synth import Params, WorldSpec


def _torch():
    import torch
    return torch


def stream_handle(stream=None) -> ctypes.c_void_p:
    """cudaStream_t of a torch stream (default: the current stream)."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def params_struct(p: Params) -> L.mc_params:
    return L.mc_params(nu=p.nu, dt=p.dt, Lambda=p.Lambda, kappa=p.kappa, k_bend=p.k_bend,
                       k_stretch=p.k_stretch, k_shear=p.k_shear, k_rep=p.k_rep, sigma=p.sigma,
                       orient=p.orient, n_pbd=int(p.n_pbd),
                       pbd_order=int(getattr(p, "pbd_order", 0)), layers=int(getattr(p, "layers", 1)),
                       layer_half=float(getattr(p, "layer_half", 0.5)), ib=int(getattr(p, "ib", 0)),
                       mdf_iters=int(getattr(p, "mdf_iters", 0)))


def default_params() -> Params:
    c = L.mc_params()
    L.check(L.load().mc_params_default(ctypes.byref(c)))
    return Params(**{k: getattr(c, k) for k, _ in L.mc_params._fields_})


_FLOAT_ARRAYS = ("x", "y", "theta", "L_rest", "theta0", "drive_amp", "drive_freq", "drive_phase")
_OPTIONAL_ARRAYS = ("f0", "len_amp", "len_freq", "len_phase", "energy")


def make_desc(spec: WorldSpec, device: bool = False):
    """mc_world_desc pointing at host (numpy) or device (torch) copies of the
    spec's arrays; returns (desc, objects that must stay alive)."""
    d = L.mc_world_desc()
    keep = []
    d.H, d.W, d.n_fil = int(spec.H), int(spec.W), int(spec.n_fil)
    fo = np.ascontiguousarray(spec.fil_off, dtype=np.int32)
    keep.append(fo)
    d.fil_off = fo.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    if device:
        torch = _torch()
        for name in _FLOAT_ARRAYS:
            t = torch.as_tensor(np.ascontiguousarray(getattr(spec, name), np.float32)).cuda()
            keep.append(t)
            setattr(d, name, ctypes.c_void_p(t.data_ptr() if t.numel() else 0))
        for name in _OPTIONAL_ARRAYS:
            v = getattr(spec, name, None)
            if v is not None:
                t = torch.as_tensor(np.ascontiguousarray(v, np.float32)).cuda()
                keep.append(t)
                setattr(d, name, ctypes.c_void_p(t.data_ptr() if t.numel() else 0))
        d.mem_kind = L.MC_MEM_DEVICE
        torch.cuda.synchronize()
    else:
        for name in _FLOAT_ARRAYS:
            a = np.ascontiguousarray(getattr(spec, name), dtype=np.float32)
            keep.append(a)
            setattr(d, name, ctypes.c_void_p(a.ctypes.data if a.size else 0))
        for name in _OPTIONAL_ARRAYS:
            v = getattr(spec, name, None)
            if v is not None:
                a = np.ascontiguousarray(v, dtype=np.float32)
                keep.append(a)
                setattr(d, name, ctypes.c_void_p(a.ctypes.data if a.size else 0))
        d.mem_kind = L.MC_MEM_HOST
    d.t0 = int(spec.t0)
    d.p = params_struct(spec.params)
    d.observe = int(bool(getattr(spec, "observe", False)))
    return d, keep


class World:
    """One world resident on the GPU.

    spec: a WorldSpec (host arrays).  With device=True the arrays are first
    moved to torch CUDA tensors and handed over as device pointers, which is
    the path the benchmark uses when inputs are already resident."""

    def __init__(self, spec: WorldSpec, stream=None, device: bool = False):
        lib = L.load()
        self.spec = spec
        d, keep = make_desc(spec, device)
        h = ctypes.c_void_p()
        L.check(lib.mc_world_create(ctypes.byref(d), stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self._lib = lib

    # -- life cycle ---------------------------------------------------------
    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("world destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.mc_world_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, stream=None) -> bytes:
        """Image of the world after the enqueued work (mc_world_save)."""
        n = ctypes.c_size_t()
        L.check(self._lib.mc_world_save_size(self.handle, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        L.check(self._lib.mc_world_save(self.handle, buf, n.value, stream_handle(stream)))
        return buf.raw

    @classmethod
    def load(cls, image: bytes, spec: WorldSpec, stream=None) -> "World":
        """A world resumed from an image of save(); spec describes it (sizes,
        for the Python-side helpers) and is not sent to the library."""
        lib = L.load()
        obj = cls.__new__(cls)
        obj.spec = spec
        obj._lib = lib
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(image, len(image))
        L.check(lib.mc_world_load(buf, len(image), stream_handle(stream), ctypes.byref(h)))
        obj._h = h
        return obj

    def info(self) -> Dict[str, int]:
        i = L.mc_world_info()
        L.check(self._lib.mc_world_info_get(self.handle, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in L.mc_world_info._fields_}

    # -- stepping -----------------------------------------------------------
    def step(self, n_steps: int = 1, stream=None):
        L.check(self._lib.mc_step(self.handle, int(n_steps), stream_handle(stream)))

    def check(self, stream=None):
        L.check(self._lib.mc_world_check(self.handle, stream_handle(stream)))

    def clear_flags(self, stream=None):
        L.check(self._lib.mc_world_clear_flags(self.handle, stream_handle(stream)))

    # -- read-out -----------------------------------------------------------
    def state(self, fluid: bool = False, stream=None) -> Dict[str, np.ndarray]:
        """Host copies: x, y [N], theta [E], disp [N, 2], and fdev [9, H, W]
        (populations minus rest weights) when fluid=True."""
        s = self.spec
        N, E = s.N, s.E
        out = {"x": np.empty(N, np.float32), "y": np.empty(N, np.float32),
               "theta": np.empty(E, np.float32), "disp": np.empty((N, 2), np.float32)}
        if fluid:
            out["fdev"] = np.empty((9, s.H, s.W), np.float32)
        ptr = lambda k: ctypes.c_void_p(out[k].ctypes.data) if k in out and out[k].size else None
        L.check(self._lib.mc_world_get_state(self.handle, ptr("x"), ptr("y"), ptr("theta"), ptr("disp"),
                                             ptr("fdev"), L.MC_MEM_HOST, stream_handle(stream)))
        return out

    def state_device(self, stream=None):
        """Device (torch) copies of x, y, theta, disp."""
        torch = _torch()
        s = self.spec
        out = {"x": torch.empty(s.N, device="cuda"), "y": torch.empty(s.N, device="cuda"),
               "theta": torch.empty(s.E, device="cuda"), "disp": torch.empty((s.N, 2), device="cuda")}
        ptr = lambda k: ctypes.c_void_p(out[k].data_ptr()) if out[k].numel() else None
        L.check(self._lib.mc_world_get_state(self.handle, ptr("x"), ptr("y"), ptr("theta"), ptr("disp"),
                                             None, L.MC_MEM_DEVICE, stream_handle(stream)))
        return out

    # -- reverse mode ---------------------------------------------------------
    def rollout_forward(self, n_steps: int, ckpt_every: int = 100, stream=None, stored: bool = False):
        """Advance n_steps recording the rollout for the reverse mode: a
        checkpoint every ckpt_every steps (the backward re-runs each segment),
        or with stored=True every step's record (the backward re-runs none)."""
        if stored:
            L.check(self._lib.mc_rollout_forward_stored(self.handle, int(n_steps), stream_handle(stream)))
        else:
            L.check(self._lib.mc_rollout_forward(self.handle, int(n_steps), int(ckpt_every), stream_handle(stream)))

    def rollout_rewind(self, stream=None):
        """Back to the start of the last recorded rollout (see mc_rollout_rewind)."""
        L.check(self._lib.mc_rollout_rewind(self.handle, stream_handle(stream)))

    def set_rest(self, theta0=None, L_rest=None, stream=None):
        """New static rest angles [J] and/or rest lengths [E] (numpy or torch CUDA)."""
        torch = _torch()
        keep, ptrs = [], []
        on_device = any(isinstance(v, torch.Tensor) and v.is_cuda for v in (theta0, L_rest) if v is not None)
        for v in (theta0, L_rest):
            if v is None:
                ptrs.append(None)
            elif on_device:
                t = torch.as_tensor(v).float().contiguous().cuda()
                keep.append(t)
                ptrs.append(ctypes.c_void_p(t.data_ptr()))
            else:
                a = np.ascontiguousarray(v, np.float32)
                keep.append(a)
                ptrs.append(ctypes.c_void_p(a.ctypes.data))
        L.check(self._lib.mc_world_set_rest(self.handle, ptrs[0], ptrs[1],
                                            L.MC_MEM_DEVICE if on_device else L.MC_MEM_HOST, stream_handle(stream)))
        if on_device:
            torch.cuda.current_stream().synchronize()

    def rollout_backward(self, dL_dx, dL_dy, stream=None):
        """dL_dx, dL_dy: torch CUDA float32 [N]; returns dL/dtheta0 as a torch CUDA tensor [J]."""
        torch = _torch()
        gx = dL_dx.contiguous().float()
        gy = dL_dy.contiguous().float()
        out = torch.empty(self.spec.J, device="cuda", dtype=torch.float32)
        L.check(self._lib.mc_rollout_backward(self.handle, ctypes.c_void_p(gx.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr() if out.numel() else 0), stream_handle(stream)))
        return out

    def rollout_backward_params(self, dL_dx, dL_dy, stream=None):
        """As rollout_backward, plus the rest-length and stiffness gradients:
        returns {"theta0": [J], "L_rest": [E], "k": [3] (k_bend, k_stretch,
        k_shear)} as torch CUDA tensors."""
        torch = _torch()
        gx = dL_dx.contiguous().float()
        gy = dL_dy.contiguous().float()
        s = self.spec
        out = {"theta0": torch.empty(s.J, device="cuda", dtype=torch.float32),
               "L_rest": torch.empty(s.E, device="cuda", dtype=torch.float32),
               "k": torch.empty(3, device="cuda", dtype=torch.float32)}
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t.numel() else 0)
        L.check(self._lib.mc_rollout_backward_params(self.handle, ctypes.c_void_p(gx.data_ptr()),
                                                     ctypes.c_void_p(gy.data_ptr()), ptr(out["theta0"]),
                                                     ptr(out["L_rest"]), ptr(out["k"]), stream_handle(stream)))
        return out

    def observables(self, stream=None) -> Dict[str, float]:
        """Behaviour descriptors E_bend, E_pos and the energy collected since
        creation (zeros unless the spec set observe)."""
        out = (ctypes.c_double * 3)()
        L.check(self._lib.mc_world_get_observables(self.handle, ctypes.cast(out, ctypes.c_void_p),
                                                   stream_handle(stream)))
        return {"e_bend": out[0], "e_pos": out[1], "energy": out[2]}

    def loss_polyline(self, poly, stream=None):
        """Folding loss against a polyline (numpy [V, 2]); returns (loss tensor [1], dL_dx, dL_dy)."""
        torch = _torch()
        pl = torch.as_tensor(np.ascontiguousarray(poly, np.float32)).cuda()
        loss = torch.zeros(1, device="cuda", dtype=torch.float32)
        gx = torch.empty(self.spec.N, device="cuda", dtype=torch.float32)
        gy = torch.empty(self.spec.N, device="cuda", dtype=torch.float32)
        L.check(self._lib.mc_loss_polyline(self.handle, ctypes.c_void_p(pl.data_ptr()), int(pl.shape[0]),
                                           ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(gx.data_ptr()),
                                           ctypes.c_void_p(gy.data_ptr()), stream_handle(stream)))
        return loss, gx, gy

    def loss_splat(self, target, sigma: float = 1.0, stream=None):
        """The splat folding loss against an R x R target image (numpy or
        torch); returns (loss tensor [1], dL_dx, dL_dy) on the GPU."""
        torch = _torch()
        tg = torch.as_tensor(np.ascontiguousarray(target, np.float32) if isinstance(target, np.ndarray) else target)
        tg = tg.float().contiguous().cuda()
        loss = torch.zeros(1, device="cuda", dtype=torch.float32)
        gx = torch.empty(self.spec.N, device="cuda", dtype=torch.float32)
        gy = torch.empty(self.spec.N, device="cuda", dtype=torch.float32)
        L.check(self._lib.mc_loss_splat(self.handle, ctypes.c_void_p(tg.data_ptr()), int(tg.shape[0]),
                                        float(sigma), ctypes.c_void_p(loss.data_ptr()),
                                        ctypes.c_void_p(gx.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                        stream_handle(stream)))
        return loss, gx, gy

    def field(self, name: str, stream=None) -> np.ndarray:
        """Host copy of one field of the last completed step (see mc_field)."""
        s = self.spec
        N, HW = s.N, s.H * s.W
        info = self.info()
        shapes = {"fel": ((N, 2), np.float32), "fs": ((N, 2), np.float32), "ubead": ((N, 2), np.float32),
                  "rho_s": ((s.H, s.W), np.float32), "rho_bar": ((s.H, s.W), np.float32),
                  "force": ((s.H, s.W, 2), np.float32), "u": ((s.H, s.W, 2), np.float32),
                  "cell": ((N,), np.int32), "bin": ((N,), np.int32), "ebead": ((N,), np.float32),
                  "bin_off": ((info["n_bins"] + 1,), np.int32), "bin_beads": ((N,), np.int32)}
        shape, dt = shapes[name]
        out = np.empty(shape, dt)
        L.check(self._lib.mc_world_get_field(self.handle, L.FIELDS[name], ctypes.c_void_p(out.ctypes.data),
                                             L.MC_MEM_HOST, stream_handle(stream)))
        return out


def step_batched(worlds: Sequence[World], n_steps: int, stream=None):
    """Advances distinct worlds together: one launch per stage per step."""
    arr = (ctypes.c_void_p * len(worlds))(*[w.handle.value for w in worlds])
    L.check(L.load().mc_step_batched(arr, len(worlds), int(n_steps), stream_handle(stream)))


def _handles(worlds: Sequence[World]):
    return (ctypes.c_void_p * len(worlds))(*[w.handle.value for w in worlds])


def _cfg_dict(c: L.mc_launch_config) -> Dict:
    return {"persistent": c.persistent, "pbd_warps": c.pbd_warps, "scan_kernels": c.scan_kernels,
            "force_kernel": c.force_kernel}


def autotune(worlds: Sequence[World], stream=None) -> Dict:
    """Tunes the launch configuration of the plan of these worlds (one world,
    or the batch as step_batched passes it) and returns the choice."""
    c = L.mc_launch_config()
    L.check(L.load().mc_autotune(_handles(worlds), len(worlds), stream_handle(stream), ctypes.byref(c)))
    return _cfg_dict(c)


def launch_config(worlds: Sequence[World]) -> Dict:
    """The launch configuration the plan of these worlds runs with."""
    c = L.mc_launch_config()
    L.check(L.load().mc_launch_config_get(_handles(worlds), len(worlds), ctypes.byref(c)))
    return _cfg_dict(c)


def set_launch_config(worlds: Sequence[World], persistent: int = 0, pbd_warps: int = 8, scan_kernels: int = 0,
                      force_kernel: int = 0):
    """Pins the launch configuration of the plan of these worlds."""
    c = L.mc_launch_config(persistent=int(persistent), pbd_warps=int(pbd_warps), scan_kernels=int(scan_kernels),
                           force_kernel=int(force_kernel))
    L.check(L.load().mc_launch_config_set(_handles(worlds), len(worlds), ctypes.byref(c)))


def _result_dict(r: L.mc_result) -> Dict:
    return {"com_disp": (r.com_disp[0], r.com_disp[1]), "e_bend": r.e_bend, "e_pos": r.e_pos,
            "energy": r.energy, "status": r.status, "n_steps": r.n_steps,
            "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns}


class Server:
    """Continuous-batching rollout server (mc_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 16 << 30, max_slots: int = 4096, steps_per_tick: int = 10,
                 max_pending: int = 1 << 20):
        self._lib = L.load()
        cfg = L.mc_server_cfg(hbm_budget_bytes=int(hbm_budget_bytes), max_slots=int(max_slots),
                              steps_per_tick=int(steps_per_tick), max_pending=int(max_pending))
        h = ctypes.c_void_p()
        L.check(self._lib.mc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, spec: WorldSpec, n_steps: int) -> int:
        d, keep = make_desc(spec)
        t = ctypes.c_uint64()
        L.check(self._lib.mc_serve_submit(self._h, ctypes.byref(d), int(n_steps), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int) -> Optional[Dict]:
        r = L.mc_result()
        st = self._lib.mc_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == 6:   # MC_ERR_BUSY
            return None
        L.check(st)
        return _result_dict(r)

    def wait(self, ticket: int, timeout_ms: int = 600000) -> Dict:
        r = L.mc_result()
        L.check(self._lib.mc_serve_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r)))
        return _result_dict(r)

    def cancel(self, ticket: int) -> bool:
        """Cancels a queued or running rollout (its result then carries status
        MC_ERR_CANCELLED); False when the ticket is not queued or running."""
        st = self._lib.mc_serve_cancel(self._h, ctypes.c_uint64(ticket))
        if st == 7:   # MC_ERR_NOT_FOUND
            return False
        L.check(st)
        return True

    def stats(self) -> Dict:
        s = L.mc_server_stats()
        L.check(self._lib.mc_server_stats_get(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in L.mc_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.mc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

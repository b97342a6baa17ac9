"""Benchmark of the filament-fluid step on GB300.

One JSON line on rank 0.  Default workload: the particle-count sweep's target
point, 2^22 beads as 64-bead filaments on a 4096 x 4096 periodic grid (0.25
bead per cell), FP32.  A "step" is one full time step (drive, PBD, binning,
steric deposit, Gaussian filter, force + spread, LBM, interpolation and
advance) of that world.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference] [--no-cpu-baseline]

value      particle-steps/s of mc_step replaying its CUDA graph, inputs
           resident in HBM (the world's state, 1.8 GB, is larger than L2).
e2e        the same metric through the C ABI from host buffers: world
           creation from host arrays (H2D), K steps, state read-back (D2H).
roofline   k_force_lbm (filter y pass, steric force, spread and LBM of a
           tile; the dominant kernel): algorithmic bytes per launch (84 B per
           cell + 36 B per bead) / its CUDA-event duration, against the
           measured HBM copy bandwidth.  traffic: DRAM bytes per launch from
           one ncu capture of this workload, reported only while the kernel's
           sources are the ones that were captured (else null).
cpu_baseline  the FP64 oracle on the host cores, one step of a 1/16 sample
           of the workload (2^18 beads on 1024^2 at the same density).
With --impl reference the oracle itself is the timed arm.
"""
from __future__ import annotations

import argparse
import copy
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the stages one step runs, with their mc_step_stage ids (the scan stage is two kernels, one when every
# world fits one scan block)
STAGES = [("pbd", 0), ("bin_scan", 1), ("bin_scatter", 2), ("deposit_x", 3), ("force_lbm", 7), ("interp_advance", 6)]
KERNELS_PER_STEP = 7
GRAPH_STEPS = 16   # mc_step replays graphs of 16 steps: PBD, then 15 x (previous advance + PBD), 16 x (scan (2),
                   # scatter, deposit, force + LBM), and the last advance = 97 kernels


def mdf_launches(steps: int, m: int) -> int:
    """Kernels of direct-forcing steps (always the unfused sequence): PBD (returns), bins, scan (2),
    scatter, deposit, steric spread, moments, predicted PBD, m passes (one tile kernel each), LBM,
    advance."""
    return steps * (11 + m)


def scan_kernels(specs) -> int:
    """The bin-offset scan is one kernel when every world's bins fit one 1024-bin scan block, else two."""
    return 1 if all((sp.H // 8) * (sp.W // 8) <= 1024 for sp in specs) else 2


def graph_launches(steps: int, scans: int = 2) -> int:
    """Kernels of a run of `steps` steps: 16-step graphs, then the leftover r steps in the same fused
    order (r PBDs, r x (scan, scatter, deposit, force + LBM), one advance; one step alone runs the
    six stages)."""
    per = 4 + scans   # PBD, scan, scatter, deposit, force + LBM per step, plus the last advance
    r = steps % GRAPH_STEPS
    return (steps // GRAPH_STEPS) * (GRAPH_STEPS * per + 1) + (per * r + 1 if r else 0)
def run_launches(steps: int, cfg: dict, scans: int) -> int:
    """Kernels of a run of `steps` steps in a launch configuration: the persistent step is one cooperative
    launch per run; otherwise the graph sequence above (two scan kernels when the configuration asks)."""
    if cfg.get("persistent"):
        return 1
    return graph_launches(steps, 2 if cfg.get("scan_kernels") == 2 else scans)


# k_force_lbm, the dominant kernel: per cell read f 36 + rho_x 4, write f' 36 + u 8;
# per bead read the binned record (position 16, F_el 8, id 4), write F_s 8
FORCE_LBM_BYTES_PER_CELL = 84
FORCE_LBM_BYTES_PER_BEAD = 36
STEP_BYTES_PER_CELL = 112        # grid traffic per step of the minimal fused form
STEP_BYTES_PER_BEAD = 32

# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant
# kernel, from an ncu capture of the workload, keyed by the fingerprint of the
# sources the kernel is built from (reported only while they are unchanged)
KERNEL_TRAFFIC = {("c3_22", "4625ff6c212d33be"): 1626334592}
KERNEL_SOURCES = ["steric_dev.cuh", "k_steric.cu", "mc_internal.cuh"]


def kernel_fingerprint() -> str:
    """SHA-1 prefix of the dominant kernel's source files."""
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2607_02954_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="c3_22",
                    help="c3_<log2 N> (default c3_22), c1, c2, dense_<log2 N> (2^N beads on 256^2), "
                         "c4 (1024 worlds: batched vs per-world launches), "
                         "served (C4 worlds as Poisson-arriving 500-step rollouts) or c5 (folding gradient: "
                         "2000-step checkpointed rollout + loss + reverse sweep)")
    ap.add_argument("--pbd-order", type=int, default=0, choices=[0, 1],
                    help="PBD pass order of the stepped world: 0 Jacobi, 1 red-black")
    ap.add_argument("--loss", default="polyline", choices=["polyline", "splat"],
                    help="c5: folding loss, distance to a polyline or the paper's splatted-density MSE (128^2)")
    ap.add_argument("--mdf-iters", type=int, default=-1,
                    help="c3/c2 workloads: couple by direct forcing with this many MDF passes (default: penalty)")
    ap.add_argument("--observe", action="store_true",
                    help="step workloads: add a rest-length drive, an energy field and the observables")
    ap.add_argument("--arrival-rate", type=float, default=2000.0, help="served: requests per second")
    ap.add_argument("--duration", type=float, default=2.0, help="served: seconds of arrivals")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch configuration (no autotuning; profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the batched (c4) and served summaries of the default line")
    ap.add_argument("--stage-steps", type=int, default=50, help="steps of the per-stage timing pass")
    return ap.parse_args()


def make_spec(name: str, seed: int, pbd_order: int = 0, observe: bool = False, mdf_iters: int = -1):
    spec, desc = _make_spec(name, seed)
    if pbd_order:
        spec.params.pbd_order = pbd_order
        desc += ", red-black PBD passes"
    if mdf_iters >= 0:
        spec.params.ib = 1
        spec.params.mdf_iters = mdf_iters
        desc += f", direct forcing with {mdf_iters} MDF passes"
    if observe:
        from paper_2607_02954_gb300 import synth
        synth.with_observables(spec, seed)
        desc += ", rest-length drive + energy field + observables"
    return spec, desc


def _make_spec(name: str, seed: int):
    from paper_2607_02954_gb300 import synth
    if name == "c1":
        return synth.world_c1(seed), "c1: 128^2 grid, 16 x 32 beads, FP32"
    if name == "c2":
        return synth.world_c2(seed), "c2: 512^2 grid, 4096 x 64 beads (262,144), FP32"
    if name.startswith("c3_"):
        n = int(name.split("_")[1])
        side = synth.c3_side(n)
        return synth.world_c3(n, seed), f"c3: 2^{n} beads as 64-bead filaments on {side}^2, FP32"
    if name.startswith("dense_"):
        n = int(name.split("_")[1])
        return (dense_spec(n, seed),
                f"dense: 2^{n} beads as 64-bead filaments on 256^2 ({2 ** n / 65536:g} per cell; the paper's "
                "scalability shape; k_rep scaled by 0.25 / density), FP32")
    raise SystemExit(f"unknown workload {name}")


def dense_spec(n: int, seed: int):
    """2^n beads on 256^2 with the steric stiffness scaled by 0.25 / (beads
    per cell), so a bead feels the steric force it feels at the sweep's
    0.25 bead per cell (the default stiffness drives the flow past the
    velocity watchdog at several beads per cell)."""
    import dataclasses
    from paper_2607_02954_gb300 import synth
    spec = synth.world_dense(256, 2 ** n, seed)
    spec.params = dataclasses.replace(spec.params, k_rep=spec.params.k_rep * 0.25 / (2 ** n / 65536.0))
    return spec


def sample_spec(name: str, seed: int, params=None):
    """Bounded sample of the workload for the CPU oracle: same density and
    filament shape, 1/16 of the area for the big sweep points."""
    from paper_2607_02954_gb300 import synth
    if name.startswith("dense_"):
        n = int(name.split("_")[1])
        spec = dense_spec(n, seed)
        if params is not None:
            spec.params = params
        return spec, f"one oracle step of the full dense world (2^{n} beads on 256^2)"
    if name.startswith("c3_"):
        n = int(name.split("_")[1])
        side = synth.c3_side(n)
        density = (2 ** n) / float(side * side)
        s_side = max(256, side // 4)
        s_n = int(round(density * s_side * s_side))
        spec = synth.world_rows(s_side, s_n, seed)
        if params is not None:
            spec.params = params
        return spec, f"one oracle step of {s_n} beads on {s_side}^2 (same density)"
    spec, _ = make_spec(name, seed)
    if params is not None:
        spec.params = params
    return spec, f"one oracle step of the full {name} world"


def max_over_ranks(x: float, dist, device) -> float:
    """Largest x over the ranks of the process group (x itself without one)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, steps: int, seconds: float, world_size: int) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank advances its own world of the same size)."""
    return world_size * units_per_rank * steps / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_cores() -> int:
    """Logical CPU cores of this host (what nproc reports)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_sample(spec, min_seconds: float, max_steps: int = 1000, threads: int = 0):
    """Times oracle steps on the sample until min_seconds of CPU work, with
    `threads` intra-op threads (0: every host core)."""
    import torch
    import oracle as O
    old = torch.get_num_threads()
    torch.set_num_threads(threads or host_cores())
    try:
        ow = O.World(spec)
        st = ow.initial_state()
        t0 = time.perf_counter()
        n = 0
        while True:
            st, _ = O.step(ow, st)
            n += 1
            el = time.perf_counter() - t0
            if el >= min_seconds or n >= max_steps:
                break
        used = torch.get_num_threads()
    finally:
        torch.set_num_threads(old)
    return spec.N * n / el, n, el, used


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    spec, desc = sample_spec(args.workload, 1)
    import torch
    import oracle as O
    torch.set_num_threads(host_cores())
    ow = O.World(spec)
    st = ow.initial_state()
    for _ in range(args.warmup):
        st, _ = O.step(ow, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, _ = O.step(ow, st)
    el = time.perf_counter() - t0
    v = spec.N * args.steps / el
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": desc, "host_cores": host_cores()},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(args, steps=None):
    """1024 uneven worlds: batched steps (one launch per stage for all worlds,
    replayed from a CUDA graph) against two per-world arms: each world's own
    16-step graph replay (mc_step(w, 16), the strongest per-world path) and
    single direct steps (mc_step(w, 1), seven launches per world and step)."""
    import torch
    from paper_2607_02954_gb300 import World, step_batched, synth
    from paper_2607_02954_gb300 import launch_config, set_launch_config
    steps = steps or args.steps
    specs = synth.batch_c4(0)
    worlds = [World(sp) for sp in specs]
    n_beads = sum(sp.N for sp in specs)
    n_cells = sum(sp.H * sp.W for sp in specs)
    stream = torch.cuda.current_stream()
    step_batched(worlds, max(args.warmup, 16))   # the first run of 16 steps tunes the batch's plan
    torch.cuda.synchronize()
    tuned = launch_config(worlds)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        step_batched(worlds, steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    batched = n_beads * steps / (ms * 1e-3)
    # each launch configuration the tuner chose from, timed on the same worlds
    configs = {}
    for name, cfg in (("stage_graph", dict(persistent=0, pbd_warps=8, scan_kernels=0)),
                      ("persistent_4", dict(persistent=4, pbd_warps=8, scan_kernels=0)),
                      ("persistent_3", dict(persistent=3, pbd_warps=8, scan_kernels=0)),
                      ("stage_graph_pbd4", dict(persistent=0, pbd_warps=4, scan_kernels=0))):
        set_launch_config(worlds, **cfg)
        step_batched(worlds, 16)
        e0.record(stream)
        step_batched(worlds, 64)
        e1.record(stream)
        torch.cuda.synchronize()
        configs[name] = e0.elapsed_time(e1) / 64
    set_launch_config(worlds, **tuned)
    # per-world graph replays: one 16-step graph per world (captured in the warm-up)
    for w in worlds:
        w.step(16)
    torch.cuda.synchronize()
    e0.record(stream)
    for w in worlds:
        w.step(16)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    plain_graph = n_beads * 16 / (ms_graph * 1e-3)
    plain_steps = 3
    for w in worlds:
        w.step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(plain_steps):
        for w in worlds:
            w.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    plain = n_beads * plain_steps / (ms_plain * 1e-3)
    for w in worlds:
        w.check()
        w.close()
    return {"metric": "particle-steps/s", "value": batched, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4", "worlds": len(specs), "beads": n_beads, "cells": n_cells,
                       "description": "1024 worlds, side ~U{64,128,256}, 1-64 filaments x 8-64 beads (log-uniform)"},
            "plain_per_world_graph": {"value": plain_graph, "ms_per_step": ms_graph / 16,
                                      "description": "each world's own 16-step CUDA graph, replayed world after world"},
            "plain_per_world": {"value": plain, "ms_per_step": ms_plain / plain_steps,
                                "launches_per_step": len(worlds) * (KERNELS_PER_STEP - 2 + scan_kernels(specs)),
                                "description": "single direct steps, world after world"},
            "batched_over_plain_graph": batched / plain_graph, "batched_over_plain": batched / plain,
            "launch_config": tuned, "config_ms_per_step": configs,
            "gpu_launches": run_launches(steps, tuned, scan_kernels(specs)),
            "clocks": clk.summary()}


def stored_bytes_per_step(spec) -> int:
    """Step record of a stored rollout (include/mc.h): 32 N + 4 E + 56 H W
    bytes (+ 8 N with two layers), before 256-byte alignment."""
    return 32 * spec.N + 4 * spec.E + 56 * spec.H * spec.W


def bench_gradient(args):
    """Folding gradient (reverse mode, the Filament Folding experiment's
    loop): a 2000-step rollout of the folding world (256^2 grid, 64 x 48
    beads) recorded with checkpoints every 100 steps, the polyline loss, and
    the reverse sweep with the gradients with respect to theta0, L_rest and
    the three stiffnesses.  value = forward particle-steps per second of the
    whole gradient (forward + loss + backward)."""
    import numpy as np
    import torch
    from paper_2607_02954_gb300 import World, synth
    spec, poly = synth.world_c5(0)
    target = synth.target_image(np.random.default_rng(0), 128)
    loss_fn = (lambda w: w.loss_splat(target, 1.0)) if args.loss == "splat" else (lambda w: w.loss_polyline(poly))
    n, K = 2000, 100
    reps = max(1, min(args.steps, 5))
    w = World(spec)
    stream = torch.cuda.current_stream()
    # the optimisation loop of the Filament Folding experiment on one world:
    # new rest angles, back to the start, rollout, loss, reverse sweep (the
    # warm-up iteration captures the sweep's graph; the timed ones replay it)
    theta0 = spec.theta0.copy()
    w.rollout_forward(n, K)
    loss, gx, gy = loss_fn(w)
    w.rollout_backward_params(gx, gy)
    torch.cuda.synchronize()
    fwd, bwd = [], []
    with ClockSampler(0) as clk:
        for _ in range(reps):
            w.rollout_rewind()
            w.set_rest(theta0=theta0)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            w.rollout_forward(n, K)
            e[1].record(stream)
            loss, gx, gy = loss_fn(w)
            g = w.rollout_backward_params(gx, gy)
            e[2].record(stream)
            torch.cuda.synchronize()
            fwd.append(e[0].elapsed_time(e[1]))
            bwd.append(e[1].elapsed_time(e[2]))
            theta0 = theta0 - 1e-3 * t2n_host(g["theta0"]).astype(np.float32)   # a gradient step
    w.check()
    grad_norm = float(torch.linalg.vector_norm(g["theta0"]).item())
    g_ck = {k: t2n_host(v).copy() for k, v in g.items()}
    # the same loop with every step's record kept (mc_rollout_forward_stored:
    # the backward re-runs no step), from the same start
    theta0 = spec.theta0.copy()
    w.rollout_rewind()
    w.set_rest(theta0=theta0)
    w.rollout_forward(n, stored=True)
    loss, gx, gy = loss_fn(w)
    w.rollout_backward_params(gx, gy)
    torch.cuda.synchronize()
    fwd_s, bwd_s = [], []
    for _ in range(reps):
        w.rollout_rewind()
        w.set_rest(theta0=theta0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        w.rollout_forward(n, stored=True)
        e[1].record(stream)
        loss, gx, gy = loss_fn(w)
        g = w.rollout_backward_params(gx, gy)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwd_s.append(e[0].elapsed_time(e[1]))
        bwd_s.append(e[1].elapsed_time(e[2]))
        theta0 = theta0 - 1e-3 * t2n_host(g["theta0"]).astype(np.float32)
    w.check()
    same = all(np.array_equal(t2n_host(g[k]), g_ck[k]) for k in g_ck)
    w.close()
    ms_fs, ms_bs = statistics.median(fwd_s), statistics.median(bwd_s)
    ms_f, ms_b = statistics.median(fwd), statistics.median(bwd)
    value = spec.N * n / ((ms_f + ms_b) * 1e-3)
    line = {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": n, "warmup": 1, "ms_per_step": (ms_f + ms_b) / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c5", "grid": [spec.H, spec.W], "beads": spec.N, "filaments": spec.n_fil,
                       "rollout_steps": n, "ckpt_every": K, "repetitions": reps,
                       "loss": args.loss,
                       "description": f"folding gradient: checkpointed forward + {args.loss} loss + reverse sweep "
                                      "(theta0, L_rest, k_bend, k_stretch, k_shear)"},
            "forward_ms": ms_f, "backward_ms": ms_b, "backward_over_forward": ms_b / ms_f,
            "stored": {"forward_ms": ms_fs, "backward_ms": ms_bs, "backward_over_forward": ms_bs / ms_fs,
                       "value": spec.N * n / ((ms_fs + ms_bs) * 1e-3), "gradients_equal_checkpointed": same,
                       "tape_bytes_per_step": stored_bytes_per_step(spec)},
            "grad_norm_theta0": grad_norm, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        m = 200
        ow = O.World(spec)
        gxt = torch.as_tensor(t2n_host(gx), dtype=torch.float64)
        gyt = torch.as_tensor(t2n_host(gy), dtype=torch.float64)
        O.parameter_gradient(ow, m, gxt, gyt)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": spec.N * m / el, "unit": "particle-steps/s", "cores": torch.get_num_threads(),
                                "kind": "oracle", "sample": f"FP64 oracle reverse mode over {m} steps of the same world "
                                                            f"({el:.1f} s)"}
    return line


def t2n_host(t):
    return t.detach().cpu().numpy()


def bench_served(args):
    """Rollout requests for C4 worlds arriving as a Poisson process; each
    asks for a 500-step rollout and reads back the displacement."""
    import random
    from paper_2607_02954_gb300 import Server, synth
    # the search workload: every rollout returns its fitness inputs (mean
    # displacement, collected energy) and behaviour descriptors
    pool = [synth.with_observables(sp, k) for k, sp in enumerate(synth.batch_c4(1, n_worlds=256))]
    rng = random.Random(7)
    srv = Server(hbm_budget_bytes=64 << 30, max_slots=4096, steps_per_tick=10)
    # warm-up: a few rollouts to load kernels
    for t in [srv.submit(pool[k], 20) for k in range(8)]:
        srv.wait(t)
    n_req = int(args.arrival_rate * args.duration)
    times, t = [], 0.0
    for _ in range(n_req):
        t += rng.expovariate(args.arrival_rate)
        times.append(t)
    tickets, sizes = [], []
    with ClockSampler(0) as clk:
        start = time.perf_counter()
        for k, at in enumerate(times):
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            sp = pool[k % len(pool)]
            tickets.append(srv.submit(sp, 500))
            sizes.append(sp.N)
        res = [srv.wait(tk) for tk in tickets]
    bad = sum(1 for r in res if r["status"] != 0)
    lat = sorted((r["t_done_ns"] - r["t_submit_ns"]) * 1e-6 for r in res)
    span = (max(r["t_done_ns"] for r in res) - min(r["t_submit_ns"] for r in res)) * 1e-9
    stats = srv.stats()
    srv.close()
    value = sum(sizes) * 500 / span
    return {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": 500, "warmup": 8, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served", "requests": n_req, "arrival_rate_per_s": args.arrival_rate,
                       "rollout_steps": 500,
                       "pool": "256 C4 worlds with rest-length drive, energy field and observables"},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1]},
            "completed_per_s": n_req / span, "failed": bad, "server": stats, "clocks": clk.summary()}


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload in ("c4", "served", "c5"):
        import torch
        torch.cuda.set_device(0)
        from paper_2607_02954_gb300 import _lib
        if not os.path.exists(_lib.LIB_PATH):
            from paper_2607_02954_gb300.build import build
            build()
        if args.workload == "c4":
            line = bench_batched(args)
        elif args.workload == "c5":
            line = bench_gradient(args)
        else:
            line = bench_served(args)
        print(json.dumps(line), flush=True)
        return 0
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2607_02954_gb300 import World, _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2607_02954_gb300.build import build
        build()
    lib = _lib.load()
    if args.no_tune:
        _lib.check(lib.mc_autotune_mode(0))

    spec, desc = make_spec(args.workload, seed=rank, pbd_order=args.pbd_order, observe=args.observe,
                           mdf_iters=args.mdf_iters)
    mdf = args.mdf_iters >= 0
    N, C = spec.N, spec.H * spec.W
    world = World(spec, device=True)
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)

    # warm-up (includes the one-time tuning of the launch configuration and the graph capture)
    world.step(max(args.warmup, 16))
    torch.cuda.synchronize()
    from paper_2607_02954_gb300 import launch_config
    tuned = launch_config([world])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K steps replayed from the CUDA graph -------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        world.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    world.check()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(N, args.steps, ms_max * 1e-3, ws)

    # ---- per-stage CUDA-event timing on the launching stream ------------
    # (direct-forcing worlds have no per-stage entry: their step runs more kernels)
    n_stage = 0 if mdf else args.stage_steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(n_stage)]
    for k in range(n_stage):
        evs[k][0].record(stream)
        for s_i, (_, sid) in enumerate(STAGES):
            _lib.check(lib.mc_step_stage(world.handle, sid, sh))
            evs[k][s_i + 1].record(stream)
    torch.cuda.synchronize()
    stage_ms = {nm: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(n_stage)) / n_stage
                for i, (nm, _) in enumerate(STAGES)} if n_stage else None
    hbm_peak, peak_kind = measured_peaks()
    top_bytes = FORCE_LBM_BYTES_PER_CELL * C + FORCE_LBM_BYTES_PER_BEAD * N
    top_gbs = top_bytes / (stage_ms["force_lbm"] * 1e-3) / 1e9 if stage_ms else None
    step_bytes = STEP_BYTES_PER_CELL * C + STEP_BYTES_PER_BEAD * N
    step_gbs = step_bytes / (ms_max / args.steps * 1e-3) / 1e9
    world.close()

    # ---- end to end through the C ABI from pinned host buffers ----------
    e2e_steps = max(16, min(args.steps, 4000))   # the timed run's step count (bounded)
    in_keys = ("x", "y", "theta", "L_rest", "theta0", "drive_amp", "drive_freq", "drive_phase")
    pinned = copy.copy(spec)
    for k in in_keys:   # page-locked copies of the input arrays (numpy views of pinned tensors)
        a = np.ascontiguousarray(getattr(spec, k), dtype=np.float32)
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        setattr(pinned, k, t.numpy())
    h2d = sum(np.asarray(getattr(spec, k)).nbytes for k in in_keys + ("fil_off",))
    d2h = N * 4 * 4   # x, y, disp (2 floats)
    barrier()
    t0 = time.perf_counter()
    w2 = World(pinned)                    # pinned host arrays -> device
    w2.step(e2e_steps)
    st = w2.state()                       # device -> host (synchronizes)
    barrier()
    e2e_s = time.perf_counter() - t0
    w2.close()
    e2e_val = whole_job_rate(N, e2e_steps, max_over_ranks(e2e_s, dist, "cuda"), ws)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "grid": [spec.H, spec.W], "beads": N,
                   "filaments": spec.n_fil, "parallelism": f"replicas x{ws}" if ws > 1 else "single world",
                   "l2": "state 1.8 GB > L2: no flush needed" if C >= 4096 * 4096 else "state may fit in L2; per-step timing includes no flush"},
        "e2e": {"value": e2e_val, "unit": "particle-steps/s", "steps": e2e_steps,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps},
        "gpu_launches": (mdf_launches(args.steps, args.mdf_iters) - (2 - scan_kernels([spec])) * args.steps if mdf
                         else run_launches(args.steps, tuned, scan_kernels([spec]))),
        "launch_config": tuned,
        "roofline": None if mdf else {
            "bound": "hbm", "kernel": "k_force_lbm", "achieved": top_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": top_gbs / hbm_peak, "peak_kind": peak_kind,
            "traffic": KERNEL_TRAFFIC.get((args.workload, kernel_fingerprint())),
            "algorithmic_bytes_per_launch": top_bytes, "launch_ms": stage_ms["force_lbm"]},
        "step_roofline": {"achieved": step_gbs, "frac": step_gbs / hbm_peak, "unit": "GB/s",
                          "algorithmic_bytes_per_step": step_bytes},
        "stage_ms": stage_ms,
        "clocks": clk.summary(),
    }
    if mdf:
        line["step_roofline"]["note"] = "penalty-step bytes: a lower bound of the direct-forcing step's traffic"
    elif line["roofline"]["traffic"]:
        # the ncu-counted DRAM bytes of one launch over the same live launch time
        line["roofline"]["achieved_dram"] = line["roofline"]["traffic"] / (stage_ms["force_lbm"] * 1e-3) / 1e9
    if not args.no_extras and ws == 1:
        # the batched and served workloads (1024 uneven worlds), summarised
        # beside the headline; each is its own line with --workload c4 / served
        b = bench_batched(args, steps=max(64, min(args.steps, 512)))
        line["batched_c4"] = {"value": b["value"], "unit": "particle-steps/s", "ms_per_step": b["ms_per_step"],
                              "steps": b["steps"], "worlds": b["config"]["worlds"],
                              "launch_config": b["launch_config"], "config_ms_per_step": b["config_ms_per_step"],
                              "plain_per_world_graph": b["plain_per_world_graph"]["value"],
                              "plain_per_world": b["plain_per_world"]["value"],
                              "batched_over_plain_graph": b["batched_over_plain_graph"],
                              "batched_over_plain": b["batched_over_plain"]}
        sv = bench_served(args)
        line["served_c4"] = {"value": sv["value"], "unit": "particle-steps/s", "latency_ms": sv["latency_ms"],
                             "requests": sv["config"]["requests"],
                             "arrival_rate_per_s": sv["config"]["arrival_rate_per_s"],
                             "rollout_steps": sv["config"]["rollout_steps"],
                             "completed_per_s": sv["completed_per_s"], "failed": sv["failed"]}
    if not args.no_cpu_baseline and ws == 1:
        sspec, sdesc = sample_spec(args.workload, 1, params=spec.params)
        v, n, el, cores = run_oracle_sample(sspec, 10.0)
        v1, n1, el1, _ = run_oracle_sample(sspec, 5.0, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{sdesc}; {n} step(s) in {el:.1f} s on {cores} threads",
                                "host_cores": host_cores(),
                                "single_thread": {"value": v1, "unit": "particle-steps/s", "cores": 1,
                                                  "sample": f"{sdesc}; {n1} step(s) in {el1:.1f} s"}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Seeded synthetic worlds shaped like the paper's workloads.

This module draws inputs only: initial bead positions and edge angles, rest
lengths and rest angles, rest-angle drive parameters and the folding target.
It holds none of the method's arithmetic.  Both the FP64 oracle and the CUDA
path consume exactly the float32 arrays it returns, so both sides start from
bit-identical inputs.

World description (the paper's statement of the world, Methods section):
  * a 2D periodic grid of H x W cells (the fluid and steric fields);
  * filaments as linear bead chains: filament f owns beads
    fil_off[f] .. fil_off[f+1]-1; edge e joins beads (a, a+1) inside one
    filament and carries an orientation angle theta and a rest length L_rest;
    joint j sits between two consecutive edges of a filament and carries a
    rest angle theta_rest;
  * the rest angle of a joint is driven in time as
    theta_rest(t) = theta0 + amp * sin(2*pi*(freq*t + phase)),
    freq in cycles per step and phase in cycles (Experiments section: the
    worm and tadpole travelling waves, the ray's single beating angle).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Params:
    """Constants of one world.  The paper names these quantities but fixes
    none of their values; the defaults are the frozen reading used throughout.

    nu: kinematic viscosity (lattice units); tau_plus = 3*nu + 1/2.
    dt: bead advance time step (the lattice time step is 1).
    Lambda: TRT "magic" parameter; tau_minus = 1/2 + Lambda/(tau_plus - 1/2).
    kappa: penalty stiffness turning the PBD correction into a force.
    k_bend, k_stretch, k_shear: PBD stiffnesses of Eqs. 1-4.
    k_rep: steric repulsion strength.
    sigma: Gaussian filter width of the steric density (cells).
    orient: 1 = the position pass also turns the edge frame toward the edge
            vector (Gauss-Newton step on the Kirchhoff-Love error), 0 = the
            literal reading where only positions move.
    n_pbd: PBD iterations (bend pass + position pass) per time step.
    pbd_order: 0 Jacobi passes, 1 red-black (two-colour Gauss-Seidel) passes.
    layers: 1 = the beads are the immersed-boundary points; 2 = two-layer
            filament, points at X +- layer_half n (n the filament normal).
    ib: 0 = penalty coupling (kappa spreads the PBD correction as a force);
        1 = direct forcing: the fluid carries the nodes, PBD corrects them,
        and mdf_iters passes of multi-direct forcing make the fluid at the
        nodes follow the corrected motion (kappa unused).
    """

    nu: float = 0.1
    dt: float = 1.0
    Lambda: float = 0.25
    kappa: float = 0.05
    k_bend: float = 0.5
    k_stretch: float = 0.5
    k_shear: float = 0.25
    k_rep: float = 0.5
    sigma: float = 1.0
    orient: float = 1.0
    n_pbd: int = 4
    pbd_order: int = 0
    layers: int = 1
    layer_half: float = 0.5
    ib: int = 0
    mdf_iters: int = 0


@dataclasses.dataclass
class WorldSpec:
    H: int
    W: int
    fil_off: np.ndarray          # int32 [n_fil + 1] bead offsets
    x: np.ndarray                # float32 [N], in [0, W)
    y: np.ndarray                # float32 [N], in [0, H)
    theta: np.ndarray            # float32 [E] edge orientation angles (unwrapped)
    L_rest: np.ndarray           # float32 [E]
    theta0: np.ndarray           # float32 [J] static part of the rest angle
    drive_amp: np.ndarray        # float32 [J]
    drive_freq: np.ndarray       # float32 [J] cycles per step
    drive_phase: np.ndarray      # float32 [J] cycles
    params: Params = dataclasses.field(default_factory=Params)
    f0: Optional[np.ndarray] = None   # float32 [9, H, W]: populations minus rest weights
    t0: int = 0
    name: str = ""
    len_amp: Optional[np.ndarray] = None     # float32 [E] rest-length drive (all three or none)
    len_freq: Optional[np.ndarray] = None    # float32 [E] cycles per step
    len_phase: Optional[np.ndarray] = None   # float32 [E] cycles
    energy: Optional[np.ndarray] = None      # float32 [H, W] energy field
    observe: bool = False                    # accumulate the behaviour descriptors and collected energy

    @property
    def n_fil(self) -> int:
        return int(len(self.fil_off) - 1)

    @property
    def N(self) -> int:
        return int(self.fil_off[-1])

    @property
    def E(self) -> int:
        return int(len(self.theta))

    @property
    def J(self) -> int:
        return int(len(self.theta0))


def _f32_wrap(v: np.ndarray, period: int) -> np.ndarray:
    """Periodic placement of float64 coordinates, returned as float32 in [0, period)."""
    w = np.mod(v, period).astype(np.float32)
    w[w >= np.float32(period)] = np.float32(0.0)
    return w


def _counts(lengths) -> tuple:
    lengths = np.asarray(lengths, dtype=np.int64)
    fil_off = np.zeros(len(lengths) + 1, dtype=np.int32)
    fil_off[1:] = np.cumsum(lengths)
    E = int(np.sum(lengths - 1))
    J = int(np.sum(np.maximum(lengths - 2, 0)))
    return fil_off, E, J


def place_rejection(rng, H, W, lengths, min_dist=2.0, max_tries=2000, spacing=1.0):
    """Straight filaments at unit spacing from random non-overlapping starts.

    Each filament gets a random start and heading; it is rejected while any of
    its beads lies closer than min_dist (periodic distance) to a bead already
    placed.  Returns (x, y, theta) or None when a filament cannot be placed.
    """
    xs, ys, th = [], [], []
    placed = np.zeros((0, 2))
    for B in lengths:
        ok = False
        for _ in range(max_tries):
            x0, y0 = rng.uniform(0, W), rng.uniform(0, H)
            h = rng.uniform(0, TWO_PI)
            k = np.arange(B)
            px = x0 + spacing * k * math.cos(h)
            py = y0 + spacing * k * math.sin(h)
            if len(placed):
                dx = px[:, None] - placed[None, :, 0]
                dy = py[:, None] - placed[None, :, 1]
                dx -= W * np.round(dx / W)
                dy -= H * np.round(dy / H)
                if np.min(dx * dx + dy * dy) < min_dist * min_dist:
                    continue
            ok = True
            break
        if not ok:
            return None
        placed = np.concatenate([placed, np.stack([np.mod(px, W), np.mod(py, H)], 1)])
        xs.append(px)
        ys.append(py)
        th.append(np.full(B - 1, h))
    x = _f32_wrap(np.concatenate(xs), W)
    y = _f32_wrap(np.concatenate(ys), H)
    theta = np.concatenate(th).astype(np.float32) if th else np.zeros(0, np.float32)
    return x, y, theta


def place_rows(rng, H, W, n_fil, B, pitch, slot=64):
    """Jittered row lattice for dense worlds: horizontal filaments in slots of
    `slot` cells along rows `pitch` cells apart, each with a random direction
    (+x or -x) and a random sub-cell offset in [0, 0.5) on both axes."""
    assert B <= slot
    per_row = W // slot
    rows = int(round(H / pitch))
    assert per_row * rows >= n_fil, "world too small for the requested filaments"
    xs, ys, th = [], [], []
    for fidx in range(n_fil):
        r, s = divmod(fidx, per_row)
        ox, oy = rng.uniform(0, 0.5), rng.uniform(0, 0.5)
        k = np.arange(B, dtype=np.float64)
        flip = rng.integers(0, 2)
        if flip:
            px = s * slot + ox + (B - 1) - k
            h = math.pi
        else:
            px = s * slot + ox + k
            h = 0.0
        py = np.full(B, r * pitch + oy)
        xs.append(px)
        ys.append(py)
        th.append(np.full(B - 1, h))
    x = _f32_wrap(np.concatenate(xs), W)
    y = _f32_wrap(np.concatenate(ys), H)
    return x, y, np.concatenate(th).astype(np.float32)


def _world(name, H, W, lengths, x, y, theta, theta0, amp, freq, phase, params=None, f0=None, t0=0):
    fil_off, E, J = _counts(lengths)
    assert len(x) == fil_off[-1] and len(theta) == E and len(theta0) == J
    return WorldSpec(H=H, W=W, fil_off=fil_off, x=x, y=y, theta=theta,
                     L_rest=np.ones(E, np.float32), theta0=theta0.astype(np.float32),
                     drive_amp=np.asarray(amp, np.float32), drive_freq=np.asarray(freq, np.float32),
                     drive_phase=np.asarray(phase, np.float32), params=params or Params(),
                     f0=f0, t0=t0, name=name)


def _per_joint(lengths, per_fil_values):
    """Expand one value per filament to one value per joint."""
    out = [np.full(max(B - 2, 0), v) for B, v in zip(lengths, per_fil_values)]
    return np.concatenate(out) if out else np.zeros(0)


def _joint_local_index(lengths):
    out = [np.arange(max(B - 2, 0)) for B in lengths]
    return np.concatenate(out) if out else np.zeros(0)


def world_c1(seed=0):
    """128x128 periodic grid, 16 filaments x 32 beads from non-overlapping
    random starts, rest angle per joint ~U[-0.3, 0.3], sinusoidal drive of
    amplitude 0.2 rad and period 200 steps with a random phase per filament."""
    rng = np.random.default_rng(seed)
    H = W = 128
    lengths = [32] * 16
    placed = place_rejection(rng, H, W, lengths)
    assert placed is not None
    x, y, theta = placed
    _, E, J = _counts(lengths)
    theta0 = rng.uniform(-0.3, 0.3, J)
    phase = _per_joint(lengths, rng.uniform(0, 1, len(lengths)))
    return _world("c1", H, W, lengths, x, y, theta, theta0,
                  np.full(J, 0.2), np.full(J, 1.0 / 200.0), phase)


def _travelling_wave(rng, lengths, amp=0.3, period=200.0, wavelength=16.0):
    J = int(sum(max(B - 2, 0) for B in lengths))
    phase_f = _per_joint(lengths, rng.uniform(0, 1, len(lengths)))
    phase = np.mod(phase_f - _joint_local_index(lengths) / wavelength, 1.0)
    return np.full(J, amp), np.full(J, 1.0 / period), phase


def world_rows(side, n_beads, seed=0, B=64, name=None):
    """Dense world of filaments of B beads on a jittered row lattice.

    Rest angles ~N(0, 0.1) plus a travelling-wave drive of amplitude 0.3 rad,
    wavelength 16 beads and period 200 steps (the period is not given by the
    workload description; 200 steps matches the other sinusoidal drives)."""
    rng = np.random.default_rng(seed)
    n_fil = n_beads // B
    assert n_fil * B == n_beads
    pitch = (side * side) // n_beads
    assert pitch >= 1 and side % pitch == 0
    lengths = [B] * n_fil
    x, y, theta = place_rows(rng, side, side, n_fil, B, pitch)
    _, E, J = _counts(lengths)
    theta0 = rng.normal(0.0, 0.1, J)
    amp, freq, phase = _travelling_wave(rng, lengths)
    return _world(name or f"rows_{side}_{n_beads}", side, side, lengths, x, y, theta,
                  theta0, amp, freq, phase)


def world_dense(side, n_beads, seed=0, B=64, name=None):
    """World denser than one bead per cell (the paper's scalability runs keep
    a 256^2 grid and go up to 500k particles, about 7.6 beads per cell):
    filaments of B beads on a jittered row lattice whose rows are
    side^2 / n_beads cells apart (below one cell, so rows interleave within a
    cell), rest angles ~N(0, 0.1) and the same travelling-wave drive as
    world_rows."""
    rng = np.random.default_rng(seed)
    n_fil = n_beads // B
    assert n_fil * B == n_beads and side % 64 == 0
    pitch = (side * side) / float(n_beads)
    lengths = [B] * n_fil
    x, y, theta = place_rows(rng, side, side, n_fil, B, pitch)
    _, E, J = _counts(lengths)
    theta0 = rng.normal(0.0, 0.1, J)
    amp, freq, phase = _travelling_wave(rng, lengths)
    return _world(name or f"dense_{side}_{n_beads}", side, side, lengths, x, y, theta,
                  theta0, amp, freq, phase)


def world_c2(seed=0):
    """512x512 grid, 4096 filaments x 64 beads (262,144 particles)."""
    return world_rows(512, 262144, seed, name="c2")


def c3_side(log2n: int) -> int:
    """Grid side of the particle-count sweep: 0.25 bead per cell where the
    side is a power of two up to 4096 (2^14 @ 256^2 ... 2^22 @ 4096^2), lower
    density for odd exponents, and 4096^2 beyond 2^22 (2^24 is 1 bead/cell)."""
    return min(4096, 2 ** int(math.ceil((log2n + 2) / 2)))


def world_c3(log2n: int, seed=0):
    """Particle-count sweep point: 2^log2n beads as 64-bead filaments."""
    side = c3_side(log2n)
    return world_rows(side, 2 ** log2n, seed, name=f"c3_2^{log2n}@{side}^2")


def world_c5(seed=0):
    """Differentiable folding world: 256x256 grid, 64 filaments x 48 beads,
    static rest angles (no drive), plus a seeded 16-vertex target polyline."""
    rng = np.random.default_rng(seed)
    H = W = 256
    lengths = [48] * 64
    placed = place_rejection(rng, H, W, lengths)
    assert placed is not None
    x, y, theta = placed
    _, E, J = _counts(lengths)
    theta0 = rng.uniform(-0.3, 0.3, J)
    w = _world("c5", H, W, lengths, x, y, theta, theta0,
               np.zeros(J), np.zeros(J), np.zeros(J))
    return w, target_polyline(rng, H, W)


def target_polyline(rng, H, W, n_vertices=16):
    """Seeded random target polyline, vertices uniform over the domain."""
    return np.stack([rng.uniform(0, W, n_vertices), rng.uniform(0, H, n_vertices)], 1).astype(np.float32)


def world_random(seed, side, n_fil, lengths=None, b_min=8, b_max=64, name=None, params=None,
                 amp_max=0.3, period=(50.0, 400.0)):
    """One world of the batched/served workload (side: int or (H, W)): log-uniform bead counts, per
    joint drive amplitude ~U[0, amp_max], period ~U[period] steps and phase
    ~U[0, 1) cycles.  Filaments are placed by rejection sampling, or on a
    jittered lattice when the world is too crowded for it."""
    rng = np.random.default_rng(seed)
    H, W = (side, side) if np.isscalar(side) else (int(side[0]), int(side[1]))
    if lengths is None:
        lengths = [int(round(math.exp(rng.uniform(math.log(b_min), math.log(b_max))))) for _ in range(n_fil)]
    lengths = [max(2, int(B)) for B in lengths]
    placed = None
    if sum(lengths) * 8 <= H * W:
        placed = place_rejection(rng, H, W, lengths, max_tries=200)
    if placed is None:
        placed = _place_dense(rng, H, W, lengths)
    x, y, theta = placed
    _, E, J = _counts(lengths)
    theta0 = rng.uniform(-0.3, 0.3, J)
    amp = rng.uniform(0, amp_max, J)
    freq = 1.0 / rng.uniform(period[0], period[1], J)
    phase = rng.uniform(0, 1, J)
    return _world(name or f"rand_{seed}", H, W, lengths, x, y, theta, theta0,
                  amp, freq, phase, params=params)


def _place_dense(rng, H, W, lengths):
    """Row placement for crowded worlds: filaments laid head to tail along rows."""
    xs, ys, th = [], [], []
    pos_x, row = 0.0, 0
    rows = []
    for B in lengths:
        if pos_x + B > W:
            row += 1
            pos_x = 0.0
        rows.append((row, pos_x))
        pos_x += B
    n_rows = row + 1
    assert n_rows <= H, "world too crowded"
    pitch = H // n_rows
    for B, (r, x0) in zip(lengths, rows):
        ox, oy = rng.uniform(0, 0.5), rng.uniform(0, 0.5)
        k = np.arange(B, dtype=np.float64)
        xs.append(x0 + ox + k)
        ys.append(np.full(B, r * pitch + oy))
        th.append(np.zeros(B - 1))
    return _f32_wrap(np.concatenate(xs), W), _f32_wrap(np.concatenate(ys), H), \
        np.concatenate(th).astype(np.float32)


def batch_c4(seed=0, n_worlds=1024):
    """The batched / served workload: n_worlds independent worlds with grid
    side ~U{64, 128, 256}, 1..64 filaments (log-uniform) of 8..64 beads
    (log-uniform) each."""
    rng = np.random.default_rng(seed)
    worlds = []
    for w in range(n_worlds):
        side = int(rng.choice([64, 128, 256]))
        n_fil = int(round(math.exp(rng.uniform(0.0, math.log(64)))))
        worlds.append(world_random(int(rng.integers(0, 2 ** 31)), side, max(1, n_fil), name=f"c4_{w}"))
    return worlds


def random_populations(rng, H, W, scale=1e-3):
    """Random population deviations (fluid state minus rest weights) for
    per-kernel parity tests."""
    return (scale * rng.standard_normal((9, H, W))).astype(np.float32)


def tiny_world(seed=0, side=16, lengths=(6, 5), params=None, amp=0.1):
    """A few short filaments on a small grid for brute-force checks."""
    rng = np.random.default_rng(seed)
    lengths = list(lengths)
    placed = place_rejection(rng, side, side, lengths, min_dist=1.5)
    assert placed is not None
    x, y, theta = placed
    _, E, J = _counts(lengths)
    theta0 = rng.uniform(-0.3, 0.3, J)
    return _world(f"tiny_{seed}", side, side, lengths, x, y, theta, theta0,
                  np.full(J, amp), np.full(J, 1.0 / 50.0), rng.uniform(0, 1, J), params=params)


def energy_packets(rng, H, W, n_packets=8, amp=(0.2, 1.0), width=(2.0, 8.0)) -> np.ndarray:
    """A persistent energy field of Gaussian packets at random positions
    (Neuroevolution experiment's chemotaxis target): the sum over packets of
    a_k exp(-|x - c_k|^2 / (2 s_k^2)) at the cell centres, periodic distance;
    a_k ~ U[amp], s_k ~ U[width].  float32 [H, W]."""
    ys, xs = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    field = np.zeros((H, W))
    for _ in range(n_packets):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        a, s = rng.uniform(*amp), rng.uniform(*width)
        dx = xs - cx
        dx -= W * np.round(dx / W)
        dy = ys - cy
        dy -= H * np.round(dy / H)
        field += a * np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
    return field.astype(np.float32)


def with_observables(spec: WorldSpec, seed: int, len_amp_max=0.2, period=(50.0, 400.0), n_packets=8) -> WorldSpec:
    """Adds what the search experiments read: a rest-length drive per edge
    (the controller's rest-length output; amplitude ~U[0, len_amp_max],
    period ~U[period] steps, phase ~U[0, 1) cycles), an energy field of
    Gaussian packets, and observe = True.  Returns spec (modified)."""
    rng = np.random.default_rng(seed + 7919)
    E = spec.E
    spec.len_amp = rng.uniform(0.0, len_amp_max, E).astype(np.float32)
    spec.len_freq = (1.0 / rng.uniform(*period, E)).astype(np.float32)
    spec.len_phase = rng.uniform(0.0, 1.0, E).astype(np.float32)
    spec.energy = energy_packets(rng, spec.H, spec.W, n_packets)
    spec.observe = True
    return spec


def target_image(rng, R=128, n_strokes=3, width=2.5) -> np.ndarray:
    """Seeded stand-in for a handwritten digit (the folding target): a few
    smooth strokes, each a quadratic Bezier curve between random points in
    the central part of an R x R image, drawn with a Gaussian profile of the
    given width in pixels; values in [0, 1].  float32 [R, R]."""
    ys, xs = np.meshgrid(np.arange(R) + 0.5, np.arange(R) + 0.5, indexing="ij")
    img = np.zeros((R, R))
    for _ in range(n_strokes):
        P = rng.uniform(0.25 * R, 0.75 * R, (3, 2))
        for t in np.linspace(0.0, 1.0, 4 * R):
            c = (1 - t) ** 2 * P[0] + 2 * (1 - t) * t * P[1] + t ** 2 * P[2]
            img = np.maximum(img, np.exp(-((xs - c[0]) ** 2 + (ys - c[1]) ** 2) / (2.0 * width ** 2)))
    return img.astype(np.float32)

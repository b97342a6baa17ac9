"""Plain FP64 oracle of one Microcosmos time step, written from the paper.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Every function below follows one passage of the paper (arXiv 2607.02954) or,
where the paper names a textbook method without its formulas, that method's
standard definition.  The paper fixes no numeric constant; the reading used
for each silent or ambiguous point is listed in the project's design notes
and repeated in the docstrings here.

Conventions (lattice units): cell centres at integer coordinates, dx = 1,
lattice time step 1, periodic in x and y.  Grids are indexed [y, x].

One step n, from state (X^n, theta^n, f^n):
  a1  rest-angle drive            theta_rest(n)
  a3  PBD (Methods, Eqs. 1-4)     (x_hat, theta_hat); F_el = kappa (x_hat - X)/dt
  a4  steric deposit (Fields)     rho_s(c) = sum_i delta_h(c - X_i)
  a5  Gaussian filter + gradient  rho_bar = G * rho_s;  grad rho_bar
  a6  steric force + IB spread    F_s,i = -k_rep sum_c delta_h grad rho_bar
                                  F(c) = sum_i delta_h(c - X_i) (F_el,i + F_s,i)
  a7  D2Q9 TRT LBM with forcing   f^{n+1}, u^n
  a8  IB interpolation + advance  U_i = sum_c delta_h u^n;  X^{n+1} = wrap(X + dt U)
"""
from __future__ import annotations

import math
import copy
import dataclasses
from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np
import torch

F64 = torch.float64

# ---------------------------------------------------------------------------
# D2Q9 lattice (Qian et al. 1992, cited for the fluid field in the Fields
# section): velocities c_i, weights w_i and the opposite direction of each.
# ---------------------------------------------------------------------------
D2Q9_C = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))
D2Q9_W = (4.0 / 9.0,) + (1.0 / 9.0,) * 4 + (1.0 / 36.0,) * 4
D2Q9_OPP = (0, 3, 4, 1, 2, 7, 8, 5, 6)


def d2q9_weights() -> torch.Tensor:
    return torch.tensor(D2Q9_W, dtype=F64)


# ---------------------------------------------------------------------------
# Topology of linear filaments (Methods, Filaments: graph of nodes and edges;
# linear chains only).  Edge e joins beads (a, a+1) of one filament; joint j
# joins edges (e, e+1) of one filament.
# ---------------------------------------------------------------------------
@dataclass
class Topology:
    N: int
    edge_a: torch.Tensor   # [E] bead index of x_1
    edge_b: torch.Tensor   # [E] bead index of x_2
    joint_e1: torch.Tensor  # [J] edge index of theta_1
    joint_e2: torch.Tensor  # [J] edge index of theta_2
    edge_color: torch.Tensor = None   # [E] parity of the edge's index within its filament
    joint_color: torch.Tensor = None  # [J] parity of the joint's index within its filament


def topology(fil_off) -> Topology:
    fil_off = [int(v) for v in fil_off]
    ea, eb, j1, j2, ec, jc = [], [], [], [], [], []
    e = 0
    for f in range(len(fil_off) - 1):
        b0, b1 = fil_off[f], fil_off[f + 1]
        n_e = b1 - b0 - 1
        for k in range(n_e):
            ea.append(b0 + k)
            eb.append(b0 + k + 1)
            ec.append(k % 2)
        for k in range(n_e - 1):
            j1.append(e + k)
            j2.append(e + k + 1)
            jc.append(k % 2)
        e += max(n_e, 0)
    as_t = lambda v: torch.tensor(v, dtype=torch.long)
    return Topology(fil_off[-1], as_t(ea), as_t(eb), as_t(j1), as_t(j2), as_t(ec), as_t(jc))


# ---------------------------------------------------------------------------
# Constants of the reading (the paper gives none).
# ---------------------------------------------------------------------------
@dataclass
class Consts:
    nu: float
    dt: float
    Lambda: float
    kappa: float
    k_bend: float
    k_stretch: float
    k_shear: float
    k_rep: float
    sigma: float
    orient: float
    n_pbd: int
    pbd_order: int = 0   # 0: Jacobi passes; 1: red-black (two-colour Gauss-Seidel) passes
    layers: int = 1      # 1: beads are the immersed-boundary points; 2: two-layer filament
    layer_half: float = 0.5   # half distance between the two layers (cells)
    ib: int = 0          # 0: penalty coupling (F_el spread); 1: direct forcing with MDF passes
    mdf_iters: int = 0   # multi-direct-forcing passes per step (ib = 1)

    @property
    def tau_plus(self) -> float:
        # LBM viscosity set by one relaxation time (Fields): nu = (tau - 1/2)/3.
        return 3.0 * self.nu + 0.5

    @property
    def tau_minus(self) -> float:
        # TRT (Ginzburg 2008): Lambda = (tau+ - 1/2)(tau- - 1/2).
        return 0.5 + self.Lambda / (self.tau_plus - 0.5)


def consts(params) -> Consts:
    """Read the constants from any object with the Params attribute names, in
    double precision after rounding each to float32 (the value the GPU sees)."""
    r = lambda v: float(np.float32(v))
    return Consts(nu=r(params.nu), dt=r(params.dt), Lambda=r(params.Lambda), kappa=r(params.kappa),
                  k_bend=r(params.k_bend), k_stretch=r(params.k_stretch), k_shear=r(params.k_shear),
                  k_rep=r(params.k_rep), sigma=r(params.sigma), orient=r(params.orient),
                  n_pbd=int(params.n_pbd), pbd_order=int(getattr(params, "pbd_order", 0)),
                  layers=int(getattr(params, "layers", 1)), layer_half=r(getattr(params, "layer_half", 0.5)),
                  ib=int(getattr(params, "ib", 0)), mdf_iters=int(getattr(params, "mdf_iters", 0)))


# ---------------------------------------------------------------------------
# a1: rest-angle drive (Experiments: sinusoidal wave of the worm and tadpole,
# single time-dependent angle of the ray).
# ---------------------------------------------------------------------------
def rest_angles(theta0, amp, freq, phase, n: int) -> torch.Tensor:
    """theta_rest,j(n) = theta0_j + A_j sin(2 pi (freq_j n + phase_j))."""
    return theta0 + amp * torch.sin(2.0 * math.pi * (freq * float(n) + phase))


# ---------------------------------------------------------------------------
# Periodic helpers.
# ---------------------------------------------------------------------------
def min_image(d: torch.Tensor, period: float) -> torch.Tensor:
    """Shortest periodic representative of a difference: d - P round(d / P)."""
    return d - period * torch.round(d / period)


def wrap(X: torch.Tensor, period: float) -> torch.Tensor:
    """X - P floor(X / P), mapped into [0, P)."""
    w = X - period * torch.floor(X / period)
    return torch.where(w >= period, w - period, w)


# ---------------------------------------------------------------------------
# a3: Position-Based Dynamics (Methods: Bending Pass Eq. 1, Position Pass
# Eqs. 2-4), Jacobi form: every correction of one pass is computed from the
# state before the pass and all are applied together.
# ---------------------------------------------------------------------------
def bend_pass(theta, theta_rest, topo: Topology, k_bend: float, color: Optional[int] = None):
    """Eq. 1: C = (theta_2 - theta_1) - theta_rest per joint;
    theta_1 += k C / 2, theta_2 -= k C / 2.  With color = 0 or 1 only the
    joints of that index parity within their filament are corrected (they
    share no edge)."""
    if topo.joint_e1.numel() == 0:
        return theta
    C = theta[topo.joint_e2] - theta[topo.joint_e1] - theta_rest
    if color is not None:
        C = torch.where(topo.joint_color == color, C, torch.zeros_like(C))
    dtheta = torch.zeros_like(theta)
    dtheta = dtheta.index_add(0, topo.joint_e1, 0.5 * k_bend * C)
    dtheta = dtheta.index_add(0, topo.joint_e2, -0.5 * k_bend * C)
    return theta + dtheta


def position_pass(x, theta, L_rest, topo: Topology, c: Consts, H: int, W: int, color: Optional[int] = None):
    """Eqs. 2-4 per edge with v = x_2 - x_1 (minimum image), d = (cos, sin)(theta):
        C_stretch = (|v| - L) v/|v|
        dx = k_stretch/2 [C_stretch + k_shear (v - L d - C_stretch)]
        x_1 += dx, x_2 -= dx.
    With orient = 1 the edge frame also turns toward v by the Gauss-Newton
    step of the Kirchhoff-Love error |v - L d(theta)|^2 scaled like Eq. 3:
        theta += orient * k_stretch k_shear / 2 * (d_perp . v) / L.
    With color = 0 or 1 only the edges of that index parity within their
    filament are corrected (they share no bead)."""
    if topo.edge_a.numel() == 0:
        return x, theta
    xa, xb = x[topo.edge_a], x[topo.edge_b]
    vx = min_image(xb[:, 0] - xa[:, 0], W)
    vy = min_image(xb[:, 1] - xa[:, 1], H)
    ell = torch.sqrt(vx * vx + vy * vy)
    csx = (ell - L_rest) * vx / ell
    csy = (ell - L_rest) * vy / ell
    dcos, dsin = torch.cos(theta), torch.sin(theta)
    dx = 0.5 * c.k_stretch * (csx + c.k_shear * (vx - L_rest * dcos - csx))
    dy = 0.5 * c.k_stretch * (csy + c.k_shear * (vy - L_rest * dsin - csy))
    delta = torch.zeros_like(x)
    d = torch.stack([dx, dy], 1)
    dtheta = c.orient * 0.5 * c.k_stretch * c.k_shear * (-dsin * vx + dcos * vy) / L_rest
    if color is not None:
        on = topo.edge_color == color
        d = torch.where(on[:, None], d, torch.zeros_like(d))
        dtheta = torch.where(on, dtheta, torch.zeros_like(dtheta))
    delta = delta.index_add(0, topo.edge_a, d)
    delta = delta.index_add(0, topo.edge_b, -d)
    return x + delta, theta + dtheta


def pbd(X, theta, theta_rest, L_rest, topo: Topology, c: Consts, H: int, W: int):
    """n_pbd iterations of (bending pass, position pass) from (X, theta)
    (Methods: "Each iteration decouples the solver into two phases").
    pbd_order 0: Jacobi passes (every correction of a pass from the state
    before it); 1: red-black passes (even-indexed joints or edges first, the
    odd ones from the updated state: a two-colour Gauss-Seidel sweep)."""
    x, th = X, theta
    for _ in range(c.n_pbd):
        if c.pbd_order == 1:
            th = bend_pass(th, theta_rest, topo, c.k_bend, color=0)
            th = bend_pass(th, theta_rest, topo, c.k_bend, color=1)
            x, th = position_pass(x, th, L_rest, topo, c, H, W, color=0)
            x, th = position_pass(x, th, L_rest, topo, c, H, W, color=1)
        else:
            th = bend_pass(th, theta_rest, topo, c.k_bend)
            x, th = position_pass(x, th, L_rest, topo, c, H, W)
    return x, th


# ---------------------------------------------------------------------------
# Diffuse interface (Fluid-filament Interaction: IBM of Peskin 2002, smoothing
# over a small neighbourhood).  Reading: Peskin's 4-point kernel, used for the
# steric deposit, the force spread and the velocity interpolation alike.
# ---------------------------------------------------------------------------
def peskin_phi(r: torch.Tensor) -> torch.Tensor:
    """phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8      for |r| <= 1
              = (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8     for 1 <= |r| <= 2
              = 0                                          otherwise."""
    a = r.abs()
    a_in = a.clamp(max=1.0)
    a_out = a.clamp(min=1.0, max=2.0)
    inner = (3.0 - 2.0 * a_in + torch.sqrt(1.0 + 4.0 * a_in - 4.0 * a_in * a_in)) / 8.0
    outer = (5.0 - 2.0 * a_out - torch.sqrt(-7.0 + 12.0 * a_out - 4.0 * a_out * a_out)) / 8.0
    return torch.where(a <= 1.0, inner, torch.where(a <= 2.0, outer, torch.zeros_like(a)))


def stencil(X: torch.Tensor, H: int, W: int):
    """The 4x4 cells around each bead: base b = floor(X) - 1, cells b..b+3 on
    each axis (wrapped), weight delta_h(c - X) = phi(c_x - X_x) phi(c_y - X_y).
    Returns flat cell indices [N, 16] and weights [N, 16]."""
    N = X.shape[0]
    offs = torch.arange(4, dtype=F64)
    bx = torch.floor(X[:, 0]).detach() - 1.0
    by = torch.floor(X[:, 1]).detach() - 1.0
    cx = bx[:, None] + offs[None, :]            # [N, 4]
    cy = by[:, None] + offs[None, :]
    wx = peskin_phi(cx - X[:, 0:1])
    wy = peskin_phi(cy - X[:, 1:2])
    ix = torch.remainder(cx.long(), W)
    iy = torch.remainder(cy.long(), H)
    idx = (iy[:, :, None] * W + ix[:, None, :]).reshape(N, 16)   # [N, 4(y), 4(x)]
    w = (wy[:, :, None] * wx[:, None, :]).reshape(N, 16)
    return idx, w


def spread(idx, w, values, H: int, W: int) -> torch.Tensor:
    """P2G: grid(c) = sum_i delta_h(c - X_i) values_i.  values [N] or [N, k]."""
    if values.dim() == 1:
        out = torch.zeros(H * W, dtype=F64)
        out = out.index_add(0, idx.reshape(-1), (w * values[:, None]).reshape(-1))
        return out.reshape(H, W)
    chans = [spread(idx, w, values[:, k], H, W) for k in range(values.shape[1])]
    return torch.stack(chans, 0)


def interpolate(idx, w, grid: torch.Tensor) -> torch.Tensor:
    """G2P: value_i = sum_c delta_h(c - X_i) grid(c).  grid [H,W] or [k,H,W]."""
    if grid.dim() == 2:
        return (w * grid.reshape(-1)[idx]).sum(1)
    return torch.stack([interpolate(idx, w, grid[k]) for k in range(grid.shape[0])], 1)


# ---------------------------------------------------------------------------
# a4-a6: steric repulsion field (Fields: positions deposited onto a grid,
# Gaussian filter, gradient gives the repulsive force).
# Reading of "Gaussian filter via FFT convolution": the sampled, normalised
# Gaussian truncated at R = ceil(4 sigma), applied as a periodic circular
# convolution along x then y (an FFT circular convolution with the same taps
# gives the same values up to rounding).
# ---------------------------------------------------------------------------
def gaussian_taps(sigma: float):
    R = int(math.ceil(4.0 * sigma))
    m = torch.arange(-R, R + 1, dtype=F64)
    g = torch.exp(-m * m / (2.0 * sigma * sigma))
    return R, g / g.sum()


def gaussian_blur(rho: torch.Tensor, sigma: float) -> torch.Tensor:
    """rho_bar(c) = sum_m g_m rho(c - m e_x), then the same along y (periodic)."""
    R, g = gaussian_taps(sigma)
    tmp = sum(g[k] * torch.roll(rho, shifts=k - R, dims=1) for k in range(2 * R + 1))
    return sum(g[k] * torch.roll(tmp, shifts=k - R, dims=0) for k in range(2 * R + 1))


def central_gradient(rho: torch.Tensor) -> torch.Tensor:
    """(d/dx, d/dy) by central differences on the periodic grid: [2, H, W]."""
    gx = 0.5 * (torch.roll(rho, shifts=-1, dims=1) - torch.roll(rho, shifts=1, dims=1))
    gy = 0.5 * (torch.roll(rho, shifts=-1, dims=0) - torch.roll(rho, shifts=1, dims=0))
    return torch.stack([gx, gy], 0)


# ---------------------------------------------------------------------------
# a7: D2Q9 lattice Boltzmann (Fields) with two-relaxation-time collision
# (TRT, Ginzburg 2008, cited in Fluid-filament Interaction) and the body force
# of the immersed boundary entering through Guo's forcing (the paper names no
# forcing scheme; Guo's, with the half-force velocity, is the reading).
# ---------------------------------------------------------------------------
def equilibrium(rho, ux, uy) -> torch.Tensor:
    """f_i^eq = w_i rho (1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u)."""
    uu = ux * ux + uy * uy
    out = []
    for (cx, cy), w in zip(D2Q9_C, D2Q9_W):
        cu = cx * ux + cy * uy
        out.append(w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu))
    return torch.stack(out, 0)


def guo_source(ux, uy, Fx, Fy) -> torch.Tensor:
    """S_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F."""
    out = []
    for (cx, cy), w in zip(D2Q9_C, D2Q9_W):
        cu = cx * ux + cy * uy
        out.append(w * (3.0 * ((cx - ux) * Fx + (cy - uy) * Fy) + 9.0 * cu * (cx * Fx + cy * Fy)))
    return torch.stack(out, 0)


def macroscopic(f, F):
    """rho = sum_i f_i; u = (sum_i c_i f_i + F/2) / rho."""
    rho = f.sum(0)
    mx = sum(cx * f[i] for i, (cx, cy) in enumerate(D2Q9_C)) + 0.5 * F[0]
    my = sum(cy * f[i] for i, (cx, cy) in enumerate(D2Q9_C)) + 0.5 * F[1]
    return rho, mx / rho, my / rho


def trt_collide(f, F, tau_p: float, tau_m: float):
    """TRT with source: with symmetric/antisymmetric parts
    g^(+/-)_i = (g_i +/- g_opp(i))/2,
    f*_i = f_i - (f+_i - feq+_i)/tau+ - (f-_i - feq-_i)/tau-
           + (1 - 1/(2 tau+)) S+_i + (1 - 1/(2 tau-)) S-_i.
    Returns (f*, ux, uy)."""
    rho, ux, uy = macroscopic(f, F)
    feq = equilibrium(rho, ux, uy)
    S = guo_source(ux, uy, F[0], F[1])
    opp = list(D2Q9_OPP)
    fp, fm = 0.5 * (f + f[opp]), 0.5 * (f - f[opp])
    ep, em = 0.5 * (feq + feq[opp]), 0.5 * (feq - feq[opp])
    sp, sm = 0.5 * (S + S[opp]), 0.5 * (S - S[opp])
    fstar = (f - (fp - ep) / tau_p - (fm - em) / tau_m
             + (1.0 - 0.5 / tau_p) * sp + (1.0 - 0.5 / tau_m) * sm)
    return fstar, ux, uy


def stream(fstar) -> torch.Tensor:
    """Periodic streaming: f_i(c, n+1) = f*_i(c - c_i)."""
    return torch.stack([torch.roll(fstar[i], shifts=(cy, cx), dims=(0, 1))
                        for i, (cx, cy) in enumerate(D2Q9_C)], 0)


def lbm_step(f, F, c: Consts):
    fstar, ux, uy = trt_collide(f, F, c.tau_plus, c.tau_minus)
    return stream(fstar), torch.stack([ux, uy], 0)


# ---------------------------------------------------------------------------
# World state and the full step.
# ---------------------------------------------------------------------------
@dataclass
class State:
    X: torch.Tensor       # [N, 2] wrapped positions
    theta: torch.Tensor   # [E]
    f: torch.Tensor       # [9, H, W] populations
    D: torch.Tensor       # [N, 2] unwrapped displacement since t0
    t: int


class World:
    """Static data of one world (topology, rest parameters, constants)."""

    def __init__(self, spec):
        self.H, self.W = int(spec.H), int(spec.W)
        self.topo = topology(spec.fil_off)
        self.c = consts(spec.params)
        as64 = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float64).copy())
        self.L_rest = as64(spec.L_rest)
        self.theta0 = as64(spec.theta0)
        self.amp = as64(spec.drive_amp)
        self.freq = as64(spec.drive_freq)
        self.phase = as64(spec.drive_phase)
        # optional: rest-length drive [E] and energy field [H, W] (search experiments)
        la = getattr(spec, "len_amp", None)
        self.len_amp = None if la is None else as64(la)
        self.len_freq = None if la is None else as64(spec.len_freq)
        self.len_phase = None if la is None else as64(spec.len_phase)
        en = getattr(spec, "energy", None)
        self.energy = None if en is None else as64(en)
        self.spec = spec

    def rest_lengths(self, n: int, L0: Optional[torch.Tensor] = None) -> torch.Tensor:
        """L_rest(n) = L0 (1 + A sin(2 pi (freq n + phase))) with a rest-length
        drive (the controller's rest-length output), else L0."""
        L0 = self.L_rest if L0 is None else L0
        if self.len_amp is None:
            return L0
        return L0 * (1.0 + self.len_amp * torch.sin(2.0 * math.pi * (self.len_freq * float(n) + self.len_phase)))

    def initial_state(self) -> State:
        s = self.spec
        X = torch.stack([torch.from_numpy(np.asarray(s.x, np.float64)),
                         torch.from_numpy(np.asarray(s.y, np.float64))], 1)
        f = d2q9_weights()[:, None, None].expand(9, self.H, self.W).clone()
        if s.f0 is not None:
            f = f + torch.from_numpy(np.asarray(s.f0, np.float64))
        return State(X=X, theta=torch.from_numpy(np.asarray(s.theta, np.float64)),
                     f=f, D=torch.zeros_like(X), t=int(s.t0))


# ---------------------------------------------------------------------------
# Two-layer filament (Fluid-filament Interaction: the single filament is
# broadcast into a two-layer version of itself so that the fluid sees a solid
# object).  Reading: the layers sit at X +- delta n, n the unit normal of the
# filament at the bead.
# ---------------------------------------------------------------------------
def bead_normals(X: torch.Tensor, topo: Topology, H: int, W: int) -> torch.Tensor:
    """n = (-t_y, t_x) with t the normalised sum of the unit vectors of the
    bead's edges (its one edge at a filament end); where the two unit vectors
    nearly cancel (|sum| < 1e-3, a chain folded back on itself) t is the
    bead's outgoing edge, the incoming one at the last bead."""
    N = X.shape[0]
    xa, xb = X[topo.edge_a], X[topo.edge_b]
    v = torch.stack([min_image(xb[:, 0] - xa[:, 0], W), min_image(xb[:, 1] - xa[:, 1], H)], 1)
    vh = v / torch.sqrt((v * v).sum(1, keepdim=True))
    out = torch.zeros(N, 2, dtype=F64).index_add(0, topo.edge_a, vh)
    inc = torch.zeros(N, 2, dtype=F64).index_add(0, topo.edge_b, vh)
    s = out + inc
    ns = torch.sqrt((s * s).sum(1, keepdim=True))
    has_out = torch.zeros(N, dtype=torch.bool)
    has_out[topo.edge_a] = True
    fallback = torch.where(has_out[:, None], out, inc)
    t = torch.where(ns >= 1e-3, s / ns.clamp_min(1e-300), fallback)
    return torch.stack([-t[:, 1], t[:, 0]], 1)


def layer_point(X: torch.Tensor, n: torch.Tensor, d: float, H: int, W: int) -> torch.Tensor:
    return torch.stack([wrap(X[:, 0] + d * n[:, 0], W), wrap(X[:, 1] + d * n[:, 1], H)], 1)


def step(world: World, st: State, theta0: Optional[torch.Tensor] = None, record: bool = False):
    """One time step in the order a1..a8 (see the module docstring).
    theta0 may be given to differentiate with respect to the rest angles.
    Returns (new state, dict of intermediates or None)."""
    if world.c.ib == 1:
        return step_direct_forcing(world, st, theta0, record)
    c, H, W, topo = world.c, world.H, world.W, world.topo
    th0 = world.theta0 if theta0 is None else theta0
    theta_rest = rest_angles(th0, world.amp, world.freq, world.phase, st.t)          # a1
    L_rest = world.rest_lengths(st.t)
    x_hat, theta_hat = pbd(st.X, st.theta, theta_rest, L_rest, topo, c, H, W)         # a3
    F_el = c.kappa * (x_hat - st.X) / c.dt
    idx, w = stencil(st.X, H, W)
    rho_s = spread(idx, w, torch.ones(st.X.shape[0], dtype=F64), H, W)                # a4
    rho_bar = gaussian_blur(rho_s, c.sigma)                                            # a5
    grad = central_gradient(rho_bar)
    F_s = -c.k_rep * interpolate(idx, w, grad)                                          # a6
    if c.layers == 2:
        # two-layer filament: each bead couples to the fluid at X +- delta n
        # with half its force, and moves with the mean of the two velocities
        nrm = bead_normals(st.X, topo, H, W)
        ip, wp = stencil(layer_point(st.X, nrm, c.layer_half, H, W), H, W)
        im, wm = stencil(layer_point(st.X, nrm, -c.layer_half, H, W), H, W)
        half = 0.5 * (F_el + F_s)
        F = spread(ip, wp, half, H, W) + spread(im, wm, half, H, W)
        f_new, u = lbm_step(st.f, F, c)                                                 # a7
        U = 0.5 * (interpolate(ip, wp, u) + interpolate(im, wm, u))                     # a8
    else:
        F = spread(idx, w, F_el + F_s, H, W)
        f_new, u = lbm_step(st.f, F, c)                                                 # a7
        U = interpolate(idx, w, u)                                                      # a8
    X_new = torch.stack([wrap(st.X[:, 0] + c.dt * U[:, 0], W), wrap(st.X[:, 1] + c.dt * U[:, 1], H)], 1)
    new = State(X=X_new, theta=theta_hat, f=f_new, D=st.D + c.dt * U, t=st.t + 1)
    rec = None
    if record:
        rec = dict(theta_rest=theta_rest, x_hat=x_hat, F_el=F_el, rho_s=rho_s, rho_bar=rho_bar,
                   F_s=F_s, F=F, u=u, U=U)
        rec.update(step_observables(world, st, idx, w, theta_rest, L_rest))
    return new, rec


# ---------------------------------------------------------------------------
# Direct forcing with Multi-Direct Forcing (Fluid-filament Interaction: the
# nodes sample the fluid velocity for their drag, the filament broadcasts its
# own velocity back onto the grid, and MDF, Wang et al. 2008, is named among
# the practices against leakage).  Reading, in the paper's order of the two
# exchanges:
#   1. the steric force F_s (a4-a6) acts on the fluid as a body force, and
#      u* = (sum_i c_i f_i + F/2)/rho is the fluid velocity before the
#      filament's forcing (the half-force velocity of Guo's scheme);
#   2. drag: each node is carried by the fluid, X~ = X + dt U*, U* = I[u*](X);
#   3. the filament's own motion: PBD from X~ gives x_hat, and the node
#      velocity is U_s = U* + (x_hat - X~)/dt;
#   4. broadcast: m passes of direct forcing make the fluid at the nodes move
#      with U_s: dF_i = 2 rho_i (U_s,i - I[u](X_i)) (rho_i = I[rho](X_i); a
#      force density F moves the half-force velocity by F/(2 rho)), then
#      F += S[dF], u += S[dF]/(2 rho);
#   5. a7 with the total F; the nodes move with their own velocity:
#      X^{n+1} = X + dt U_s.
# The per-node force the filament exerts is sum over the passes of dF_i.
# ---------------------------------------------------------------------------
def step_direct_forcing(world: World, st: State, theta0: Optional[torch.Tensor] = None, record: bool = False):
    c, H, W, topo = world.c, world.H, world.W, world.topo
    th0 = world.theta0 if theta0 is None else theta0
    theta_rest = rest_angles(th0, world.amp, world.freq, world.phase, st.t)          # a1
    L_rest = world.rest_lengths(st.t)
    idx, w = stencil(st.X, H, W)
    rho_s = spread(idx, w, torch.ones(st.X.shape[0], dtype=F64), H, W)                # a4
    rho_bar = gaussian_blur(rho_s, c.sigma)                                            # a5
    grad = central_gradient(rho_bar)
    F_s = -c.k_rep * interpolate(idx, w, grad)                                          # a6
    F = spread(idx, w, F_s, H, W)
    rho, ux, uy = macroscopic(st.f, F)                                                  # 1
    u = torch.stack([ux, uy], 0)
    U_star = interpolate(idx, w, u)
    X_pred = torch.stack([wrap(st.X[:, 0] + c.dt * U_star[:, 0], W),                  # 2
                          wrap(st.X[:, 1] + c.dt * U_star[:, 1], H)], 1)
    x_hat, theta_hat = pbd(X_pred, st.theta, theta_rest, L_rest, topo, c, H, W)       # 3
    U_s = U_star + (x_hat - X_pred) / c.dt
    F_ib = torch.zeros_like(U_s)
    for _ in range(c.mdf_iters):                                                        # 4
        r = interpolate(idx, w, rho)
        dF = 2.0 * r[:, None] * (U_s - interpolate(idx, w, u))
        G = spread(idx, w, dF, H, W)
        F = F + G
        u = u + G / (2.0 * rho)
        F_ib = F_ib + dF
    f_new, u_new = lbm_step(st.f, F, c)                                                 # 5
    X_new = torch.stack([wrap(st.X[:, 0] + c.dt * U_s[:, 0], W), wrap(st.X[:, 1] + c.dt * U_s[:, 1], H)], 1)
    new = State(X=X_new, theta=theta_hat, f=f_new, D=st.D + c.dt * U_s, t=st.t + 1)
    rec = None
    if record:
        rec = dict(theta_rest=theta_rest, x_hat=x_hat, F_el=F_ib, rho_s=rho_s, rho_bar=rho_bar,
                   F_s=F_s, F=F, u=u_new, U=U_s, U_star=U_star, u_mdf=u)
        rec.update(step_observables(world, st, idx, w, theta_rest, L_rest))
    return new, rec


def step_observables(world: World, st: State, idx, w, theta_rest, L_rest) -> Dict[str, torch.Tensor]:
    """What one step adds to the search observables (QD Search: Eqs. 5, 6;
    Neuroevolution: energy sampled at the nodes):
      e_bend = sum_j (theta_rest(t-1) - theta_rest(t))^2,
      e_pos  = sum_e (L_rest(t-1) - L_rest(t))^2   (both 0 at t = 0),
      e_bead = energy field at each bead (start of step, interpolation kernel),
      energy = sum of e_bead."""
    t = st.t
    zero = torch.zeros((), dtype=F64)
    if t >= 1:
        prev = rest_angles(world.theta0, world.amp, world.freq, world.phase, t - 1)
        e_bend = ((prev - theta_rest) ** 2).sum()
        e_pos = ((world.rest_lengths(t - 1) - L_rest) ** 2).sum()
    else:
        e_bend, e_pos = zero, zero
    if world.energy is not None:
        e_bead = interpolate(idx, w, world.energy)
        energy = e_bead.sum()
    else:
        e_bead, energy = None, zero
    return dict(e_bend=e_bend, e_pos=e_pos, e_bead=e_bead, energy=energy)


def observables(world: World, n_steps: int) -> Dict[str, float]:
    """E_bend, E_pos and the energy collected over n_steps from the initial state."""
    st = world.initial_state()
    tot = {"e_bend": 0.0, "e_pos": 0.0, "energy": 0.0}
    for _ in range(n_steps):
        st, rec = step(world, st, record=True)
        for k in tot:
            tot[k] += float(rec[k])
    return tot


def rollout(world: World, n_steps: int, st: Optional[State] = None, theta0=None) -> State:
    st = world.initial_state() if st is None else st
    for _ in range(n_steps):
        st, _ = step(world, st, theta0)
    return st


# ---------------------------------------------------------------------------
# Cell and bin indexing (the binned deposition's data structure).  Computed on
# float32 positions so that both sides floor identical numbers.
# ---------------------------------------------------------------------------
def cell_and_bin(x32: np.ndarray, y32: np.ndarray, H: int, W: int, tile: int):
    """cell = (floor(Y) mod H) W + (floor(X) mod W); bin = tile row-major
    index of the tile x tile block holding the cell; bin_off = exclusive
    prefix sum of the bead count per bin."""
    cx = np.mod(np.floor(x32.astype(np.float64)).astype(np.int64), W)
    cy = np.mod(np.floor(y32.astype(np.float64)).astype(np.int64), H)
    ntx = (W + tile - 1) // tile
    nty = (H + tile - 1) // tile
    cell = cy * W + cx
    b = (cy // tile) * ntx + (cx // tile)
    counts = np.bincount(b, minlength=ntx * nty)
    off = np.zeros(ntx * nty + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    return cell, b, off


# ---------------------------------------------------------------------------
# Folding loss (Filament Folding experiment; the MNIST image target is
# replaced by a seeded random polyline): mean over beads of the squared
# distance from the unwrapped bead position X^0 + D to the nearest segment.
# ---------------------------------------------------------------------------
def point_segment_dist2(P: torch.Tensor, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Squared distance of points P [N,2] to segments (A_s, B_s) [S,2]: [N, S]."""
    AB = B - A
    AP = P[:, None, :] - A[None, :, :]
    tt = (AP * AB[None]).sum(-1) / (AB * AB).sum(-1)[None]
    tt = tt.clamp(0.0, 1.0)
    Q = A[None] + tt[..., None] * AB[None]
    d = P[:, None, :] - Q
    return (d * d).sum(-1)


def polyline_loss(P: torch.Tensor, poly: torch.Tensor) -> torch.Tensor:
    d2 = point_segment_dist2(P, poly[:-1], poly[1:])
    return d2.min(1).values.mean()


def folding_loss(world: World, n_steps: int, poly, theta0: Optional[torch.Tensor] = None):
    st = rollout(world, n_steps, theta0=theta0)
    X0 = world.initial_state().X
    poly = torch.as_tensor(np.asarray(poly, np.float64))
    return polyline_loss(X0 + st.D, poly), st


# ---------------------------------------------------------------------------
# The paper's folding loss (Filament Folding experiment): mean squared error
# between the Gaussian-splatted particle density at the final step and a
# target image of R x R pixels covering the periodic domain.  Readings: pixel
# (px, py) has its centre at ((px + 1/2) W/R, (py + 1/2) H/R); a bead at image
# coordinates u = (X R/W, Y R/H) adds exp(-|c - u|^2 / (2 s^2)) to the
# (2K + 1)^2 pixels c with px in floor(u_x) - K .. floor(u_x) + K (same in y,
# periodic), K = ceil(4 s), s in pixels; no normalisation.
# ---------------------------------------------------------------------------
def splat_image(X: torch.Tensor, H: int, W: int, R: int, s: float) -> torch.Tensor:
    K = int(math.ceil(4.0 * s))
    ux = X[:, 0] * (R / W)
    uy = X[:, 1] * (R / H)
    offs = torch.arange(-K, K + 1, dtype=F64)
    px = torch.floor(ux).detach()[:, None] + offs[None, :]      # [N, 2K+1]
    py = torch.floor(uy).detach()[:, None] + offs[None, :]
    gx = torch.exp(-((px + 0.5 - ux[:, None]) ** 2) / (2.0 * s * s))
    gy = torch.exp(-((py + 0.5 - uy[:, None]) ** 2) / (2.0 * s * s))
    ix = torch.remainder(px.long(), R)
    iy = torch.remainder(py.long(), R)
    idx = (iy[:, :, None] * R + ix[:, None, :]).reshape(X.shape[0], -1)
    val = (gy[:, :, None] * gx[:, None, :]).reshape(X.shape[0], -1)
    img = torch.zeros(R * R, dtype=F64).index_add(0, idx.reshape(-1), val.reshape(-1))
    return img.reshape(R, R)


def splat_loss(X: torch.Tensor, target: torch.Tensor, H: int, W: int, s: float) -> torch.Tensor:
    R = int(target.shape[0])
    d = splat_image(X, H, W, R, s) - target
    return (d * d).mean()


def splat_folding_loss(world: World, n_steps: int, target, s: float, theta0: Optional[torch.Tensor] = None):
    st = rollout(world, n_steps, theta0=theta0)
    target = torch.as_tensor(np.asarray(target, np.float64))
    return splat_loss(st.X, target, world.H, world.W, s), st


def folding_gradient(world: World, n_steps: int, poly):
    """dL/dtheta0 by reverse-mode automatic differentiation of the FP64
    rollout (the paper differentiates its simulator end to end with JAX;
    here torch.autograd plays that role)."""
    th0 = world.theta0.clone().requires_grad_(True)
    loss, _ = folding_loss(world, n_steps, poly, th0)
    (g,) = torch.autograd.grad(loss, th0)
    return float(loss.detach()), g


def parameter_gradient(world: World, n_steps: int, gx: torch.Tensor, gy: torch.Tensor):
    """Gradient of <g, X^0 + D^n> with respect to theta0, the rest lengths
    L_rest and the PBD stiffnesses (k_bend, k_stretch, k_shear), by
    reverse-mode automatic differentiation of the FP64 rollout with those
    parameters as leaves (Methods, Filaments: the quantities the searches
    and the folding optimisation act on)."""
    th0 = world.theta0.clone().requires_grad_(True)
    L = world.L_rest.clone().requires_grad_(True)
    ks = [torch.tensor(v, dtype=F64, requires_grad=True)
          for v in (world.c.k_bend, world.c.k_stretch, world.c.k_shear)]
    w2 = copy.copy(world)
    w2.L_rest = L
    w2.c = dataclasses.replace(world.c, k_bend=ks[0], k_stretch=ks[1], k_shear=ks[2])
    st = rollout(w2, n_steps, theta0=th0)
    obj = (st.D[:, 0] * gx).sum() + (st.D[:, 1] * gy).sum()
    g = torch.autograd.grad(obj, [th0, L] + ks, allow_unused=True)
    z = lambda v, like: torch.zeros_like(like) if v is None else v
    return {"theta0": z(g[0], th0), "L_rest": z(g[1], L),
            "k": torch.stack([z(gi, k) for gi, k in zip(g[2:], ks)])}


def final_position_gradient(world: World, n_steps: int, gx: torch.Tensor, gy: torch.Tensor):
    """Gradient of <g, X^0 + D^n> with respect to theta0 for fixed weights g
    (the cotangent the C-ABI backward call receives)."""
    th0 = world.theta0.clone().requires_grad_(True)
    st = rollout(world, n_steps, theta0=th0)
    obj = (st.D[:, 0] * gx).sum() + (st.D[:, 1] * gy).sum()
    (g,) = torch.autograd.grad(obj, th0)
    return g

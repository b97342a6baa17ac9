"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a closed
form, an invariant, a textbook special case or a brute-force sum, chosen so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  All run on the CPU.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import oracle_one_step, t2n

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _consts(**kw):
    return O.consts(synth.Params(**kw))


def _chain(xs, ys):
    topo = O.topology([0, len(xs)])
    X = torch.tensor(np.stack([xs, ys], 1), dtype=F64)
    return topo, X


# ---------------------------------------------------------------------------
# Golden fixtures: Peskin kernel closed forms and the D2Q9 lattice.
# ---------------------------------------------------------------------------
def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_peskin_golden_values():
    for row in _read_golden("peskin_phi.txt"):
        r, expr = row[0], "".join(row[1:])
        want = eval(expr, {"sqrt": math.sqrt})
        got = float(O.peskin_phi(torch.tensor([float(r)], dtype=F64))[0])
        assert abs(got - want) < 1e-15, (r, got, want)


def test_d2q9_golden_lattice():
    rows = _read_golden("d2q9.txt")
    for i, cx, cy, w, opp in rows:
        i = int(i)
        assert O.D2Q9_C[i] == (int(cx), int(cy))
        assert abs(O.D2Q9_W[i] - eval(w)) < 1e-16
        assert O.D2Q9_OPP[i] == int(opp)
    # isotropy moments of the lattice: sum w = 1, sum w c_a c_b = delta_ab / 3
    W = np.array(O.D2Q9_W)
    C = np.array(O.D2Q9_C, dtype=float)
    assert abs(W.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", W, C, C), np.eye(2) / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia->a", W, C), 0, atol=1e-16)


# ---------------------------------------------------------------------------
# T5: kernel moments and exact interpolation of linear fields.
# ---------------------------------------------------------------------------
def test_T5_peskin_moments():
    r = torch.rand(200, dtype=F64) * 10 - 5
    j = torch.arange(-10, 11, dtype=F64)
    phi = O.peskin_phi(r[:, None] - j[None, :])
    assert torch.allclose(phi.sum(1), torch.ones(200, dtype=F64), atol=1e-14)
    assert torch.allclose(((r[:, None] - j[None, :]) * phi).sum(1), torch.zeros(200, dtype=F64), atol=1e-14)
    # the 4-point kernel's even/odd sums and sum of squares are fixed constants
    even = torch.where((j.long() % 2 == 0)[None, :], phi, torch.zeros_like(phi)).sum(1)
    assert torch.allclose(even, torch.full((200,), 0.5, dtype=F64), atol=1e-14)
    assert torch.allclose((phi * phi).sum(1), torch.full((200,), 3.0 / 8.0, dtype=F64), atol=1e-14)


def test_T5_interpolation_of_linear_field_is_exact():
    H = W = 32
    X = torch.tensor([[10.3, 12.8], [15.0, 15.5], [20.71, 9.02]], dtype=F64)
    idx, w = O.stencil(X, H, W)
    yy, xx = torch.meshgrid(torch.arange(H, dtype=F64), torch.arange(W, dtype=F64), indexing="ij")
    field = 0.7 + 0.3 * xx - 0.2 * yy
    got = O.interpolate(idx, w, field)
    want = 0.7 + 0.3 * X[:, 0] - 0.2 * X[:, 1]
    assert torch.allclose(got, want, atol=1e-13)
    # partition of unity: sum of the 16 weights is one
    assert torch.allclose(w.sum(1), torch.ones(3, dtype=F64), atol=1e-14)


def test_stencil_cells_brute_force():
    """Cells receiving non-zero weight are exactly those within distance 2 on
    both axes (periodic), each listed once."""
    H, W = 16, 24
    rng = np.random.default_rng(3)
    X = torch.tensor(np.stack([rng.uniform(0, W, 50), rng.uniform(0, H, 50)], 1), dtype=F64)
    idx, w = O.stencil(X, H, W)
    for i in range(50):
        got = {}
        for k in range(16):
            got[int(idx[i, k])] = got.get(int(idx[i, k]), 0.0) + float(w[i, k])
        for y in range(H):
            for x in range(W):
                dx = float(O.min_image(torch.tensor(x - X[i, 0].item(), dtype=F64), W))
                dy = float(O.min_image(torch.tensor(y - X[i, 1].item(), dtype=F64), H))
                want = float(O.peskin_phi(torch.tensor(dx, dtype=F64)) * O.peskin_phi(torch.tensor(dy, dtype=F64)))
                assert abs(got.get(y * W + x, 0.0) - want) < 1e-14


# ---------------------------------------------------------------------------
# T6: adjointness of the transfer operators.
# ---------------------------------------------------------------------------
def test_T6_spread_interp_adjoint():
    H, W = 20, 28
    rng = np.random.default_rng(0)
    X = torch.tensor(np.stack([rng.uniform(0, W, 40), rng.uniform(0, H, 40)], 1), dtype=F64)
    idx, w = O.stencil(X, H, W)
    Fb = torch.randn(40, dtype=F64)
    g = torch.randn(H, W, dtype=F64)
    lhs = (O.spread(idx, w, Fb, H, W) * g).sum()
    rhs = (Fb * O.interpolate(idx, w, g)).sum()
    assert abs(float(lhs - rhs)) < 1e-12 * float(abs(lhs) + 1)


def test_T6_blur_symmetric_and_mass_preserving():
    H, W = 18, 22
    a, b = torch.randn(H, W, dtype=F64), torch.randn(H, W, dtype=F64)
    Ga, Gb = O.gaussian_blur(a, 1.0), O.gaussian_blur(b, 1.0)
    assert abs(float((Ga * b).sum() - (a * Gb).sum())) < 1e-12
    assert abs(float(Ga.sum() - a.sum())) < 1e-12
    # a delta blurs into the separable sampled Gaussian
    d = torch.zeros(H, W, dtype=F64)
    d[5, 7] = 1.0
    Gd = O.gaussian_blur(d, 1.0)
    R, g = O.gaussian_taps(1.0)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            want = math.exp(-(dx * dx) / 2) * math.exp(-(dy * dy) / 2) / (sum(math.exp(-m * m / 2) for m in range(-R, R + 1)) ** 2)
            assert abs(float(Gd[(5 + dy) % H, (7 + dx) % W]) - want) < 1e-15


def test_T6_stream_moves_population_along_its_velocity():
    H, W = 8, 8
    for i, (cx, cy) in enumerate(O.D2Q9_C):
        f = torch.zeros(9, H, W, dtype=F64)
        f[i, 3, 4] = 1.0
        out = O.stream(f)
        assert float(out[i, (3 + cy) % H, (4 + cx) % W]) == 1.0
        assert float(out.sum()) == 1.0


# ---------------------------------------------------------------------------
# T3: PBD closed forms (Eqs. 1-4).
# ---------------------------------------------------------------------------
def test_T3_stretch_exact_with_unit_stiffness():
    c = _consts(k_stretch=1.0, k_shear=0.0, n_pbd=1)
    topo, X = _chain([3.0, 4.7], [5.0, 6.1])
    theta = torch.tensor([0.4], dtype=F64)
    L = torch.tensor([1.3], dtype=F64)
    x, th = O.position_pass(X, theta, L, topo, c, 32, 32)
    v = x[1] - x[0]
    assert abs(float(v.norm()) - 1.3) < 1e-14
    assert torch.allclose(x.mean(0), X.mean(0), atol=1e-15)      # symmetric update
    v0 = X[1] - X[0]
    assert abs(float(v[0] * v0[1] - v[1] * v0[0])) < 1e-14       # direction kept


def test_T3_full_kirchhoff_love_with_unit_shear():
    c = _consts(k_stretch=1.0, k_shear=1.0, orient=0.0)
    topo, X = _chain([3.0, 4.7], [5.0, 6.1])
    theta = torch.tensor([0.4], dtype=F64)
    L = torch.tensor([1.3], dtype=F64)
    x, th = O.position_pass(X, theta, L, topo, c, 32, 32)
    v = x[1] - x[0]
    assert torch.allclose(v, 1.3 * torch.tensor([math.cos(0.4), math.sin(0.4)], dtype=F64), atol=1e-14)
    assert float(th[0]) == 0.4


def test_T3_bend_pass_closed_form():
    theta = torch.tensor([0.1, 0.5], dtype=F64)
    topo = O.topology([0, 3])
    rest = torch.tensor([0.15], dtype=F64)
    for k in (0.3, 0.5, 1.0):
        th = O.bend_pass(theta, rest, topo, k)
        C0 = float(theta[1] - theta[0] - rest[0])
        C1 = float(th[1] - th[0] - rest[0])
        assert abs(C1 - (1 - k) * C0) < 1e-15
        assert abs(float(th.sum() - theta.sum())) < 1e-15


def test_T3_bend_alternating_mode_factor():
    n_e = 40
    topo = O.topology([0, n_e + 1])
    rest = torch.zeros(n_e - 1, dtype=F64)
    theta = torch.tensor([0.05 * ((k // 1) % 2) for k in range(n_e)], dtype=F64)
    k = 0.3
    C0 = theta[1:] - theta[:-1]
    th = O.bend_pass(theta, rest, topo, k)
    C1 = th[1:] - th[:-1]
    assert torch.allclose(C1[1:-1], (1 - 2 * k) * C0[1:-1], atol=1e-15)


def test_T3_orientation_follows_edge_at_fixed_point():
    """Position pass alone (no bending) converges to an edge frame aligned
    with the edge vector and an edge of rest length."""
    c = _consts(k_stretch=0.5, k_shear=0.5, orient=1.0)
    topo, X = _chain([3.0, 4.0], [5.0, 5.9])
    theta = torch.tensor([-0.3], dtype=F64)
    L = torch.tensor([1.0], dtype=F64)
    x, th = X, theta
    for _ in range(400):
        x, th = O.position_pass(x, th, L, topo, c, 32, 32)
    v = x[1] - x[0]
    assert abs(float(torch.atan2(v[1], v[0]) - th[0])) < 1e-10
    assert abs(float(v.norm()) - 1.0) < 1e-10


def test_T3_rigid_motion_equivariance():
    """Rotating beads and frames rotates every correction; translating changes nothing."""
    c = _consts()
    rng = np.random.default_rng(1)
    n = 7
    xs = np.cumsum(rng.uniform(0.7, 1.3, n))
    ys = rng.uniform(-0.3, 0.3, n) + 10
    topo, X = _chain(xs + 10, ys)
    theta = torch.tensor(rng.uniform(-0.4, 0.4, n - 1), dtype=F64)
    rest = torch.tensor(rng.uniform(-0.3, 0.3, n - 2), dtype=F64)
    L = torch.ones(n - 1, dtype=F64)
    x1, th1 = O.pbd(X, theta, rest, L, topo, c, 256, 256)
    a = 0.7
    Rm = torch.tensor([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]], dtype=F64)
    ctr = torch.tensor([40.0, 50.0], dtype=F64)
    X2 = X @ Rm.T + ctr
    x2, th2 = O.pbd(X2, theta + a, rest, L, topo, c, 256, 256)
    assert torch.allclose(x2 - X2, (x1 - X) @ Rm.T, atol=1e-13)
    assert torch.allclose(th2 - a, th1, atol=1e-13)


def test_T3_jacobi_is_order_free():
    c = _consts()
    w = synth.tiny_world(2, side=32, lengths=(9, 7))
    ow = O.World(w)
    X = ow.initial_state().X
    th = ow.initial_state().theta
    rest = O.rest_angles(ow.theta0, ow.amp, ow.freq, ow.phase, 3)
    x1, t1 = O.pbd(X, th, rest, ow.L_rest, ow.topo, c, 32, 32)
    perm_e = torch.randperm(ow.topo.edge_a.numel())
    perm_j = torch.randperm(ow.topo.joint_e1.numel())
    topo2 = O.Topology(ow.topo.N, ow.topo.edge_a[perm_e], ow.topo.edge_b[perm_e],
                       ow.topo.joint_e1[perm_j], ow.topo.joint_e2[perm_j])
    # permuting the edge list must also permute per-edge data; undo it afterwards
    inv = torch.argsort(perm_e)
    remap = inv  # new index of old edge k is inv[k]
    topo2 = O.Topology(ow.topo.N, ow.topo.edge_a[perm_e], ow.topo.edge_b[perm_e],
                       remap[ow.topo.joint_e1[perm_j]], remap[ow.topo.joint_e2[perm_j]])
    x2, t2 = O.pbd(X, th[perm_e], rest[perm_j], ow.L_rest[perm_e], topo2, c, 32, 32)
    assert torch.allclose(x1, x2, atol=1e-14)
    assert torch.allclose(t1, t2[inv], atol=1e-14)


# ---------------------------------------------------------------------------
# T1: a filament at its rest shape with no drive and no repulsion stays put.
# ---------------------------------------------------------------------------
def _rest_world(curved):
    B = 12
    if curved:
        rng = np.random.default_rng(5)
        rest = rng.uniform(-0.2, 0.2, B - 2)
        th = np.concatenate([[0.3], 0.3 + np.cumsum(rest)])
        px = 10.25 + np.concatenate([[0], np.cumsum(np.cos(th))])
        py = 12.5 + np.concatenate([[0], np.cumsum(np.sin(th))])
    else:
        rest = np.zeros(B - 2)
        th = np.zeros(B - 1)
        px = 5.5 + np.arange(B)
        py = np.full(B, 9.5)
    p = synth.Params(k_rep=0.0)
    J = B - 2
    return synth._world("rest", 32, 32, [B], px.astype(np.float32), py.astype(np.float32),
                        th.astype(np.float32), rest.astype(np.float32), np.zeros(J), np.zeros(J),
                        np.zeros(J), params=p)


def test_T1_rest_fixed_point_straight():
    w = O.World(_rest_world(False))
    st = w.initial_state()
    X0 = st.X.clone()
    for _ in range(5):
        st, rec = O.step(w, st, record=True)
        assert torch.equal(rec["F_el"], torch.zeros_like(rec["F_el"]))
        assert torch.equal(rec["F"], torch.zeros_like(rec["F"]))
        assert torch.equal(rec["u"], torch.zeros_like(rec["u"]))
    assert torch.equal(st.X, X0)
    assert float((st.f - O.d2q9_weights()[:, None, None]).abs().max()) < 1e-15


def test_T1_rest_fixed_point_curved():
    spec = _rest_world(True)
    w = O.World(spec)
    st = w.initial_state()
    # float32 inputs: the rest shape holds to the rounding of the inputs
    # (coordinates in [8, 32) carry up to 1e-6 of rounding), against forces of
    # order 1e-3 for a shape away from rest
    st, rec = O.step(w, st, record=True)
    assert float(rec["F_el"].abs().max()) < w.c.kappa * 1e-5
    for _ in range(20):
        st, rec = O.step(w, st, record=True)
    assert float(st.D.abs().max()) < 1e-5


# ---------------------------------------------------------------------------
# T2: internal forces sum to zero (the swimmer is force-free).
# ---------------------------------------------------------------------------
def test_T2_force_free():
    w = O.World(synth.world_c1(4))
    st = w.initial_state()
    for _ in range(3):
        st, rec = O.step(w, st, record=True)
    scale_el = float(rec["F_el"].abs().max())
    scale_s = float(rec["F_s"].abs().max())
    assert scale_el > 1e-4 and scale_s > 1e-3
    assert float(rec["F_el"].sum(0).abs().max()) < 1e-13 * w.topo.N * scale_el + 1e-16
    assert float(rec["F_s"].sum(0).abs().max()) < 1e-13 * w.topo.N * scale_s
    # the spread conserves the total force (partition of unity)
    tot = (rec["F_el"] + rec["F_s"]).sum(0)
    assert torch.allclose(rec["F"].sum((1, 2)), tot, atol=1e-13)


# ---------------------------------------------------------------------------
# T8: steric repulsion through the field equals an explicit pairwise sum.
# ---------------------------------------------------------------------------
def _pairwise_steric(P, H, W, c):
    """F_s,i = -k_rep sum_j K(X_i, X_j) with
    K = sum_{c, c'} delta_h(c - X_i) grad G(c - c') delta_h(c' - X_j),
    summed explicitly over the 16 x 16 stencil cell pairs of every bead pair."""
    n = len(P)
    R = int(math.ceil(4 * c.sigma))
    taps = [math.exp(-m * m / (2 * c.sigma ** 2)) for m in range(-R, R + 1)]
    norm = sum(taps)

    def g1(d, period):  # periodic 1D filter tap for offset d (no aliasing: 2R+1 < period)
        d = (d + period // 2) % period - period // 2
        return taps[d + R] / norm if abs(d) <= R else 0.0

    def weights(p):
        out = []
        for a in range(4):
            for b in range(4):
                cx = math.floor(p[0]) - 1 + a
                cy = math.floor(p[1]) - 1 + b
                wgt = float(O.peskin_phi(torch.tensor(cx - p[0], dtype=F64))
                            * O.peskin_phi(torch.tensor(cy - p[1], dtype=F64)))
                out.append((cx, cy, wgt))
        return out

    brute = np.zeros((n, 2))
    for i in range(n):
        for j in range(n):
            for (cx, cy, wi) in weights(P[i]):
                for (qx, qy, wj) in weights(P[j]):
                    dx, dy = cx - qx, cy - qy
                    gx = 0.5 * (g1(dx + 1, W) - g1(dx - 1, W)) * g1(dy, H)
                    gy = 0.5 * (g1(dy + 1, H) - g1(dy - 1, H)) * g1(dx, W)
                    brute[i, 0] += -c.k_rep * wi * wj * gx
                    brute[i, 1] += -c.k_rep * wi * wj * gy
    return brute


def test_T8_steric_matches_pairwise_brute_force():
    H = W = 16
    c = _consts()
    rng = np.random.default_rng(11)
    n = 6
    P = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1)
    X = torch.tensor(P, dtype=F64)
    idx, w = O.stencil(X, H, W)
    rho = O.spread(idx, w, torch.ones(n, dtype=F64), H, W)
    grad = O.central_gradient(O.gaussian_blur(rho, c.sigma))
    field_force = -c.k_rep * O.interpolate(idx, w, grad)
    brute = _pairwise_steric(P, H, W, c)
    assert np.allclose(field_force.numpy(), brute, atol=1e-14)
    # repulsive: two isolated beads push each other apart
    X2 = torch.tensor([[7.3, 8.0], [8.6, 8.2]], dtype=F64)
    idx2, w2 = O.stencil(X2, H, W)
    rho2 = O.spread(idx2, w2, torch.ones(2, dtype=F64), H, W)
    f2 = -c.k_rep * O.interpolate(idx2, w2, O.central_gradient(O.gaussian_blur(rho2, c.sigma)))
    assert float(f2[0, 0]) < 0 < float(f2[1, 0])


# ---------------------------------------------------------------------------
# T4: lattice Boltzmann invariants and closed forms.
# ---------------------------------------------------------------------------
def _rand_f(H, W, seed=0):
    g = torch.Generator().manual_seed(seed)
    return O.d2q9_weights()[:, None, None] * (1 + 0.05 * torch.randn(9, H, W, generator=g, dtype=F64))


def test_T4_mass_and_momentum():
    c = _consts()
    H, W = 12, 16
    f = _rand_f(H, W)
    F = 1e-3 * torch.randn(2, H, W, dtype=F64)
    fn, u = O.lbm_step(f, F, c)
    assert abs(float(fn.sum() - f.sum())) < 1e-12
    cx = torch.tensor([q[0] for q in O.D2Q9_C], dtype=F64)[:, None, None]
    cy = torch.tensor([q[1] for q in O.D2Q9_C], dtype=F64)[:, None, None]
    jx0, jy0 = float((cx * f).sum()), float((cy * f).sum())
    jx1, jy1 = float((cx * fn).sum()), float((cy * fn).sum())
    assert abs(jx1 - jx0 - float(F[0].sum())) < 1e-13
    assert abs(jy1 - jy0 - float(F[1].sum())) < 1e-13


def test_T4_equilibrium_is_fixed_point():
    c = _consts()
    H, W = 8, 8
    rho = torch.full((H, W), 1.03, dtype=F64)
    ux = torch.full((H, W), 0.02, dtype=F64)
    uy = torch.full((H, W), -0.015, dtype=F64)
    feq = O.equilibrium(rho, ux, uy)
    fn, u = O.lbm_step(feq, torch.zeros(2, H, W, dtype=F64), c)
    assert torch.allclose(fn, feq, atol=1e-15)
    assert torch.allclose(u[0], ux, atol=1e-15) and torch.allclose(u[1], uy, atol=1e-15)


def test_T4_trt_with_equal_times_is_bgk():
    H, W = 6, 10
    tau = 0.8
    c = _consts(nu=(tau - 0.5) / 3, Lambda=(tau - 0.5) ** 2)
    assert abs(c.tau_minus - c.tau_plus) < 1e-6
    f = _rand_f(H, W, 2)
    F = 1e-3 * torch.randn(2, H, W, dtype=F64)
    got, _, _ = O.trt_collide(f, F, c.tau_plus, c.tau_plus)
    # BGK with Guo forcing written directly
    rho = f.sum(0)
    cs = O.D2Q9_C
    ux = (sum(cs[i][0] * f[i] for i in range(9)) + F[0] / 2) / rho
    uy = (sum(cs[i][1] * f[i] for i in range(9)) + F[1] / 2) / rho
    for i in range(9):
        cu = cs[i][0] * ux + cs[i][1] * uy
        feq = O.D2Q9_W[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
        S = O.D2Q9_W[i] * (3 * ((cs[i][0] - ux) * F[0] + (cs[i][1] - uy) * F[1])
                           + 9 * cu * (cs[i][0] * F[0] + cs[i][1] * F[1]))
        want = f[i] - (f[i] - feq) / c.tau_plus + (1 - 0.5 / c.tau_plus) * S
        assert torch.allclose(got[i], want, atol=1e-15)


def test_T4_uniform_force_accelerates_fluid():
    """Uniform body force on a periodic box: momentum grows by F each step and
    the half-force velocity is u^n = (n + 1/2) F / rho."""
    c = _consts()
    H, W = 8, 8
    f = O.d2q9_weights()[:, None, None].expand(9, H, W).clone()
    F = torch.zeros(2, H, W, dtype=F64)
    F[0] = 2e-5
    F[1] = -1e-5
    for n in range(20):
        f, u = O.lbm_step(f, F, c)
        assert torch.allclose(u[0], torch.full((H, W), (n + 0.5) * 2e-5, dtype=F64), atol=1e-15)
        assert torch.allclose(u[1], torch.full((H, W), -(n + 0.5) * 1e-5, dtype=F64), atol=1e-15)


def test_T4_shear_wave_decay():
    """u_x = U0 sin(2 pi y / H) decays as exp(-nu k^2 t)."""
    nu = 0.1
    c = _consts(nu=nu)
    H, W = 32, 4
    k = 2 * math.pi / H
    y = torch.arange(H, dtype=F64)[:, None].expand(H, W)
    U0 = 1e-4
    f = O.equilibrium(torch.ones(H, W, dtype=F64), U0 * torch.sin(k * y), torch.zeros(H, W, dtype=F64))
    Fz = torch.zeros(2, H, W, dtype=F64)
    amps = []
    for n in range(301):
        f, u = O.lbm_step(f, Fz, c)
        if n in (100, 300):
            amps.append(float((u[0][:, 0] * torch.sin(k * y[:, 0])).sum() * 2 / H))
    rate = math.log(amps[0] / amps[1]) / 200.0
    assert abs(rate / (nu * k * k) - 1) < 0.01


def test_T4_kolmogorov_steady_state():
    """Steady flow under F_x = F0 sin(k y): u_x = F0 sin(k y) / (nu k^2)."""
    nu = 0.1
    c = _consts(nu=nu)
    H, W = 32, 4
    k = 2 * math.pi / H
    y = torch.arange(H, dtype=F64)[:, None].expand(H, W)
    F0 = 1e-6
    F = torch.stack([F0 * torch.sin(k * y), torch.zeros(H, W, dtype=F64)], 0)
    f = O.d2q9_weights()[:, None, None].expand(9, H, W).clone()
    for _ in range(2500):
        f, u = O.lbm_step(f, F, c)
    want = F0 * torch.sin(k * y) / (nu * k * k)
    assert float((u[0] - want).abs().max()) < 0.01 * F0 / (nu * k * k)
    assert float(u[1].abs().max()) < 1e-12


# ---------------------------------------------------------------------------
# T7: scallop theorem (Hand-designed Locomotion: reciprocal strokes give no net
# displacement at high viscosity; non-reciprocal ones swim).
# ---------------------------------------------------------------------------
def _swimmer(kind, nu, kappa, B=16, side=48, amp=0.5, period=100):
    J = B - 2
    x = (np.arange(B) + side / 2 - B / 2 + 0.25).astype(np.float32)
    y = np.full(B, side / 2 + 0.25, np.float32)
    phase = np.zeros(J) if kind == "reciprocal" else -np.arange(J) / J
    p = synth.Params(nu=nu, kappa=kappa)
    return synth._world(kind, side, side, [B], x, y, np.zeros(B - 1, np.float32), np.zeros(J),
                        np.full(J, amp), np.full(J, 1.0 / period), phase, params=p)


@pytest.mark.slow
def test_T7_reciprocal_stroke_does_not_swim():
    # nu = 2 is the top of the paper's viscosity sweep; the coupling stiffness
    # is scaled with the viscosity so that the body follows its drive.
    per_cycle = {}
    for kind in ("reciprocal", "wave"):
        w = O.World(_swimmer(kind, 2.0, 2.0))
        st = w.initial_state()
        marks = []
        for n in range(1500):
            st, _ = O.step(w, st)
            if (n + 1) % 100 == 0:
                marks.append(st.D.mean(0).numpy().copy())
        per_cycle[kind] = np.linalg.norm(np.diff(np.array(marks), axis=0), axis=1)
    wave, recip = per_cycle["wave"], per_cycle["reciprocal"]
    assert wave[-1] > 0.01                           # the travelling wave swims
    assert abs(wave[-1] / wave[-4] - 1) < 0.05       # ... at a steady speed
    assert recip[-1] < 0.05 * wave[-1]               # the reciprocal stroke does not
    assert recip[-1] < recip[-4]                     # (what remains is a decaying transient)


# ---------------------------------------------------------------------------
# Drive, periodic helpers, cell and bin indices.
# ---------------------------------------------------------------------------
def test_drive_is_periodic_and_bounded():
    th0 = torch.tensor([0.1, -0.2], dtype=F64)
    amp = torch.tensor([0.3, 0.2], dtype=F64)
    freq = torch.tensor([1 / 50, 1 / 8], dtype=F64)
    ph = torch.tensor([0.25, 0.0], dtype=F64)
    r0 = O.rest_angles(th0, amp, freq, ph, 0)
    assert torch.allclose(r0, torch.tensor([0.4, -0.2], dtype=F64), atol=1e-15)   # sin(pi/2), sin(0)
    assert torch.allclose(O.rest_angles(th0, amp, freq, ph, 400), r0, atol=1e-13)


def test_wrap_and_min_image():
    W = 16.0
    X = torch.tensor([-0.5, 0.0, 15.999, 16.0, 33.25], dtype=F64)
    assert torch.allclose(O.wrap(X, W), torch.tensor([15.5, 0.0, 15.999, 0.0, 1.25], dtype=F64))
    d = torch.tensor([15.5, -15.5, 7.9, -8.1], dtype=F64)
    assert torch.allclose(O.min_image(d, W), torch.tensor([-0.5, 0.5, 7.9, 7.9], dtype=F64))


def test_cell_and_bin_brute_force():
    rng = np.random.default_rng(7)
    H, W, T = 40, 72, 16
    x = rng.uniform(0, W, 500).astype(np.float32)
    y = rng.uniform(0, H, 500).astype(np.float32)
    x[:5] = np.float32(np.nextafter(np.float32(W), np.float32(0)))
    cell, b, off = O.cell_and_bin(x, y, H, W, T)
    ntx = (W + T - 1) // T
    counts = {}
    for i in range(500):
        cx, cy = int(math.floor(float(x[i]))), int(math.floor(float(y[i])))
        assert cell[i] == cy * W + cx
        bb = (cy // T) * ntx + (cx // T)
        assert b[i] == bb
        counts[bb] = counts.get(bb, 0) + 1
    for bb in range(len(off) - 1):
        assert off[bb + 1] - off[bb] == counts.get(bb, 0)


# ---------------------------------------------------------------------------
# T10 (oracle half): reverse-mode gradient against FP64 central differences.
# ---------------------------------------------------------------------------
def test_T10_oracle_gradient_matches_finite_differences():
    spec = synth.tiny_world(1, side=16, lengths=(7, 6))
    w = O.World(spec)
    rng = np.random.default_rng(0)
    poly = synth.target_polyline(rng, 16, 16, 6)
    n_steps = 12
    loss, g = O.folding_gradient(w, n_steps, poly)
    eps = 1e-5
    for k in range(8):
        d = torch.tensor(rng.standard_normal(g.numel()), dtype=F64)
        d /= d.norm()
        lp, _ = O.folding_loss(w, n_steps, poly, w.theta0 + eps * d)
        lm, _ = O.folding_loss(w, n_steps, poly, w.theta0 - eps * d)
        fd = float(lp - lm) / (2 * eps)
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-8) + 1e-11, (k, fd, ad)


# ---------------------------------------------------------------------------
# Red-black (two-colour Gauss-Seidel) PBD ordering: closed forms.
# ---------------------------------------------------------------------------
def test_red_black_bend_pass_closed_form():
    """Three edges at (0, a, 0), rest angles 0, h = k_bend/2.  Joint 0 first:
    theta_0 = h a, theta_1 = a (1 - h); then joint 1 from the updated theta_1:
    C_1 = -a (1 - h), theta_1 = a (1 - h)^2, theta_2 = h a (1 - h).  (Jacobi
    gives (h a, a (1 - 2h), h a).)"""
    topo = O.topology([0, 4])
    a, k = 0.3, 0.6
    h = k / 2
    th = torch.tensor([0.0, a, 0.0], dtype=F64)
    tr = torch.zeros(2, dtype=F64)
    th = O.bend_pass(th, tr, topo, k, color=0)
    th = O.bend_pass(th, tr, topo, k, color=1)
    want = [h * a, a * (1 - h) ** 2, h * a * (1 - h)]
    assert np.allclose(t2n(th), want, rtol=0, atol=1e-15)
    jac = O.bend_pass(torch.tensor([0.0, a, 0.0], dtype=F64), tr, topo, k)
    assert np.allclose(t2n(jac), [h * a, a * (1 - 2 * h), h * a], rtol=0, atol=1e-15)


def test_red_black_position_pass_closed_form():
    """Beads at x = 0, 2, 4 on a line, L = 1, k_stretch = 1, no shear or
    turning.  Edge 0 first: correction (2 - 1)/2 moves beads 0, 1 to 0.5, 1.5;
    edge 1 then sees |v| = 2.5 and moves beads 1, 2 by 0.75: (0.5, 2.25, 3.25).
    Jacobi moves both edges from the start: (0.5, 2, 3.5)."""
    c = _consts(k_stretch=1.0, k_shear=0.0, orient=0.0)
    topo, X = _chain([0.0, 2.0, 4.0], [5.0, 5.0, 5.0])
    th = torch.zeros(2, dtype=F64)
    L = torch.ones(2, dtype=F64)
    x, _ = O.position_pass(X, th, L, topo, c, 32, 32, color=0)
    x, _ = O.position_pass(x, th, L, topo, c, 32, 32, color=1)
    assert np.allclose(t2n(x[:, 0]), [0.5, 2.25, 3.25], rtol=0, atol=1e-15)
    xj, _ = O.position_pass(X, th, L, topo, c, 32, 32)
    assert np.allclose(t2n(xj[:, 0]), [0.5, 2.0, 3.5], rtol=0, atol=1e-15)


def test_red_black_colours_are_local_to_each_filament():
    """Colours follow the index within the filament: a second filament's first
    joint and edge are colour 0 whatever the first filament's length."""
    topo = O.topology([0, 4, 9])   # 3 + 4 edges, 2 + 3 joints
    assert t2n(topo.edge_color).tolist() == [0, 1, 0, 0, 1, 0, 1]
    assert t2n(topo.joint_color).tolist() == [0, 1, 0, 1, 0]


def test_red_black_rest_state_is_a_fixed_point():
    """T1 for the red-black order: a straight filament at its rest shape with
    no drive stays where it is, bitwise."""
    spec = synth.tiny_world(0, side=32, lengths=(12,))
    spec.theta = np.zeros(spec.E, np.float32)
    spec.x = (5.0 + np.arange(12)).astype(np.float32)
    spec.y = np.full(12, 7.0, np.float32)
    spec.theta0 = np.zeros(spec.J, np.float32)
    spec.drive_amp = np.zeros(spec.J, np.float32)
    spec.params = synth.Params(k_rep=0.0, pbd_order=1)
    w = O.World(spec)
    st = w.initial_state()
    x_hat, th = O.pbd(st.X, st.theta, torch.zeros(spec.J, dtype=F64), w.L_rest, w.topo, w.c, 32, 32)
    assert torch.equal(x_hat, st.X) and torch.equal(th, st.theta)


# ---------------------------------------------------------------------------
# Search observables (QD Search Eqs. 5, 6; the Neuroevolution energy field).
# ---------------------------------------------------------------------------
def _observed_world(A=0.2, a=0.1, nu=0.25, energy=None):
    spec = synth.tiny_world(3, side=32, lengths=(6, 5, 4))
    spec.drive_amp = np.full(spec.J, A, np.float32)
    spec.drive_freq = np.full(spec.J, nu, np.float32)
    spec.drive_phase = np.zeros(spec.J, np.float32)
    spec.len_amp = np.full(spec.E, a, np.float32)
    spec.len_freq = np.full(spec.E, nu, np.float32)
    spec.len_phase = np.zeros(spec.E, np.float32)
    spec.energy = energy
    spec.observe = True
    return spec


def test_behaviour_descriptors_closed_form():
    """Drive and rest-length drive at frequency 1/4 cycle per step, phase 0:
    sin(2 pi t / 4) runs 0, 1, 0, -1, so every step t >= 1 changes each rest
    angle by A and each rest length by L0 a in magnitude.  Over n steps from
    t = 0: E_bend = (n - 1) J A^2 and E_pos = (n - 1) E (L0 a)^2."""
    A, a, n = 0.2, 0.1, 9
    spec = _observed_world(A, a)
    obs = O.observables(O.World(spec), n)
    L0 = float(spec.L_rest[0])
    A, a = float(np.float32(A)), float(np.float32(a))   # the inputs are float32
    assert abs(obs["e_bend"] - (n - 1) * spec.J * A * A) < 1e-12
    assert abs(obs["e_pos"] - (n - 1) * spec.E * (L0 * a) ** 2) < 1e-12
    assert obs["energy"] == 0.0


def test_energy_collected_from_a_constant_field_is_exact():
    """The interpolation weights of a bead sum to one: a constant field E0
    gives N E0 per step whatever the positions."""
    E0, n = 0.37, 5
    spec = _observed_world(energy=np.full((32, 32), E0, np.float32))
    obs = O.observables(O.World(spec), n)
    assert abs(obs["energy"] - n * spec.N * float(np.float32(E0))) < 1e-10


def test_energy_sample_of_a_linear_field_is_the_field_at_the_bead():
    """Peskin's kernel reproduces linear functions: on E(c) = 0.01 c_x +
    0.02 c_y + 0.5 (cell centres, beads away from the periodic seam) each
    bead samples exactly 0.01 X + 0.02 Y + 0.5."""
    ys, xs = np.meshgrid(np.arange(32.0), np.arange(32.0), indexing="ij")
    field = (0.01 * xs + 0.02 * ys + 0.5).astype(np.float64)
    spec = _observed_world(energy=field)
    spec.x = (8.0 + np.linspace(0, 12, spec.N)).astype(np.float32)
    spec.y = (10.0 + np.linspace(0, 9, spec.N)).astype(np.float32)
    w = O.World(spec)
    st = w.initial_state()
    _, rec = O.step(w, st, record=True)
    want = 0.01 * t2n(st.X[:, 0]) + 0.02 * t2n(st.X[:, 1]) + 0.5
    assert np.allclose(t2n(rec["e_bead"]), want, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# The splat folding loss (Filament Folding experiment).
# ---------------------------------------------------------------------------
def test_splat_of_one_bead_closed_form():
    """A bead at a pixel centre: the pixel reads exp(0) = 1, the pixel
    (a, b) away reads exp(-(a^2 + b^2) / (2 s^2)), the total is
    (sum_k exp(-k^2 / (2 s^2)))^2 over |k| <= ceil(4 s), also across the
    periodic seam."""
    H = W = 64
    R, s = 32, 1.3
    K = int(math.ceil(4 * s))
    g1 = sum(math.exp(-k * k / (2 * s * s)) for k in range(-K, K + 1))
    for px, py in ((10, 20), (0, 31)):
        X = torch.tensor([[(px + 0.5) * W / R, (py + 0.5) * H / R]], dtype=F64)
        img = O.splat_image(X, H, W, R, s)
        assert abs(float(img[py, px]) - 1.0) < 1e-15
        assert abs(float(img[(py + 2) % R, (px - 1) % R]) - math.exp(-5 / (2 * s * s))) < 1e-15
        assert abs(float(img.sum()) - g1 * g1) < 1e-12


def test_splat_translates_with_the_bead():
    """Moving every bead by one pixel (W/R cells) rolls the image by one pixel."""
    H, W, R, s = 48, 64, 32, 0.9
    rng = np.random.default_rng(3)
    X = torch.tensor(np.stack([rng.uniform(0, W, 7), rng.uniform(0, H, 7)], 1), dtype=F64)
    a = O.splat_image(X, H, W, R, s)
    b = O.splat_image(X + torch.tensor([W / R, 0.0], dtype=F64), H, W, R, s)
    assert torch.allclose(torch.roll(a, 1, dims=1), b, rtol=0, atol=1e-13)


def test_splat_loss_gradient_matches_finite_differences():
    H = W = 64
    R, s = 32, 1.1
    rng = np.random.default_rng(4)
    X = torch.tensor(np.stack([rng.uniform(10, 50, 9), rng.uniform(10, 50, 9)], 1), dtype=F64, requires_grad=True)
    target = torch.tensor(synth.target_image(rng, R), dtype=F64)
    loss = O.splat_loss(X, target, H, W, s)
    (g,) = torch.autograd.grad(loss, X)
    eps = 1e-6
    for i in range(3):
        for k in range(2):
            Xp = X.detach().clone()
            Xm = X.detach().clone()
            Xp[i, k] += eps
            Xm[i, k] -= eps
            fd = float(O.splat_loss(Xp, target, H, W, s) - O.splat_loss(Xm, target, H, W, s)) / (2 * eps)
            assert abs(fd - float(g[i, k])) <= 1e-6 * abs(float(g[i, k])) + 1e-12
    # the target equal to the splat of X: zero loss and zero gradient
    own = O.splat_image(X.detach(), H, W, R, s)
    l0 = O.splat_loss(X, own, H, W, s)
    (g0,) = torch.autograd.grad(l0, X)
    assert float(l0) == 0.0 and float(g0.abs().max()) == 0.0


# ---------------------------------------------------------------------------
# Two-layer filament.
# ---------------------------------------------------------------------------
def test_bead_normals_closed_form():
    """A straight chain at angle phi has normal (-sin phi, cos phi) at every
    bead; a right-angle corner has the bisector's normal (-1, 1)/sqrt 2; a
    chain folded back on itself takes its outgoing edge."""
    phi = 0.7
    xs = 5.0 + np.arange(5) * math.cos(phi)
    ys = 6.0 + np.arange(5) * math.sin(phi)
    topo, X = _chain(xs, ys)
    n = t2n(O.bead_normals(X, topo, 32, 32))
    assert np.allclose(n, [[-math.sin(phi), math.cos(phi)]] * 5, rtol=0, atol=1e-14)
    topo, X = _chain([5.0, 6.0, 6.0], [5.0, 5.0, 6.0])
    n = t2n(O.bead_normals(X, topo, 32, 32))
    assert np.allclose(n[1], [-1 / math.sqrt(2), 1 / math.sqrt(2)], rtol=0, atol=1e-15)
    topo, X = _chain([5.0, 6.0, 5.0], [5.0, 5.0, 5.0])
    n = t2n(O.bead_normals(X, topo, 32, 32))
    assert np.allclose(n[0], [0.0, 1.0], rtol=0, atol=1e-15)    # edge (1, 0)
    assert np.allclose(n[1], [0.0, -1.0], rtol=0, atol=1e-15)   # folded: its outgoing edge (-1, 0)
    assert np.allclose(n[2], [0.0, -1.0], rtol=0, atol=1e-15)   # last bead: incoming edge (-1, 0)


def test_two_layers_at_zero_separation_equal_one_layer():
    spec = synth.tiny_world(4, side=32, lengths=(9, 6))
    one = oracle_one_step(spec)[3]
    spec.params = synth.Params(layers=2, layer_half=0.0)
    two = oracle_one_step(spec)[3]
    for k in ("F", "u", "U"):
        assert torch.allclose(one[k], two[k], rtol=0, atol=1e-15), k


def test_two_layer_coupling_keeps_momentum_and_reproduces_linear_flow():
    """The spread force sums to the beads' total force, and the mean of the
    two layer velocities of a linear velocity field is its value at the bead."""
    spec = synth.tiny_world(5, side=48, lengths=(12, 9))
    spec.params = synth.Params(layers=2, layer_half=1.3)
    _, st0, _, rec = oracle_one_step(spec)
    tot = (rec["F_el"] + rec["F_s"]).sum(0)
    assert torch.allclose(rec["F"].sum((1, 2)), tot, rtol=0, atol=1e-13)
    w = O.World(spec)
    nrm = O.bead_normals(st0.X, w.topo, 48, 48)
    ys, xs = torch.meshgrid(torch.arange(48, dtype=F64), torch.arange(48, dtype=F64), indexing="ij")
    u = torch.stack([0.01 * xs - 0.02 * ys + 0.1, 0.03 * xs + 0.005 * ys], 0)
    ip, wp = O.stencil(O.layer_point(st0.X, nrm, 1.3, 48, 48), 48, 48)
    im, wm = O.stencil(O.layer_point(st0.X, nrm, -1.3, 48, 48), 48, 48)
    U = 0.5 * (O.interpolate(ip, wp, u) + O.interpolate(im, wm, u))
    X = st0.X
    want = torch.stack([0.01 * X[:, 0] - 0.02 * X[:, 1] + 0.1, 0.03 * X[:, 0] + 0.005 * X[:, 1]], 1)
    assert torch.allclose(U, want, rtol=0, atol=1e-13)


def _objective(w, n_steps, gx, gy, L_rest=None, ks=None):
    import copy
    import dataclasses
    w2 = copy.copy(w)
    if L_rest is not None:
        w2.L_rest = L_rest
    if ks is not None:
        w2.c = dataclasses.replace(w.c, k_bend=ks[0], k_stretch=ks[1], k_shear=ks[2])
    st = O.rollout(w2, n_steps)
    return float((st.D[:, 0] * gx).sum() + (st.D[:, 1] * gy).sum())


@pytest.mark.parametrize("order,layers,ib", [(0, 1, 0), (1, 1, 0), (0, 2, 0), (0, 1, 1)])
def test_T10_parameter_gradient_matches_finite_differences(order, layers, ib):
    """Gradients with respect to the rest lengths and the three stiffnesses
    against FP64 central differences of the same objective, with Jacobi and
    with red-black PBD passes, for a two-layer filament, and with direct
    forcing (two MDF passes)."""
    spec = synth.tiny_world(2, side=16, lengths=(7, 6))
    spec.params = synth.Params(k_bend=0.6, k_stretch=0.7, k_shear=0.4, orient=1.0, pbd_order=order,
                               layers=layers, layer_half=0.7, ib=ib, mdf_iters=2)
    w = O.World(spec)
    rng = np.random.default_rng(5)
    gx = torch.tensor(rng.standard_normal(spec.N), dtype=F64)
    gy = torch.tensor(rng.standard_normal(spec.N), dtype=F64)
    n_steps = 8
    g = O.parameter_gradient(w, n_steps, gx, gy)
    eps = 1e-6
    for k in range(4):
        d = torch.tensor(rng.standard_normal(spec.E), dtype=F64)
        d /= d.norm()
        fd = (_objective(w, n_steps, gx, gy, L_rest=w.L_rest + eps * d)
              - _objective(w, n_steps, gx, gy, L_rest=w.L_rest - eps * d)) / (2 * eps)
        ad = float((g["L_rest"] * d).sum())
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-6), (k, fd, ad)
    base = [w.c.k_bend, w.c.k_stretch, w.c.k_shear]
    for i in range(3):
        kp = list(base)
        km = list(base)
        kp[i] += eps
        km[i] -= eps
        fd = (_objective(w, n_steps, gx, gy, ks=kp) - _objective(w, n_steps, gx, gy, ks=km)) / (2 * eps)
        ad = float(g["k"][i])
        assert abs(ad) > 1e-8
        # the floor is the central difference's FP64 rounding: |objective|
        # (order 1) x 2^-52 / eps
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-9, (i, fd, ad)
    # theta0 part equals the dedicated routine
    assert torch.allclose(g["theta0"], O.final_position_gradient(w, n_steps, gx, gy), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# Step-level wiring: each stage of one full step checked by a closed form or a
# physical property of the whole step.
# ---------------------------------------------------------------------------
def test_position_pass_turns_frame_toward_edge():
    """With the edge at angle theta + eps and |v| = L, one pass with unit
    stiffnesses turns the frame toward the edge by less than eps."""
    c = _consts(k_stretch=1.0, k_shear=1.0, orient=1.0)
    for eps in (0.3, -0.2, 0.05):
        topo, X = _chain([3.0, 3.0 + math.cos(0.4 + eps)], [5.0, 5.0 + math.sin(0.4 + eps)])
        x, th = O.position_pass(X, torch.tensor([0.4], dtype=F64), torch.tensor([1.0], dtype=F64),
                                topo, c, 32, 32)
        turn = float(th[0]) - 0.4
        assert turn * eps > 0 and abs(turn) < abs(eps)


def _dimer_world(sep, y=8.0):
    p = synth.Params(k_rep=0.0)
    return synth._world("dimer", 24, 24, [2], np.array([10.0, 10.0 + sep], np.float32),
                        np.array([y, y], np.float32), np.zeros(1, np.float32), np.zeros(0),
                        np.zeros(0), np.zeros(0), np.zeros(0), params=p)


def test_step_stretched_dimer_contracts_along_its_axis():
    """The elastic force pulls a stretched edge back toward its rest length
    through the fluid: the beads approach each other along the edge; the flow
    is mirror-symmetric about the edge so nothing moves across it."""
    w = O.World(_dimer_world(2.0))
    st = w.initial_state()
    dist = [1.0]
    for _ in range(40):
        st, rec = O.step(w, st, record=True)
        d = float(st.X[1, 0] - st.X[0, 0])
        assert d < dist[-1] + 1e-12 if len(dist) > 1 else d < 2.0
        dist.append(d)
    assert dist[-1] < 1.9
    assert float(rec["F_el"][0, 0]) > 0 > float(rec["F_el"][1, 0])
    assert float(st.D[:, 1].abs().max()) < 1e-13


def test_step_uniform_flow_advects_beads():
    """A fluid at rest-density equilibrium with uniform velocity u0 and no
    filament forces carries every bead by dt u0 per step."""
    spec = _dimer_world(1.0, y=8.3)
    spec.params = synth.Params(k_rep=0.0)
    u0 = (0.01, -0.004)
    H, W = spec.H, spec.W
    feq = O.equilibrium(torch.ones(H, W, dtype=F64), torch.full((H, W), u0[0], dtype=F64),
                        torch.full((H, W), u0[1], dtype=F64))
    spec.f0 = (feq - O.d2q9_weights()[:, None, None]).numpy().astype(np.float32)
    w = O.World(spec)
    st = w.initial_state()
    X0 = st.X.clone()
    for n in range(5):
        st, rec = O.step(w, st, record=True)
    # f0 was rounded to float32: the flow is u0 to that rounding
    assert torch.allclose(st.D[:, 0], torch.full((2,), 5 * u0[0], dtype=F64), atol=1e-8)
    assert torch.allclose(st.D[:, 1], torch.full((2,), 5 * u0[1], dtype=F64), atol=1e-8)
    assert torch.allclose(st.X, X0 + st.D, atol=1e-12)


def test_step_steric_force_is_pairwise_repulsion():
    """The steric force a full step applies equals the explicit pairwise sum
    for the step's own positions."""
    p = synth.Params()
    x = np.array([3.2, 4.1, 9.6, 10.4, 7.3, 8.05], np.float32)
    y = np.array([5.1, 5.3, 6.0, 6.7, 11.2, 11.0], np.float32)
    spec = synth._world("pairs", 16, 16, [2, 2, 2], x, y, np.zeros(3, np.float32), np.zeros(0),
                        np.zeros(0), np.zeros(0), np.zeros(0), params=p)
    w = O.World(spec)
    st = w.initial_state()
    _, rec = O.step(w, st, record=True)
    brute = _pairwise_steric(np.stack([x.astype(np.float64), y.astype(np.float64)], 1), 16, 16, w.c)
    assert np.allclose(rec["F_s"].numpy(), brute, atol=1e-14)


# ---------------------------------------------------------------------------
# Direct forcing with multi-direct forcing passes (Fluid-filament Interaction).
# ---------------------------------------------------------------------------
def _uniform_flow_f0(H, W, u0):
    feq = O.equilibrium(torch.ones(H, W, dtype=F64), torch.full((H, W), u0[0], dtype=F64),
                        torch.full((H, W), u0[1], dtype=F64))
    return (feq - O.d2q9_weights()[:, None, None]).numpy().astype(np.float32)


def test_direct_forcing_rest_filament_rides_a_uniform_flow():
    """A straight filament at its rest shape in a uniform flow: the fluid
    already moves every node with the filament's own velocity, so the direct
    forcing is zero, the flow stays uniform and every node moves by dt u."""
    B = 8
    x = np.float32(4.25) + np.arange(B, dtype=np.float32)
    y = np.full(B, 9.6, np.float32)
    spec = synth._world("rest", 24, 24, [B], x, y, np.zeros(B - 1, np.float32), np.zeros(B - 2),
                        np.zeros(B - 2), np.zeros(B - 2), np.zeros(B - 2),
                        params=synth.Params(k_rep=0.0, ib=1, mdf_iters=4))
    spec.f0 = _uniform_flow_f0(24, 24, (0.02, -0.013))
    w = O.World(spec)
    st = w.initial_state()
    rho, ux, uy = O.macroscopic(st.f, torch.zeros(2, 24, 24, dtype=F64))
    f0 = st.f.clone()
    for _ in range(3):
        st, rec = O.step(w, st, record=True)
        assert float(rec["F_el"].abs().max()) < 1e-12
    assert torch.allclose(st.f, f0, atol=1e-14)
    assert torch.allclose(st.D[:, 0], torch.full((B,), 3 * float(ux[0, 0]), dtype=F64), atol=1e-13)
    assert torch.allclose(st.D[:, 1], torch.full((B,), 3 * float(uy[0, 0]), dtype=F64), atol=1e-13)


@pytest.mark.parametrize("m", [1, 2, 5])
def test_mdf_pass_shrinks_an_isolated_node_residual_by_55_over_64(m):
    """Fluid at rest (rho = 1) and two nodes whose stencils do not overlap:
    one pass changes the velocity interpolated at a node by
    sum_c delta_h(c - X)^2 (U_s - U) = (3/8)^2 (U_s - U) (the Peskin kernel's
    sum of squares is 3/8 per axis), so after m passes the node velocity
    misses U_s by (1 - 9/64)^m of the initial miss."""
    x = np.array([5.3, 16.8], np.float32)
    y = np.array([7.45, 7.2], np.float32)
    spec = synth._world("iso", 24, 24, [2], x, y, np.zeros(1, np.float32), np.zeros(0), np.zeros(0),
                        np.zeros(0), np.zeros(0), params=synth.Params(k_rep=0.0, ib=1, mdf_iters=m))
    spec.L_rest = np.array([10.0], np.float32)   # stretched: PBD moves the nodes
    w = O.World(spec)
    st = w.initial_state()
    _, rec = O.step(w, st, record=True)
    idx, wt = O.stencil(st.X, 24, 24)
    U_end = O.interpolate(idx, wt, rec["u_mdf"])
    miss0 = rec["U_star"] - rec["U"]
    assert float(miss0.abs().max()) > 1e-3
    assert torch.allclose(U_end - rec["U"], (55.0 / 64.0) ** m * miss0, atol=1e-13)


def test_direct_forcing_changes_fluid_momentum_by_the_total_force():
    """Guo forcing adds the force density to the momentum of every cell, and
    the spread keeps the sum of the node forces: over one step the fluid
    momentum changes by sum_i (F_s,i + F_ib,i)."""
    spec = synth.tiny_world(4, side=16, lengths=(6, 5, 4))
    spec.params = synth.Params(ib=1, mdf_iters=3)
    w = O.World(spec)
    st = w.initial_state()

    def momentum(f):
        return torch.stack([sum(cx * f[i] for i, (cx, cy) in enumerate(O.D2Q9_C)).sum(),
                            sum(cy * f[i] for i, (cx, cy) in enumerate(O.D2Q9_C)).sum()])

    new, rec = O.step(w, st, record=True)
    total = (rec["F_s"] + rec["F_el"]).sum(0)
    assert float(rec["F_el"].abs().max()) > 1e-4
    assert torch.allclose(momentum(new.f) - momentum(st.f), total, atol=1e-13)


def test_direct_forcing_dimer_in_shear_is_carried_then_restored():
    """A vertical dimer at its rest length in the shear flow u = (g (y - yc), 0):
    the fluid carries the nodes to X~ (stretching the edge), the stretch pass
    with unit stiffness restores the length along the carried edge, and the
    nodes end there: X^{n+1} = X~ -/+ (l - L)/2 e_hat, |X1 - X0| = L."""
    g, yc, L = 0.01, 13.7, 3.0
    H = W = 32
    yy = torch.arange(H, dtype=F64)[:, None].expand(H, W)
    feq = O.equilibrium(torch.ones(H, W, dtype=F64), g * (yy - yc), torch.zeros(H, W, dtype=F64))
    x = np.array([10.3, 10.3], np.float32)
    y = np.array([12.2, 12.2 + L], np.float32)
    p = synth.Params(k_rep=0.0, k_stretch=1.0, k_shear=0.0, k_bend=0.0, ib=1, mdf_iters=2)
    spec = synth._world("shear", H, W, [2], x, y, np.array([math.pi / 2], np.float32), np.zeros(0),
                        np.zeros(0), np.zeros(0), np.zeros(0), params=p)
    spec.L_rest = np.array([L], np.float32)
    spec.f0 = (feq - O.d2q9_weights()[:, None, None]).numpy().astype(np.float32)
    w = O.World(spec)
    st = w.initial_state()
    new, rec = O.step(w, st, record=True)
    X = st.X
    Xt = X + torch.stack([g * (X[:, 1] - yc), torch.zeros(2, dtype=F64)], 1)   # dt = 1
    e = Xt[1] - Xt[0]
    ell = float(torch.sqrt((e * e).sum()))
    assert ell > L + 1e-5
    eh = e / ell
    want = torch.stack([Xt[0] + 0.5 * (ell - L) * eh, Xt[1] - 0.5 * (ell - L) * eh])
    assert torch.allclose(new.X, want, atol=1e-8)       # f0 rounded to float32
    d = new.X[1] - new.X[0]
    assert abs(float(torch.sqrt((d * d).sum())) - L) < 1e-12

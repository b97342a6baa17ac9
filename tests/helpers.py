"""Shared test helpers: oracle runs on seeded worlds and comparisons."""
import numpy as np
import torch

import oracle as O


def oracle_one_step(spec):
    w = O.World(spec)
    st0 = w.initial_state()
    st1, rec = O.step(w, st0, record=True)
    return w, st0, st1, rec


def max_err(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (got.shape, want.shape)
    if want.size == 0:
        return 0.0, 0.0
    return float(np.max(np.abs(got - want))), float(np.max(np.abs(want)))


def assert_field(name, got, want, rtol, floor=1e-12):
    """|got - want| <= rtol * max|want| + floor, element by element; and on
    every entry of at least 1% of the field's scale, |got - want| <=
    100 rtol |want| + floor (FP32 sums of terms up to the field's scale round
    at about rtol of the scale, so an entry of 1% of it keeps 100 rtol of its
    own value)."""
    err, scale = max_err(got, want)
    assert err <= rtol * scale + floor, f"{name}: max err {err:.3e} vs scale {scale:.3e} (rtol {rtol})"
    g = np.asarray(got, np.float64).ravel()
    w = np.asarray(want, np.float64).ravel()
    big = np.abs(w) >= 0.01 * scale
    if big.any():
        rel = np.abs(g[big] - w[big]) - floor
        bad = rel > 100 * rtol * np.abs(w[big])
        assert not bad.any(), (f"{name}: {int(bad.sum())} entries above 1% of the scale off by more than "
                               f"{100 * rtol:g} of their value (worst {np.max(rel / np.abs(w[big])):.3e})")
    return err, scale


def periodic_diff(a, b, period):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return d - period * np.round(d / period)


def t2n(t):
    return t.detach().cpu().numpy()


def crop_world(spec, cx, cy, radius=16, side=256):
    """Sub-world of `spec` around the point (cx, cy) for checking one bead of
    a world too large for the oracle.

    Keeps every filament with a bead within periodic Chebyshev distance
    `radius` of the point, whole, translated by an integer so that the point
    sits near the centre of a side x side periodic grid (translation by an
    integer is exact in float32).  With the fluid at rest initially, one step
    of a bead within 4 cells of the point, and of the grid cells within 2
    cells of it, depends only on beads within 13 cells (stencil 2, gradient
    1, filter R = 4, deposit 2, and the spread and interpolation stencils),
    all of them kept, so the sub-world reproduces those values exactly.
    Returns (sub-spec, index of each kept bead in `spec`, integer shift)."""
    from paper_2607_02954_gb300 import synth
    bx, by = int(np.floor(cx)), int(np.floor(cy))
    dx = periodic_diff(spec.x, bx, spec.W)
    dy = periodic_diff(spec.y, by, spec.H)
    near = np.maximum(np.abs(dx), np.abs(dy)) <= radius
    fil_of = np.repeat(np.arange(spec.n_fil), np.diff(spec.fil_off))
    fils = np.unique(fil_of[near])
    lengths = np.diff(spec.fil_off)[fils]
    beads = np.concatenate([np.arange(spec.fil_off[f], spec.fil_off[f + 1]) for f in fils])
    edges = np.concatenate([np.arange(spec.fil_off[f] - f, spec.fil_off[f + 1] - f - 1) for f in fils])
    joints = np.concatenate([np.arange(spec.fil_off[f] - 2 * f, spec.fil_off[f + 1] - 2 * f - 2) for f in fils])
    half = side // 2
    x = half + dx[beads]
    y = half + dy[beads]
    assert x.min() >= 0 and x.max() < side and y.min() >= 0 and y.max() < side
    sub = synth._world(f"crop of {spec.name}", side, side, list(lengths), x, y, spec.theta[edges],
                       spec.theta0[joints], spec.drive_amp[joints], spec.drive_freq[joints],
                       spec.drive_phase[joints], params=spec.params, t0=spec.t0)
    sub.L_rest = spec.L_rest[edges].copy()
    assert spec.f0 is None
    return sub, beads, (bx - half, by - half)

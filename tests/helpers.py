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
    """|got - want| <= rtol * max|want| + floor, element by element."""
    err, scale = max_err(got, want)
    assert err <= rtol * scale + floor, f"{name}: max err {err:.3e} vs scale {scale:.3e} (rtol {rtol})"
    return err, scale


def periodic_diff(a, b, period):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return d - period * np.round(d / period)


def t2n(t):
    return t.detach().cpu().numpy()

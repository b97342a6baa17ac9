"""The sampled checks of full-size worlds rest on `crop_world`: one oracle
step of a small sub-world around a bead must reproduce that bead's values
(and the grid values around it) of one oracle step of the whole world.
Checked here, on the CPU, on a world small enough for the whole-world oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import crop_world, oracle_one_step, t2n


@pytest.mark.parametrize("seed", [0, 1])
def test_crop_reproduces_the_whole_world_step(seed):
    spec = synth.world_rows(256, 16384, seed=seed)       # 256^2 grid, 0.25 bead per cell
    _, _, st1, rec = oracle_one_step(spec)
    rng = np.random.default_rng(seed)
    picks = list(rng.choice(spec.N, 3, replace=False)) + [int(np.argmin(spec.x)), int(np.argmax(spec.y))]
    for i in picks:
        sub, beads, (sx, sy) = crop_world(spec, spec.x[i], spec.y[i], side=192)
        _, _, sst1, srec = oracle_one_step(sub)
        k = int(np.nonzero(beads == i)[0][0])
        for name in ("F_el", "F_s", "U"):
            np.testing.assert_allclose(t2n(srec[name])[k], t2n(rec[name])[i], rtol=0, atol=1e-12)
        cx, cy = int(np.floor(spec.x[i])), int(np.floor(spec.y[i]))
        for gy in range(cy - 2, cy + 3):
            for gx in range(cx - 2, cx + 3):
                a = t2n(rec["F"])[:, gy % spec.H, gx % spec.W]
                b = t2n(srec["F"])[:, (gy - sy) % sub.H, (gx - sx) % sub.W]
                np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)
                a = t2n(rec["u"])[:, gy % spec.H, gx % spec.W]
                b = t2n(srec["u"])[:, (gy - sy) % sub.H, (gx - sx) % sub.W]
                np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)

"""Tile capacity under crowding: two uncharged streams converge on the middle
of a periodic box, so the tiles there come to hold about twice their
particles.  With almost no capacity slack the library must re-lay the tiles
out as they fill (pic_step's periodic check) instead of losing particles,
and the run must be exactly the run with ample slack (which never re-lays),
particle for particle."""
import numpy as np
import pytest

from gpu_harness import Case
from paper_2602_15939_gb300 import pic as P
from paper_2602_15939_gb300 import workloads as W


def converging(slack, nsteps=200, v=0.1):
    n = (64, 32, 1)
    cfg = P.make_config(box=P.PIC_BOX_PERIODIC, nx=n[0], ny=n[1], nz=1, ndim=2, plane=P.PIC_PLANE_XY, order=1,
                        precision=P.PIC_FP32, capacity_slack=slack)
    sp = W.uniform_plasma(n, 8, seed=5, uth=0.0, charges=(0.0,), q=0.0, ignorable=2)[0]
    sp["u"][:, 0] = np.where(sp["x"][:, 0] < n[0] / 2, v, -v) / np.sqrt(1 - (v / 0.45) ** 2)  # u = gamma v
    box = P.Box(cfg)
    try:
        z = np.zeros((3, 1, n[1], n[0]))
        box.set_fields(z, z)
        box.load(0, 0.0, 1.0, sp["x"], sp["u"], sp["id"])
        cap0 = P.pic_get_capacity(box.h, 0)
        box.step(nsteps)
        d = box.diagnostics()
        x, u, ids, _ = box.particles(0)
        cap1 = P.pic_get_capacity(box.h, 0)
    finally:
        box.close()
    o = np.argsort(ids)
    return d, x[o], u[o], ids[o], cap0, cap1, sp


@pytest.mark.gpu
def test_crowded_tiles_are_relaid_not_lost():
    d, x, u, ids, cap0, cap1, sp = converging(0.02)
    assert d.error_word == 0 and d.count[0] == len(sp["x"])
    assert cap1[2] >= 1 and cap1[0] > cap0[0]  # re-laid out, with more slots per tile
    # ballistic motion, exactly as with generous capacity (no re-layout)
    d2, x2, u2, ids2, _, cap2, _ = converging(3.0)
    assert cap2[2] == 0
    assert np.array_equal(ids, ids2) and np.array_equal(x, x2) and np.array_equal(u, u2)
    v = 0.1
    x0 = sp["x"][ids]
    xe = (x0[:, 0] + np.where(x0[:, 0] < 32, v, -v) * 200) % 64
    dx = x[:, 0] - xe
    dx -= 64 * np.round(dx / 64)
    assert np.abs(dx).max() < 1e-3

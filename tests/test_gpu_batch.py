"""Batches (pic_batch_*): boxes of one kind but different grids, parameters
and particle counts, stepped together by one persistent particle kernel per
step under graph replay (and, for the unsheared kinds, with every box's grid
work in one launch per grid kernel), give exactly the results of stepping
each box on its own (FP32 bit for bit; FP64 to rounding, its current being
summed with double atomics), and one of them matches the FP64 oracle like
any box."""
import dataclasses

import numpy as np
import pytest

from gpu_harness import Case, inputs, rel_maxerr, run_oracle, current_scale
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_S, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY

EXPAND = [
    Case("e0", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=200, ppc=4),
    Case("e1", BOX_E, (24, 16, 16), order=2, rate=(0.0, 2e-3, 1e-3), step0=10, ppc=6, seed=5, uth=0.2),
    Case("e2", BOX_E, (8, 8, 8), order=2, rate=(1e-3, 1e-3, 1e-3), ppc=8, seed=9),
]
LEAKY = [
    Case("l0", BOX_L, (32, 24, 1), ndim=2, plane=P.PIC_PLANE_XY, order=2, ppc=6, esc_mode=2, p_esc=0.05, theta_inj=1.0),
    Case("l1", BOX_L, (48, 32, 1), ndim=2, plane=P.PIC_PLANE_XY, order=2, ppc=4, esc_mode=2, p_esc=0.02, theta_inj=0.3,
         seed=3),
]
PERIODIC = [
    Case("p0", BOX_P, (16, 12, 8), order=1, ppc=3),
    Case("p1", BOX_P, (12, 20, 16), order=1, ppc=4, seed=6, uth=0.25),
]
PERIODIC_XZ = [
    Case("q0", BOX_P, (32, 1, 24), ndim=2, plane=P.PIC_PLANE_XZ, order=1, ppc=5),
    Case("q1", BOX_P, (24, 1, 40), ndim=2, plane=P.PIC_PLANE_XZ, order=1, ppc=3, seed=8, uth=0.3),
    Case("q2", BOX_P, (8, 1, 8), ndim=2, plane=P.PIC_PLANE_XZ, order=1, ppc=7, seed=2),
]
SHEAR = [
    Case("s0", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37),
    Case("s1", BOX_S, (16, 16, 16), order=2, s=1.2, Omega0=2e-3, step0=5, seed=4, ppc=3),
]


def load(case, fp64):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    box.set_fields(E, B)
    for i, d in enumerate(sp):
        box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
    box.set_step(case.step0)
    return box, len(sp)


def state(box, nsp):
    parts = []
    for i in range(nsp):
        x, u, ids, _ = box.particles(i)
        o = np.argsort(ids)
        parts.append((x[o], u[o], ids[o]))
    return parts, box.fields(), box.diagnostics()


def run_alone(case, nsteps, fp64):
    box, nsp = load(case, fp64)
    try:
        box.step(nsteps)
        return state(box, nsp)
    finally:
        box.close()


def run_batched(cases, nsteps, fp64, chunks=None):
    loaded = [load(c, fp64) for c in cases]
    try:
        with P.Batch([b for b, _ in loaded]) as bt:
            for k in (chunks or [nsteps]):
                bt.step(k)
            bt.sync()
            # members are refused to pic_step while batched
            with pytest.raises(P.PicError):
                loaded[0][0].step(1)
        return [state(b, n) for b, n in loaded]
    finally:
        for b, _ in loaded:
            b.close()


def assert_same(a, b, exact, tol=1e-12):
    (pa, fa, da), (pb, fb, db) = a, b
    assert da.step == db.step and da.error_word == 0 and db.error_word == 0
    assert list(da.count[:2]) == list(db.count[:2])
    assert da.escaped_total == db.escaped_total
    for (xa, ua, ia), (xb, ub, ib) in zip(pa, pb):
        assert np.array_equal(ia, ib)
        if exact:
            assert np.array_equal(xa, xb) and np.array_equal(ua, ub)
        else:
            assert np.abs(ua - ub).max() <= tol * np.abs(ua).max()
    for x, y in zip(fa, fb):
        if exact:
            assert np.array_equal(x, y)
        else:
            assert np.abs(x - y).max() <= tol * max(np.abs(y).max(), 1e-30)


@pytest.mark.gpu
@pytest.mark.parametrize("cases", [EXPAND, LEAKY, SHEAR, PERIODIC, PERIODIC_XZ],
                         ids=["expand3d", "leaky2d", "shear3d", "periodic3d_o1", "periodic2dxz_o1"])
def test_fp32_batch_equals_boxes_alone(cases):
    n = 5  # two graph-replayed pairs and one plain step
    got = run_batched(cases, n, False, chunks=[2, 3])
    for c, g in zip(cases, got):
        assert_same(g, run_alone(c, n, False), exact=True)


@pytest.mark.gpu
def test_fp32_batch_regroup_cycles_equal_boxes_alone():
    # 3D FP32 batches regroup every 3 steps: plain steps, then graph-replayed
    # cycles (a regroup and three steps), then a tail; and with regrouping off
    n = 14
    got = run_batched(EXPAND, n, False, chunks=[2, 9, 3])
    alone = [run_alone(c, n, False) for c in EXPAND]
    for g, a in zip(got, alone):
        assert_same(g, a, exact=True)
    loaded = [load(c, False) for c in EXPAND]
    try:
        with P.Batch([b for b, _ in loaded]) as bt:
            bt.set_regroup_interval(0)
            bt.step(n)
            bt.sync()
        for (b, nsp), a in zip(loaded, alone):
            assert_same(state(b, nsp), a, exact=True)
    finally:
        for b, _ in loaded:
            b.close()


@pytest.mark.gpu
def test_fp64_batch_equals_boxes_alone():
    got = run_batched(EXPAND, 3, True)
    for c, g in zip(EXPAND, got):
        assert_same(g, run_alone(c, 3, True), exact=False)


@pytest.mark.gpu
def test_more_boxes_than_one_launch_holds():
    m = P.pic_batch_max_boxes_per_launch() + 3
    cases = [dataclasses.replace(EXPAND[2], name=f"b{k}", seed=100 + k, ppc=2 + k % 3) for k in range(m)]
    got = run_batched(cases, 4, False)
    for c, g in zip(cases, got):
        assert_same(g, run_alone(c, 4, False), exact=True)


@pytest.mark.gpu
def test_batched_box_matches_oracle():
    """A batched box against the oracle over a graph-replayed pair of steps
    (regrouping off, so the batch's first cycle is a captured pair; FP32
    tolerances doubled for two steps)."""
    c = EXPAND[0]
    loaded = [load(x, False) for x in EXPAND]
    try:
        with P.Batch([b for b, _ in loaded]) as bt:
            bt.set_regroup_interval(0)
            bt.step(2)
            bt.sync()
        got = state(*loaded[0])
    finally:
        for b, _ in loaded:
            b.close()
    st, _ = run_oracle(c, 2)
    (parts, (E, B, J), _) = got
    for (x, u, ids), d in zip(parts, st.species):
        o = np.argsort(d["id"])
        assert np.array_equal(ids, d["id"][o])
        assert rel_maxerr(u, d["u"][o]) <= 2e-6
        dx = x - d["x"][o]
        dx -= np.asarray(c.n) * np.round(dx / np.asarray(c.n))
        assert np.abs(dx).max() <= 4e-6
    jref = current_scale(c)
    assert rel_maxerr(J, st.J, jref) <= 2e-6
    assert rel_maxerr(E, st.E, 4 * np.pi * jref) <= 2e-6
    assert rel_maxerr(B, st.B, 4 * np.pi * jref) <= 2e-6


@pytest.mark.gpu
def test_batch_rejects_mixed_kinds():
    a, _ = load(EXPAND[0], False)
    b, _ = load(SHEAR[0], False)
    try:
        with pytest.raises(P.PicError):
            P.Batch([a, b])
        a.step(1)  # a failed batch leaves its boxes free
    finally:
        a.close()
        b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("lanes", [1, 2, 5])
def test_lane_counts_give_the_same_results(lanes, monkeypatch):
    """Unsheared batches run their boxes in lanes (chains of batched launches
    on streams of their own); any lane count gives the boxes-alone results."""
    monkeypatch.setenv("PIC_BATCH_LANES", str(lanes))
    cases = [dataclasses.replace(EXPAND[k % 3], name=f"x{k}", seed=200 + k, ppc=2 + k % 4) for k in range(7)]
    got = run_batched(cases, 7, False, chunks=[1, 6])
    for c, g in zip(cases, got):
        assert_same(g, run_alone(c, 7, False), exact=True)


@pytest.mark.gpu
def test_members_on_different_automatic_tiles_are_batched():
    """Small boxes take 4^3 tiles automatically and large ones 8^3; a batch
    runs its members on the plain 8^3 tiles (re-laid out) and still gives the
    boxes-alone results (which do not depend on the tile shape)."""
    cases = [dataclasses.replace(EXPAND[2], name="s16", n=(16, 16, 16), ppc=2, seed=31),
             dataclasses.replace(EXPAND[2], name="s64", n=(64, 64, 64), ppc=1, seed=32)]
    loaded = [load(c, False) for c in cases]
    try:
        tiles = [b.tile() for b, _ in loaded]
        with P.Batch([b for b, _ in loaded]) as bt:
            bt.step(4)
            bt.sync()
        assert all(b.tile() == (8, 8, 8) for b, _ in loaded)
        got = [state(b, n) for b, n in loaded]
    finally:
        for b, _ in loaded:
            b.close()
    if tiles[0] != tiles[1]:  # the automatic choice differed (the usual case on a 152-SM part)
        assert tiles[0] == (4, 4, 4)
    for c, g in zip(cases, got):
        assert_same(g, run_alone(c, 4, False), exact=True)

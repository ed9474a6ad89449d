"""Regrouping by cell (pic_set_regroup_interval): every few steps each tile's
particles are rewritten into the other buffer in cell order.  It only
reorders particles within their tiles, so FP32 runs (integer current, per-
particle states) are bit-identical at every interval, with and without graph
replay, in batches too; FP64 runs agree to rounding; a regrouped run still
matches the oracle."""
import numpy as np
import pytest

from gpu_harness import Case, current_scale, inputs, rel_maxerr, run_oracle
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_S, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY

CASES = [
    Case("expand3d_o2", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=50, ppc=6, uth=0.3),
    Case("shear3d_o2", BOX_S, (16, 16, 8), order=2, s=1.5, Omega0=3e-3, step0=11, ppc=5, uth=0.3),
    # leaky displacement rule: the displacement arrays move with the particles
    Case("leaky2dxy_disp", BOX_L, (40, 24, 1), ndim=2, plane=P.PIC_PLANE_XY, order=2, ppc=6, esc_mode=1,
         l_esc=0.25, theta_inj=0.5, uth=0.3),
    Case("periodic2dxz_o1", BOX_P, (24, 1, 20), ndim=2, plane=P.PIC_PLANE_XZ, order=1, ppc=8, uth=0.3),
]


def run(case, every, chunks, fp64=False):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    try:
        P.pic_set_regroup_interval(box.h, every)
        assert P.pic_get_regroup_interval(box.h) == every
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.set_step(case.step0)
        for k in chunks:
            box.step(k)
        parts = []
        for i in range(len(sp)):
            x, u, ids, dr = box.particles(i, want_dr=case.esc_mode == 1)
            o = np.argsort(ids)
            parts.append((x[o], u[o], ids[o], None if dr is None else dr[o]))
        return parts, box.fields(), box.diagnostics()
    finally:
        box.close()


def same(a, b):
    (pa, fa, da), (pb, fb, db) = a, b
    assert da.error_word == 0 and db.error_word == 0 and da.step == db.step
    assert list(da.count[:2]) == list(db.count[:2]) and da.escaped_total == db.escaped_total
    for qa, qb in zip(pa, pb):
        for x, y in zip(qa, qb):
            assert (x is None and y is None) or np.array_equal(x, y)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fp32_regrouped_runs_are_bit_identical(case):
    # 13 steps: plain steps, then graph-replayed regroup cycles, then a tail
    ref = run(case, 0, [13])
    for every, chunks in ((1, [13]), (2, [3, 10]), (3, [1, 12]), (5, [13])):
        same(run(case, every, chunks), ref)


@pytest.mark.gpu
def test_fp64_regrouped_run_agrees_to_rounding():
    case = CASES[0]
    a = run(case, 0, [7], fp64=True)
    b = run(case, 2, [7], fp64=True)
    (pa, fa, _), (pb, fb, _) = a, b
    for (xa, ua, ia, _), (xb, ub, ib, _) in zip(pa, pb):
        assert np.array_equal(ia, ib)
        assert np.abs(ua - ub).max() <= 1e-12 * np.abs(ua).max()
    for x, y in zip(fa, fb):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1e-30)


@pytest.mark.gpu
def test_regrouped_run_matches_oracle():
    # interval 1: the second step runs on regrouped particles.  Two FP32 steps:
    # the one-step bounds (1e-6 on u and J, 2e-6 on positions, E and B),
    # tripled for the second step
    case = CASES[0]
    parts, (E, B, J), d = run(case, 1, [2])
    st, _ = run_oracle(case, 2)
    for (x, u, ids, _), sp in zip(parts, st.species):
        o = np.argsort(sp["id"])
        assert np.array_equal(ids, sp["id"][o])
        assert rel_maxerr(u, sp["u"][o]) <= 3e-6
        dx = x - sp["x"][o]
        dx -= np.asarray(case.n) * np.round(dx / np.asarray(case.n))
        assert np.abs(dx).max() <= 6e-6
    jref = current_scale(case)
    assert rel_maxerr(J, st.J, jref) <= 3e-6
    assert rel_maxerr(E, st.E, 4 * np.pi * jref) <= 6e-6
    assert rel_maxerr(B, st.B, 4 * np.pi * jref) <= 6e-6


@pytest.mark.gpu
def test_regroup_interval_arguments():
    box = P.Box(CASES[0].gpu_config(False))
    try:
        assert P.pic_get_regroup_interval(box.h) == 3  # 3D FP32 default
        with pytest.raises(P.PicError):
            P.pic_set_regroup_interval(box.h, -1)
    finally:
        box.close()
    box = P.Box(CASES[0].gpu_config(True))
    try:
        assert P.pic_get_regroup_interval(box.h) == 0  # FP64 default
    finally:
        box.close()


def run_species(cfg, sp, every, nsteps):
    box = P.Box(cfg)
    try:
        P.pic_set_regroup_interval(box.h, every)
        n = (cfg.nx, cfg.ny, cfg.nz)
        z = np.zeros((3, n[2], n[1], n[0]))
        box.set_fields(z, z)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.step(nsteps)
        out = []
        for i in range(len(sp)):
            x, u, ids, _ = box.particles(i)
            o = np.argsort(ids)
            out.append((x[o], u[o], ids[o]))
        return out, box.fields(), box.diagnostics(), P.pic_get_capacity(box.h, 0)
    finally:
        box.close()


@pytest.mark.gpu
def test_regroup_edge_cases_empty_tiles_and_oversized_tiles():
    # (a) half the tiles empty: particles only in x < 8 of a 16-cell box
    n = (16, 8, 8)
    cfg = P.make_config(box=BOX_P, nx=n[0], ny=n[1], nz=n[2], ndim=3, order=2, precision=P.PIC_FP32)
    sp = [dict(q=-0.05, m=1.0, x=np.random.default_rng(3).uniform(0, 1, (4000, 3)) * [8, 8, 8],
               u=np.random.default_rng(4).normal(0, 0.05, (4000, 3)), id=np.arange(4000, dtype=np.uint32))]
    a = run_species(cfg, sp, 0, 7)
    b = run_species(cfg, sp, 1, 7)
    assert a[2].error_word == 0 and b[2].error_word == 0
    for (xa, ua, ia), (xb, ub, ib) in zip(a[0], b[0]):
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(ua, ub)
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    # (b) one 8^3 tile holding more slots than the in-shared-memory sort takes
    # (tcap >= 65536): the regroup copies that species in order instead
    cfg = P.make_config(box=BOX_P, nx=8, ny=8, nz=8, ndim=3, order=1, precision=P.PIC_FP32, tile=(8, 8, 8))
    N = 512 * 130
    r = np.random.default_rng(5)
    sp = [dict(q=-0.01, m=1.0, x=r.uniform(0, 8, (N, 3)), u=r.normal(0, 0.05, (N, 3)),
               id=np.arange(N, dtype=np.uint32))]
    a = run_species(cfg, sp, 0, 4)
    b = run_species(cfg, sp, 1, 4)
    assert b[3][0] >= 65536  # slots per tile
    assert a[2].error_word == 0 and b[2].error_word == 0
    for (xa, ua, ia), (xb, ub, ib) in zip(a[0], b[0]):
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(ua, ub)
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)

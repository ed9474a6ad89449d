"""Particle tile shapes (2D: 8 x 8, 16 x 16 or, in FP32, 32 x 32 cells; 3D:
4 x 4 x 4 or 8 x 8 x 8).  The
tile only decides where a particle is stored and which CTA moves it, so a box
on 8 x 8 or 32 x 32 tiles matches the oracle like any box, and gives bit for
bit the FP32 results of the same box on 16 x 16 tiles (its current is an
integer sum, exact in any order); so does a box switched between shapes
mid-run (pic_set_tile) or by the tile autotuner, and a batch of such boxes."""
import dataclasses

import numpy as np
import pytest

from gpu_harness import Case, compare, inputs
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_S, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY
BOX_SE = P.PIC_BOX_SHEAR_EXPAND
XY, XZ = P.PIC_PLANE_XY, P.PIC_PLANE_XZ

# grids that are not multiples of 32: ragged tiles on the high sides
WIDE = [
    Case("leaky2d_prob_o1", BOX_L, (72, 40, 1), ndim=2, plane=XY, order=1, ppc=6, esc_mode=2, p_esc=0.05,
         theta_inj=1.0, tile=(32, 32, 0)),
    Case("leaky2d_disp_o2", BOX_L, (40, 72, 1), ndim=2, plane=XY, order=2, ppc=5, esc_mode=1, l_esc=0.35,
         theta_inj=0.2, tile=(32, 32, 0)),
    Case("periodic2dxz_o2", BOX_P, (40, 1, 36), ndim=2, plane=XZ, order=2, ppc=6, tile=(32, 0, 32)),
    Case("expand2dxy_o1", BOX_E, (48, 33, 1), ndim=2, plane=XY, order=1, ppc=6, rate=(2e-3, 1e-3, 0.0), step0=50,
         tile=(32, 32, 0)),
    Case("shear2dxz_o1", BOX_S, (64, 1, 40), ndim=2, plane=XZ, order=1, ppc=6, s=1.5, Omega0=4e-3, step0=11,
         tile=(32, 0, 32)),
]
IDS = [c.name for c in WIDE]


def with_side(case, side):
    return dataclasses.replace(case, tile=(side, 0, side) if case.plane == XZ else (side, side, 0))


def narrow(case):
    return with_side(case, 16)


def load(case, fp64=False):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    box.set_fields(E, B)
    for i, d in enumerate(sp):
        box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
    box.set_step(case.step0)
    return box, len(sp)


def state(box, nsp, with_dr):
    parts = []
    for i in range(nsp):
        x, u, ids, dr = box.particles(i, want_dr=with_dr)
        o = np.argsort(ids)
        parts.append((x[o], u[o], ids[o], None if dr is None else dr[o]))
    return parts, box.fields(), box.diagnostics()


def assert_identical(a, b):
    (pa, fa, da), (pb, fb, db) = a, b
    assert da.step == db.step and da.error_word == 0 and db.error_word == 0
    assert da.escaped_total == db.escaped_total
    for (xa, ua, ia, ra), (xb, ub, ib, rb) in zip(pa, pb):
        assert np.array_equal(ia, ib)
        assert np.array_equal(xa, xb) and np.array_equal(ua, ub)
        if ra is not None:
            assert np.array_equal(ra, rb)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


def run(case, plan):
    """Step a box through `plan`: ints are step counts, ("tile", s) switches
    the tile side, ("tune", k) runs the tile autotuner with k trial steps."""
    box, nsp = load(case)
    try:
        for item in plan:
            if isinstance(item, int):
                box.step(item)
            elif item[0] == "tile":
                box.set_tile(item[1])
            else:
                best, ms = box.autotune_tile(item[1])
                assert best in (8, 16, 32) and box.tile()[0] == best
                assert sorted(ms) == [8, 16, 32] and all(v > 0 for v in ms.values())
        return state(box, nsp, case.esc_mode == 1), box.tile()
    finally:
        box.close()


@pytest.mark.gpu
@pytest.mark.parametrize("side", [8, 32])
@pytest.mark.parametrize("case", WIDE, ids=IDS)
def test_tile_shapes_match_oracle(case, side):
    r = compare(with_side(case, side), 1, fp64=False)
    assert r["error_word"] == 0, r
    assert r["u"] <= 1e-6 and r["x"] <= 2e-6, r
    assert r["E"] <= 1e-6 and r["B"] <= 1e-6 and r["J"] <= 1e-6, r
    assert r["escaped_gpu"] == r["escaped_oracle"], r


@pytest.mark.gpu
@pytest.mark.parametrize("case", WIDE, ids=IDS)
def test_small_tiles_match_oracle_fp64(case):
    r = compare(with_side(case, 8), 1, fp64=True)
    assert r["error_word"] == 0, r
    assert r["u"] <= 1e-12 and r["x"] <= 1e-11, r
    assert r["E"] <= 1e-12 and r["B"] <= 1e-12 and r["J"] <= 1e-12, r
    assert r["escaped_gpu"] == r["escaped_oracle"], r


@pytest.mark.gpu
@pytest.mark.parametrize("side", [8, 32])
@pytest.mark.parametrize("case", WIDE, ids=IDS)
def test_tile_shapes_equal_16x16_tiles(case, side):
    (a, ta), (b, tb) = run(with_side(case, side), [6]), run(narrow(case), [6])
    assert ta == (side, 1 if case.plane == XZ else side, side if case.plane == XZ else 1)
    assert tb[0] == 16
    assert_identical(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("case", [WIDE[0], WIDE[1], WIDE[2]], ids=IDS[:3])
def test_switching_tiles_mid_run_changes_nothing(case):
    c = narrow(case)
    got, t = run(c, [2, ("tile", 32), 3, ("tile", 8), 2, ("tile", 16), 1, ("tile", 32), 1])
    assert t[0] == 32
    want, _ = run(c, [9])
    assert_identical(got, want)


@pytest.mark.gpu
def test_tile_autotuner_keeps_the_simulation():
    c = narrow(WIDE[0])
    box, nsp = load(c)
    try:
        best, ms = box.autotune_tile(2)
        assert best in (8, 16, 32) and box.tile()[0] == best
        assert sorted(ms) == [8, 16, 32] and all(v > 0 for v in ms.values())
        box.step(1)
        got = state(box, nsp, False)
    finally:
        box.close()
    steps = got[2].step - c.step0
    want, _ = run(c, [int(steps)])
    assert_identical(got, want)


@pytest.mark.gpu
def test_batch_of_wide_tile_boxes_equals_boxes_alone():
    cases = [WIDE[0], dataclasses.replace(WIDE[0], name="l1", n=(64, 64, 1), seed=4, ppc=4),
             dataclasses.replace(WIDE[0], name="l2", n=(33, 97, 1), seed=7, p_esc=0.02)]
    loaded = [load(c) for c in cases]
    try:
        with P.Batch([b for b, _ in loaded]) as bt:
            bt.step(2)
            bt.step(3)
            bt.sync()
        got = [state(b, n, False) for b, n in loaded]
    finally:
        for b, _ in loaded:
            b.close()
    for c, g in zip(cases, got):
        want, _ = run(c, [5])
        assert_identical(g, want)


@pytest.mark.gpu
def test_tile_shape_errors():
    c = WIDE[0]
    with pytest.raises(P.PicError) as e:  # 32 x 32 tiles are FP32 only
        P.Box(c.gpu_config(True))
    assert e.value.status == P.PIC_ERR_ARG
    for bad in ((24, 24, 0), (32, 16, 0), (16, 32, 0)):
        with pytest.raises(P.PicError) as e:
            P.Box(dataclasses.replace(c, tile=bad).gpu_config(False))
        assert e.value.status == P.PIC_ERR_ARG
    box = P.Box(narrow(c).gpu_config(False))
    try:
        for bad in (24, 4, 64):
            with pytest.raises(P.PicError):
                box.set_tile(bad)
    finally:
        box.close()
    box64 = P.Box(narrow(c).gpu_config(True))
    try:
        with pytest.raises(P.PicError):  # no FP64 kernels for 32 x 32 tiles
            box64.set_tile(32)
        box64.set_tile(8)
        assert box64.tile() == (8, 8, 1)
    finally:
        box64.close()
    box3 = P.Box(Case("p3", BOX_P, (8, 8, 8), tile=(8, 8, 8)).gpu_config(False))
    try:
        assert box3.tile() == (8, 8, 8)
        for bad in (16, 2, 32):
            with pytest.raises(P.PicError):
                box3.set_tile(bad)
        box3.set_tile(4)
        assert box3.tile() == (4, 4, 4)
    finally:
        box3.close()
    for bad in ((4, 8, 8), (8, 8, 16), (16, 16, 16)):
        with pytest.raises(P.PicError):
            P.Box(Case("p3", BOX_P, (8, 8, 8), tile=bad).gpu_config(False))
    boxes = [load(c)[0], load(narrow(c))[0]]
    try:
        with P.Batch(boxes) as bt:  # a batch's members run on the plain tiles
            bt.sync()
            assert boxes[0].tile() == boxes[1].tile() == (16, 16, 1)
    finally:
        for b in boxes:
            b.close()


@pytest.mark.gpu
def test_fp64_tile_autotuner_tries_8_and_16():
    c = narrow(WIDE[2])
    box, nsp = load(c, fp64=True)
    try:
        best, ms = box.autotune_tile(1)
        assert best in (8, 16) and box.tile()[0] == best
        assert sorted(ms) == [8, 16] and all(v > 0 for v in ms.values())
    finally:
        box.close()


@pytest.mark.gpu
def test_automatic_tile_side_follows_the_box_size():
    """With the tile left open, pic_init takes 8 x 8 tiles when 16 x 16 ones
    would leave fewer than two per SM, 32 x 32 (FP32) when those still give
    eight per SM, else 16 x 16; 3D boxes keep 8 x 8 x 8."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for n, fp64, want in (((64, 64, 1), False, 8), ((64, 64, 1), True, 8), ((512, 512, 1), False, 16),
                          ((2048, 2048, 1), False, 32), ((2048, 2048, 1), True, 16), ((64, 1, 2048), False, 16)):
        plane = XZ if n[1] == 1 else XY
        tiles16 = -(-n[0] // 16) * -(-(n[2] if plane == XZ else n[1]) // 16)
        tiles32 = -(-n[0] // 32) * -(-(n[2] if plane == XZ else n[1]) // 32)
        expect = 8 if tiles16 < 2 * sms else (32 if not fp64 and tiles32 >= 8 * sms else 16)
        assert expect == want or sms != 152
        cfg = P.make_config(box=BOX_P, nx=n[0], ny=n[1], nz=n[2], ndim=2, plane=plane, order=1,
                            precision=P.PIC_FP64 if fp64 else P.PIC_FP32)
        box = P.Box(cfg)
        try:
            t = box.tile()
            assert t[0] == expect and (t[2] if plane == XZ else t[1]) == expect
        finally:
            box.close()
    # 3D: 4^3 tiles when 8^3 ones would be fewer than two per SM
    for n, want in (((16, 16, 16), 4 if 8 < 2 * sms else 8), ((64, 64, 64), 8 if 512 >= 2 * sms else 4)):
        box = P.Box(P.make_config(box=BOX_P, nx=n[0], ny=n[1], nz=n[2], order=1, precision=P.PIC_FP32))
        try:
            assert box.tile() == (want,) * 3
        finally:
            box.close()


CUBES = [
    Case("expand3d_o2", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=20, ppc=4),
    Case("shear3d_o2", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37, ppc=4),
    Case("leaky3d_disp_o1", BOX_L, (12, 10, 9), order=1, esc_mode=1, esc_dims=3, l_esc=0.3, theta_inj=0.3, ppc=4),
    Case("shearexp3d_o1_esc", BOX_SE, (16, 16, 8), order=1, s=1.2, Omega0=2e-3, rate=(0.0, 1e-3, 1e-3),
         step0=101, fp_iters=3, esc_mode=2, p_esc=0.05, theta_inj=0.3, ppc=4),
]


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [False, True], ids=["fp32", "fp64"])
@pytest.mark.parametrize("case", CUBES, ids=[c.name for c in CUBES])
def test_small_3d_tiles_match_oracle(case, fp64):
    """4 x 4 x 4 tiles (small 3D boxes) against the oracle, on grids that are
    not multiples of the tile."""
    r = compare(dataclasses.replace(case, tile=(4, 4, 4)), 1, fp64=fp64)
    tol, tx = (1e-12, 1e-11) if fp64 else (1e-6, 2e-6)
    assert r["error_word"] == 0, r
    assert r["u"] <= tol and r["x"] <= tx, r
    assert r["E"] <= tol and r["B"] <= tol and r["J"] <= tol, r
    assert r["escaped_gpu"] == r["escaped_oracle"], r


@pytest.mark.gpu
@pytest.mark.parametrize("case", CUBES, ids=[c.name for c in CUBES])
def test_small_3d_tiles_equal_8x8x8_tiles(case):
    """FP32 on 4^3 tiles equals FP32 on 8^3 tiles bit for bit over six steps
    (regrouping every 3), and so does a box switched between the two."""
    a, ta = run(dataclasses.replace(case, tile=(4, 4, 4)), [6])
    b, tb = run(dataclasses.replace(case, tile=(8, 8, 8)), [6])
    c, tc = run(dataclasses.replace(case, tile=(8, 8, 8)), [2, ("tile", 4), 3, ("tile", 8), 1])
    assert ta == (4, 4, 4) and tb == (8, 8, 8) and tc == (8, 8, 8)
    assert_identical(a, b)
    assert_identical(c, b)

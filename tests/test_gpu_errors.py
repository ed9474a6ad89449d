"""Device-side errors reach the caller as status codes, and the handle stays
usable.  The FP32 current is accumulated in int32 fixed point whose range is
max(512, 16 n0) c q_max: a current beyond half of it (here 600 particles at one
node moving together at nearly c) must be reported as PIC_ERR_NUMERIC by the
next synchronising call; after pic_clear_error and a fresh load the same
handle steps bit-identically to a new one."""
import numpy as np
import pytest

from paper_2602_15939_gb300 import pic as P
from paper_2602_15939_gb300 import workloads as W

N = (16, 16, 16)
C = 0.45


def _cfg():
    return P.make_config(nx=N[0], ny=N[1], nz=N[2], order=1, precision=P.PIC_FP32, c=C)


def _sane(box):
    sp = W.uniform_plasma(N, 2, seed=4, uth=0.1, q=0.05)
    for i, d in enumerate(sp):
        box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
    box.set_uniform_fields((0.0, 0.0, 0.0), (0.0, 0.0, 0.1))
    box.set_step(0)


@pytest.mark.gpu
def test_fixed_point_current_beyond_range_is_reported_and_handle_recovers():
    box = P.Box(_cfg())
    try:
        n = 600
        x = np.tile(np.array([5.0, 6.0, 7.0]), (n, 1))  # on a node: all of J_x on one face per particle
        u = np.tile(np.array([20.0 * C, 0.0, 0.0]), (n, 1))  # gamma ~ 20, v ~ 0.9988 c along x
        box.load(0, 0.05, 1.0, x, u, np.arange(n, dtype=np.uint32))
        box.set_uniform_fields((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
        # J_x at one face ~ 600 x 0.449 q = 269 q, above half the range 256 c q = 115 q
        box.step(1)
        with pytest.raises(P.PicError) as err:
            box.diagnostics()
        assert err.value.status == P.PIC_ERR_NUMERIC
        assert "fixed-point range" in str(err.value)
        with pytest.raises(P.PicError):
            box.step(1)  # the error stays recorded until cleared
            box.diagnostics()
        box.clear_error()
        _sane(box)
        box.step(3)
        d = box.diagnostics()
        assert d.error_word == 0 and d.step == 3
        got = [box.particles(i) for i in range(2)]
    finally:
        box.close()
    fresh = P.Box(_cfg())
    try:
        _sane(fresh)
        fresh.step(3)
        want = [fresh.particles(i) for i in range(2)]
    finally:
        fresh.close()
    for (xg, ug, ig, _), (xw, uw, iw, _) in zip(got, want):
        og, ow = np.argsort(ig), np.argsort(iw)
        np.testing.assert_array_equal(ig[og], iw[ow])
        np.testing.assert_array_equal(xg[og], xw[ow])
        np.testing.assert_array_equal(ug[og], uw[ow])


@pytest.mark.gpu
def test_displacement_escape_is_the_leaky_boxs_only():
    """The probabilistic escape runs in every box; the displacement rule is
    defined for the leaky box alone, so other boxes refuse it."""
    for box in (P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_SHEAR_EXPAND, P.PIC_BOX_PERIODIC):
        cfg = P.make_config(box=box, nx=8, ny=8, nz=8, order=1, precision=P.PIC_FP32, s=1.5, Omega0=1e-3,
                            escape_mode=P.PIC_ESC_DISPLACEMENT, l_esc=2.0, theta_inj=0.2)
        with pytest.raises(P.PicError) as e:
            P.Box(cfg)
        assert e.value.status == P.PIC_ERR_ARG
        cfg.escape_mode = P.PIC_ESC_PROBABILISTIC
        cfg.p_esc = 0.01
        P.Box(cfg).close()

"""Continuous batching on the GPU: a mixed stream of runs (shearing,
expanding, leaky, periodic; 2D and 3D; FP32) served under an HBM budget that
forces queueing, with runs admitted while others step; every result must
equal the same run served alone (FP32 state is bitwise reproducible; the
kinetic-energy sum is compared to 1e-12 because its summation order follows
the device's particle order)."""
import time

import numpy as np
import pytest

from paper_2602_15939_gb300 import pic as P


def _mix():
    XY, XZ = P.PIC_PLANE_XY, P.PIC_PLANE_XZ
    specs = []
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_SHEAR, ndim=2, plane=XZ, nx=32, ny=1, nz=32, order=1,
                                               precision=P.PIC_FP32, s=1.5, Omega0=2e-3), 24, 8, 0.1,
                                 q=(-0.05, 0.05), B0=(0, 0, 0.3), load_seed=1))
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_EXPAND, nx=16, ny=16, nz=16, order=2,
                                               precision=P.PIC_FP32, rate=(0, 1e-3, 1e-3)), 20, 8, 0.05,
                                 q=(-0.05, 0.05), B0=(0.2, 0.2, 0), load_seed=2))
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_LEAKY, ndim=2, plane=XY, nx=32, ny=32, nz=1, order=1,
                                               precision=P.PIC_FP32, escape_mode=P.PIC_ESC_PROBABILISTIC,
                                               p_esc=0.02, theta_inj=1.0, seed=5), 30, 8, 1.0,
                                 q=(-0.05, 0.05), B0=(0, 0, 0.2), load_seed=3))
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_SHEAR, nx=16, ny=16, nz=16, order=2,
                                               precision=P.PIC_FP32, s=1.5, Omega0=3e-3), 16, 4, 0.3,
                                 q=(-0.05, 0.05), B0=(0, 0, 0.1), noise_sigma=1e-3, load_seed=4))
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_PERIODIC, nx=24, ny=16, nz=8, order=2,
                                               precision=P.PIC_FP32), 12, 8, 0.05, q=(-0.05, 0.05),
                                 B0=(0, 0, 0.2), load_seed=5))
    specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_LEAKY, ndim=2, plane=XY, nx=32, ny=32, nz=1, order=2,
                                               precision=P.PIC_FP32, escape_mode=P.PIC_ESC_DISPLACEMENT, l_esc=2.0,
                                               theta_inj=0.2, seed=6), 18, 8, 0.2, q=(-0.05, 0.05),
                                 B0=(0, 0, 0.2), load_seed=6))
    return specs


def _key(d):
    return (np.array(d.field_energy_E[:]), np.array(d.field_energy_B[:]), np.array(d.kinetic_energy[:2]),
            d.escaped_total, d.step)


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    specs = _mix()
    foot = [P.pic_run_footprint(s) for s in specs]
    budget = int(sum(sorted(foot)[-3:]) * 1.05)  # about three runs at a time
    with P.Server(hbm_budget_bytes=budget, max_active=8, steps_per_round=4) as srv:
        tickets = []
        for s in specs:
            tickets.append(srv.submit(s))
            time.sleep(0.005)  # arrivals while others are stepping
        srv.wait(0, 300)
        info = srv.stats()
        mixed = [srv.poll(t) for t in tickets]
    assert info.completed == len(specs)
    assert info.peak_active >= 2
    assert info.peak_bytes <= budget
    for i, s in enumerate(specs):
        with P.Server(hbm_budget_bytes=1 << 40, max_active=1, steps_per_round=3) as alone:
            t = alone.submit(s)
            alone.wait(t, 300)
            d_alone, _ = alone.poll(t)
        d_mix, lat = mixed[i]
        a, b = _key(d_alone), _key(d_mix)
        assert b[4] == s.nsteps and a[4] == s.nsteps
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        np.testing.assert_allclose(a[2], b[2], rtol=1e-12)
        assert a[3] == b[3]
        assert lat > 0


@pytest.mark.gpu
def test_failed_run_reports_its_error_without_stopping_others():
    bad = P.make_run_spec(P.make_config(nx=4, ny=8, nz=8), 5, 4, 0.05)  # nx < 8: rejected by pic_init
    good = _mix()[4]
    with P.Server(hbm_budget_bytes=1 << 34, max_active=4) as srv:
        tb = srv.submit(bad)
        tg = srv.submit(good)
        srv.wait(0, 120)
        with pytest.raises(P.PicError):
            srv.poll(tb)
        d, _ = srv.poll(tg)
        assert d.step == good.nsteps

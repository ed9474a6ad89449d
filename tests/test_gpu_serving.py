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
            time.sleep(0.001)  # arrivals while others are stepping
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


def _alone(spec):
    """The run of `spec` stepped alone through pic_step: the same device
    Maxwellian load (per-species seed and id offsets as the server makes
    them), uniform fields, nsteps steps."""
    box = P.Box(spec.cfg)
    per_species = spec.ppc * spec.cfg.nx * spec.cfg.ny * spec.cfg.nz
    for k in range(spec.nspecies):
        box.load_maxwellian(k, spec.q[k], spec.m[k], spec.ppc, spec.theta, tuple(spec.drift), spec.noise_sigma,
                            spec.load_seed + 7919 * k, k * per_species)
    box.set_uniform_fields(tuple(spec.E0), tuple(spec.B0))
    return box


def _state(box, nspecies):
    out = []
    for k in range(nspecies):
        x, u, ids, dr = box.particles(k, want_dr=True)
        o = np.argsort(ids)
        out.append((x[o], u[o], ids[o], dr[o]))
    return out, box.fields()


@pytest.mark.gpu
def test_served_states_equal_the_runs_stepped_alone():
    """Element by element: every served run's final particles (matched by id)
    and fields (E, B and the last step's J) equal those of the same run stepped
    alone through pic_step, bit for bit (FP32 results do not depend on
    particle order or on what else runs on the GPU)."""
    specs = _mix()
    for s in specs:
        s.keep_state = 1
    foot = [P.pic_run_footprint(s) for s in specs]
    budget = int(sum(foot) * 1.05)
    with P.Server(hbm_budget_bytes=budget, max_active=8, steps_per_round=4) as srv:
        tickets = []
        for s in specs:
            tickets.append(srv.submit(s))
            time.sleep(0.003)
        srv.wait(0, 300)
        assert srv.stats().peak_active >= 2
        served = []
        for t, s in zip(tickets, specs):
            b = srv.take(t)
            with pytest.raises(P.PicError):
                srv.take(t)  # handed over once
            served.append(_state(b, s.nspecies))
            assert b.diagnostics().step == s.nsteps
            b.close()
    for s, (sp_s, f_s) in zip(specs, served):
        box = _alone(s)
        box.step(s.nsteps)
        sp_a, f_a = _state(box, s.nspecies)
        box.close()
        for (xs, us, is_, ds), (xa, ua, ia, da) in zip(sp_s, sp_a):
            np.testing.assert_array_equal(is_, ia)
            np.testing.assert_array_equal(xs, xa)
            np.testing.assert_array_equal(us, ua)
            np.testing.assert_array_equal(ds, da)
        for a, b in zip(f_s, f_a):
            np.testing.assert_array_equal(a, b)


@pytest.mark.gpu
def test_a_served_run_matches_the_oracle():
    """One served run (2D x-y leaky box, probabilistic escape, FP32, two steps)
    against the FP64 oracle started from the same initial particles (read back
    from a box given the same device load): momenta, positions and fields
    within the FP32 tolerances of the parity tests, escape counts equal."""
    import oracle as O

    cfg = P.make_config(box=P.PIC_BOX_LEAKY, ndim=2, plane=P.PIC_PLANE_XY, nx=32, ny=24, nz=1, order=1,
                        precision=P.PIC_FP32, escape_mode=P.PIC_ESC_PROBABILISTIC, p_esc=0.05, theta_inj=0.5, seed=9)
    q = 0.05
    spec = P.make_run_spec(cfg, 2, 6, 0.05, q=(-q, q), B0=(0.0, 0.0, 0.2), load_seed=11, keep_state=True)
    with P.Server(hbm_budget_bytes=1 << 34, max_active=2) as srv:
        t = srv.submit(spec)
        srv.wait(t, 120)
        b = srv.take(t)
        (sp_s, (E, B, J)) = _state(b, 2)
        esc = b.diagnostics().escaped_total
        b.close()
    box = _alone(spec)
    init = [box.particles(k) for k in range(2)]
    box.close()
    n = (32, 24, 1)
    p = O.make_params(*n, cfg.c, order=1, box=O.BOX_LEAKY, esc_mode=O.ESC_PROBABILISTIC, p_esc=0.05,
                      theta_inj=0.5, seed=9)
    E0 = np.zeros((3, 1, 24, 32))
    B0 = np.zeros_like(E0)
    B0[2] = 0.2
    species = [{"q": qq, "m": 1.0, "x": x, "u": u, "id": ids} for qq, (x, u, ids, _) in zip((-q, q), init)]
    st = O.State(p, E0, B0, species)
    info = st.step(2)
    assert esc == info["escaped"]
    jref = q * cfg.c * 2 * 6
    for d, (xs, us, ids, _) in zip(st.species, sp_s):
        o = np.argsort(d["id"])
        np.testing.assert_array_equal(ids, d["id"][o])
        dx = xs - d["x"][o]
        dx -= np.array(n, dtype=float) * np.round(dx / np.array(n, dtype=float))
        assert np.abs(dx[:, :2]).max() <= 4e-6
        assert np.abs(us - d["u"][o]).max() <= 2e-6 * np.abs(d["u"]).max()
    for a, r in ((E, st.E), (B, st.B), (J, st.J)):
        floor = jref if a is J else 4 * np.pi * jref
        assert np.abs(a - r).max() <= 2e-6 * max(np.abs(r).max(), floor)


def _kinds_mix():
    """Three runs each of three kinds, with different grids, loads and step
    counts, so that cohorts form, dissolve as their shortest runs finish and
    regroup."""
    XY, XZ = P.PIC_PLANE_XY, P.PIC_PLANE_XZ
    specs = []
    for k, (n, steps) in enumerate(((16, 12), (24, 20), (16, 27))):
        specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_EXPAND, nx=n, ny=n, nz=n, order=2,
                                                   precision=P.PIC_FP32, rate=(0, 1e-3, 1e-3)), steps, 6 + k, 0.05,
                                     q=(-0.05, 0.05), B0=(0.2, 0.2, 0), load_seed=20 + k))
        specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_LEAKY, ndim=2, plane=XY, nx=2 * n, ny=2 * n, nz=1,
                                                   order=1, precision=P.PIC_FP32,
                                                   escape_mode=P.PIC_ESC_PROBABILISTIC, p_esc=0.02, theta_inj=1.0,
                                                   seed=30 + k), steps + 3, 8, 1.0, q=(-0.05, 0.05),
                                     B0=(0, 0, 0.2), load_seed=30 + k))
        specs.append(P.make_run_spec(P.make_config(box=P.PIC_BOX_SHEAR, ndim=2, plane=XZ, nx=2 * n, ny=1, nz=2 * n,
                                                   order=1, precision=P.PIC_FP32, s=1.5, Omega0=2e-3), steps + 1,
                                     8, 0.1, q=(-0.05, 0.05), B0=(0, 0, 0.3), load_seed=40 + k))
    return specs


@pytest.mark.gpu
@pytest.mark.parametrize("policy", [0, 1])
def test_batched_serving_equals_the_runs_stepped_alone(policy, monkeypatch):
    """With batching on, runs of one kind are stepped as batches (cohorts):
    policy 1 (the default) groups runs admitted together, policy 0 regroups
    every run of a kind with steps enough left; every served run's final
    particles and fields still equal the same run stepped alone, bit for
    bit."""
    monkeypatch.setenv("PIC_SERVER_COHORT_POLICY", str(policy))
    specs = _kinds_mix()
    for s in specs:
        s.keep_state = 1
    # cohorts take runs with at least 4 x steps_per_round = 8 steps left
    with P.Server(hbm_budget_bytes=1 << 36, max_active=16, steps_per_round=2, min_batch=2) as srv:
        tickets = [srv.submit(s) for s in specs]
        srv.wait(0, 300)
        if policy == 0:  # runs drain until they can be grouped
            assert srv.stats().cohorts_formed >= 3
        served = []
        for t, s in zip(tickets, specs):
            d, _ = srv.poll(t)
            assert d.step == s.nsteps
            b = srv.take(t)
            served.append(_state(b, s.nspecies))
            b.close()
    for s, (sp_s, f_s) in zip(specs, served):
        box = _alone(s)
        box.step(s.nsteps)
        sp_a, f_a = _state(box, s.nspecies)
        box.close()
        for (xs, us, is_, ds), (xa, ua, ia, da) in zip(sp_s, sp_a):
            np.testing.assert_array_equal(is_, ia)
            np.testing.assert_array_equal(xs, xa)
            np.testing.assert_array_equal(us, ua)
            np.testing.assert_array_equal(ds, da)
        for a, b in zip(f_s, f_a):
            np.testing.assert_array_equal(a, b)


@pytest.mark.gpu
def test_batching_argument_checks():
    with P.Server(hbm_budget_bytes=1 << 30, max_active=2) as srv:
        for bad in (-1, 1):
            with pytest.raises(P.PicError):
                srv.set_batching(bad)
        srv.set_batching(0)
        srv.set_batching(4)

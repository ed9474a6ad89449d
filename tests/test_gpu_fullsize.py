"""Parity at the full sizes of the measured configurations, in the launch
configuration bench.py times (device Maxwellian load, uniform B0, the same
tiles and threads), against the FP64 oracle:

- the 2D shearing box in FP64 (64 x 64, 131,072 particles): the whole state
  against the oracle after three steps;
- the 3D expanding box (128^3, 134M particles), the 3D shearing box (256^3,
  1.07e9 particles) and the 2D leaky box (2048^2, 5.4e8 particles, on 16 x 16
  and on 32 x 32 tiles): a fixed
  id-sampled subset of particles followed through one step and recomputed one
  by one by the oracle in the device's own fields (gather, push, move,
  boundary and, for the leaky box, the escape decision and reinjection);
- for the 3D expanding box also charge continuity of the device current on a
  sub-box, from the oracle's charge density of every particle around it.

FP32 tolerances as in the small-grid parity tests: momenta 1e-6 of the
largest, positions 2e-6 cells; continuity residual 1e-5 of J_ref = |q| c n0.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_15939_gb300 import pic as P
from paper_2602_15939_gb300 import workloads as W

BOXMAP = {0: O.BOX_PERIODIC, 1: O.BOX_SHEAR, 2: O.BOX_EXPAND, 3: O.BOX_LEAKY}


def oracle_params(w, seed=0):
    kw = w.config_kwargs()
    return O.make_params(*w.n, w.c, order=w.order, box=BOXMAP[w.box], s=w.s, Omega0=kw["Omega0"], rate=kw["rate"],
                         esc_mode=w.escape_mode, p_esc=kw.get("p_esc", 0.0), l_esc=kw.get("l_esc", 0.0),
                         theta_inj=w.theta_inj, seed=seed)


def follow_sample(w, box, modulus, steps_before, seed=0, remainder=3):
    """Step `steps_before` steps, take the id-sampled particles and the
    fields, step once more, and recompute the sample with the oracle."""
    box.step(steps_before)
    E, B, _ = box.fields()
    before = [box.particles_sampled(s, modulus, remainder, 1 << 18) for s in (0, 1)]
    box.step(1)
    after = [box.particles_sampled(s, modulus, remainder, 1 << 18) for s in (0, 1)]
    p = oracle_params(w, seed)
    qs = (-w.units.q, w.units.q)
    errs = {"u": 0.0, "x": 0.0, "n": 0, "escaped": 0}
    active = [a for a in range(3) if not (w.ndim == 2 and a == (2 if w.plane == 0 else 1))]
    n = np.asarray(w.n, dtype=float)
    for s in (0, 1):
        xb, ub, ib, _ = before[s]
        xa, ua, ia, _ = after[s]
        assert len(ib) > 100 and len(ib) == len(ia)
        ob, oa = np.argsort(ib), np.argsort(ia)
        assert np.array_equal(ib[ob], ia[oa])
        xo, uo, _, info = O.advance_particles(p, E, B, steps_before, qs[s], 1.0, ib[ob], xb[ob], ub[ob])
        dx = xa[oa] - xo
        dx -= n * np.round(dx / n)
        errs["x"] = max(errs["x"], float(np.abs(dx[:, active]).max()))
        errs["u"] = max(errs["u"], float(np.abs(ua[oa] - uo).max() / np.abs(uo).max()))
        errs["n"] += len(ib)
        errs["escaped"] += info["escaped"]
    return errs


@pytest.mark.gpu
def test_shear2d_fp64_full_state_three_steps():
    w = W.SHEAR_2D_FP64
    sp = W.host_maxwellian(w, seed=11)
    r = np.random.default_rng(12)
    E = r.normal(0, 1e-3, (3, w.n[2], w.n[1], w.n[0]))
    B = np.zeros_like(E)
    for c, v in enumerate(w.b0()):
        B[c] += v
    st = O.State(oracle_params(w), E, B, sp)
    st.step(3)
    box = P.Box(P.make_config(precision=P.PIC_FP64, **w.config_kwargs()))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.step(3)
        Eg, Bg, Jg = box.fields()
        parts = [box.particles(i) for i in range(2)]
    finally:
        box.close()
    for d, (x, u, ids, _) in zip(st.species, parts):
        og, oo = np.argsort(ids), np.argsort(d["id"])
        dx = x[og] - d["x"][oo]
        dx -= np.asarray(w.n) * np.round(dx / np.asarray(w.n))
        assert np.abs(dx[:, [0, 2]]).max() < 1e-10
        assert np.abs(u[og] - d["u"][oo]).max() < 1e-11 * np.abs(d["u"]).max()
    for a, b in ((Eg, st.E), (Bg, st.B), (Jg, st.J)):
        assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()


@pytest.mark.gpu
def test_expand3d_128_sampled_particles_and_continuity():
    w = W.EXPAND_3D_FP32
    box = W.setup_box(w, device=0, seed=0)
    try:
        errs = follow_sample(w, box, 65537, 2)
        assert errs["u"] <= 1e-6 and errs["x"] <= 2e-6, errs
        # charge continuity of the device current around a sub-box: every
        # particle within 4 cells of it, before and after one more step
        full_b = [box.particles(s) for s in (0, 1)]
        box.step(1)
        _, _, J = box.fields()
        full_a = [box.particles(s) for s in (0, 1)]
    finally:
        box.close()
    lo, hi = 40, 56
    p = oracle_params(w)
    rho0 = np.zeros((1,) + J.shape[1:])
    rho1 = np.zeros_like(rho0)
    qs = (-w.units.q, w.units.q)
    for s in (0, 1):
        xb, _, ib, _ = full_b[s]
        xa, _, ia, _ = full_a[s]
        inv = np.empty(ia.max() + 1, dtype=np.int64)
        inv[ia] = np.arange(len(ia))
        sel = np.all((xb >= lo - 4) & (xb < hi + 4), axis=1)
        for row_b, row_a in zip(xb[sel], xa[inv[ib[sel]]]):
            O.deposit_rho(p, rho0, 0.0, qs[s], row_b)
            O.deposit_rho(p, rho1, 0.0, qs[s], row_a)
    div = ((J[0] - np.roll(J[0], 1, axis=2)) + (J[1] - np.roll(J[1], 1, axis=1)) + (J[2] - np.roll(J[2], 1, axis=0)))
    res = (rho1[0] - rho0[0] + div)[lo + 2:hi - 2, lo + 2:hi - 2, lo + 2:hi - 2]
    jref = w.units.q * w.c * w.units.n0
    assert np.abs(res).max() <= 1e-5 * jref, np.abs(res).max() / jref


@pytest.mark.gpu
def test_shear3d_256_sampled_particles():
    w = W.SHEAR_3D_FP32
    box = W.setup_box(w, device=0, seed=0)
    try:
        errs = follow_sample(w, box, 1000003, 1)
    finally:
        box.close()
    assert errs["u"] <= 1e-6 and errs["x"] <= 2e-6, errs


@pytest.mark.gpu
@pytest.mark.parametrize("side", [16, 32])
def test_leaky2d_2048_sampled_particles_and_escapes(side):
    # 32 x 32 tiles with launch variant 2: the shape and variant the bench's
    # tile autotuner keeps at this size
    w = W.LEAKY_2D_FP32
    box = W.setup_box(w, device=0, seed=0)
    try:
        box.set_tile(side)
        P.pic_set_kernel_variant(box.h, 2)
        assert box.tile() == (side, side, 1)
        d0 = box.diagnostics()
        errs = follow_sample(w, box, 10007, 1)
        d1 = box.diagnostics()
    finally:
        box.close()
    # reinjected momenta agree too, so every escape decision in the sample matched
    assert errs["u"] <= 1e-6 and errs["x"] <= 2e-6, errs
    assert errs["escaped"] > 0
    p = 1.0 / (w.t_esc_Lc * w.n[0] / w.c)
    total = d1.escaped_total - d0.escaped_total
    N = w.n_particles * 2  # two steps
    assert abs(total - N * p) < 6 * np.sqrt(N * p)

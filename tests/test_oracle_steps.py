"""Pins of the oracle's whole step (no GPU): invariants and reductions of the
three box methods (Secs. 2.2, 3.2, 4.1) on small synthetic plasmas."""
import math

import numpy as np
import pytest

import oracle as O

C = 0.45


def plasma(n, ppc, seed, uth=0.1, q=0.05):
    """Two species of opposite charge, uniform in the box, Gaussian momenta."""
    r = np.random.default_rng(seed)
    ncell = n[0] * n[1] * n[2]
    sp = []
    for s, sign in enumerate((-1.0, 1.0)):
        N = ncell * ppc
        x = r.uniform(0, 1, (N, 3)) * np.array(n, dtype=float)
        u = r.normal(0, uth, (N, 3))
        sp.append({"q": sign * q, "m": 1.0, "x": x, "u": u, "id": np.arange(N) + s * N})
    return sp


def div_node(F):
    return ((F[0] - np.roll(F[0], 1, axis=2)) + (F[1] - np.roll(F[1], 1, axis=1))
            + (F[2] - np.roll(F[2], 1, axis=0)))


def rho_nodes(p, st):
    return O.rho_of(p, [(d["q"], d["x"]) for d in st.species])


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("n", [(6, 5, 4), (8, 1, 6)])
def test_gauss_law_preserved_by_full_steps(order, n):
    """div E - 4 pi rho stays constant: the charge-conserving deposit and the
    Yee update together (standard PIC, and the leaky box, Sec. 4.1)."""
    p = O.make_params(*n, C, order=order)
    r = np.random.default_rng(1)
    E = r.normal(0, 0.01, (3, n[2], n[1], n[0]))
    B = r.normal(0, 0.05, (3, n[2], n[1], n[0]))
    st = O.State(p, E, B, plasma(n, 4, 2))
    g0 = div_node(st.E) - 4 * math.pi * rho_nodes(p, st)
    st.step(5)
    g1 = div_node(st.E) - 4 * math.pi * rho_nodes(p, st)
    assert np.abs(g1 - g0).max() < 1e-12


def test_expanding_box_with_zero_rate_is_standard_pic():
    n = (6, 5, 4)
    r = np.random.default_rng(3)
    E = r.normal(0, 0.01, (3, 4, 5, 6))
    B = r.normal(0, 0.05, (3, 4, 5, 6))
    a = O.State(O.make_params(*n, C, order=2), E, B, plasma(n, 3, 4))
    b = O.State(O.make_params(*n, C, order=2, box=O.BOX_EXPAND, rate=(0, 0, 0)), E, B, plasma(n, 3, 4))
    a.step(3)
    b.step(3)
    np.testing.assert_allclose(b.E, a.E, atol=1e-15)
    np.testing.assert_allclose(b.B, a.B, atol=1e-15)
    for sa, sb in zip(a.species, b.species):
        np.testing.assert_allclose(sb["x"], sa["x"], atol=1e-13)
        np.testing.assert_allclose(sb["u"], sa["u"], atol=1e-15)


def test_shearing_box_particle_phase_reduces_to_standard_pic():
    """With Omega0 = 0 the shearing-box push, position update and (advected)
    current equal the standard ones; only the field solver differs."""
    n = (6, 5, 4)
    r = np.random.default_rng(5)
    E = r.normal(0, 0.01, (3, 4, 5, 6))
    B = r.normal(0, 0.05, (3, 4, 5, 6))
    a = O.State(O.make_params(*n, C, order=1), E, B, plasma(n, 3, 6))
    b = O.State(O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=1.5, Omega0=0.0), E, B, plasma(n, 3, 6))
    a.step(1)
    b.step(1)
    np.testing.assert_allclose(b.J, a.J, atol=1e-16)
    for sa, sb in zip(a.species, b.species):
        np.testing.assert_allclose(sb["x"], sa["x"], atol=1e-13)
        np.testing.assert_allclose(sb["u"], sa["u"], atol=1e-16)


def test_shearing_box_particle_at_rest_rides_the_shear_flow():
    """u' = 0 and no fields: the particle stays at rest in the shearing frame
    and its lab position moves with v_s = -s Omega0 x e_y (Sec. 2.1)."""
    n = (16, 32, 1)
    s, Om = 1.5, 0.01
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=s, Omega0=Om)
    x0 = np.array([[12.25, 20.0, 0.5], [3.5, 5.0, 0.5]])
    sp = [{"q": 1e-9, "m": 1.0, "x": x0, "u": np.zeros((2, 3))}]
    st = O.State(p, np.zeros((3, 1, 32, 16)), np.zeros((3, 1, 32, 16)), sp)
    st.step(10)
    xc = x0[:, 0] - 8
    want_y = np.mod(x0[:, 1] - s * Om * xc * 10, 32)
    np.testing.assert_allclose(st.species[0]["x"][:, 1], want_y, atol=1e-10)
    np.testing.assert_allclose(st.species[0]["x"][:, 0], x0[:, 0], atol=1e-12)


def test_shearing_box_boundary_crossing_shifts_y():
    """A particle leaving through x_o re-enters at x_i with y + Dy_s(t^{n+1}),
    and through x_i with y - Dy_s, with u' unchanged (the particle counterpart
    of X(x_i, y) = X(x_o, y - Dy_s))."""
    n = (8, 20, 1)
    s, Om = 1.5, 0.003
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=s, Omega0=Om)
    step0 = 40
    u = np.array([[0.3, 0.0, 0.0], [-0.3, 0.0, 0.0]])
    x0 = np.array([[7.9, 10.0, 0.5], [0.1, 10.0, 0.5]])
    sp = [{"q": 1e-12, "m": 1.0, "x": x0, "u": u}]
    st = O.State(p, np.zeros((3, 1, 20, 8)), np.zeros((3, 1, 20, 8)), sp, step=step0)
    st.step(1)
    dys = O.shear_shift(p, step0 + 1.0)
    uu = st.species[0]["u"]
    g = np.sqrt(1 + (uu**2).sum(axis=1) / C**2)
    xp = x0[:, 0] + uu[:, 0] / g
    xc0 = x0[:, 0] - 4
    y_sh = x0[:, 1] + uu[:, 1] / g - s * Om * ((xp - 4) + xc0) / 2
    got = st.species[0]["x"]
    assert got[0, 0] == pytest.approx(xp[0] - 8, abs=1e-12)
    assert got[1, 0] == pytest.approx(xp[1] + 8, abs=1e-12)
    assert got[0, 1] == pytest.approx(np.mod(y_sh[0] + dys, 20), abs=1e-10)
    assert got[1, 1] == pytest.approx(np.mod(y_sh[1] - dys, 20), abs=1e-10)


def test_leaky_displacement_escape_is_ballistic_exact():
    """E = B = 0: a particle of velocity v escapes at the first step n with
    n |v_x| dt >= l_esc; it is reinjected at the same position with Dr = 0."""
    n = (8, 8, 1)
    v = 0.2
    u = v / math.sqrt(1 - (v / C) ** 2)
    g = math.sqrt(1 + (u / C) ** 2)
    vstep = u / g
    l_esc = 2.3
    p = O.make_params(*n, C, order=1, box=O.BOX_LEAKY, esc_mode=O.ESC_DISPLACEMENT,
                      l_esc=l_esc, theta_inj=0.1, seed=9)
    sp = [{"q": 1e-12, "m": 1.0, "x": np.array([[1.0, 4.0, 0.5]]), "u": np.array([[u, 0.0, 0.0]])}]
    st = O.State(p, np.zeros((3, 1, 8, 8)), np.zeros((3, 1, 8, 8)), sp)
    first = math.ceil(l_esc / vstep - 1e-12)
    for k in range(1, first + 1):
        x_before = st.species[0]["x"].copy()
        info = st.step(1)
        if k < first:
            assert info["escaped"] == 0
            assert st.species[0]["dr"][0, 0] == pytest.approx(k * vstep, rel=1e-13)
        else:
            assert info["escaped"] == 1
            assert np.all(st.species[0]["dr"][0] == 0.0)
            np.testing.assert_allclose(st.species[0]["x"][0, 0], np.mod(x_before[0, 0] + vstep, 8), atol=1e-13)
            assert not np.allclose(st.species[0]["u"][0], [u, 0, 0])


def test_leaky_probabilistic_survival_is_binomial():
    """Probabilistic escape at p = dt / t_esc per step: the fraction of
    particles never reinjected after n steps is (1 - p)^n ~ exp(-t/t_esc);
    checked at 5 sigma.  Particles start at rest without fields, so a particle
    has been reinjected iff its momentum is non-zero (uncharged test
    particles, so no field ever acts on them)."""
    n = (4, 4, 1)
    N = 8000
    p_esc = 0.02
    p = O.make_params(*n, C, order=1, box=O.BOX_LEAKY, esc_mode=O.ESC_PROBABILISTIC,
                      p_esc=p_esc, theta_inj=0.2, seed=5)
    r = np.random.default_rng(0)
    sp = [{"q": 0.0, "m": 1.0, "x": r.uniform(0, 4, (N, 3)) * [1, 1, 0.25], "u": np.zeros((N, 3))}]
    st = O.State(p, np.zeros((3, 1, 4, 4)), np.zeros((3, 1, 4, 4)), sp)
    steps = 40
    st.step(steps)
    surv = np.all(st.species[0]["u"] == 0.0, axis=1).sum()
    pr = (1 - p_esc) ** steps
    assert abs(surv - N * pr) < 5 * math.sqrt(N * pr * (1 - pr))


OTHER_BOXES = [
    dict(box=O.BOX_SHEAR, s=1.5, Omega0=3e-3),
    dict(box=O.BOX_EXPAND, rate=(0.0, 1e-3, 2e-3)),
    dict(box=O.BOX_SHEAR_EXPAND, s=1.2, Omega0=2e-3, rate=(1e-3, 2e-3, 5e-4)),
]


@pytest.mark.parametrize("kw", OTHER_BOXES, ids=["shear", "expand", "shear_expand"])
def test_probabilistic_escape_in_other_boxes_follows_the_move(kw):
    """The leaky box's probabilistic escape combined with the shearing,
    expanding and combined boxes (Sec. 5): it acts at the end of the step.
    With p = 1 every particle escapes: its position and the step's current
    and fields are those of the step without escape (the move and deposit
    came first), and its momentum is the Maxwell-Juettner draw keyed on (id,
    seed, step).  With p = 0 nothing changes."""
    n = (6, 5, 4)
    p_none = O.make_params(*n, C, order=2, seed=4, **kw)
    sp = plasma(n, 3, seed=2, uth=0.15)
    r = np.random.default_rng(1)
    E = r.normal(0, 0.01, (3, n[2], n[1], n[0]))
    B = r.normal(0, 0.01, (3, n[2], n[1], n[0])) + np.array([0, 0, 0.2])[:, None, None, None]
    ref = O.State(p_none, E, B, sp, step=7)
    ref.step(1)
    for p_esc in (0.0, 1.0):
        p = O.make_params(*n, C, order=2, seed=4, esc_mode=O.ESC_PROBABILISTIC, p_esc=p_esc, theta_inj=0.3, **kw)
        st = O.State(p, E, B, sp, step=7)
        info = st.step(1)
        for a, b in zip(st.species, ref.species):
            assert np.array_equal(a["x"], b["x"])
            if p_esc == 0.0:
                assert np.array_equal(a["u"], b["u"])
            else:
                want = np.array([O.sample_mj(int(i), 4, 7, 0.3, C)[0] for i in a["id"]])
                np.testing.assert_array_equal(a["u"], want)
        assert np.array_equal(st.E, ref.E) and np.array_equal(st.B, ref.B) and np.array_equal(st.J, ref.J)
        assert info["escaped"] == (0 if p_esc == 0.0 else sum(len(d["id"]) for d in sp))


@pytest.mark.parametrize("kw", OTHER_BOXES, ids=["shear", "expand", "shear_expand"])
def test_probabilistic_escape_in_other_boxes_is_binomial(kw):
    """Survival of uncharged test particles under escape at p per step, in
    the shearing, expanding and combined boxes: a particle never reinjected
    has exactly the momentum of the same particle stepped without escape;
    their number after n steps is binomial(N, (1 - p)^n), checked at 5
    sigma."""
    n = (4, 4, 3)
    N = 6000
    p_esc = 0.03
    r = np.random.default_rng(3)
    sp = [{"q": 0.0, "m": 1.0, "x": r.uniform(0, 1, (N, 3)) * np.array(n, dtype=float),
           "u": r.normal(0, 0.1, (N, 3)), "id": np.arange(N)}]
    z = np.zeros((3, n[2], n[1], n[0]))
    steps = 30
    ref = O.State(O.make_params(*n, C, order=1, seed=8, **kw), z, z, sp)
    ref.step(steps)
    st = O.State(O.make_params(*n, C, order=1, seed=8, esc_mode=O.ESC_PROBABILISTIC, p_esc=p_esc, theta_inj=0.2,
                               **kw), z, z, sp)
    st.step(steps)
    surv = np.all(st.species[0]["u"] == ref.species[0]["u"], axis=1).sum()
    pr = (1 - p_esc) ** steps
    assert abs(surv - N * pr) < 5 * math.sqrt(N * pr * (1 - pr))


def test_threaded_step_equals_the_plain_loop():
    """The timed CPU baseline runs the oracle's particle loop on several
    threads (per-thread currents added in thread order): the same step as the
    plain loop up to the rounding order of the current sums."""
    from paper_2602_15939_gb300 import workloads as W

    n = (8, 8, 8)
    sp = W.uniform_plasma(n, 4, seed=3, uth=0.2, q=0.05)
    E, B = W.random_fields(n, 4, b0=(0.0, 0.0, 0.2))
    p = O.make_params(*n, 0.45, order=2, box=O.BOX_SHEAR, s=1.5, Omega0=3e-3)
    out = []
    try:
        for th in (1, 3):
            O.set_threads(th)
            st = O.State(p, E, B, sp, step=5)
            info = st.step(2)
            out.append((st, info))
    finally:
        O.set_threads(1)
    (a, ia), (b, ib) = out
    assert ia == ib
    for da, db in zip(a.species, b.species):
        dx = da["x"] - db["x"]
        dx -= np.asarray(n, dtype=float) * np.round(dx / np.asarray(n, dtype=float))
        assert np.abs(dx).max() < 1e-12
        np.testing.assert_allclose(da["u"], db["u"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(a.J, b.J, rtol=0, atol=1e-14 * np.abs(a.J).max())
    np.testing.assert_allclose(a.E, b.E, rtol=0, atol=1e-14 * np.abs(a.E).max())


@pytest.mark.parametrize("box", [O.BOX_SHEAR, O.BOX_SHEAR_EXPAND])
def test_superluminal_counter_counts_the_shear_flow(box):
    """Sec. 2.1: particles move with the effective velocity u'/gamma' + v_s,
    v_s = -s Omega0 x e_y, which can exceed c far from the box centre.  A
    particle at rest in the shearing frame with no fields stays at rest (every
    push term is proportional to u' or E), so the count over one step is the
    number of particles with s Omega0 |x - nx/2| >= c, x the physical radial
    coordinate: l_1(t^n) times the expanding coordinate in the combined box."""
    n = (16, 4, 4)
    s, Om = 1.5, 0.05
    step0, rate = 10, 0.02
    kw = dict(box=box, s=s, Omega0=Om)
    l1 = 1.0
    if box == O.BOX_SHEAR_EXPAND:
        kw["rate"] = (rate, 0.0, 0.0)
        l1 = math.exp(rate * step0)
    p = O.make_params(*n, C, order=1, **kw)
    xi = np.arange(n[0]) + 0.5                  # one particle per x column
    N = xi.size
    x = np.stack([xi, np.full(N, 1.5), np.full(N, 2.5)], axis=1)
    sp = [{"q": 0.05, "m": 1.0, "x": x, "u": np.zeros((N, 3)), "id": np.arange(N)}]
    z = np.zeros((3, n[2], n[1], n[0]))
    st = O.State(p, z, z, sp, step=step0)
    info = st.step(1)
    speed = s * Om * np.abs(l1 * (xi - n[0] / 2))  # |v_s| of each particle
    want = int((speed >= C).sum())
    assert 0 < want < N and np.abs(speed - C).min() > 0.01  # some, not all, and no ties
    assert info["superluminal"] == want
    np.testing.assert_array_equal(st.species[0]["u"], 0.0)


def _yee_curl(F, forward):
    """Yee curl of a [3][nz][ny][nx] periodic field: forward differences
    (E at B locations) or backward ones (B at E locations)."""
    d = (lambda A, ax: np.roll(A, -1, axis=ax) - A) if forward else (lambda A, ax: A - np.roll(A, 1, axis=ax))
    return np.stack([d(F[2], 1) - d(F[1], 0), d(F[0], 0) - d(F[2], 2), d(F[1], 2) - d(F[0], 1)])


def test_isotropic_expansion_is_yee_in_conformal_time():
    """Secs. 3.1-3.2 with L = l(t) I: the expanding-frame fields X' = ell L^-1 X
    = l^2 X obey the vacuum Maxwell equations with c / l in place of c (the
    conformal time of the expansion).  The transformed leapfrog must then be
    the textbook Yee leapfrog on E', B' with c / l at the level of each of its
    three half updates: t^n, t^{n+1/2}, t^{n+1}.  Two whole steps of an
    expanding box without particles, from step 7."""
    n = (6, 5, 4)
    rate, step0 = 0.05, 7
    p = O.make_params(*n, C, order=1, box=O.BOX_EXPAND, rate=(rate, rate, rate))
    r = np.random.default_rng(12)
    E = r.normal(0, 0.1, (3, n[2], n[1], n[0]))
    B = r.normal(0, 0.1, (3, n[2], n[1], n[0]))
    st = O.State(p, E, B, [], step=step0)
    st.step(2)
    lv = lambda t: math.exp(rate * t)
    Ep, Bp = lv(step0) ** 2 * E, lv(step0) ** 2 * B
    for t in (step0, step0 + 1):
        Bp = Bp - C / (2 * lv(t)) * _yee_curl(Ep, True)
        Ep = Ep + C / lv(t + 0.5) * _yee_curl(Bp, False)
        Bp = Bp - C / (2 * lv(t + 1)) * _yee_curl(Ep, True)
    l2 = lv(step0 + 2) ** 2
    np.testing.assert_allclose(st.E, Ep / l2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(st.B, Bp / l2, rtol=0, atol=1e-14)


def test_combined_box_current_advection_integer_shift_is_a_roll():
    """The combined box advects the collected current along xi_y by
    v_{s,y} dt / (2 l_2) = -s Omega0 (l_1/l_2)(xi_x - nx/2) / 2, with l_1/l_2
    at t^{n+1/2}.  Choosing s Omega0 so that this is exactly one cell for the
    J_y column two cells right of the centre makes that column an exact roll
    (and the mirror column the opposite roll, the centre column unmoved);
    l_1/l_2 taken at another time level gives a fractional shift instead."""
    n = (8, 8, 1)
    t, r0, r1 = 4.0, 0.03, -0.02
    vf = math.exp((r0 - r1) * (t + 0.5))
    p = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=1.0, Omega0=1.0 / vf, rate=(r0, r1, 0.0))
    r = np.random.default_rng(4)
    J = r.normal(size=(3, n[2], n[1], n[0]))
    J0 = J.copy()
    O.sxe_advect_current(p, J, t)
    # J_y sits at x = i: the shift of column i is -(i - 4) / 2 * s Omega0 vf = -(i - 4) / 2
    np.testing.assert_allclose(J[1, :, :, 6], np.roll(J0[1, :, :, 6], -1, axis=1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(J[1, :, :, 2], np.roll(J0[1, :, :, 2], 1, axis=1), rtol=0, atol=1e-14)
    np.testing.assert_array_equal(J[1, :, :, 4], J0[1, :, :, 4])


@pytest.mark.parametrize("dims", [2, 3])
def test_displacement_rule_watches_each_axis(dims):
    """Sec. 4.1: a particle escapes once its displacement since injection
    reaches l_esc along a watched axis: x and y in 2D, x, y and z in 3D.  With
    no fields the momenta stay put, so particles moving along one axis at
    0.25 cells per step have covered 2.0 cells after 8 steps and 2.25 after 9:
    with l_esc = 2.1 the x and y movers (and in 3D the z mover) escape on the
    ninth step, a particle at rest never, and escape resets the displacement
    and replaces the momentum."""
    n = (16, 16, 16)
    v = 0.25
    u0 = v / math.sqrt(1 - (v / C) ** 2)
    u = np.zeros((4, 3))
    u[0, 0], u[1, 1], u[2, 2] = u0, -u0, u0
    x = np.full((4, 3), 8.3)
    sp = [{"q": 0.0, "m": 1.0, "x": x, "u": u, "id": np.arange(4)}]  # uncharged: no fields arise
    z = np.zeros((3, n[2], n[1], n[0]))
    p = O.make_params(*n, C, box=O.BOX_LEAKY, esc_mode=O.ESC_DISPLACEMENT, esc_dims=dims, l_esc=2.1,
                      theta_inj=0.1, seed=9)
    st = O.State(p, z, z, sp)
    counts = [st.step(1)["escaped"] for _ in range(9)]
    movers = 3 if dims == 3 else 2
    assert counts == [0] * 8 + [movers]
    d = st.species[0]
    gone = [0, 1, 2][:movers]
    kept = [q for q in range(4) if q not in gone]
    np.testing.assert_array_equal(d["dr"][gone], 0.0)
    assert np.all(np.any(d["u"][gone] != u[gone], axis=1))
    np.testing.assert_array_equal(d["u"][kept], u[kept])


@pytest.mark.parametrize("box", [O.BOX_LEAKY, O.BOX_SHEAR, O.BOX_EXPAND, O.BOX_SHEAR_EXPAND])
def test_probabilistic_escape_uses_the_draws_of_the_step_taken(box):
    """Sec. 4.1 with the probabilistic rule: in the step n -> n+1 a particle
    escapes when its escape draw keyed on step n says so, and its momentum is
    replaced by the reinjection sample keyed on the same step (both draws are
    pinned above).  Uncharged particles in zero fields keep their momenta
    otherwise (the shearing and expanding pushes leave u = 0 at rest)."""
    n = (8, 8, 8)
    N, step0, p_esc, theta, seed = 400, 6, 0.3, 0.2, 21
    kw = {}
    if box in (O.BOX_SHEAR, O.BOX_SHEAR_EXPAND):
        kw.update(s=1.5, Omega0=1e-3)
    if box in (O.BOX_EXPAND, O.BOX_SHEAR_EXPAND):
        kw.update(rate=(0.01, 0.0, -0.01))
    p = O.make_params(*n, C, box=box, esc_mode=O.ESC_PROBABILISTIC, p_esc=p_esc, theta_inj=theta, seed=seed, **kw)
    r = np.random.default_rng(2)
    x = r.uniform(0, 8, (N, 3))
    ids = np.arange(N) * 7 + 3
    sp = [{"q": 0.0, "m": 1.0, "x": x, "u": np.zeros((N, 3)), "id": ids}]
    z = np.zeros((3, n[2], n[1], n[0]))
    st = O.State(p, z, z, sp, step=step0)
    info = st.step(1)
    esc = np.array([O.escape_draw(int(i), seed, step0, p_esc) for i in ids])
    assert 0 < esc.sum() < N and info["escaped"] == esc.sum()
    want = np.zeros((N, 3))
    for q in np.flatnonzero(esc):
        want[q] = O.sample_mj(int(ids[q]), seed, step0, theta, C)[0]
    np.testing.assert_array_equal(st.species[0]["u"], want)


def test_combined_box_pushes_with_the_physical_radial_coordinate():
    """The combined box carries xi = L^-1 x (Sec. 3.1), but the shear terms of
    the push (Sec. 2.2: a2 = s Omega0 x / c) take the physical distance from
    the box centre, x = l_1(t^n) (xi_x - nx/2).  In uniform fields the gather
    returns the fields themselves, so one step's momentum is the pinned
    combined push at that coordinate."""
    n = (16, 8, 8)
    rate, step0, s, Om = (0.05, 0.01, -0.02), 10, 1.5, 0.01
    p = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=s, Omega0=Om, rate=rate)
    Eu, Bu = np.array([0.03, -0.05, 0.02]), np.array([0.1, 0.2, -0.3])
    E = np.broadcast_to(Eu[:, None, None, None], (3, n[2], n[1], n[0])).copy()
    B = np.broadcast_to(Bu[:, None, None, None], (3, n[2], n[1], n[0])).copy()
    x0 = np.array([[13.2, 4.1, 3.7], [2.6, 1.5, 6.2]])
    u0 = np.array([[0.1, 0.2, -0.05], [-0.15, 0.05, 0.1]])
    sp = [{"q": 0.05, "m": 1.0, "x": x0, "u": u0, "id": np.arange(2)}]
    st = O.State(p, E, B, sp, step=step0)
    st.step(1)
    l1 = math.exp(rate[0] * step0)
    Lam = [-0.5 * r for r in rate]
    for q in range(2):
        want, _ = O.push_sxe(0.05, 1.0, C, s, Om, l1 * (x0[q, 0] - n[0] / 2), Lam, Eu, Bu, u0[q])
        np.testing.assert_allclose(st.species[0]["u"][q], want, rtol=1e-13, atol=1e-16)

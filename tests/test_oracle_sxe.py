"""Pins of the oracle's combined shearing + expanding box (the combination the
paper leaves for future work, Sec. 5): the KSB-OA system of Sec. 2 written in
the expanding coordinates xi = L^{-1} x of Sec. 3.  Each part is fixed by
something other than itself: its reductions to the two pinned boxes, a closed
form of the discrete push, quadrature of the shear shift, exact uniform-field
evolutions, and the chain rule applied to the continuum shearing-box
equations."""
import math

import numpy as np
import pytest

import oracle as O

C = 0.45
E_STAG = np.array([[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5]])
B_STAG = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])


def _rng_vec(r, scale):
    return r.normal(size=3) * scale


# ---- push -----------------------------------------------------------------------------

def test_push_without_expansion_is_the_shearing_box_push():
    """Lambda = 0: the combined discrete equation is Sec. 2.2's, solved there
    by the closed form (Sherman-Morrison on the Boris operator) and here by
    elimination: the two agree to round-off, gbar included."""
    r = np.random.default_rng(1)
    for _ in range(200):
        E, B, u = _rng_vec(r, 0.05), _rng_vec(r, 0.3), _rng_vec(r, 0.3)
        xc, s, Om = r.uniform(-20, 20), r.uniform(0.5, 1.8), r.uniform(1e-4, 5e-3)
        q = r.choice([-0.05, 0.05])
        u1, g1 = O.push_ksb(q, 1.0, C, s, Om, xc, E, B, u)
        u2, g2 = O.push_sxe(q, 1.0, C, s, Om, xc, (0.0, 0.0, 0.0), E, B, u)
        np.testing.assert_allclose(u2, u1, rtol=0, atol=2e-15 * np.abs(u1).max())
        assert g2 == pytest.approx(g1, rel=1e-15)


def test_push_without_shear_is_the_expanding_box_push():
    """Omega0 = s = 0: the expanding-box equation of Sec. 3.2, equal to its
    direct solve for any diagonal Lambda and to the printed closed form for an
    isotropic one."""
    r = np.random.default_rng(2)
    for k in range(200):
        E, B, u = _rng_vec(r, 0.05), _rng_vec(r, 0.3), _rng_vec(r, 0.3)
        lam = -0.5 * r.uniform(0, 2e-2, 3) if k % 2 else -0.5 * np.full(3, r.uniform(0, 2e-2))
        q = r.choice([-0.05, 0.05])
        u_keb = O.push_keb(q, 1.0, C, lam, E, B, u, exact=True)
        u_sxe, _ = O.push_sxe(q, 1.0, C, 0.0, 0.0, 7.0, lam, E, B, u)
        np.testing.assert_allclose(u_sxe, u_keb, rtol=0, atol=2e-15 * np.abs(u_keb).max())
        if k % 2 == 0:
            u_cf = O.push_keb(q, 1.0, C, lam, E, B, u, exact=False)
            np.testing.assert_allclose(u_sxe, u_cf, rtol=0, atol=4e-15 * np.abs(u_cf).max())


def test_epicycles_in_an_isotropically_expanding_box():
    """E = B = 0, isotropic Lambda = lam: the (u_x, u_y) system is
    ((1 - lam) I - K) u+ = ((1 + lam) I + K) u- with K the epicycle generator
    (eigenvalues +-i theta, theta = kappa dt / 2, kappa^2 = 2 (2 - s) Omega0^2).
    So each step turns the epicycle phase by atan(theta/(1+lam)) +
    atan(theta/(1-lam)) and multiplies Q = (2-s) u_x^2 + 2 u_y^2 by
    ((1+lam)^2 + theta^2) / ((1-lam)^2 + theta^2); u_z scales by
    (1+lam)/(1-lam)."""
    s, Om, rate = 1.5, 2e-2, 3e-3
    lam = -0.5 * rate
    theta = math.sqrt(2 * (2 - s)) * Om / 2
    u = np.array([0.1, -0.05, 0.07])
    u0 = u.copy()
    nsteps = 300
    for _ in range(nsteps):
        u, _ = O.push_sxe(0.0, 1.0, C, s, Om, 3.0, (lam, lam, lam), (0, 0, 0), (0, 0, 0), u)
    Q = lambda v: (2 - s) * v[0] ** 2 + 2 * v[1] ** 2
    rq = ((1 + lam) ** 2 + theta**2) / ((1 - lam) ** 2 + theta**2)
    assert Q(u) == pytest.approx(Q(u0) * rq**nsteps, rel=1e-12)
    assert u[2] == pytest.approx(u0[2] * ((1 + lam) / (1 - lam)) ** nsteps, rel=1e-12)
    ph = lambda v: math.atan2(math.sqrt(2) * v[1], math.sqrt(2 - s) * v[0])
    dphi = nsteps * (math.atan(theta / (1 + lam)) + math.atan(theta / (1 - lam)))
    turned = (ph(u0) - ph(u)) % (2 * math.pi)
    assert turned == pytest.approx(dphi % (2 * math.pi), abs=1e-11)


# ---- shear shift ----------------------------------------------------------------------------

def test_shear_shift_is_the_integral_of_the_face_velocity():
    """Dxi_s(t) = s Omega0 nx int_0^t l_1/l_2 dt' (mod ny): with l_1 = l_2 the
    shearing box's s Omega0 Lx t; otherwise the quadrature of
    exp((r_1 - r_2) t')."""
    from scipy.integrate import quad

    n = (16, 24, 8)
    s, Om = 1.5, 2e-3
    p_sh = O.make_params(*n, C, box=O.BOX_SHEAR, s=s, Omega0=Om)
    p_eq = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=s, Omega0=Om, rate=(1e-3, 1e-3, 1e-3))
    for t in (0.0, 3.5, 117.0, 2500.0):
        assert O.shear_shift(p_eq, t) == pytest.approx(O.shear_shift(p_sh, t), abs=1e-10)
    for r1, r2 in ((0.0, 1e-3), (2e-3, 0.0), (1e-4, 7e-4)):
        p = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=s, Omega0=Om, rate=(r1, r2, 0.0))
        for t in (1.0, 40.0, 900.0):
            I, _ = quad(lambda x: math.exp((r1 - r2) * x), 0.0, t, epsabs=1e-13, epsrel=1e-13)
            want = (s * Om * n[0] * I) % n[1]
            assert O.shear_shift(p, t) == pytest.approx(want, abs=1e-9)


# ---- fields ----------------------------------------------------------------------------------

def test_fields_without_expansion_are_the_shearing_box_solve():
    n = (8, 10, 6)
    r = np.random.default_rng(3)
    E, B, J = (r.normal(size=(3, 6, 10, 8)) for _ in range(3))
    kw = dict(s=1.5, Omega0=4e-3, fp_iters=4)
    p1 = O.make_params(*n, C, box=O.BOX_SHEAR, **kw)
    p4 = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, **kw)
    for t in (0.0, 37.0):
        FE1, FB1 = O.ksb_rhs(p1, E, B, J, t)
        FE4, FB4 = O.sxe_rhs(p4, E, B, J, t)
        np.testing.assert_array_equal(FE1, FE4)
        np.testing.assert_array_equal(FB1, FB4)
        E1, B1, E4, B4 = E.copy(), B.copy(), E.copy(), B.copy()
        O.ksb_field_solve(p1, E1, B1, J, t)
        O.sxe_field_solve(p4, E4, B4, J, t)
        np.testing.assert_array_equal(E1, E4)
        np.testing.assert_array_equal(B1, B4)
        J1, J4 = J.copy(), J.copy()
        O.ksb_advect_current(p1, J1)
        O.sxe_advect_current(p4, J4, t)
        np.testing.assert_array_equal(J1, J4)


def test_uniform_fields_scale_with_l_over_ell_and_wind_up():
    """Uniform fields, no current: curls and advection vanish, so
    X^ = ell L^{-1} X changes only through the shear term,
    dB^_y/dt = -s Omega0 (l_1/l_2) B^_x, which the implicit midpoint rule
    integrates exactly with l_1/l_2 at the midpoint; every other component
    keeps X^, i.e. X_i ~ l_i / ell (Sec. 3.1)."""
    n = (6, 6, 6)
    s, Om, rates = 1.5, 5e-3, (2e-3, 5e-4, 1e-3)
    p = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=s, Omega0=Om, rate=rates, fp_iters=4)
    E = np.zeros((3, 6, 6, 6))
    B = np.zeros_like(E)
    E0 = np.array([0.01, -0.02, 0.03])
    B0 = np.array([0.4, 0.1, 1.0])
    for c in range(3):
        E[c], B[c] = E0[c], B0[c]
    l = lambda t: np.exp(np.array(rates) * t)
    Eh = np.prod(l(0.0)) / l(0.0) * E0
    Bh = np.prod(l(0.0)) / l(0.0) * B0
    for step in range(5):
        t = float(step)
        O.sxe_field_solve(p, E, B, np.zeros_like(E), t)
        lh = l(t + 0.5)
        Bh = Bh.copy()
        Bh[1] -= s * Om * (lh[0] / lh[1]) * Bh[0]
        l1 = l(t + 1.0)
        for c in range(3):
            np.testing.assert_allclose(E[c], l1[c] / np.prod(l1) * Eh[c], rtol=1e-13, atol=0)
            np.testing.assert_allclose(B[c], l1[c] / np.prod(l1) * Bh[c], rtol=1e-13, atol=0)


def _fields_and_continuum_rhs(n, sO, rates, t, kvec):
    """Smooth expanding-frame fields X^ (periodic on the xi grid) and the
    right-hand sides the combined box must have: ell L^{-1} times the
    shearing-box right-hand sides of Sec. 2.1 evaluated, by the chain rule,
    on the physical fields X = L X^ / ell over x = L xi (d/dx_b = (1/l_b)
    d/dxi_b), with V = -s Omega0 x, x = l_1 (xi_x - nx/2)."""
    l = np.exp(np.array(rates) * t)
    ell = np.prod(l)
    kx, ky, kz = kvec
    ph = np.array([[0.3, 1.1, 2.0], [0.7, 0.2, 1.4], [1.9, 0.5, 0.9], [0.4, 0.8, 1.7], [1.2, 0.6, 0.1], [0.9, 1.5, 0.3]])

    def f(idx, x, y, z):
        return np.sin(kx * x + ph[idx, 0]) * np.cos(ky * y + ph[idx, 1]) * np.cos(kz * z + ph[idx, 2])

    def df(idx, x, y, z, ax):  # derivative along xi_ax
        s1, c1 = np.sin(kx * x + ph[idx, 0]), np.cos(kx * x + ph[idx, 0])
        s2, c2 = np.sin(ky * y + ph[idx, 1]), np.cos(ky * y + ph[idx, 1])
        s3, c3 = np.sin(kz * z + ph[idx, 2]), np.cos(kz * z + ph[idx, 2])
        return [kx * c1 * c2 * c3, -ky * s1 * s2 * c3, -kz * s1 * c2 * s3][ax]

    def grid(fn, stag):
        k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        return np.stack([fn(c, i + stag[c][0], j + stag[c][1], k + stag[c][2]) for c in range(3)])

    Eh = grid(lambda c, x, y, z: f(c, x, y, z), E_STAG)
    Bh = grid(lambda c, x, y, z: 0.7 * f(3 + c, x, y, z), B_STAG)

    # physical field X_a = l_a X^_a / ell and its physical derivatives
    dE = lambda a, b, x, y, z: l[a] / ell / l[b] * df(a, x, y, z, b)
    dB = lambda a, b, x, y, z: l[a] / ell / l[b] * 0.7 * df(3 + a, x, y, z, b)
    Bphys = lambda a, x, y, z: l[a] / ell * 0.7 * f(3 + a, x, y, z)
    V = lambda x: -sO * l[0] * (x - n[0] / 2)

    def curl(d, a, x, y, z):
        b, c = (a + 1) % 3, (a + 2) % 3
        return d(c, b, x, y, z) - d(b, c, x, y, z)

    def FE(c, x, y, z):
        v = V(x)
        adv = [v * dE(0, 1, x, y, z) - v * dE(1, 0, x, y, z),
               -v * (dE(0, 0, x, y, z) + dE(1, 1, x, y, z) + dE(2, 2, x, y, z)),
               v * dE(2, 1, x, y, z) - v * dE(1, 2, x, y, z)][c]
        return ell / l[c] * (C * curl(dB, c, x, y, z) + adv)

    def FB(c, x, y, z):
        out = -C * curl(dE, c, x, y, z) - V(x) * dB(c, 1, x, y, z)
        if c == 1:
            out = out - sO * Bphys(0, x, y, z)
        return ell / l[c] * out

    return Eh, Bh, grid(FE, E_STAG), grid(FB, B_STAG)


def test_rhs_is_the_shearing_box_rhs_in_expanding_coordinates():
    """On smooth fields the discrete right-hand sides approach ell L^{-1}
    times the shearing-box ones written through the coordinate change (at
    least first order under refinement, away from the x seam, Dy = 0 at
    t = 0 is not needed: the fields are periodic and the shift only matters
    across the seam, excluded); a misplaced factor l_a leaves an O(1) error."""
    rates = (2e-3, 5e-3, -1e-3)
    t = 60.0  # l of order 1.1-1.35 and anisotropic
    errs = []
    for N in (16, 32, 64):
        n = (N, N, N // 2)
        kvec = (2 * math.pi / N, 2 * math.pi * 2 / N, 2 * math.pi / (N // 2))
        sO = 0.2 / N
        p = O.make_params(*n, C, box=O.BOX_SHEAR_EXPAND, s=1.0, Omega0=sO, rate=rates)
        Eh, Bh, FEc, FBc = _fields_and_continuum_rhs(n, sO, rates, t, kvec)
        FE, FB = O.sxe_rhs(p, Eh, Bh, np.zeros_like(Eh), t)
        inner = slice(2, N - 2)
        err = max(np.abs(FE - FEc)[..., inner].max(), np.abs(FB - FBc)[..., inner].max())
        scale = max(np.abs(FEc).max(), np.abs(FBc).max())
        errs.append(err / scale)
    assert errs[-1] < 0.03
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6


# ---- whole steps --------------------------------------------------------------------------------

def _step_state(box, n, rates, s, Om, step0=11, keb_exact=0):
    from paper_2602_15939_gb300 import workloads as W

    sp = W.uniform_plasma(n, 3, seed=5, uth=0.15, q=0.05)
    E, B = W.random_fields(n, 6, b0=(0.0, 0.0, 0.2))
    p = O.make_params(*n, C, order=2, box=box, s=s, Omega0=Om, rate=rates, keb_exact=keb_exact)
    st = O.State(p, E, B, sp, step=step0)
    st.step(1)
    return st


def test_step_without_expansion_is_the_shearing_box_step():
    n = (8, 8, 8)
    a = _step_state(O.BOX_SHEAR, n, (0, 0, 0), 1.5, 3e-3)
    b = _step_state(O.BOX_SHEAR_EXPAND, n, (0, 0, 0), 1.5, 3e-3)
    for da, db in zip(a.species, b.species):
        np.testing.assert_allclose(db["u"], da["u"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(db["x"], da["x"], rtol=0, atol=1e-13)
    # the two pushes solve the same equation by different algorithms: positions
    # differ at round-off, and so do the currents they deposit
    np.testing.assert_allclose(b.J, a.J, rtol=0, atol=1e-12 * np.abs(a.J).max())
    np.testing.assert_allclose(b.E, a.E, rtol=0, atol=1e-12 * np.abs(a.E).max())


def test_particles_without_shear_move_like_the_expanding_box():
    """Omega0 = s = 0: push (exact variant), comoving move and deposit are the
    expanding box's, so particles and current after one step agree; only the
    field solve differs (implicit midpoint here, leapfrog there)."""
    n = (8, 8, 8)
    rates = (0.0, 2e-3, 1e-3)
    a = _step_state(O.BOX_EXPAND, n, rates, 0.0, 0.0, keb_exact=1)
    b = _step_state(O.BOX_SHEAR_EXPAND, n, rates, 0.0, 0.0)
    for da, db in zip(a.species, b.species):
        np.testing.assert_allclose(db["u"], da["u"], rtol=0, atol=2e-15)
        np.testing.assert_allclose(db["x"], da["x"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b.J, a.J, rtol=0, atol=1e-14 * np.abs(a.J).max())


def test_particles_at_rest_follow_the_shear_flow_in_xi():
    """u = 0 and no fields: a particle rides the shear flow, dxi_y/dt =
    v_{s,y}/l_2 = -s Omega0 (l_1/l_2)(xi_x - nx/2), taken at each step's
    midpoint; across the x faces it re-enters shifted by Dxi_s."""
    n = (8, 16, 4)
    s, Om, rates = 1.5, 2e-2, (1e-3, 3e-3, 0.0)
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR_EXPAND, s=s, Omega0=Om, rate=rates)
    x = np.array([[1.25, 3.0, 2.0], [6.5, 9.0, 1.0]])
    u = np.zeros_like(x)
    z = np.zeros((3, 4, 16, 8))
    want = x.copy()
    for step in range(40):
        x, u, _, _ = O.advance_particles(p, z, z, step, 0.0, 1.0, [0, 1], x, u)
        vf = math.exp((rates[0] - rates[1]) * (step + 0.5))
        want[:, 1] = (want[:, 1] - s * Om * vf * (want[:, 0] - n[0] / 2)) % n[1]
    np.testing.assert_allclose(x, want, atol=1e-11)
    assert np.all(u == 0)

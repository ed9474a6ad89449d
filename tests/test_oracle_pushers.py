"""Pins of the oracle's particle pushers against what the paper and the
mathematics fix (no GPU).  Each test is chosen so that a plausible slip in the
oracle (a dropped factor, a wrong sign, a transposed operand) fails it.

Paper sections: the Boris operator and the shearing-box push (Sec. 2.2),
the expanding-box push (Sec. 3.2).
"""
import math

import numpy as np
import pytest

import oracle as O

C = 0.45


def _rng(seed=1):
    return np.random.default_rng(seed)


# ---- P1: Boris in a pure magnetic field ------------------------------------

def test_boris_pure_B_rotation_angle_and_norm():
    """|u| is conserved and u turns by exactly 2 atan(|tau|) per step,
    tau = q dt B / (2 m c gamma): the closed form of the Boris rotation."""
    q, m = 0.7, 1.3
    B = np.array([0.2, -0.1, 0.35])
    u = np.cross(B, [1.0, 0.0, 0.0])  # perpendicular to B
    u *= 0.3 / np.linalg.norm(u)
    gamma = math.sqrt(1 + np.dot(u, u) / C**2)
    tau = q * np.linalg.norm(B) / (2 * m * C * gamma)
    expected = 2 * math.atan(tau)
    for _ in range(500):
        un = O.push_boris(q, m, C, [0, 0, 0], B, u)
        ang = math.atan2(np.linalg.norm(np.cross(u, un)), np.dot(u, un))
        assert ang == pytest.approx(expected, rel=1e-12)
        u = un
    assert np.linalg.norm(u) == pytest.approx(0.3, rel=1e-13)


# ---- P2: E x B drift ----------------------------------------------------------

def test_boris_ExB_drift():
    """Mean velocity over whole gyro-periods tends to c E x B / B^2."""
    q, m = 1.0, 1.0
    B0, E0 = 0.05, 0.0005
    E = np.array([E0, 0.0, 0.0])
    B = np.array([0.0, 0.0, B0])
    vd = C * np.cross(E, B) / B0**2  # = (0, -c E0/B0, 0)
    u = np.zeros(3)
    omega = q * B0 / (m * C)  # gyro-frequency per step (gamma ~ 1)
    period = 2 * math.pi / (2 * math.atan(omega / 2))  # steps per discrete gyration
    nper = 100
    nsteps = int(round(nper * period))
    x = np.zeros(3)
    for _ in range(nsteps):
        u = O.push_boris(q, m, C, E, B, u)
        g = math.sqrt(1 + np.dot(u, u) / C**2)
        x += u / g
    vmean = x / nsteps
    assert vmean[1] == pytest.approx(vd[1], rel=1e-3)
    assert abs(vmean[0]) < 2e-3 * abs(vd[1])


# ---- P3: shearing-box epicycle -------------------------------------------------

def test_ksb_epicycle_phase_and_invariant():
    """With E = B = 0 the shearing-box momentum equation reduces to
    du_x/dt = 2 Omega0 u_y, du_y/dt = -(2 - s) Omega0 u_x: epicycles with
    kappa^2 = 2 (2 - s) Omega0^2.  The discrete push is the implicit midpoint
    rule for that system, so (2-s) u_x^2 + 2 u_y^2 is conserved to round-off
    and the phase advances by exactly 2 atan(kappa dt / 2) per step."""
    s, Om = 1.5, 0.05
    kappa = math.sqrt(2 * (2 - s)) * Om
    u = np.array([0.1, 0.0, 0.03])
    inv0 = (2 - s) * u[0] ** 2 + 2 * u[1] ** 2

    def angle(v):
        return math.atan2(math.sqrt(2) * v[1], math.sqrt(2 - s) * v[0])

    total = 0.0
    for _ in range(1000):
        un, _ = O.push_ksb(1.0, 1.0, C, s, Om, 0.0, [0, 0, 0], [0, 0, 0], u)
        d = angle(u) - angle(un)  # rotates clockwise in (sqrt(2-s) ux, sqrt2 uy)
        d = (d + math.pi) % (2 * math.pi) - math.pi
        assert d == pytest.approx(2 * math.atan(kappa / 2), rel=1e-11)
        total += d
        u = un
    inv = (2 - s) * u[0] ** 2 + 2 * u[1] ** 2
    assert inv == pytest.approx(inv0, rel=1e-13)
    assert u[2] == pytest.approx(0.03, rel=1e-15)


# ---- P4: shearing-box closed form vs the defining linear system ------------------

def _ksb_direct(q, m, c, s, Om, xc, E, B, u):
    """Solve the discretised shearing-box momentum equation of Sec. 2.2,
    (I - T - S) u+ = (I + T + S) u-, T v = v x tt, by a library 3x3 solve."""
    E, B, u = map(np.asarray, (E, B, u))
    eps = q * E / (2 * m)
    um = u + eps
    a1 = s * Om / 2
    a2 = s * Om * xc / c
    gbar, _ = O.ksb_gamma_bar(c, a1, a2, um, eps)
    et = eps / (c * gbar)
    tt = q * B / (2 * m * c) / gbar + np.array([0, 0, Om])
    T = np.array([[0, tt[2], -tt[1]], [-tt[2], 0, tt[0]], [tt[1], -tt[0], 0]])
    S = np.zeros((3, 3))
    S[1] = [a1 + a2 * et[0], a2 * et[1], a2 * et[2]]
    I = np.eye(3)
    up = np.linalg.solve(I - T - S, (I + T + S) @ um)
    return up + eps


@pytest.mark.parametrize("seed", range(6))
def test_ksb_closed_form_equals_direct_solve(seed):
    r = _rng(seed)
    q, m = r.choice([-1.0, 1.0]) * 0.3, 1.0
    s, Om = 1.5, 0.02 * r.random() + 0.001
    xc = r.uniform(-30, 30)
    E, B = r.normal(0, 0.05, 3), r.normal(0, 0.3, 3)
    u = r.normal(0, 0.3, 3)
    got, _ = O.push_ksb(q, m, C, s, Om, xc, E, B, u)
    want = _ksb_direct(q, m, C, s, Om, xc, E, B, u)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.linalg.norm(want))


# ---- P5: reductions -------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_reductions_to_boris(seed):
    """Omega0 = 0 (S = 0) and Lambda = 0 both give back the Boris push."""
    r = _rng(100 + seed)
    q, m = -0.4, 1.0
    E, B, u = r.normal(0, 0.05, 3), r.normal(0, 0.3, 3), r.normal(0, 0.4, 3)
    ub = O.push_boris(q, m, C, E, B, u)
    uk, _ = O.push_ksb(q, m, C, 1.5, 0.0, 12.0, E, B, u)
    ue = O.push_keb(q, m, C, [0, 0, 0], E, B, u)
    ux = O.push_keb(q, m, C, [0, 0, 0], E, B, u, exact=True)
    np.testing.assert_allclose(uk, ub, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ue, ub, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ux, ub, rtol=0, atol=2e-15)


def test_ksb_boris_when_no_force_terms_except_shear_row_zero():
    """alpha1 = alpha2 = 0 gives gbar = gamma^- (the standard Boris factor)."""
    r = _rng(7)
    um, eps = r.normal(0, 0.4, 3), r.normal(0, 0.01, 3)
    g, res = O.ksb_gamma_bar(C, 0.0, 0.0, um, eps)
    assert g == pytest.approx(math.sqrt(1 + np.dot(um, um) / C**2), rel=1e-15)


# ---- P6: the gamma-bar cubic -----------------------------------------------------

def test_ksb_gamma_bar_root_and_small_omega_approximation():
    """gbar solves its defining relation to round-off, and the paper's
    small-Omega0 approximation is second-order accurate in Omega0."""
    r = _rng(3)
    um, eps = r.normal(0, 0.5, 3), r.normal(0, 0.05, 3)
    errs = []
    for Om in (1e-2, 5e-3, 2.5e-3):
        a1, a2 = 1.5 * Om / 2, 1.5 * Om * 40.0 / C
        g, res = O.ksb_gamma_bar(C, a1, a2, um, eps)
        assert res < 1e-15
        assert g >= 1.0
        gm = math.sqrt(1 + np.dot(um, um) / C**2)
        approx = gm + (a1 * um[0] * um[1] * gm + a2 * np.dot(um, eps) * um[1]) / (C * gm) ** 2
        errs.append(abs(g - approx))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


# ---- P7 / P8: expanding-box push ------------------------------------------------------

def test_keb_free_decay_exact_and_continuum():
    """E = B = 0: u_i^{n+1/2} = [(1 + L_ii)/(1 - L_ii)]^n u_i exactly; with
    Lambda = -(dt/2) r, the continuum law u_i ~ 1/l_i = exp(-r_i t) is met to
    O((r dt)^3) per step."""
    rate = np.array([0.0, 1e-2, 3e-2])
    Lam = -0.5 * rate
    u0 = np.array([0.2, -0.3, 0.1])
    u = u0.copy()
    n = 200
    for _ in range(n):
        u = O.push_keb(1.0, 1.0, C, Lam, [0, 0, 0], [0, 0, 0], u)
    fac = ((1 + Lam) / (1 - Lam)) ** n
    np.testing.assert_allclose(u, u0 * fac, rtol=1e-13)
    cont = u0 * np.exp(-rate * n)
    # per-step error (r^3/12) accumulated over n steps
    np.testing.assert_allclose(u, cont, rtol=n * (rate.max() ** 3) / 12 * 1.01 + 1e-15)
    assert u[0] == pytest.approx(u0[0], rel=1e-15)  # non-expanding axis untouched


@pytest.mark.parametrize("seed", range(4))
def test_keb_closed_form_isotropic_equals_exact_solve(seed):
    r = _rng(200 + seed)
    lam = -r.uniform(1e-4, 5e-2)
    E, B, u = r.normal(0, 0.05, 3), r.normal(0, 0.3, 3), r.normal(0, 0.4, 3)
    a = O.push_keb(0.5, 1.0, C, [lam] * 3, E, B, u)
    b = O.push_keb(0.5, 1.0, C, [lam] * 3, E, B, u, exact=True)
    np.testing.assert_allclose(a, b, rtol=0, atol=2e-15 * np.linalg.norm(b))


def test_keb_exact_mode_solves_the_defining_system():
    """The exact mode satisfies u+ - L u+ - u+ x tau = u- + L u- + u- x tau,
    with the gbar and tau of Sec. 3.2; the closed form differs only at
    O(Lambda tau) for anisotropic Lambda."""
    r = _rng(9)
    q, m = 0.5, 1.0
    Lam = np.array([0.0, -0.01, -0.01])
    E, B, u = r.normal(0, 0.05, 3), r.normal(0, 0.3, 3), r.normal(0, 0.4, 3)
    eps = q * E / (2 * m)
    um = u + eps
    gbar = math.sqrt(1 + np.dot((1 + Lam) * um, (1 + Lam) * um) / C**2)
    tau = q * B / (2 * gbar * m * C)
    up = O.push_keb(q, m, C, Lam, E, B, u, exact=True) - eps
    lhs = up - Lam * up - np.cross(up, tau)
    rhs = um + Lam * um + np.cross(um, tau)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-15)
    closed = O.push_keb(q, m, C, Lam, E, B, u)
    diff = np.linalg.norm(closed - (up + eps)) / np.linalg.norm(up)
    assert 1e-6 < diff < 2 * np.abs(Lam).max() * np.linalg.norm(tau)

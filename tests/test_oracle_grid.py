"""Pins of the oracle's grid operators (no GPU): gather, charge-conserving
deposit, shearing-periodic identification, field solvers.

Paper sections: standard PIC ingredients (Sec. 1), KSB-OA boundaries and
Maxwell solve (Secs. 2.1-2.2), KEB field transforms and solve (Secs. 3.1-3.2).
"""
import math

import numpy as np
import pytest

import oracle as O

C = 0.45
E_STAG = np.array([[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5]])
B_STAG = np.array([[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])


def grid_coords(n):
    """node coordinates of a (nz, ny, nx) grid, as broadcastable arrays"""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.astype(float), j.astype(float), k.astype(float)


def field_from(fn, n, stag):
    """sample fn(x, y, z, comp) at each component's staggered location"""
    i, j, k = grid_coords(n)
    F = np.zeros((3,) + i.shape)
    for c in range(3):
        F[c] = fn(i + stag[c][0], j + stag[c][1], k + stag[c][2], c)
    return F


# ---- gather ----------------------------------------------------------------------

@pytest.mark.parametrize("order", [1, 2])
def test_gather_reproduces_linear_fields(order):
    """B-spline shapes of order 1 and 2 reproduce linear functions exactly, so
    a linear field is gathered exactly at any interior point -- provided each
    component is sampled at its own staggered location."""
    n = (16, 12, 10)
    p = O.make_params(*n, C, order=order)
    a = np.array([[0.3, -0.2, 0.7, 0.1], [0.5, 0.4, -0.3, 0.2], [-0.6, 0.1, 0.2, 0.9]])
    lin = lambda x, y, z, c: a[c, 0] + a[c, 1] * x + a[c, 2] * y + a[c, 3] * z
    E = field_from(lin, n, E_STAG)
    B = field_from(lambda x, y, z, c: 2 * lin(x, y, z, c), n, B_STAG)
    r = np.random.default_rng(0)
    for _ in range(50):
        x = r.uniform([3, 3, 3], [12, 8, 6])
        Ep, Bp = O.gather(p, E, B, 0.0, x)
        want = a[:, 0] + a[:, 1] * x[0] + a[:, 2] * x[1] + a[:, 3] * x[2]
        np.testing.assert_allclose(Ep, want, atol=1e-12)
        np.testing.assert_allclose(Bp, 2 * want, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_gather_second_moment(order):
    """Gathering f = (x - x0)^2 returns the shape's second moment about the
    particle: w (1 - w) for linear (w the offset from the node), 1/4 for the
    quadratic spline (variance of three unit boxes)."""
    n = (20, 1, 1)
    p = O.make_params(*n, C, order=order)
    r = np.random.default_rng(1)
    for _ in range(20):
        xp = np.array([r.uniform(5, 14), r.random(), r.random()])
        sq = lambda x, y, z, c: (x - xp[0]) ** 2 if c == 1 else 0.0 * x
        E = field_from(sq, n, E_STAG)  # E_y sits on x-nodes
        Ep, _ = O.gather(p, E, np.zeros_like(E), 0.0, xp)
        w = xp[0] - math.floor(xp[0])
        want = w * (1 - w) if order == 1 else 0.25
        assert Ep[1] == pytest.approx(want, abs=1e-12)


# ---- deposit -----------------------------------------------------------------------

def divergence(J):
    """node divergence of a Yee current, periodic"""
    return ((J[0] - np.roll(J[0], 1, axis=2)) + (J[1] - np.roll(J[1], 1, axis=1))
            + (J[2] - np.roll(J[2], 1, axis=0)))


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("n", [(8, 7, 6), (9, 1, 8), (10, 9, 1)])
def test_deposit_charge_conservation(order, n):
    """(rho^{n+1} - rho^n) + div J = 0 in every cell, to round-off, for moves
    below one cell per axis, across the periodic boundaries; 2D runs use a
    one-cell ignorable axis."""
    p = O.make_params(*n, C, order=order)
    r = np.random.default_rng(2)
    J = np.zeros((3, n[2], n[1], n[0]))
    rho0 = np.zeros((1, n[2], n[1], n[0]))
    rho1 = np.zeros_like(rho0)
    for _ in range(40):
        x0 = r.uniform([0, 0, 0], n)
        x1 = x0 + r.uniform(-0.95, 0.95, 3)
        q = r.choice([-1.0, 1.0]) * r.uniform(0.5, 2)
        O.deposit_current(p, J, 0.0, q, x0, x1)
        O.deposit_rho(p, rho0, 0.0, q, x0)
        O.deposit_rho(p, rho1, 0.0, q, np.mod(x1, n))
    res = (rho1[0] - rho0[0]) + divergence(J)
    assert np.abs(res).max() < 1e-13


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_total_current(order):
    """Summed over the grid, J equals q times the displacement (q v dt)."""
    n = (8, 8, 8)
    p = O.make_params(*n, C, order=order)
    r = np.random.default_rng(3)
    for _ in range(10):
        J = np.zeros((3, 8, 8, 8))
        x0 = r.uniform(0, 8, 3)
        d = r.uniform(-0.9, 0.9, 3)
        O.deposit_current(p, J, 0.0, 1.7, x0, x0 + d)
        np.testing.assert_allclose(J.reshape(3, -1).sum(axis=1), 1.7 * d, atol=1e-14)


def test_deposit_order1_matches_villasenor_buneman():
    """For a move inside one cell the linear-shape deposit equals the
    Villasenor-Buneman charge-conserving current (the method the paper cites):
    J_x on the four x-edges of the cell is q dx [(1-yb)(1-zb) + dy dz/12],
    q dx [yb(1-zb) - dy dz/12], q dx [(1-yb) zb - dy dz/12],
    q dx [yb zb + dy dz/12], with yb, zb the midpoint offsets in the cell."""
    n = (6, 6, 6)
    p = O.make_params(*n, C, order=1)
    r = np.random.default_rng(4)
    for _ in range(20):
        cell = r.integers(1, 4, 3)
        a = r.uniform(0.05, 0.95, 3)
        b = r.uniform(0.05, 0.95, 3)
        x0, x1 = cell + a, cell + b
        J = np.zeros((3, 6, 6, 6))
        q = 0.8
        O.deposit_current(p, J, 0.0, q, x0, x1)
        d = b - a
        mid = (a + b) / 2
        i, j, k = cell
        for comp, (u, v) in ((0, (1, 2)), (1, (0, 2)), (2, (0, 1))):
            mu, mv = mid[u], mid[v]
            cross = d[u] * d[v] / 12
            want = q * d[comp] * np.array([(1 - mu) * (1 - mv) + cross, mu * (1 - mv) - cross,
                                           (1 - mu) * mv - cross, mu * mv + cross])
            idx = np.array([i, j, k])

            def at(du, dv):
                ix = idx.copy()
                ix[u] += du
                ix[v] += dv
                return J[comp, ix[2], ix[1], ix[0]]

            got = np.array([at(0, 0), at(1, 0), at(0, 1), at(1, 1)])
            np.testing.assert_allclose(got, want, atol=1e-15)
            assert abs(J[comp]).sum() == pytest.approx(abs(want).sum(), abs=1e-14)


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_1d_motion_fixed_by_continuity(order):
    """For motion along x only, continuity fixes J_x uniquely (it vanishes far
    from the particle): J_x(i+1/2) = -sum_{i'<=i} (rho1 - rho0)(i')."""
    n = (12, 5, 5)
    p = O.make_params(*n, C, order=order)
    x0 = np.array([5.3, 2.2, 2.7])
    x1 = x0 + np.array([0.7, 0.0, 0.0])
    J = np.zeros((3, 5, 5, 12))
    rho0 = np.zeros((1, 5, 5, 12))
    rho1 = np.zeros_like(rho0)
    O.deposit_current(p, J, 0.0, 1.0, x0, x1)
    O.deposit_rho(p, rho0, 0.0, 1.0, x0)
    O.deposit_rho(p, rho1, 0.0, 1.0, x1)
    want = -np.cumsum(rho1[0] - rho0[0], axis=2)
    np.testing.assert_allclose(J[0], want, atol=1e-15)
    assert np.abs(J[1]).max() == 0 and np.abs(J[2]).max() == 0


# ---- shearing-periodic identification -------------------------------------------

def test_shear_integer_shift_is_a_roll():
    """With Dy_s a whole number m of cells the ghost values across x are the
    interior values rolled by m in y (X(x_i, y) = X(x_o, y - Dy_s)); check via
    a particle gathered just past the outer edge."""
    n = (8, 10, 4)
    Om = 0.01
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=1.5, Omega0=Om)
    t = 3.0 / (1.5 * Om * n[0])  # Dy_s = 3 exactly
    assert O.shear_shift(p, t) == pytest.approx(3.0, abs=1e-12)
    r = np.random.default_rng(5)
    E = r.normal(size=(3, 4, 10, 8))
    B = r.normal(size=(3, 4, 10, 8))
    pp = O.make_params(*n, C, order=1)  # plain periodic
    for _ in range(10):
        x = np.array([r.uniform(7.6, 7.99), r.uniform(0, 10), r.uniform(0, 4)])
        Ep, Bp = O.gather(p, E, B, t, x)
        # equivalent: x beyond x_o maps to x - Lx with y + Dy_s ; here the stencil
        # straddles both, so compare with a periodic box whose x-ghost columns
        # carry the rolled values
        Er = E.copy(); Br = B.copy()
        big_E = np.concatenate([E, np.roll(E, -3, axis=2)], axis=3)
        big_B = np.concatenate([B, np.roll(B, -3, axis=2)], axis=3)
        pbig = O.make_params(16, 10, 4, C, order=1)
        Eb, Bb = O.gather(pbig, np.ascontiguousarray(big_E), np.ascontiguousarray(big_B), 0.0, x)
        np.testing.assert_allclose(Ep, Eb, atol=1e-14)
        np.testing.assert_allclose(Bp, Bb, atol=1e-14)
    del pp, Er, Br


def test_shear_fold_conserves_current_and_charge_for_integer_shift():
    n = (8, 10, 4)
    Om = 0.01
    p = O.make_params(*n, C, order=2, box=O.BOX_SHEAR, s=1.5, Omega0=Om)
    t = 2.0 / (1.5 * Om * n[0])  # Dy_s = 2
    r = np.random.default_rng(6)
    J = np.zeros((3, 4, 10, 8))
    rho0 = np.zeros((1, 4, 10, 8))
    rho1 = np.zeros_like(rho0)
    for _ in range(30):
        x0 = np.array([r.choice([r.uniform(0, 1.5), r.uniform(6.5, 8)]), r.uniform(0, 10), r.uniform(0, 4)])
        x1 = x0 + r.uniform(-0.9, 0.9, 3)
        O.deposit_current(p, J, t, 1.0, x0, x1)
        O.deposit_rho(p, rho0, t, 1.0, x0)
        O.deposit_rho(p, rho1, t, 1.0, x1)
    # the divergence must use the same shear identification for the x-neighbour
    shift = 2
    Jxm = np.roll(J[0], 1, axis=2)
    Jxm[:, :, 0] = np.roll(J[0][:, :, -1], shift, axis=1)  # x_i - 1/2 ghost = J(x_o - 1/2, y - Dy_s)
    div = (J[0] - Jxm) + (J[1] - np.roll(J[1], 1, axis=1)) + (J[2] - np.roll(J[2], 1, axis=0))
    assert np.abs(rho1[0] - rho0[0] + div).max() < 1e-13


def test_shear_fractional_fetch_is_linear_interpolation():
    n = (6, 9, 3)
    Om = 0.004
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=1.5, Omega0=Om)
    t = 37.0
    dys = O.shear_shift(p, t)
    assert dys == pytest.approx((1.5 * Om * 6 * 37.0) % 9, abs=1e-12)
    # a field linear in y (periodic image ignored away from the y seam) gathered
    # past x_o equals the interior field at y + Dy_s
    j = np.arange(9, dtype=float)
    E = np.zeros((3, 3, 9, 6))
    E[2] = (j[None, :, None] * 0.1)  # E_z = 0.1 y, uniform in x and z
    B = np.zeros_like(E)
    x = np.array([6.3, 1.2, 1.5])  # already past x_o; the stencil is fully outside
    Ep, _ = O.gather(p, E, B, t, x)
    yy = x[1] + dys
    assert yy < 7.5
    assert Ep[2] == pytest.approx(0.1 * yy, abs=1e-12)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("t", [37.0, 45.0])
def test_shear_fractional_fold_is_adjoint_of_fetch(order, t):
    """Across the shearing-periodic seam a ghost current is folded back into
    the box with the transpose of the interpolation that fetches ghost field
    values (the identification X(x_i, y) = X(x_o, y - Dy_s) of Sec. 2.1 read
    as one linear map).  Then, for any field F and any particle position x,
    sum_grid rho_c F_c = q F_c(x) exactly, where rho_c is the particle's shape
    deposited at the stagger of component c and F_c(x) the gathered value.
    Dy_s has fractional part 0.33 (t = 37) and 0.62 (t = 45), and particles sit
    on both sides of the seam, so ghost points at both images (fractional
    parts f and 1 - f) are exercised."""
    n = (6, 9, 4)
    Om = 0.004
    p = O.make_params(*n, C, order=order, box=O.BOX_SHEAR, s=1.5, Omega0=Om)
    dys = O.shear_shift(p, t)
    assert 0.1 < dys % 1.0 < 0.9
    r = np.random.default_rng(11 + order)
    F = r.normal(size=(3, 4, 9, 6))
    zero = np.zeros_like(F)
    for trial in range(24):
        xs = r.uniform(0.0, 1.6) if trial % 2 else r.uniform(4.4, 6.0)
        x = np.array([xs, r.uniform(0, 9), r.uniform(0, 4)])
        Eg, _ = O.gather(p, F, zero, t, x)
        _, Bg = O.gather(p, zero, F, t, x)
        for stag, got in ((E_STAG, Eg), (B_STAG, Bg)):
            for comp in range(3):
                rho = np.zeros((1, 4, 9, 6))
                O.deposit_rho(p, rho, t, 1.0, x - stag[comp])
                assert rho.sum() == pytest.approx(1.0, abs=1e-13)
                assert (rho[0] * F[comp]).sum() == pytest.approx(got[comp], abs=1e-13)


def _v_rows(n, sO):
    """transport velocity of each advected row at each x column: V at the
    component's own x location for the B rows and the E'_y row, -V for the
    E'_x and E'_z rows (their advection term enters with a plus sign)."""
    V = lambda x: -sO * (x - n[0] / 2)
    i = np.arange(n[0], dtype=float)
    vB = [V(i + B_STAG[c][0]) for c in range(3)]
    vE = [-V(i + 0.5), V(i), -V(i)]
    return vB, vE


@pytest.mark.parametrize("field", ["B", "E"])
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_ksb_advection_responds_downstream_of_a_step(field, comp):
    """Sec. 2.2 upwinds the y-advection terms in the local direction of the
    transport velocity, so a step in y changes only the first point on its
    downstream side, at rate -v times the jump; the point just upstream of
    the step does not change.  Profiles uniform in x and z leave every other
    term of the row at zero (curls of the other field vanish; the
    off-stagger V-terms differentiate in x or z)."""
    n = (8, 12, 4)
    sO = 0.04
    p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.0, Omega0=sO)
    j0 = 6
    prof = (np.arange(12) >= j0).astype(float)
    X = np.zeros((3, 4, 12, 8))
    X[comp] = prof[None, :, None]
    zero = np.zeros_like(X)
    if field == "B":
        FE, FB = O.ksb_rhs(p, zero, X, zero, 0.0)
        rhs, v = FB[comp], _v_rows(n, sO)[0][comp]
    else:
        FE, FB = O.ksb_rhs(p, X, zero, zero, 0.0)
        rhs, v = FE[comp], _v_rows(n, sO)[1][comp]
    for i in range(8):
        down, up = (j0, j0 - 1) if v[i] > 0 else (j0 - 1, j0)
        if v[i] == 0:
            assert np.all(rhs[:, :, i] == 0)
            continue
        np.testing.assert_allclose(rhs[:, down, i], -v[i], rtol=1e-13)
        assert np.all(rhs[:, up, i] == 0)


@pytest.mark.parametrize("field", ["B", "E"])
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_ksb_advection_step_does_not_raise_the_l2_norm(field, comp):
    """Pure advection (c = 0, no current, one component with a random profile
    in y, uniform in x and z): the implicit midpoint rule is neutral and the
    first-order upwind difference dissipates, so one field solve lowers the
    discrete L2 norm of every x column that moves (a downwind difference would
    raise it)."""
    n = (8, 16, 3)
    sO = 0.05
    p = O.make_params(*n, 0.0, box=O.BOX_SHEAR, s=1.0, Omega0=sO, fp_iters=4)
    r = np.random.default_rng(20 + comp)
    E = np.zeros((3, 3, 16, 8))
    B = np.zeros_like(E)
    X = B if field == "B" else E
    X[comp] = r.normal(size=16)[None, :, None]
    before = (X[comp] ** 2).sum(axis=(0, 1))
    # t = -1/2 puts the solve's midpoint at t = 0, where Dy_s = 0, so the
    # profile is also uniform across the x seam and no x-derivative appears
    O.ksb_field_solve(p, E, B, np.zeros_like(E), -0.5)
    after = (X[comp] ** 2).sum(axis=(0, 1))
    v = _v_rows(n, sO)[0 if field == "B" else 1][comp]
    for i in range(8):
        if v[i] == 0:
            assert after[i] == pytest.approx(before[i], rel=1e-15)
        else:
            assert after[i] < before[i] * (1 - 1e-3 * abs(v[i]))
    # B rows and the E'_z row stay uncoupled (B_y is wound up by B_x, the
    # -s Omega0 B_x term).  An advected E'_x or E'_y is sheared in x by the
    # x-dependent V, so the -V d_x terms couple E'_x and E'_y from the second
    # sweep on; that coupling is left to the continuum-convergence pin.
    if field == "B" or comp == 2:
        others = [c for c in range(3) if c != comp and not (field == "B" and comp == 0 and c == 1)]
        assert np.abs(X[others]).max() == 0 and np.abs((E if field == "B" else B)).max() == 0


def test_ksb_current_advection_direction_and_conservation():
    """J' is moved along y by v_{s,y} dt/2 = -s Omega0 x dt / 2: towards -y
    for x > 0 (right of the centre), +y for x < 0; column sums unchanged."""
    n = (8, 16, 2)
    Om = 0.5
    p = O.make_params(*n, C, order=1, box=O.BOX_SHEAR, s=1.5, Omega0=Om)
    J = np.zeros((3, 2, 16, 8))
    J[2, 0, 8, 6] = 1.0  # J_z on node x = 6, i.e. xc = +2: shift -1.5 Om = -0.75 cells
    J[2, 0, 8, 1] = 1.0  # xc = -3: shift +1.125 cells
    O.ksb_advect_current(p, J)
    np.testing.assert_allclose(J[2, 0, :, 6].sum(), 1.0)
    np.testing.assert_allclose(J[2, 0, :, 1].sum(), 1.0)
    ycen6 = (np.arange(16) * J[2, 0, :, 6]).sum()
    ycen1 = (np.arange(16) * J[2, 0, :, 1]).sum()
    assert ycen6 == pytest.approx(8 - 0.75)
    assert ycen1 == pytest.approx(8 + 1.125)


# ---- Yee leapfrog --------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_yee_standing_wave_dispersion(axis):
    """A vacuum standing wave evolves as cos(omega n) with the Yee relation
    sin(omega dt / 2) = c dt sin(k dx / 2) / dx."""
    N = 16
    n = [4, 4, 4]
    n[axis] = N
    n = tuple(n)
    p = O.make_params(*n, C)
    kk = 2 * math.pi * 3 / N
    comp = (axis + 1) % 3  # transverse E component
    E = np.zeros((3, n[2], n[1], n[0]))
    coords = grid_coords(n)
    E[comp] = np.cos(kk * (coords[axis] + E_STAG[comp][axis]))
    E0 = E.copy()
    B = np.zeros_like(E)
    J = np.zeros_like(E)
    omega = 2 * math.asin(C * math.sin(kk / 2))
    for step in range(1, 61):
        O.yee_update(p, E, B, J)
    np.testing.assert_allclose(E, E0 * math.cos(omega * 60), atol=1e-11)


# ---- expanding box fields ---------------------------------------------------------

def test_keb_uniform_fields_scale_with_l_over_ell():
    """With no current, uniform B' and E' stay constant, so the lab fields
    obey B_i ~ l_i / ell: for expansion of y and z, B_x ~ a^-2, B_y, B_z ~ a^-1."""
    n = (4, 4, 4)
    rate = (0.0, 2e-3, 2e-3)
    p = O.make_params(*n, C, box=O.BOX_EXPAND, rate=rate)
    E = np.zeros((3, 4, 4, 4))
    B = np.zeros_like(E)
    B0 = np.array([0.3, -0.2, 0.5])
    E0 = np.array([0.01, 0.02, -0.03])
    for c in range(3):
        B[c] = B0[c]
        E[c] = E0[c]
    J = np.zeros_like(E)
    for step in range(50):
        O.keb_field_update(p, E, B, J, float(step))
    a = math.exp(2e-3 * 50)
    want = np.array([1 / a**2, 1 / a, 1 / a])
    np.testing.assert_allclose(B.reshape(3, -1).mean(axis=1), B0 * want, rtol=1e-13)
    np.testing.assert_allclose(E.reshape(3, -1).mean(axis=1), E0 * want, rtol=1e-13)


def test_keb_field_update_reduces_to_yee():
    n = (6, 5, 4)
    r = np.random.default_rng(7)
    E, B, J = (r.normal(size=(3, 4, 5, 6)) for _ in range(3))
    E2, B2 = E.copy(), B.copy()
    O.keb_field_update(O.make_params(*n, C, box=O.BOX_EXPAND), E, B, J, 5.0)
    O.yee_update(O.make_params(*n, C), E2, B2, J)
    np.testing.assert_allclose(E, E2, atol=1e-14)
    np.testing.assert_allclose(B, B2, atol=1e-14)


def test_keb_gauss_law_in_primed_variables():
    """div' E' - 4 pi (ell rho') is constant when the deposited ell J' obeys
    continuity: E' = ell L^-1 E, and the primed leapfrog is a standard one."""
    n = (6, 6, 6)
    rate = (0.0, 1e-2, 2e-2)
    p = O.make_params(*n, C, order=1, box=O.BOX_EXPAND, rate=rate)
    r = np.random.default_rng(8)
    E = r.normal(size=(3, 6, 6, 6)) * 0.01
    B = r.normal(size=(3, 6, 6, 6)) * 0.01
    x0 = r.uniform(0, 6, (20, 3))
    x1 = x0 + r.uniform(-0.8, 0.8, (20, 3))

    def gauss(E, t, xs):
        l = np.exp(np.array(rate) * t)
        ell = l.prod()
        Ep = np.stack([ell / l[c] * E[c] for c in range(3)])
        rho = np.zeros((1, 6, 6, 6))
        for x in xs:
            O.deposit_rho(p, rho, t, 1.0, np.mod(x, 6))
        return divergence(Ep) - 4 * math.pi * rho[0]

    g0 = gauss(E, 3.0, x0)
    J = np.zeros_like(E)
    for a, b in zip(x0, x1):
        O.deposit_current(p, J, 3.5, 1.0, a, b)
    O.keb_field_update(p, E, B, J, 3.0)
    g1 = gauss(E, 4.0, x1)
    assert np.abs(g1 - g0).max() < 1e-12


# ---- shearing-box Maxwell solve -----------------------------------------------------

def test_ksb_rhs_omega0_zero_is_maxwell():
    """With Omega0 = 0 the shearing-box right-hand sides are c curl B - 4 pi J
    and -c curl E, the Yee curls written here with numpy rolls from the
    staggering (independently of the oracle's loops)."""
    n = (6, 5, 4)
    r = np.random.default_rng(9)
    E, B, J = (r.normal(size=(3, 4, 5, 6)) for _ in range(3))
    p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.5, Omega0=0.0)
    FE, FB = O.ksb_rhs(p, E, B, J, 0.0)
    # compare against numpy Yee curls written from the staggering
    def curlE(E):
        Ex, Ey, Ez = E
        return np.stack([(np.roll(Ez, -1, 1) - Ez) - (np.roll(Ey, -1, 0) - Ey),
                         (np.roll(Ex, -1, 0) - Ex) - (np.roll(Ez, -1, 2) - Ez),
                         (np.roll(Ey, -1, 2) - Ey) - (np.roll(Ex, -1, 1) - Ex)])

    def curlB(B):
        Bx, By, Bz = B
        return np.stack([(Bz - np.roll(Bz, 1, 1)) - (By - np.roll(By, 1, 0)),
                         (Bx - np.roll(Bx, 1, 0)) - (Bz - np.roll(Bz, 1, 2)),
                         (By - np.roll(By, 1, 2)) - (Bx - np.roll(Bx, 1, 1))])
    np.testing.assert_allclose(FB, -C * curlE(E), atol=1e-14)
    np.testing.assert_allclose(FE, C * curlB(B) - 4 * math.pi * J, atol=1e-13)


def _continuum_rhs(n, sO, k):
    """Fields periodic in x, y, z with wavenumbers k; returns sampled fields
    and the exact right-hand sides of the shearing-box equations (Sec. 2.1)
    at each component's Yee location, with V = -s Omega0 (x - nx/2), c = C."""
    kx, ky, kz = k
    ph = np.array([[0.3, 1.1, 2.0], [0.7, 0.2, 1.4], [1.9, 0.5, 0.9]])

    def e(c, x, y, z):
        return np.sin(kx * x + ph[c, 0]) * np.cos(ky * y + ph[c, 1]) * np.cos(kz * z + ph[c, 2])

    def de(c, x, y, z, ax):
        s1 = np.sin(kx * x + ph[c, 0]); c1 = np.cos(kx * x + ph[c, 0])
        s2 = np.sin(ky * y + ph[c, 1]); c2 = np.cos(ky * y + ph[c, 1])
        s3 = np.sin(kz * z + ph[c, 2]); c3 = np.cos(kz * z + ph[c, 2])
        if ax == 0:
            return kx * c1 * c2 * c3
        if ax == 1:
            return -ky * s1 * s2 * c3
        return -kz * s1 * c2 * s3

    b = lambda c, x, y, z: e((c + 1) % 3, x, y, z) * 0.7
    db = lambda c, x, y, z, ax: de((c + 1) % 3, x, y, z, ax) * 0.7
    E = field_from(lambda x, y, z, c: e(c, x, y, z), n, E_STAG)
    B = field_from(lambda x, y, z, c: b(c, x, y, z), n, B_STAG)
    V = lambda x: -sO * (x - n[0] / 2)

    def FE(x, y, z, c):
        curlB = [db(2, x, y, z, 1) - db(1, x, y, z, 2), db(0, x, y, z, 2) - db(2, x, y, z, 0),
                 db(1, x, y, z, 0) - db(0, x, y, z, 1)][c]
        v = V(x)
        if c == 0:
            return C * curlB + v * de(0, x, y, z, 1) - v * de(1, x, y, z, 0)
        if c == 1:
            return C * curlB - v * de(1, x, y, z, 1) - v * (de(0, x, y, z, 0) + de(2, x, y, z, 2))
        return C * curlB + v * de(2, x, y, z, 1) - v * de(1, x, y, z, 2)

    def FB(x, y, z, c):
        curlE = [de(2, x, y, z, 1) - de(1, x, y, z, 2), de(0, x, y, z, 2) - de(2, x, y, z, 0),
                 de(1, x, y, z, 0) - de(0, x, y, z, 1)][c]
        out = -C * curlE - V(x) * db(c, x, y, z, 1)
        if c == 1:
            out = out - sO * b(0, x, y, z)
        return out

    return E, B, field_from(FE, n, E_STAG), field_from(FB, n, B_STAG)


def test_ksb_rhs_converges_to_the_continuum_equations():
    """On smooth periodic fields (Dy_s = 0 at t = 0, so any periodic field is
    admissible) the discrete right-hand sides approach the continuum ones of
    Sec. 2.1; the error falls at least first order under refinement (the
    upwinded advection), away from the x seam where V jumps.  A wrong sign,
    component or stagger leaves an O(1) error."""
    errs = []
    for N in (16, 32, 64):
        n = (N, N, N // 2)
        k = (2 * math.pi / N, 2 * math.pi * 2 / N, 2 * math.pi / (N // 2))
        sO = 0.2 / N  # keeps V = O(0.1) across the box
        p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.0, Omega0=sO)
        E, B, FEc, FBc = _continuum_rhs(n, sO, k)
        FE, FB = O.ksb_rhs(p, E, B, np.zeros_like(E), 0.0)
        inner = slice(2, N - 2)
        err = max(np.abs(FE - FEc)[..., inner].max(), np.abs(FB - FBc)[..., inner].max())
        scale = max(np.abs(FEc).max(), np.abs(FBc).max())
        errs.append(err / scale)
    assert errs[-1] < 0.025
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6


def test_ksb_uniform_Bx_winds_up_By_exactly():
    """Uniform fields: curls and advection vanish, leaving dB_y/dt = -s Omega0 B_x
    (the shear term of Sec. 2.1); the implicit midpoint step is exact for it."""
    n = (6, 6, 6)
    sO = 0.015
    p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.5, Omega0=sO / 1.5, fp_iters=4)
    E = np.zeros((3, 6, 6, 6))
    B = np.zeros_like(E)
    B[0] = 0.4
    B[2] = 1.0
    O.ksb_field_solve(p, E, B, np.zeros_like(E), 0.0)
    np.testing.assert_allclose(B[1], -sO * 0.4, rtol=1e-14)
    np.testing.assert_allclose(B[0], 0.4, rtol=1e-15)
    np.testing.assert_allclose(E, 0.0, atol=1e-18)


@pytest.mark.parametrize("nsweeps", [1, 2, 3, 4, 7])
def test_ksb_fixed_point_iteration_polynomial(nsweeps):
    """N fixed-point sweeps of the implicit midpoint rule give
    X^(N) = (I + 2 sum_{m=1..N} (dt A / 2)^m) X^n for the linear operator A
    (here A applied through the oracle's own right-hand side at Omega0 = 0,
    whose curls are pinned above)."""
    n = (5, 4, 3)
    r = np.random.default_rng(10)
    E, B = r.normal(size=(3, 3, 4, 5)), r.normal(size=(3, 3, 4, 5))
    J = np.zeros_like(E)
    p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.5, Omega0=0.0, fp_iters=nsweeps)
    E1, B1 = E.copy(), B.copy()
    O.ksb_field_solve(p, E1, B1, J, 0.0)
    termE, termB = E.copy(), B.copy()
    accE, accB = E.copy(), B.copy()
    for _ in range(nsweeps):
        FE, FB = O.ksb_rhs(p, termE, termB, J, 0.0)
        termE, termB = FE / 2, FB / 2
        accE += 2 * termE
        accB += 2 * termB
    np.testing.assert_allclose(E1, accE, atol=1e-12)
    np.testing.assert_allclose(B1, accB, atol=1e-12)


@pytest.mark.parametrize("term", ["bx4", "dxEy", "divxz", "dzEy"])
def test_ksb_rhs_averaged_shear_terms_on_a_sinusoid(term):
    """The shear terms of Sec. 2.1 that need a field at another component's
    location (B_x in the B_y row; d_x E'_y, d_x E'_x + d_z E'_z and d_z E'_y
    in the E'_x, E'_y and E'_z rows) are centred differences averaged over the
    two neighbouring y rows.  On a product of sinusoids both steps have closed
    forms: [sin(a + h/2) + sin(a - h/2)] / 2 = cos(h/2) sin(a) and
    sin(a + h/2) - sin(a - h/2) = 2 sin(h/2) cos(a).  With one field component
    nonzero the row reduces to that term alone (its curl, current and
    upwinded terms vanish), so the right-hand side is known exactly; an
    average over the wrong rows or a difference at the wrong points is not."""
    n = (16, 12, 8)
    kx, ky, kz = 2 * math.pi * 2 / n[0], 2 * math.pi / n[1], 2 * math.pi / n[2]
    sO = 0.01
    p = O.make_params(*n, C, box=O.BOX_SHEAR, s=1.0, Omega0=sO)
    i, j, k = grid_coords(n)
    E = np.zeros((3,) + i.shape)
    B = np.zeros_like(E)
    VN = -sO * (i - n[0] / 2)
    VH = -sO * (i + 0.5 - n[0] / 2)
    cy = math.cos(ky / 2)
    if term == "bx4":  # B_x at (i, j+1/2, k+1/2), wanted at B_y's (i+1/2, j, k+1/2)
        B = field_from(lambda x, y, z, c: (c == 0) * np.sin(kx * x) * np.sin(ky * y), n, B_STAG)
        comp, F = 1, "B"
        want = -sO * math.cos(kx / 2) * np.sin(kx * (i + 0.5)) * cy * np.sin(ky * j)
    elif term == "dxEy":  # E'_y at (i, j+1/2, k), d_x wanted at E'_x's (i+1/2, j, k)
        E = field_from(lambda x, y, z, c: (c == 1) * np.sin(kx * x) * np.sin(ky * y), n, E_STAG)
        comp, F = 0, "E"
        want = -VH * 2 * math.sin(kx / 2) * np.cos(kx * (i + 0.5)) * cy * np.sin(ky * j)
    elif term == "divxz":  # E'_x at (i+1/2, j, k), d_x wanted at E'_y's (i, j+1/2, k)
        E = field_from(lambda x, y, z, c: (c == 0) * np.sin(kx * x) * np.sin(ky * y), n, E_STAG)
        comp, F = 1, "E"
        want = -VN * 2 * math.sin(kx / 2) * np.cos(kx * i) * cy * np.sin(ky * (j + 0.5))
    else:  # E'_y at (i, j+1/2, k), d_z wanted at E'_z's (i, j, k+1/2)
        E = field_from(lambda x, y, z, c: (c == 1) * np.sin(kz * z) * np.sin(ky * y), n, E_STAG)
        comp, F = 2, "E"
        want = -VN * 2 * math.sin(kz / 2) * np.cos(kz * (k + 0.5)) * cy * np.sin(ky * j)
    FE, FB = O.ksb_rhs(p, E, B, np.zeros_like(E), 0.0)
    got = (FE if F == "E" else FB)[comp]
    assert np.abs(want).max() > 1e-3
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)

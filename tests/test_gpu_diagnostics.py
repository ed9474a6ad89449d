"""pic_diagnostics (the FP64 global sums) against independent sums of the
same state: the field energies sum_c F_c^2 / (8 pi) and the kinetic energies
sum m c^2 (gamma - 1), computed here with numpy in FP64 over the arrays that
pic_get_fields and pic_get_particles read back (FP32 device values convert to
FP64 exactly).  FP64 boxes agree to 1e-12; FP32 boxes to 1e-12 for the field
energies (FP64 sums of exact squares) and to 1e-6 for the kinetic energies
(gamma - 1 is formed per particle in the particles' precision)."""
import math

import numpy as np
import pytest

from gpu_harness import Case, inputs
from paper_2602_15939_gb300 import pic as P

CASES = [
    Case("expand3d_o2", P.PIC_BOX_EXPAND, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=20),
    Case("shear3d_o2", P.PIC_BOX_SHEAR, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37),
    Case("leaky2d_prob_o1", P.PIC_BOX_LEAKY, (32, 24, 1), ndim=2, plane=P.PIC_PLANE_XY, order=1, ppc=6,
         esc_mode=2, p_esc=0.05, theta_inj=1.0),
    Case("periodic2dxz_o2", P.PIC_BOX_PERIODIC, (24, 1, 20), ndim=2, plane=P.PIC_PLANE_XZ, order=2, ppc=6),
]


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [True, False], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_diagnostics_equal_independent_sums(case, fp64):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.set_step(case.step0)
        box.step(3)
        diag = box.diagnostics()
        Eg, Bg, _ = box.fields()
        parts = [box.particles(i) for i in range(len(sp))]
    finally:
        box.close()
    assert diag.error_word == 0
    want_E = (Eg.reshape(3, -1) ** 2).sum(axis=1) / (8 * math.pi)
    want_B = (Bg.reshape(3, -1) ** 2).sum(axis=1) / (8 * math.pi)
    np.testing.assert_allclose(np.array(diag.field_energy_E[:]), want_E, rtol=1e-12, atol=0)
    np.testing.assert_allclose(np.array(diag.field_energy_B[:]), want_B, rtol=1e-12, atol=0)
    c = case.c
    for i, (d, (x, u, ids, _)) in enumerate(zip(sp, parts)):
        assert diag.count[i] == len(ids) == len(d["id"])
        u2 = (u ** 2).sum(axis=1) / c**2
        kin = d["m"] * c**2 * (u2 / (np.sqrt(1.0 + u2) + 1.0)).sum()
        np.testing.assert_allclose(diag.kinetic_energy[i], kin, rtol=1e-12 if fp64 else 1e-6, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [True, False], ids=["fp64", "fp32"])
@pytest.mark.parametrize("box_kind", [P.PIC_BOX_SHEAR, P.PIC_BOX_SHEAR_EXPAND], ids=["shear", "shear_expand"])
def test_superluminal_count_matches_oracle_and_closed_form(box_kind, fp64):
    """The superluminal counter (Sec. 2.1: the effective velocity u'/gamma' +
    v_s, v_s = -s Omega0 x e_y, can exceed c far from the centre).  Particles
    at rest in the shearing frame with no fields stay at rest, so each step
    counts those with s Omega0 |x - nx/2| >= c, x the physical coordinate
    (l_1(t^n) times the expanding coordinate in the combined box).  The
    device's total over three steps must equal the oracle's and the closed
    form."""
    import oracle as O

    # the library admits shear flows with c + s Omega0 nx/2 < 1 cell per step,
    # so the edge speed (0.52 here) sits between c and 1 - c
    n = (16, 8, 8)
    s, Om, c, step0, rate = 1.5, 0.065 / 1.5, 0.45, 10, 0.01
    rates = (rate, 0.0, 0.0) if box_kind == P.PIC_BOX_SHEAR_EXPAND else (0.0, 0.0, 0.0)
    xi = np.arange(n[0]) + 0.5
    N = xi.size
    x = np.stack([xi, np.full(N, 1.5), np.full(N, 2.5)], axis=1)
    u = np.zeros((N, 3))
    ids = np.arange(N, dtype=np.uint32)
    z = np.zeros((3, n[2], n[1], n[0]))
    want = 0
    for t in range(step0, step0 + 3):
        l1 = math.exp(rates[0] * t)
        speed = s * Om * np.abs(l1 * (xi - n[0] / 2))
        assert np.abs(speed - c).min() > 0.01  # no particle near the threshold
        want += int((speed >= c).sum())
    st = O.State(O.make_params(*n, c, box=box_kind, s=s, Omega0=Om, rate=rates), z, z,
                 [{"q": 0.05, "m": 1.0, "x": x, "u": u, "id": ids}], step=step0)
    assert st.step(3)["superluminal"] == want
    cfg = P.make_config(box=box_kind, nx=n[0], ny=n[1], nz=n[2], c=c, order=1,
                        precision=P.PIC_FP64 if fp64 else P.PIC_FP32, s=s, Omega0=Om, rate=rates)
    box = P.Box(cfg)
    try:
        box.set_fields(z, z)
        box.load(0, 0.05, 1.0, x, u, ids)
        box.set_step(step0)
        box.step(3)
        diag = box.diagnostics()
    finally:
        box.close()
    assert diag.error_word == 0
    assert 0 < want < 3 * N
    assert diag.superluminal_total == want

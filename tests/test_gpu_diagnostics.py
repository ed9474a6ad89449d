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

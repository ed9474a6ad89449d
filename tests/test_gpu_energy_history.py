"""FP32 against FP64 over long runs: the total energy history (field energy
plus kinetic energy of both species) of the FP32 path stays within 1% of the
FP64 path's on the same seeded inputs, for the expanding, shearing and leaky
boxes.  Individual particle orbits separate over hundreds of steps (rounding
is amplified by the dynamics), so the comparison is on the box's totals."""
import numpy as np
import pytest

from gpu_harness import Case, inputs
from paper_2602_15939_gb300 import pic as P

BOX_S, BOX_E, BOX_L = P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY

CASES = [
    Case("expand3d_o2", BOX_E, (24, 16, 16), order=2, rate=(0.0, 1e-3, 1e-3), ppc=8, uth=0.2),
    Case("shear3d_o2", BOX_S, (24, 16, 16), order=2, s=1.5, Omega0=3e-3, ppc=8, uth=0.2),
    Case("leaky2d_prob_o1", BOX_L, (64, 48, 1), ndim=2, plane=P.PIC_PLANE_XY, order=1, ppc=16, esc_mode=2,
         p_esc=0.01, theta_inj=0.3, uth=0.3),
]
STEPS, EVERY = 400, 20


def energy_history(case, fp64):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    hist = []
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        for _ in range(STEPS // EVERY):
            box.step(EVERY)
            dg = box.diagnostics()
            assert dg.error_word == 0
            hist.append(sum(dg.field_energy_E) + sum(dg.field_energy_B) + sum(dg.kinetic_energy[:2]))
    finally:
        box.close()
    return np.array(hist)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fp32_energy_history_within_one_percent(case):
    h32 = energy_history(case, False)
    h64 = energy_history(case, True)
    rel = np.abs(h32 - h64) / np.abs(h64)
    assert rel.max() <= 0.01, (rel.max(), h32, h64)

"""Charge conservation of the device current, cell by cell: after a step,
(rho^{n+1} - rho^n) + div J = 0 (dt = dx = 1), with rho computed by the
oracle's node deposit from the device's own particle positions before and
after the step, and J read from the device.  Every box whose particle move is
the one the current is deposited along (standard, leaky, expanding -- the
shearing box deposits on the comoving move and then advects J'), in 3D and
both 2D planes.  FP32: within 1e-5 of J_ref = |q| c n0 (fixed-point current
and FP32 shape weights); FP64: 1e-11."""
import numpy as np
import pytest

import oracle as O
from gpu_harness import Case, current_scale, inputs
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY
XY, XZ = P.PIC_PLANE_XY, P.PIC_PLANE_XZ

CASES = [
    Case("periodic3d_o1", BOX_P, (16, 12, 8), order=1, uth=0.3),
    Case("periodic3d_o2", BOX_P, (16, 12, 8), order=2, uth=0.3),
    Case("periodic2dxy_o2", BOX_P, (32, 24, 1), ndim=2, plane=XY, order=2, ppc=6, uth=0.3),
    Case("periodic2dxz_o1", BOX_P, (24, 1, 20), ndim=2, plane=XZ, order=1, ppc=6, uth=0.3),
    Case("expand3d_o2", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 2e-3), step0=30, uth=0.3),
    Case("leaky2d_prob_o1", BOX_L, (32, 24, 1), ndim=2, plane=XY, order=1, ppc=6, esc_mode=2, p_esc=0.05,
         theta_inj=0.5, uth=0.3),
]


def residual(case, fp64):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.set_step(case.step0)
        box.step(2)
        before = [box.particles(i) for i in range(len(sp))]
        box.step(1)
        after = [box.particles(i) for i in range(len(sp))]
        _, _, J = box.fields()
        assert box.diagnostics().error_word == 0
    finally:
        box.close()
    p = case.oracle_params()
    rho0 = np.zeros((1,) + J.shape[1:])
    rho1 = np.zeros_like(rho0)
    for d, (xb, _, ib, _), (xa, _, ia, _) in zip(sp, before, after):
        ob, oa = np.argsort(ib), np.argsort(ia)
        assert np.array_equal(ib[ob], ia[oa])
        for rb, ra in zip(xb[ob], xa[oa]):
            O.deposit_rho(p, rho0, 0.0, d["q"], rb)
            O.deposit_rho(p, rho1, 0.0, d["q"], ra)
    div = (J[0] - np.roll(J[0], 1, axis=2)) + (J[1] - np.roll(J[1], 1, axis=1)) + (J[2] - np.roll(J[2], 1, axis=0))
    res = rho1[0] - rho0[0] + div
    return np.abs(res).max() / current_scale(case), np.abs(div).max() / current_scale(case)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
@pytest.mark.parametrize("fp64,tol", [(False, 1e-5), (True, 1e-11)], ids=["fp32", "fp64"])
def test_charge_continuity_per_cell(case, fp64, tol):
    res, div = residual(case, fp64)
    assert div > 1e-3  # the current is not trivially zero
    assert res <= tol, res

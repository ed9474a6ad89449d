"""GPU parity: libpic (through its C ABI) against the FP64 CPU oracle on the
same seeded inputs, element by element, for every box (periodic, leaky,
shearing, expanding), geometry (3D, 2D x-y, 2D x-z), shape order and
precision.  Grids span several tiles with a ragged last tile.

Tolerances (max-norm errors relative to the largest reference value):
FP64 1e-12 for momenta, fields and currents after one step (rounding order
only).  FP32 1e-6 for one step (single-precision momenta, in-cell offsets and
fields; fixed-point current units of about 2e-7 of a particle charge), with
positions compared in cells; for J the reference is at least the physical
current scale J_ref = |q| c n0 and for E and B at least 4 pi J_ref, the field
change such a current drives in one step.  Escape decisions of the
probabilistic leaky box are integer comparisons and must agree exactly.
"""
import pytest

from gpu_harness import Case, compare
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_S, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY
BOX_SE = P.PIC_BOX_SHEAR_EXPAND
XY, XZ = P.PIC_PLANE_XY, P.PIC_PLANE_XZ

CASES = [
    Case("periodic3d_o1", BOX_P, (16, 12, 8), order=1),
    Case("periodic3d_o2", BOX_P, (16, 12, 8), order=2),
    Case("periodic2dxy_o1", BOX_P, (32, 24, 1), ndim=2, plane=XY, order=1, ppc=6),
    Case("periodic2dxy_o2", BOX_P, (32, 24, 1), ndim=2, plane=XY, order=2, ppc=6),
    Case("periodic2dxz_o2", BOX_P, (24, 1, 20), ndim=2, plane=XZ, order=2, ppc=6),
    Case("leaky2d_disp_o1", BOX_L, (32, 24, 1), ndim=2, plane=XY, order=1, ppc=6, esc_mode=1, l_esc=0.35,
         theta_inj=0.2),
    Case("leaky2d_prob_o2", BOX_L, (32, 24, 1), ndim=2, plane=XY, order=2, ppc=6, esc_mode=2, p_esc=0.05,
         theta_inj=1.0),
    Case("leaky3d_disp_o2", BOX_L, (16, 12, 8), order=2, esc_mode=1, esc_dims=3, l_esc=0.3, theta_inj=0.3),
    Case("shear3d_o2", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37),
    Case("shear3d_o1", BOX_S, (16, 16, 8), order=1, s=1.5, Omega0=2e-3, step0=101, fp_iters=3),
    Case("shear2dxz_o1", BOX_S, (32, 1, 24), ndim=2, plane=XZ, order=1, ppc=6, s=1.5, Omega0=4e-3, step0=11),
    Case("expand3d_o2", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=200),
    Case("expand3d_o2_exact", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 2e-3), step0=150, keb_exact=1),
    Case("expand2dxy_o1", BOX_E, (32, 24, 1), ndim=2, plane=XY, order=1, ppc=6, rate=(2e-3, 1e-3, 0.0), step0=50),
    # electron-ion plasmas, m_i / m_e = 25 (the expanding-box example of Sec. 3.3)
    Case("expand3d_o2_ion25", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=20, masses=(1.0, 25.0)),
    Case("shear3d_o2_ion25", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=7, masses=(1.0, 25.0)),
    Case("leaky2d_prob_o1_ion25", BOX_L, (32, 24, 1), ndim=2, plane=XY, order=1, ppc=6, esc_mode=2, p_esc=0.05,
         theta_inj=0.5, masses=(1.0, 25.0)),
    # shearing box that also expands (the combination of Sec. 5): fractional shear shifts at these steps
    Case("shearexp3d_o2", BOX_SE, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, rate=(1e-3, 2e-3, 5e-4), step0=37),
    Case("shearexp3d_o1", BOX_SE, (16, 16, 8), order=1, s=1.2, Omega0=2e-3, rate=(0.0, 1e-3, 1e-3), step0=101,
         fp_iters=3),
    Case("shearexp2dxy_o2", BOX_SE, (32, 24, 1), ndim=2, plane=XY, order=2, ppc=6, s=1.5, Omega0=4e-3,
         rate=(2e-3, 1e-3, 0.0), step0=11),
    # the leaky box's probabilistic escape combined with the other boxes (Sec. 4.1 with Sec. 5)
    Case("shear3d_o2_esc", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37, esc_mode=2, p_esc=0.05,
         theta_inj=0.3),
    Case("shear2dxz_o1_esc", BOX_S, (32, 1, 24), ndim=2, plane=XZ, order=1, ppc=6, s=1.5, Omega0=4e-3, step0=11,
         esc_mode=2, p_esc=0.05, theta_inj=0.5),
    Case("expand3d_o2_esc", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=20, esc_mode=2, p_esc=0.05,
         theta_inj=0.2),
    Case("shearexp3d_o1_esc", BOX_SE, (16, 16, 8), order=1, s=1.2, Omega0=2e-3, rate=(0.0, 1e-3, 1e-3),
         step0=101, fp_iters=3, esc_mode=2, p_esc=0.05, theta_inj=0.3),
]

IDS = [c.name for c in CASES]


def _check(r, tol_rel, tol_x):
    assert r["error_word"] == 0, r
    assert r["u"] <= tol_rel, r
    assert r["x"] <= tol_x, r
    assert r["E"] <= tol_rel, r
    assert r["B"] <= tol_rel, r
    assert r["J"] <= tol_rel, r
    assert r["escaped_gpu"] == r["escaped_oracle"], r


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp64_one_step(case):
    r = compare(case, 1, fp64=True)
    _check(r, 1e-12, 1e-11)
    assert r["dr"] <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp64_three_steps(case):
    r = compare(case, 3, fp64=True)
    _check(r, 1e-11, 1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp32_one_step(case):
    r = compare(case, 1, fp64=False)
    _check(r, 1e-6, 2e-6)

"""Every particle-kernel variant (threads per CTA x private copies of the
shared current box) against the FP64 oracle, and against each other.

The variants change only how the work is laid out on the GPU, so a
particle's state after a step does not depend on the variant at all (bit for
bit), and neither does the FP32 current: it is summed in int32 fixed point,
which is exact and order-independent.  FP64 currents are summed with double
atomics in an order that depends on scheduling, so there the variants agree to
rounding (1e-12 relative).
"""
import dataclasses

import numpy as np
import pytest

from gpu_harness import Case, compare, run_gpu
from paper_2602_15939_gb300 import pic as P

BOX_P, BOX_S, BOX_E, BOX_L = P.PIC_BOX_PERIODIC, P.PIC_BOX_SHEAR, P.PIC_BOX_EXPAND, P.PIC_BOX_LEAKY

CASES = [
    Case("expand3d_o2", BOX_E, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), step0=200, ppc=8),
    Case("shear3d_o2", BOX_S, (16, 12, 8), order=2, s=1.5, Omega0=3e-3, step0=37, ppc=8),
    Case("leaky2d_prob_o2", BOX_L, (32, 24, 1), ndim=2, plane=P.PIC_PLANE_XY, order=2, ppc=12, esc_mode=2,
         p_esc=0.05, theta_inj=1.0),
    Case("periodic2dxz_o1", BOX_P, (24, 1, 20), ndim=2, plane=P.PIC_PLANE_XZ, order=1, ppc=12),
]


def fitting_variants(case, fp64):
    """Variants (1-based) whose shared memory fits the case's configuration."""
    out = []
    for k in range(1, P.pic_kernel_variant_count() + 1):
        try:
            b = P.Box(dataclasses.replace(case, variant=k).gpu_config(fp64))
        except P.PicError:
            continue
        assert P.pic_get_kernel_variant(b.h) == k
        b.close()
        out.append(k)
    return out


def by_id(parts):
    res = []
    for x, u, ids, _ in parts:
        o = np.argsort(ids)
        res.append((x[o], u[o], ids[o]))
    return res


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_fp32_variants_match_oracle_and_each_other(case):
    ks = fitting_variants(case, False)
    assert len(ks) == P.pic_kernel_variant_count()  # every variant fits an FP32 tile
    ref = None
    for k in ks:
        cv = dataclasses.replace(case, variant=k)
        r = compare(cv, 1, fp64=False)
        assert r["error_word"] == 0 and r["u"] <= 1e-6 and r["x"] <= 2e-6, (k, r)
        assert r["E"] <= 1e-6 and r["B"] <= 1e-6 and r["J"] <= 1e-6, (k, r)
        assert r["escaped_gpu"] == r["escaped_oracle"], (k, r)
        parts, (E, B, J), _ = run_gpu(cv, 2, False)
        got = (by_id(parts), E, B, J)
        if ref is None:
            ref = got
            continue
        for (xa, ua, ia), (xb, ub, ib) in zip(ref[0], got[0]):
            assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(ua, ub), k
        for a, b in zip(ref[1:], got[1:]):
            assert np.array_equal(a, b), k


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES[:2], ids=[c.name for c in CASES[:2]])
def test_fp64_variants_match_oracle(case):
    ks = fitting_variants(case, True)
    assert 1 in ks and 2 in ks
    for k in ks:
        r = compare(dataclasses.replace(case, variant=k), 1, fp64=True)
        assert r["error_word"] == 0 and r["u"] <= 1e-12 and r["J"] <= 1e-12 and r["E"] <= 1e-12, (k, r)


@pytest.mark.gpu
def test_switch_variant_on_a_live_box():
    case = CASES[0]
    parts_ref, fields_ref, _ = run_gpu(dataclasses.replace(case, variant=2), 3, False)
    from gpu_harness import inputs

    sp, E, B = inputs(case)
    box = P.Box(dataclasses.replace(case, variant=1).gpu_config(False))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.set_step(case.step0)
        box.step(1)
        P.pic_set_kernel_variant(box.h, 4)
        box.step(1)
        P.pic_set_kernel_variant(box.h, 2)
        box.step(1)
        parts = [box.particles(i) for i in range(len(sp))]
        fields = box.fields()
    finally:
        box.close()
    for (xa, ua, ia), (xb, ub, ib) in zip(by_id(parts_ref), by_id(parts)):
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(ua, ub)
    for a, b in zip(fields_ref, fields):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_autotune_steps_are_ordinary_steps():
    """The autotuner's trial steps advance the box exactly like pic_step: the
    state after autotune + k steps equals that of a fixed variant run for the
    same total number of steps, bit for bit (FP32)."""
    from gpu_harness import inputs

    case = CASES[0]
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(False))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.set_step(case.step0)
        best, ms, taken = box.autotune(2)
        assert 1 <= best <= P.pic_kernel_variant_count()
        assert all(v is not None and v > 0 for v in ms)
        assert ms[best - 1] == min(ms)
        assert P.pic_get_kernel_variant(box.h) == best
        box.step(1)
        parts = [box.particles(i) for i in range(len(sp))]
        fields = box.fields()
        assert box.diagnostics().step == case.step0 + taken + 1
    finally:
        box.close()
    parts_ref, fields_ref, _ = run_gpu(dataclasses.replace(case, variant=1), taken + 1, False)
    for (xa, ua, ia), (xb, ub, ib) in zip(by_id(parts_ref), by_id(parts)):
        assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(ua, ub)
    for a, b in zip(fields_ref, fields):
        assert np.array_equal(a, b)


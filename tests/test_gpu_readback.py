"""pic_get_particles writes pinned host and device buffers in place (the
compaction kernel stores straight into them) and stages pageable ones
through device temporaries; the three give the same arrays."""
import numpy as np
import pytest

from gpu_harness import Case, inputs
from paper_2602_15939_gb300 import pic as P

CASES = [
    Case("leaky2dxy_disp", P.PIC_BOX_LEAKY, (40, 24, 1), ndim=2, plane=P.PIC_PLANE_XY, order=2, ppc=6, esc_mode=1,
         l_esc=0.25, theta_inj=0.5, uth=0.3),
    Case("expand3d_o2", P.PIC_BOX_EXPAND, (16, 12, 8), order=2, rate=(0.0, 1e-3, 1e-3), ppc=6, uth=0.3),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_readback_pinned_device_and_pageable_agree(case):
    torch = pytest.importorskip("torch")
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(False))
    try:
        box.set_fields(E, B)
        for i, d in enumerate(sp):
            box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
        box.step(3)
        lib = P.lib()
        for s in range(len(sp)):
            x, u, ids, dr = box.particles(s, want_dr=True)  # pageable numpy buffers: staged copies
            n = len(ids)
            for kw in (dict(pin_memory=True), dict(device="cuda")):
                bx = torch.full((n, 3), -1.0, dtype=torch.float64, **kw)
                bu = torch.full((n, 3), -1.0, dtype=torch.float64, **kw)
                bi = torch.zeros((n,), dtype=torch.int32, **kw)
                bd = torch.full((n, 3), -1.0, dtype=torch.float64, **kw)
                st = lib.pic_get_particles(box.h, s, P.C.cast(bx.data_ptr(), P._D), P.C.cast(bu.data_ptr(), P._D),
                                           P.C.cast(bi.data_ptr(), P._U32), P.C.cast(bd.data_ptr(), P._D))
                assert st == P.PIC_OK, P.pic_last_error(box.h)
                torch.cuda.synchronize()
                assert np.array_equal(bx.cpu().numpy(), x) and np.array_equal(bu.cpu().numpy(), u)
                assert np.array_equal(bi.cpu().numpy().view(np.uint32), ids)
                assert np.array_equal(bd.cpu().numpy(), dr)
            if case.ndim == 2:
                ig = case.ignorable
                assert np.all(x[:, ig] == 0.5)
    finally:
        box.close()

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


@pytest.mark.gpu
def test_load_and_readback_across_staging_chunks():
    # more particles per species than one staging chunk (2^23): a load and a
    # read-back each take two chunks.  Species 0 brings shuffled ids, species 1
    # none (ids are then the input positions 0..n-1, also across chunks).
    n3 = (48, 48, 48)
    ppc = 80
    N = n3[0] * n3[1] * n3[2] * ppc
    assert N > (1 << 23)
    cfg = P.make_config(box=P.PIC_BOX_PERIODIC, nx=n3[0], ny=n3[1], nz=n3[2], ndim=3, order=1, precision=P.PIC_FP32)
    r = np.random.default_rng(11)
    x = r.uniform(0.0, 1.0, (N, 3)) * np.asarray(n3, dtype=float)
    u = r.normal(0.0, 0.1, (N, 3))
    ids = r.permutation(N).astype(np.uint32)
    box = P.Box(cfg)
    try:
        z = np.zeros((3, n3[2], n3[1], n3[0]))
        box.set_fields(z, z)
        box.load(0, -0.01, 1.0, x, u, ids)
        box.load(1, 0.01, 1.0, x, u)
        for s, want_ids in ((0, ids), (1, np.arange(N, dtype=np.uint32))):
            xo, uo, io, _ = box.particles(s)
            assert len(io) == N
            o = np.argsort(io)
            assert np.array_equal(io[o], np.arange(N, dtype=np.uint32))
            back = np.empty(N, dtype=np.int64)
            back[want_ids] = np.arange(N)  # input row of each id
            xi, ui = x[back], u[back]
            assert np.abs(xo[o] - xi).max() <= 1e-5  # FP32 in-cell offsets
            assert np.abs(uo[o] - ui).max() <= 1e-6 * np.abs(ui).max()
        box.step(1)
        for s in (0, 1):
            xo, uo, io, _ = box.particles(s)
            xs, us, is_, _ = box.particles_sampled(s, 997, 5, max_out=N // 900)
            o = np.argsort(io)
            k = np.searchsorted(io[o], is_)
            assert np.array_equal(io[o][k], is_)
            assert np.array_equal(xo[o][k], xs) and np.array_equal(uo[o][k], us)
    finally:
        box.close()


@pytest.mark.gpu
@pytest.mark.parametrize("source", ["pageable", "pinned", "device", "pageable_restaged"])
def test_load_paths_give_the_same_box(source, monkeypatch):
    """A load of three staging chunks (more than 2 x 2^23 particles) from
    pageable or pinned host memory (copies overlapping the kernels, positions
    kept on the device between the two passes, or copied twice when that is
    switched off) or from device memory (read in place) lays out the same
    particles, and the box steps to the same state bit for bit."""
    torch = pytest.importorskip("torch")
    if source == "pageable_restaged":
        monkeypatch.setenv("PIC_LOAD_RESIDENT_POSITIONS", "0")
    n3 = (64, 48, 48)
    ppc = 115
    N = n3[0] * n3[1] * n3[2] * ppc
    assert N > 2 * (1 << 23)
    cfg = P.make_config(box=P.PIC_BOX_PERIODIC, nx=n3[0], ny=n3[1], nz=n3[2], ndim=3, order=1, precision=P.PIC_FP32)
    r = np.random.default_rng(5)
    # cell-ordered positions (the order the loader's aggregated tile counters favour), shuffled ids
    cells = np.repeat(np.arange(n3[0] * n3[1] * n3[2]), ppc)
    ci, cj, ck = cells % n3[0], (cells // n3[0]) % n3[1], cells // (n3[0] * n3[1])
    x = np.stack([ci, cj, ck], axis=1) + r.uniform(0.0, 1.0, (N, 3))
    u = r.normal(0.0, 0.1, (N, 3))
    ids = r.permutation(N).astype(np.uint32)
    box = P.Box(cfg)
    try:
        z = np.zeros((3, n3[2], n3[1], n3[0]))
        box.set_fields(z, z)
        if source in ("pageable", "pageable_restaged"):
            box.load(0, -0.01, 1.0, x, u, ids)
        else:
            kw = dict(pin_memory=True) if source == "pinned" else dict(device="cuda")
            tx = torch.from_numpy(x).to(**kw) if source == "device" else torch.from_numpy(x).pin_memory()
            tu = torch.from_numpy(u).to(**kw) if source == "device" else torch.from_numpy(u).pin_memory()
            ti = torch.from_numpy(ids.view(np.int32)).to(**kw) if source == "device" else \
                torch.from_numpy(ids.view(np.int32)).pin_memory()
            torch.cuda.synchronize()
            st = P.lib().pic_load_particles(box.h, 0, -0.01, 1.0, N, P.C.cast(tx.data_ptr(), P._D),
                                            P.C.cast(tu.data_ptr(), P._D), P.C.cast(ti.data_ptr(), P._U32))
            assert st == P.PIC_OK, P.pic_last_error(box.h)
        xo, uo, io, _ = box.particles(0)
        o = np.argsort(io)
        back = np.empty(N, dtype=np.int64)
        back[ids] = np.arange(N)
        assert np.array_equal(io[o], np.arange(N, dtype=np.uint32))
        assert np.abs(xo[o] - x[back]).max() <= 1e-5
        assert np.array_equal(uo[o], u[back].astype(np.float32).astype(np.float64))
        box.step(2)
        xo, uo, io, _ = box.particles(0)
        o = np.argsort(io)
        E, B, J = box.fields()
        # the same particles stepped from a pageable load (the reference path)
        ref = P.Box(cfg)
        try:
            ref.set_fields(z, z)
            ref.load(0, -0.01, 1.0, x, u, ids)
            ref.step(2)
            xr, ur, ir, _ = ref.particles(0)
            orr = np.argsort(ir)
            assert np.array_equal(xo[o], xr[orr]) and np.array_equal(uo[o], ur[orr])
            for a_, b_ in zip((E, B, J), ref.fields()):
                assert np.array_equal(a_, b_)
        finally:
            ref.close()
    finally:
        box.close()

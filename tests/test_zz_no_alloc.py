"""pic_field_energy_noalloc: the field energy for callers that cannot
allocate device memory (their memory is owned by a pool allocator, or
allocation is not allowed in their loop or callback), computed with scratch
compiled into the library.  Checked through the C ABI against the field
energies pic_diagnostics reports for the same fields, on two calls in a row
(E, then B) that reuse the shared static scratch.  Kept in its own file, which
pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_2602_15939_gb300 import build as B
from paper_2602_15939_gb300 import pic as P
from paper_2602_15939_gb300 import workloads as W


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [True, False])
def test_noalloc_field_energy_matches_diagnostics(fp64):
    import torch

    B.build()
    n = (24, 16, 12)
    box = P.Box(P.make_config(nx=n[0], ny=n[1], nz=n[2], order=2,
                              precision=P.PIC_FP64 if fp64 else P.PIC_FP32))
    try:
        E, Bf = W.random_fields(n, seed=3, b0=(0.1, 0.0, 0.3))
        box.set_fields(E, Bf)
        diag = box.diagnostics()
        Eg, Bg, _ = box.fields()  # the device values, as stored
    finally:
        box.close()
    dtype = torch.float64 if fp64 else torch.float32
    prec = P.PIC_FP64 if fp64 else P.PIC_FP32
    stream = torch.cuda.current_stream()
    lib = P.lib()
    tol = 1e-12 if fp64 else 1e-6
    for arr, want in ((Eg, diag.field_energy_E), (Bg, diag.field_energy_B)):
        dev = torch.from_numpy(np.ascontiguousarray(arr.reshape(3, -1))).to("cuda", dtype=dtype)
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.pic_field_energy_noalloc(ctypes.c_void_p(dev.data_ptr()), prec, dev.shape[1], 3,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == P.PIC_OK, P.pic_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, np.array(want[:]), rtol=tol, atol=0)
        # and against a sum written here: FP64 squares of the stored values
        indep = (arr.reshape(3, -1).astype(np.float64) ** 2).sum(axis=1) / (8 * np.pi)
        np.testing.assert_allclose(got, indep, rtol=1e-12, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [True, False])
def test_noalloc_large_then_small_call(fp64):
    """A field larger than the scratch's 1024 blocks of 256 threads cover in
    one pass (one 128^3 component per slot, all 8 slots: each block strides
    over the array), then a small single-component call on the same stream,
    which must not see the larger call's leftover partial sums.  Both against
    FP64 numpy sums of squares / 8 pi."""
    import torch

    B.build()
    dtype = torch.float64 if fp64 else torch.float32
    prec = P.PIC_FP64 if fp64 else P.PIC_FP32
    g = torch.Generator(device="cpu").manual_seed(5)
    big = torch.randn((8, 128 ** 3), generator=g, dtype=torch.float64).to(dtype)
    small = torch.randn((1, 1000), generator=g, dtype=torch.float64).to(dtype)
    stream = torch.cuda.current_stream()
    lib = P.lib()
    outs = []
    for host in (big, small):
        dev = host.to("cuda")
        out = torch.full((host.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.pic_field_energy_noalloc(ctypes.c_void_p(dev.data_ptr()), prec, host.shape[1], host.shape[0],
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == P.PIC_OK, P.pic_last_error(None)
        outs.append((out, dev, host))
    torch.cuda.synchronize()
    for out, _, host in outs:
        want = (host.double().numpy() ** 2).sum(axis=1) / (8 * np.pi)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_noalloc_rejects_too_many_components():
    import torch

    B.build()
    dev = torch.zeros(9 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    st = P.lib().pic_field_energy_noalloc(ctypes.c_void_p(dev.data_ptr()), P.PIC_FP64, 4, 9,
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == P.PIC_ERR_ARG
    assert "PIC_NOALLOC_MAX_COMPONENTS" in P.pic_last_error(None)

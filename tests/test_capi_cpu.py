"""The C-ABI library loads and exports every symbol include/pic.h declares,
and host-side validation rejects bad configurations -- no GPU needed."""
import ctypes

import pytest

from paper_2602_15939_gb300 import build as B
from paper_2602_15939_gb300 import pic as P


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_exports_every_declared_symbol():
    names = P.header_functions()
    assert len(names) >= 19
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(P.header_functions()) <= set(P._SIGS)


def test_version():
    assert P.pic_abi_version() == 1
    assert "sm_103a" in P.pic_version()


@pytest.mark.parametrize("kw,msg", [
    (dict(ndim=4), "ndim"),
    (dict(nx=4), "at least 8"),
    (dict(order=3), "shape_order"),
    (dict(c=0.7), "Courant"),
    (dict(ndim=2, plane=P.PIC_PLANE_XY, nz=8), "nz = 1"),
    (dict(box=P.PIC_BOX_LEAKY, escape_mode=P.PIC_ESC_DISPLACEMENT, l_esc=0.0, theta_inj=1.0), "l_esc"),
    (dict(box=P.PIC_BOX_SHEAR, s=1.5, Omega0=0.5, nx=64), "shear speed"),
])
def test_validation_rejects_bad_configs(kw, msg):
    base = dict(nx=8, ny=8, nz=8)
    base.update(kw)
    cfg = P.make_config(**base)
    with pytest.raises(P.PicError) as e:
        P.pic_init(cfg)
    assert e.value.status == P.PIC_ERR_ARG
    assert msg in str(e.value)


def test_null_handle_calls_fail_cleanly():
    lib = P.lib()
    assert lib.pic_step(None, 1) == P.PIC_ERR_ARG
    assert lib.pic_destroy(None) == P.PIC_OK
    assert lib.pic_synchronize(None) == P.PIC_ERR_ARG
    # capacity, regrouping and batch controls check their handles before any CUDA call
    k = ctypes.c_int32()
    n = ctypes.c_int64()
    assert lib.pic_set_regroup_interval(None, 3) == P.PIC_ERR_ARG
    assert lib.pic_get_regroup_interval(None, ctypes.byref(k)) == P.PIC_ERR_ARG
    assert lib.pic_set_capacity_check(None, 8, 1) == P.PIC_ERR_ARG
    assert lib.pic_rebalance(None, 0, ctypes.byref(k)) == P.PIC_ERR_ARG
    assert lib.pic_get_capacity(None, 0, ctypes.byref(n), None, None) == P.PIC_ERR_ARG
    assert lib.pic_batch_set_regroup_interval(None, 3) == P.PIC_ERR_ARG
    assert lib.pic_batch_step(None, 1) == P.PIC_ERR_ARG


def test_kernel_variant_table():
    n = P.pic_kernel_variant_count()
    assert n == 7
    shapes = [P.pic_kernel_variant_info(k) for k in range(1, n + 1)]
    assert shapes == [(256, 0, 1), (512, 0, 1), (512, 1, 1), (256, 1, 1), (256, 0, 2), (256, 1, 2), (512, 0, 4)]
    for bad in (0, n + 1):
        with pytest.raises(P.PicError):
            P.pic_kernel_variant_info(bad)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with libpic absent, loading the binding and creating a
    box both raise."""
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "libpic.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(P.LibraryMissing):
        P.lib()
    with pytest.raises(P.LibraryMissing):
        P.Box(P.make_config())

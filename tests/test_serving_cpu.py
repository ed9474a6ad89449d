"""Host-side logic of the run server (no GPU): the admission rule (FIFO
prefix that fits the HBM budget and the free slots; a lone run is always
admitted) and the device-footprint estimate used by it."""
import pytest

from paper_2602_15939_gb300 import build as B
from paper_2602_15939_gb300 import pic as P


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_admission_takes_fifo_prefix_within_budget():
    assert P.pic_admission_count(100, 0, 0, 8, [30, 30, 30, 30]) == 3
    assert P.pic_admission_count(100, 50, 1, 8, [30, 30, 30]) == 1
    assert P.pic_admission_count(100, 0, 0, 2, [10, 10, 10]) == 2          # slots
    assert P.pic_admission_count(100, 0, 6, 8, [10, 10, 10]) == 2          # slots in use
    assert P.pic_admission_count(100, 90, 2, 8, [20, 5]) == 0              # head-of-line waits
    assert P.pic_admission_count(100, 0, 0, 8, []) == 0


def test_admission_runs_an_oversized_job_alone():
    assert P.pic_admission_count(100, 0, 0, 8, [500, 10]) == 1
    assert P.pic_admission_count(100, 10, 1, 8, [500]) == 0


def _spec(**kw):
    base = dict(box=P.PIC_BOX_EXPAND, nx=32, ny=32, nz=32, order=2, precision=P.PIC_FP32, rate=(0, 1e-4, 1e-4))
    base.update(kw.pop("cfg", {}))
    return P.make_run_spec(P.make_config(**base), kw.pop("nsteps", 10), kw.pop("ppc", 16), 0.05, **kw)


def test_footprint_scales_with_particles_and_precision():
    small = P.pic_run_footprint(_spec(ppc=8))
    big = P.pic_run_footprint(_spec(ppc=32))
    f64 = P.pic_run_footprint(_spec(ppc=8, cfg=dict(precision=P.PIC_FP64)))
    assert big > small and f64 > small
    # particle arrays dominate: ~2 species x 2 buffers x 1.3 slack x 32 B x 32^3 x 32
    est = 2 * 2 * 1.3 * 32 * 32**3 * 32
    assert 0.9 * est < big < 1.6 * est


def test_footprint_rejects_bad_specs():
    with pytest.raises(P.PicError):
        P.pic_run_footprint(_spec(ppc=-1))

"""The benchmark's roofline arithmetic on CPU (no GPU): the algorithmic bytes
per particle-step of each configuration, the bytes per particle-kernel launch
that `roofline.achieved` divides by the launch time, the id and regroup
overhead, the issue-rate ceiling, and the reading of the committed ncu
summaries (used only while they were taken on the current kernel source).

The per-unit figures are those the step's definition fixes: each particle's
state (int32 cell, in-cell offsets of the active axes, three momentum
components; the id only where random numbers are drawn) read once and
written once, plus about 15 words per cell per field sweep of grid traffic,
shared by the particles of that cell."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2602_15939_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("name,particle,step", [
    # 3D FP32: 4 + 3*4 + 3*4 = 28 B, twice; 4 implicit sweeps x 60 B/cell over 64 particles per cell
    ("ksb3d_256_fp32", 56.0, 56.0 + 4 * 60 / 64),
    # 3D FP32, one leapfrog per step
    ("keb3d_128_fp32", 56.0, 56.0 + 60 / 64),
    # 2D FP32 with probabilistic escape: 4 + 2*4 + 3*4 + 4 (the id keys the escape draws) = 28 B
    ("leaky2d_2048_fp32", 56.0, 56.0 + 60 / 128),
    # 2D FP64: 4 + 2*8 + 3*8 = 44 B; 4 sweeps x 120 B/cell over 32 particles per cell
    ("ksb2d_64x64_fp64", 88.0, 88.0 + 4 * 120 / 32),
])
def test_bytes_per_particle_step(name, particle, step):
    m = bench.bytes_model(W.SUITE[name], 0)
    assert m["particle_bytes_per_particle_step"] == particle
    assert m["step_bytes_per_particle_step"] == pytest.approx(step, rel=1e-15)


def test_kernel_bytes_per_launch_of_the_headline():
    """256^3 cells, 32 particles per cell per species: 56 B per particle plus
    the kernel's own E, B reads and J write, 9 FP32 words per cell."""
    w = W.SUITE["ksb3d_256_fp32"]
    assert w.n_particles == 2 * 32 * 256 ** 3
    m = bench.bytes_model(w, 2)
    assert m["kernel_bytes_per_launch"] == 56 * w.n_particles + 36 * 256 ** 3 == 60733521920


@pytest.mark.parametrize("every,regroup", [(0, 0.0), (2, 32.0), (3, 64 / 3)])
def test_overhead_of_stored_id_and_regroup(every, regroup):
    """The layout stores the 4-byte id for read-back even where no random
    numbers are drawn (8 B per particle-step, read and written); a regroup
    every k steps copies the 32 stored bytes once (read and write) per k."""
    m = bench.bytes_model(W.SUITE["ksb3d_256_fp32"], every)["overhead_bytes_per_particle_step"]
    assert m["stored_id_and_unused_components"] == 8
    assert m["regroup_pass"] == pytest.approx(regroup, rel=1e-15)


def test_issue_roofline_arithmetic(monkeypatch):
    """Warp instructions per launch (per 32 particles, times the particles)
    over the launch time, against one warp instruction per scheduler (4 per
    SM) per cycle."""
    import torch

    class Props:
        multi_processor_count = 152

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda *_: Props())
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    r = bench.issue_roofline(1711.0, 2 ** 30, 70.4, 2070.0)
    assert r["achieved"] == pytest.approx(1711.0 * 2 ** 30 / 32 / 0.0704, rel=1e-15)
    assert r["peak"] == 152 * 4 * 2070e6
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-15)
    assert bench.issue_roofline(None, 2 ** 30, 70.4, 2070.0) is None


def test_stored_traffic_follows_the_kernel_source(monkeypatch):
    """The committed summaries give the DRAM bytes per full-size launch for
    the launch variant (and 2D tile side) they were taken on, and only while
    the particle kernel's sources hash to the profiled version."""
    hashes = set()
    for name in W.SUITE:
        p = os.path.join(ROOT, "profiles", f"tile_kernel_{name}.md")
        if os.path.exists(p):
            for line in open(p):
                if line.startswith("kernel_source_hash:"):
                    hashes.add(line.split(":")[1].strip())
    if hashes != {bench.kernel_source_hash()}:
        pytest.skip("the kernel sources changed since the summaries were taken (traffic reported as null)")
    assert bench.stored_traffic("ksb3d_256_fp32", 7) == pytest.approx(6.707e10)
    assert bench.stored_traffic("ksb3d_256_fp32", 3) is None        # a variant that was not captured
    assert bench.stored_traffic("leaky2d_2048_fp32", 2, 32) is not None
    assert bench.stored_traffic("leaky2d_2048_fp32", 2, 16) is None  # another tile side
    assert bench.stored_instructions("ksb3d_256_fp32", 7) == 1711.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.stored_traffic("ksb3d_256_fp32", 7) is None
    assert bench.stored_instructions("ksb3d_256_fp32", 7) is None


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 2, 500.0) == 1000 * 4 * 2 / 0.5
    assert math.isclose(bench.whole_job_rate(2 ** 30, 20, 1, 81.0 * 20), 2 ** 30 / 0.081)


def test_l2_note_tells_which_configurations_fit_in_l2():
    """Timed steps on a state larger than the 129 MB L2 need no flush; the
    64^2 FP64 box's 12 MiB state stays in L2 and is labelled so."""
    assert bench.l2_note(W.SUITE["ksb3d_256_fp32"]).startswith("inputs larger than L2 (64.0 GiB")
    assert bench.l2_note(W.SUITE["ksb2d_64x64_fp64"]).startswith("inputs fit in L2 (12 MiB")

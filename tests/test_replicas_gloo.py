"""The N>1 path of bench.py on CPU: world-size-2 gloo process groups.

The PIC box does not shard (replicas only), so the multi-rank logic is the
timing reduction (max over ranks), the whole-job rate (units every rank
processed over that time), per-rank replica seeds, and the reference arm's
rank-0-only rule.  Each rank here runs a tiny oracle replica on its own seed.
"""
import json
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, fn, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, fn(rank, world)))
    except Exception as e:  # reported to the parent, which fails the test
        out.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def _run(fn, world=2, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, fn, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=timeout) for _ in ps)
    for p in ps:
        p.join(timeout)
        assert p.exitcode == 0
    return [res[r] for r in range(world)]


def _timing(rank, world):
    import bench

    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    ms = bench.max_over_ranks(10.0 + 7.5 * rank, w)
    return {"ms": ms, "value": bench.whole_job_rate(1000, 4, w, ms), "seed": bench.replica_seed(r)}


def test_max_over_ranks_and_whole_job_rate():
    res = _run(_timing)
    assert all(r["ms"] == 17.5 for r in res), res
    # 2 ranks x 1000 units x 4 steps in the slowest rank's 17.5 ms
    assert all(abs(r["value"] - 8000 / 17.5e-3) < 1e-6 for r in res), res
    assert res[0]["seed"] != res[1]["seed"]


def _replica(rank, world):
    """One oracle step of a tiny shearing box on the rank's own seed; the
    ranks share nothing but the timing and the gathered checksums."""
    import torch
    import torch.distributed as dist

    import bench
    import oracle as O
    from paper_2602_15939_gb300 import workloads as W

    w = W.SHEAR_2D_FP64
    n = (8, 1, 8)
    sp = W.host_maxwellian(w, bench.replica_seed(rank), n=n, ppc=2)
    kw = w.config_kwargs()
    p = O.make_params(*n, w.c, order=w.order, box=O.BOX_SHEAR, s=w.s, Omega0=kw["Omega0"])
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    for c, v in enumerate(w.b0()):
        B[c] = v
    st = O.State(p, E, B, sp)
    st.step(1)
    npart = sum(len(d["x"]) for d in st.species)
    chk = float(sum(np.abs(d["u"]).sum() for d in st.species))
    t = torch.tensor([chk, float(npart)], dtype=torch.float64)
    allv = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(allv, t)
    return {"checksums": [float(a[0]) for a in allv], "counts": [int(a[1]) for a in allv]}


def test_replicas_are_independent():
    res = _run(_replica)
    assert res[0] == res[1]
    cs, counts = res[0]["checksums"], res[0]["counts"]
    assert counts[0] == counts[1] == 2 * 2 * 64
    assert cs[0] != cs[1]


def _reference_arm(rank, world):
    import contextlib
    import io

    import bench

    args = type("A", (), {"workload": "ksb2d_64x64_fp64", "steps": 1, "warmup": 0, "gpus": world})()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(args)
    return {"rc": rc, "out": buf.getvalue()}


@pytest.mark.slow
def test_reference_arm_rank0_only():
    res = _run(_reference_arm, timeout=300)
    assert res[0]["rc"] == 0 and res[1]["rc"] == 0
    assert res[1]["out"] == ""
    line = json.loads(res[0]["out"].strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"

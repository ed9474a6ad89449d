#!/usr/bin/env python
"""Throughput benchmark of the PIC step (particle-steps/s) on GB300.

Default workload: the 3D expanding-box pair plasma, 128^3 cells, 32 particles
per cell per species (134,217,728 particles), quadratic shapes, FP32 particle
state (int32 cell + float offsets) with FP64 expansion factors -- a seeded
synthetic stand-in shaped like the paper's expanding-box setup (Sec. 3.3).
A "step" is one full PIC step: sort-in-place, gather, push, deposit, current
fold and the transformed Maxwell update.  Inputs (4.3 GB of particles) are
larger than the L2 cache, so no flush is needed between steps.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (weak scaling;
the box does not shard), timing is the max over ranks of CUDA-event time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit), FP32 vs FP64; ensemble p99 latency"
UNIT = "particle-steps/s"


BOX_NAMES = {0: "periodic", 1: "shearing", 2: "expanding", 3: "leaky"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="keb3d_128_fp32")
    ap.add_argument("--grid", default=None, help="override the grid, e.g. 64,64,64 (profiling a smaller case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-runs", type=int, default=64)
    ap.add_argument("--kernel-only", action="store_true", help="warmup + timed steps only (for profiler runs)")
    ap.add_argument("--batch-legs-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--seed", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--variant", type=int, default=0,
                    help="particle-kernel variant (1-based); 0 = autotune on the box after warm-up")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank):
    """Seed of the replica a rank runs: independent boxes, no shared data."""
    return 1000 * rank


def max_over_ranks(x, world, device="cpu"):
    """Maximum of a per-rank scalar over all ranks: the job's time is that of
    its slowest replica.  Works on any process-group backend (NCCL on the GPU,
    gloo in the CPU tests)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, world, ms):
    """Whole-job throughput: units every rank processed per second of the
    (max-over-ranks) timed region."""
    return units_per_rank * steps * world / (ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("particle.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2602_15939_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stored_traffic(workload, variant):
    """DRAM bytes per launch of the particle kernel (launch variant `variant`)
    from the committed ncu summary, if it was taken on the current kernel
    source."""
    p = os.path.join(ROOT, "profiles", f"tile_kernel_{workload}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_launch_full_size\[v%d\]:\s*([0-9.eE+]+)" % variant, txt)
    if not m_hash or not m_b or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(w, n_sub, steps, seed=0):
    """Particle-steps/s of the FP64 CPU oracle on a sub-box of workload w."""
    import numpy as np

    import oracle as O
    from paper_2602_15939_gb300 import workloads as W

    sp = W.host_maxwellian(w, seed, n=n_sub)
    wp = w.units.omega_p
    box = {0: O.BOX_PERIODIC, 1: O.BOX_SHEAR, 2: O.BOX_EXPAND, 3: O.BOX_LEAKY}[w.box]
    kw = w.config_kwargs()
    p = O.make_params(*n_sub, w.c, order=w.order, box=box, s=w.s, Omega0=w.Omega0_wp * wp,
                      rate=tuple(r * wp for r in w.rate_wp), esc_mode=w.escape_mode,
                      p_esc=kw.get("p_esc", 0.0), l_esc=kw.get("l_esc", 0.0), theta_inj=w.theta_inj)
    E = np.zeros((3, n_sub[2], n_sub[1], n_sub[0]))
    B = np.zeros_like(E)
    for c, v in enumerate(w.b0()):
        B[c] = v
    st = O.State(p, E, B, sp)
    npart = sum(len(d["x"]) for d in sp)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st.step(1)
        times.append(time.perf_counter() - t0)
    return npart, times


def sub_box(w):
    if w.ndim == 3:
        return (16, 16, 16)
    return (64, 64, 1) if w.plane == 0 else (64, 1, 64)


def run_reference(args):
    from paper_2602_15939_gb300 import workloads as W

    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = W.SUITE[args.workload]
    n_sub = sub_box(w)
    npart, _ = oracle_rate(w, n_sub, 0)
    _, wt = oracle_rate(w, n_sub, args.warmup + args.steps)
    times = wt[args.warmup:]
    tot = sum(times)
    value = npart * len(times) / tot
    sample = f"{n_sub[0]}x{n_sub[1]}x{n_sub[2]} sub-box of {w.name}, {w.ppc} ppc/species ({npart} particles), " \
             f"{len(times)} timed steps after {args.warmup} warm-up"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": sample, "box": "expanding" if w.box == 2 else str(w.box)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def particle_bytes(fp64, ndim, leaky_disp):
    """Algorithmic bytes per particle-step of the fused kernel: the particle
    state read once and written once (cell index, in-cell offsets, momentum,
    id, and the leaky displacement when tracked)."""
    es = 8 if fp64 else 4
    state = 4 + ndim * es + 3 * es + 4 + (3 * es if leaky_disp else 0)
    return 2 * state


def setup_box(w, device, stream, fp64=None, seed=0):
    from paper_2602_15939_gb300 import workloads as W

    return W.setup_box(w, device=device, stream=stream, fp64=fp64, seed=seed)


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2602_15939_gb300 import build as libbuild
    from paper_2602_15939_gb300 import pic as P
    from paper_2602_15939_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    libbuild.build()
    w = W.SUITE[args.workload]
    if args.grid:
        w = W.scaled(w, tuple(int(v) for v in args.grid.split(",")))
    stream = torch.cuda.Stream()
    box = setup_box(w, local, stream.cuda_stream, seed=replica_seed(rank))
    npart = w.n_particles
    box.step(args.warmup)
    # particle-kernel launch variant: autotuned on this machine (trial steps are
    # ordinary, untimed steps) unless forced
    if args.variant:
        P.pic_set_kernel_variant(box.h, args.variant)
        tune = {"chosen": args.variant, "how": "forced"}
    else:
        best, ms_v, taken = box.autotune(4)
        tune = {"chosen": best, "how": f"autotuned on {taken} untimed steps",
                "particle_ms_per_variant": [None if v is None else round(v, 4) for v in ms_v]}
    nt_, st_, jc_ = P.pic_kernel_variant_info(tune["chosen"])
    tune.update({"threads_per_cta": nt_, "stable_order": bool(st_), "current_copies": jc_})
    box.sync()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # timed region: K steps (CUDA-graph replay), CUDA events on the box's stream
    sampler = ClockSampler(local)
    sampler.start()
    P.pic_reset_profile(box.h)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    gpu_launches = int(P.pic_get_profile(box.h).launches)
    # second pass with per-kernel-group events (no graphs) for the roofline
    P.pic_set_profiling(box.h, True)
    P.pic_reset_profile(box.h)
    box.step(args.steps)
    box.sync()
    prof = P.pic_get_profile(box.h)
    P.pic_set_profiling(box.h, False)
    diag = box.diagnostics()
    assert diag.error_word == 0, diag.error_word
    ms = max_over_ranks(ms, world, device="cuda")
    value = whole_job_rate(npart, args.steps, world, ms)
    particle_ms = prof.ms_particle / max(1, prof.particle_launches)

    peak, peak_kind = measured_peaks()
    ncell = w.n[0] * w.n[1] * w.n[2]
    bpp = particle_bytes(w.fp64, w.ndim, w.escape_mode == 1)
    es = 8 if w.fp64 else 4
    alg_bytes = npart * bpp + ncell * (6 + 3) * es
    achieved = alg_bytes / (particle_ms / 1e3) / 1e9
    traffic = stored_traffic(w.name, tune["chosen"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "kernel": "tile_kernel (fused gather+push+deposit+sort)",
                "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_particle": bpp,
                "avg_launch_ms": particle_ms}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w.fp64 else "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.n), "ppc_per_species": w.ppc, "particles": npart,
                       "shape_order": w.order, "box": BOX_NAMES.get(w.box, str(w.box)), "expansion_rate_wp": list(w.rate_wp),
                       "precision": ("int32 cell + fp64 offsets/momenta" if w.fp64 else
                                     "int32 cell + fp32 offsets/momenta, fp64 l(t)"),
                       "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}",
                       "kernel_variant": tune, "regroup_every": P.pic_get_regroup_interval(box.h)},
            "particle_phase": {"value": npart / (particle_ms / 1e3), "unit": UNIT, "avg_launch_ms": particle_ms},
            "profile_ms_per_step": {"particle": prof.ms_particle / args.steps, "field": prof.ms_field / args.steps,
                                    "other": prof.ms_other / args.steps,
                                    "other_is": "loose kernel, tile bookkeeping, regroup by cell"},
            "gpu_launches": gpu_launches, "roofline": roofline, "clocks": clocks}

    # FP64 path on the same workload (the plain FP64 method), a few steps
    if not args.no_fp64 and not args.kernel_only:
        box.close()
        torch.cuda.synchronize()
        b64 = setup_box(w, local, stream.cuda_stream, fp64=True, seed=replica_seed(rank))
        b64.step(2)
        b64.sync()
        k64 = max(2, min(args.steps, 5))
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        b64.step(k64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        line["fp64"] = {"value": npart * k64 / (ms64 / 1e3), "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64}
        b64.close()
        box = None
    elif box is not None:
        box.close()

    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e and not args.kernel_only:
        line["e2e"] = run_e2e(w, local, stream, args.steps, rank)

    if not args.no_serving and not args.kernel_only:
        line["serving"] = run_serving(local, seed=rank, runs=args.serve_runs)
        line["batched_ensemble"] = batch_legs_subprocess(local, rank)

    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.kernel_only:
        n_sub = sub_box(w)
        n_o, times = oracle_rate(w, n_sub, 5)
        line["cpu_baseline"] = {"value": n_o * len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n_sub[0]}x{n_sub[1]}x{n_sub[2]} sub-box of {w.name} at {w.ppc} "
                                          f"ppc/species ({n_o} particles), 5 steps, single-threaded FP64 C"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving(device, seed=0, runs=64):
    """A bounded sample of the served-ensemble workload: a Poisson stream of
    independent shearing / expanding / leaky runs (2D and 3D, FP32) submitted
    to libpic's continuous-batching server; runs/s and time to result."""
    import threading

    import numpy as np

    from paper_2602_15939_gb300 import pic as P
    from paper_2602_15939_gb300 import workloads as W

    runs = W.served_ensemble(runs, seed=seed)
    specs = [W.run_spec_of(r) for r in runs]
    work = sum(2 * r["ppc"] * r["n"][0] * r["n"][1] * r["n"][2] * r["steps"] for r in runs)
    srv = P.Server(device=device, hbm_budget_bytes=96 << 30, max_active=32, steps_per_round=10)
    tickets = []
    t0 = time.perf_counter()

    def feeder():
        for r, spec in zip(runs, specs):
            dt = r["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(spec))

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    srv.wait(0, 600)
    wall = time.perf_counter() - t0
    lat = sorted(srv.poll(t)[1] for t in tickets)
    info = srv.stats()
    srv.close()
    return {"runs": len(runs), "runs_per_s": len(runs) / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "particle_steps_per_s": work / wall,
            "peak_active": int(info.peak_active), "wall_s": wall,
            "sample": "Poisson arrivals (mean gap 2 ms); shearing/expanding/leaky x 2D (32^2-128^2) / 3D (16^3-32^3); "
                      "8-32 ppc/species; 20-100 steps; FP32"}


def run_batch_leg(device, steps=20, seed=0, nbox=16, sizes=(32, 48, 64)):
    """Batched against separate stepping of an ensemble of one kind: nbox 3D
    expanding boxes with grids drawn from `sizes` (cubes) at 8-32 ppc per
    species (FP32, quadratic shapes).  Batched: one Batch, one persistent
    particle kernel per step, graph-replayed.  Separate: each box with its own
    graphs, either one after another on one stream or all at once on their
    own streams."""
    import torch

    from paper_2602_15939_gb300 import pic as P
    from paper_2602_15939_gb300 import workloads as W

    runs = W.ensemble_of_kind(nbox, box=2, ndim=3, seed=seed, sizes=sizes)
    npart = sum(2 * r["ppc"] * r["n"][0] * r["n"][1] * r["n"][2] for r in runs)
    out = {"boxes": len(runs), "particles": npart, "steps": steps,
           "grids": sorted(set(r["n"][0] for r in runs)),
           "sample": f"{nbox} x 3D expanding box, {min(sizes)}^3-{max(sizes)}^3, 8-32 ppc/species"}

    def timed(fn, stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    s = torch.cuda.Stream()
    boxes = [W.box_of_run(r, device, s.cuda_stream) for r in runs]
    for b in boxes:
        b.step(2)
    ms = timed(lambda: [b.step(steps) for b in boxes], s)
    out["separate_one_stream"] = npart * steps / (ms / 1e3)
    streams = [torch.cuda.Stream() for _ in boxes]
    for b, st in zip(boxes, streams):
        P.pic_set_stream(b.h, st.cuda_stream)
        b.step(2)
    torch.cuda.synchronize()

    def concurrent():
        ev = torch.cuda.Event()
        ev.record(s)
        for st in streams:
            st.wait_event(ev)
        for b in boxes:
            b.step(steps)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            s.wait_event(e)

    ms = timed(concurrent, s)
    out["separate_concurrent_streams"] = npart * steps / (ms / 1e3)
    with P.Batch(boxes) as bt:
        bt.step(2)
        bt.sync()
        t0 = time.perf_counter()
        bt.step(steps)
        bt.sync()
        ms = 1e3 * (time.perf_counter() - t0)
    out["batched"] = npart * steps / (ms / 1e3)
    out["unit"] = UNIT
    for b in boxes:
        b.close()
    return out


def batch_legs_subprocess(device, rank):
    """The batched-ensemble comparison, run in a child process of its own (its
    own CUDA context), so that nothing it does can affect this run's line."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", str(device)))
    cmd = [sys.executable, os.path.abspath(__file__), "--batch-legs-only", "--seed", str(rank)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env)
        if r.returncode == 0 and r.stdout.strip():
            return json.loads(r.stdout.strip().splitlines()[-1])
        return {"error": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"}
    except Exception as e:  # a failed comparison leg is reported, not fatal
        return {"error": repr(e)[:300]}


def run_e2e(w, device, stream, steps, rank):
    """Same metric through the public API with host buffers: load the whole
    particle state from pinned host memory, K x (step + diagnostics read-back),
    read the final particle state back; all inside the timed region."""
    import numpy as np
    import torch

    from paper_2602_15939_gb300 import pic as P
    from paper_2602_15939_gb300 import workloads as W

    sp = W.host_maxwellian(w, 7 + rank)
    pinned = []
    for d in sp:
        n = len(d["x"])
        tx = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        tu = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        ti = torch.empty((n,), dtype=torch.int32, pin_memory=True)
        tx.numpy()[:] = d["x"]
        tu.numpy()[:] = d["u"]
        ti.numpy()[:] = d["id"].view(np.int32)
        pinned.append((d["q"], tx, tu, ti))
    del sp
    # pinned like the inputs (empty_like would give pageable memory)
    outs = [(torch.empty(tx.shape, dtype=tx.dtype, pin_memory=True), torch.empty(tu.shape, dtype=tu.dtype, pin_memory=True),
             torch.empty(ti.shape, dtype=ti.dtype, pin_memory=True)) for _, tx, tu, ti in pinned]
    cfg = P.make_config(precision=P.PIC_FP64 if w.fp64 else P.PIC_FP32, device=device, **w.config_kwargs())
    box = P.Box(cfg)
    P.pic_set_stream(box.h, stream.cuda_stream)
    npart = sum(len(t[1]) for t in pinned)
    lib = P.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, (q, tx, tu, ti) in enumerate(pinned):
        P._check(box.h, lib.pic_load_particles(box.h, s, q, 1.0, len(tx), P.C.cast(tx.data_ptr(), P._D),
                                               P.C.cast(tu.data_ptr(), P._D), P.C.cast(ti.data_ptr(), P._U32)))
    box.set_uniform_fields((0.0, 0.0, 0.0), w.b0())
    for _ in range(steps):
        box.step(1)
        box.diagnostics()
    for s, (ox, ou, oi) in enumerate(outs):
        P._check(box.h, lib.pic_get_particles(box.h, s, P.C.cast(ox.data_ptr(), P._D), P.C.cast(ou.data_ptr(), P._D),
                                              P.C.cast(oi.data_ptr(), P._U32), None))
    box.sync()
    dt = time.perf_counter() - t0
    box.close()
    h2d = sum(tx.numel() * 8 + tu.numel() * 8 + ti.numel() * 4 for _, tx, tu, ti in pinned)
    d2h = h2d + steps * P.C.sizeof(P.pic_diag)
    return {"value": npart * steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "steps": steps, "seconds": dt,
            "includes": "pic_load_particles from pinned host memory, per step pic_step + pic_diagnostics, "
                        "final pic_get_particles"}


def main():
    args = parse()
    if args.batch_legs_only:
        import torch

        torch.cuda.set_device(0)
        from paper_2602_15939_gb300 import build as libbuild

        libbuild.build()
        out = {"medium": run_batch_leg(0, seed=args.seed),
               "small": run_batch_leg(0, seed=args.seed, nbox=64, sizes=(16, 24, 32))}
        print(json.dumps(out), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())

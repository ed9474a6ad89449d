"""Seeded synthetic inputs shaped like the paper's setups.

This module holds only input generation and unit bookkeeping (no part of the
PIC method's arithmetic); both the CUDA path and the CPU oracle are fed from
it.  Units are code units: dx = dt = 1, c = Courant number.  The paper's
simulation data are not available, so every workload here is a seeded
stand-in with the same kind of plasma: a pair plasma (e-, e+) with total
density n0 = 2 ppc per cell, plasma frequency omega_p = c / d_e (d_e the skin
depth in cells), macro mass 1 and macro charge q = omega_p sqrt(1/(4 pi n0)),
guide field B0 from the cold magnetisation sigma = B0^2 / (4 pi n0 m c^2),
or from the plasma beta = n0 theta m c^2 / (B0^2 / 8 pi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class PairUnits:
    c: float
    skin_depth: float
    ppc: int  # per species

    @property
    def n0(self) -> float:
        return 2.0 * self.ppc

    @property
    def omega_p(self) -> float:
        return self.c / self.skin_depth

    @property
    def q(self) -> float:
        return self.omega_p * math.sqrt(1.0 / (4.0 * math.pi * self.n0))

    def b0_from_sigma(self, sigma: float) -> float:
        return math.sqrt(sigma * 4.0 * math.pi * self.n0 * self.c**2)

    def b0_from_beta(self, beta: float, theta: float) -> float:
        return math.sqrt(8.0 * math.pi * self.n0 * theta * self.c**2 / beta)


def uniform_plasma(n, ppc, seed, uth=0.1, drift=(0.0, 0.0, 0.0), charges=(-1.0, 1.0), q=0.05, ignorable=None):
    """Species dicts with ppc particles per cell uniformly placed, Gaussian
    momenta of deviation uth (cells/step) per component.  `ignorable` is the
    2D ignorable axis (its coordinate is set to 0.5)."""
    r = np.random.default_rng(seed)
    ncell = int(n[0]) * int(n[1]) * int(n[2])
    out = []
    next_id = 0
    for sign in charges:
        N = ncell * ppc
        x = r.uniform(0.0, 1.0, (N, 3)) * np.asarray(n, dtype=float)
        if ignorable is not None:
            x[:, ignorable] = 0.5
        u = r.normal(0.0, uth, (N, 3)) + np.asarray(drift, dtype=float)
        out.append({"q": sign * q, "m": 1.0, "x": x, "u": u,
                    "id": np.arange(next_id, next_id + N, dtype=np.uint32)})
        next_id += N
    return out


def random_fields(n, seed, e_amp=0.01, b_amp=0.05, b0=(0.0, 0.0, 0.0)):
    """E, B arrays [3][nz][ny][nx] with independent Gaussian values plus a
    uniform B0 (a single step is defined for any field)."""
    r = np.random.default_rng(seed)
    shape = (3, n[2], n[1], n[0])
    E = r.normal(0.0, e_amp, shape)
    B = r.normal(0.0, b_amp, shape)
    for c in range(3):
        B[c] += b0[c]
    return E, B


def smooth_fields(n, seed, e_amp=0.01, b_amp=0.05, modes=(1, 2), b0=(0.0, 0.0, 0.0)):
    """Sum of a few random-phase Fourier modes per component (periodic)."""
    r = np.random.default_rng(seed)
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    E = np.zeros((3, nz, ny, nx))
    B = np.zeros((3, nz, ny, nx))
    for arr, amp in ((E, e_amp), (B, b_amp)):
        for c in range(3):
            for m in modes:
                ph = r.uniform(0, 2 * math.pi, 3)
                kx = 2 * math.pi * m / nx
                ky = 2 * math.pi * m / ny if ny > 1 else 0.0
                kz = 2 * math.pi * m / nz if nz > 1 else 0.0
                arr[c] += amp * np.cos(kx * i + ph[0]) * np.cos(ky * j + ph[1]) * np.cos(kz * k + ph[2])
    for c in range(3):
        B[c] += b0[c]
    return E, B


@dataclass
class Workload:
    """A configuration of the paper-shaped benchmark suite."""
    name: str
    box: int
    ndim: int
    plane: int
    n: tuple
    ppc: int
    theta: float
    order: int
    fp64: bool
    steps: int
    c: float = 0.45
    skin_depth: float = 5.0
    sigma: float | None = None
    beta: float | None = None
    b_dir: tuple = (0.0, 0.0, 1.0)
    s: float = 0.0
    Omega0_wp: float = 0.0       # Omega0 in units of omega_p
    rate_wp: tuple = (0.0, 0.0, 0.0)  # expansion rates in units of omega_p
    escape_mode: int = 0
    t_esc_Lc: float = 0.0        # t_esc in units of L/c
    l_esc_L: float = 0.0         # l_esc in units of L
    theta_inj: float = 0.0
    noise: float = 0.0           # Gaussian momentum noise, units of c
    extra: dict = field(default_factory=dict)

    @property
    def units(self) -> PairUnits:
        return PairUnits(self.c, self.skin_depth, self.ppc)

    @property
    def n_particles(self) -> int:
        return 2 * self.ppc * self.n[0] * self.n[1] * self.n[2]

    def b0(self):
        u = self.units
        if self.sigma is not None:
            mag = u.b0_from_sigma(self.sigma)
        elif self.beta is not None:
            mag = u.b0_from_beta(self.beta, self.theta)
        else:
            mag = 0.0
        d = np.asarray(self.b_dir, dtype=float)
        return tuple(mag * d / np.linalg.norm(d))

    def config_kwargs(self):
        u = self.units
        wp = u.omega_p
        L = float(self.n[0])
        kw = dict(box=self.box, nx=self.n[0], ny=self.n[1], nz=self.n[2], ndim=self.ndim, plane=self.plane,
                  c=self.c, order=self.order, s=self.s, Omega0=self.Omega0_wp * wp,
                  rate=tuple(r * wp for r in self.rate_wp), escape_mode=self.escape_mode,
                  theta_inj=self.theta_inj)
        if self.escape_mode == 2:
            kw["p_esc"] = 1.0 / (self.t_esc_Lc * L / self.c)
        if self.escape_mode == 1:
            kw["l_esc"] = self.l_esc_L * L
        return kw


# The benchmark suite: synthetic stand-ins for the paper's three example
# setups (Sec. 2.3 MRI shearing box, Sec. 3.3 expanding firehose box, Sec. 4.2
# leaky turbulence box), with the sizes of the measured configurations.
SHEAR_2D_FP64 = Workload("ksb2d_64x64_fp64", box=1, ndim=2, plane=1, n=(64, 1, 64), ppc=16, theta=0.1, order=1,
                         fp64=True, steps=100, sigma=1.0, b_dir=(0, 0, 1), s=1.5, Omega0_wp=1e-3)
EXPAND_3D_FP32 = Workload("keb3d_128_fp32", box=2, ndim=3, plane=0, n=(128, 128, 128), ppc=32, theta=0.05, order=2,
                          fp64=False, steps=2000, sigma=0.5, b_dir=(1, 1, 0), rate_wp=(0.0, 1e-4, 1e-4))
SHEAR_3D_FP32 = Workload("ksb3d_256_fp32", box=1, ndim=3, plane=0, n=(256, 256, 256), ppc=32, theta=0.3, order=2,
                         fp64=False, steps=5000, beta=1e3, b_dir=(0, 0, 1), s=1.5, Omega0_wp=2e-3, noise=1e-3)
LEAKY_2D_FP32 = Workload("leaky2d_2048_fp32", box=3, ndim=2, plane=0, n=(2048, 2048, 1), ppc=64, theta=1.0, order=1,
                         fp64=False, steps=10000, sigma=0.1, b_dir=(0, 0, 1), escape_mode=2, t_esc_Lc=1.0,
                         theta_inj=1.0)

SUITE = {w.name: w for w in (SHEAR_2D_FP64, EXPAND_3D_FP32, SHEAR_3D_FP32, LEAKY_2D_FP32)}


def scaled(w: Workload, n, ppc=None, name=None) -> Workload:
    """The same workload on another grid (and optionally ppc)."""
    from dataclasses import replace
    return replace(w, n=tuple(n), ppc=ppc or w.ppc, name=name or f"{w.name}@{'x'.join(map(str, n))}")


def host_maxwellian(w: Workload, seed: int, n=None, ppc=None):
    """Host-side load of workload w (or a sub-box n): positions uniform,
    momenta isotropic with Gaussian components of variance theta c^2 for
    theta < 0.2 (nonrelativistic) -- an input recipe, not the reinjection law."""
    n = n or w.n
    ppc = ppc or w.ppc
    u = w.units
    uth = math.sqrt(w.theta) * w.c
    ign = None
    if w.ndim == 2:
        ign = 2 if w.plane == 0 else 1
    sp = uniform_plasma(n, ppc, seed, uth=uth, q=u.q, ignorable=ign)
    if w.noise:
        r = np.random.default_rng(seed + 1)
        for d in sp:
            d["u"] += r.normal(0.0, w.noise * w.c, d["u"].shape)
    return sp


def host_maxwellian_into(w: Workload, seed: int, x_out, u_out, id_out, id_base=0, chunk=1 << 22):
    """One species of workload w written straight into caller arrays
    (x_out[n][3], u_out[n][3], id_out[n], n = ppc x cells), chunk by chunk so
    that no temporary grows with n: positions uniform in the box (the 2D
    ignorable coordinate 0.5), momenta Gaussian with variance theta c^2 per
    component plus the workload's noise, ids id_base + 0..n-1.  An input recipe
    for host-side loads of large boxes, not the reinjection law."""
    n = len(x_out)
    r = np.random.default_rng(seed)
    ext = np.asarray(w.n, dtype=float)
    uth = math.sqrt(w.theta) * w.c
    sd = math.sqrt(uth * uth + (w.noise * w.c) ** 2)
    ign = None
    if w.ndim == 2:
        ign = 2 if w.plane == 0 else 1
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        x = r.random((b - a, 3)) * ext
        if ign is not None:
            x[:, ign] = 0.5
        x_out[a:b] = x
        u_out[a:b] = r.normal(0.0, sd, (b - a, 3))
        id_out[a:b] = np.arange(id_base + a, id_base + b, dtype=np.uint32)


def random_phase_dB(n, seed, modes=(2, 3, 4), amplitude=1.0):
    """In-plane magnetic perturbation of a 2D x-y box from a random-phase
    vector potential A_z(i, j) = sum a cos(k.x + phi) on the nodes, over mode
    numbers with |n| in `modes`: B_x(i, j+1/2) = A(i, j+1) - A(i, j) and
    B_y(i+1/2, j) = A(i, j) - A(i+1, j), so the Yee divergence vanishes
    identically; scaled to the given rms.  Returns the [3][1][ny][nx] array."""
    nx, ny = n[0], n[1]
    r = np.random.default_rng(seed)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A = np.zeros((ny, nx))
    for mx in range(-max(modes), max(modes) + 1):
        for my in range(-max(modes), max(modes) + 1):
            m2 = mx * mx + my * my
            if m2 == 0 or int(round(math.sqrt(m2))) not in modes:
                continue
            A += r.normal() * np.cos(2 * math.pi * (mx * i / nx + my * j / ny) + r.uniform(0, 2 * math.pi))
    bx = np.roll(A, -1, axis=0) - A
    by = A - np.roll(A, -1, axis=1)
    rms = math.sqrt((bx**2 + by**2).mean())
    B = np.zeros((3, 1, ny, nx))
    if rms > 0:
        B[0, 0] = bx * amplitude / rms
        B[1, 0] = by * amplitude / rms
    return B


def setup_box(w: Workload, device=0, stream=None, fp64=None, seed=0):
    """A libpic box for workload w on `device`, loaded as the benchmark
    does: the device Maxwellian loader for both species, uniform B0 (plus the
    random-phase dB of a leaky turbulence box), E = 0."""
    from . import pic as P

    fp64 = w.fp64 if fp64 is None else fp64
    cfg = P.make_config(precision=P.PIC_FP64 if fp64 else P.PIC_FP32, device=device, seed=seed,
                        **w.config_kwargs())
    box = P.Box(cfg)
    if stream is not None:
        P.pic_set_stream(box.h, stream)
    u = w.units
    box.load_maxwellian(0, -u.q, 1.0, w.ppc, w.theta, noise_sigma=w.noise * w.c, seed=seed, id_base=0)
    box.load_maxwellian(1, u.q, 1.0, w.ppc, w.theta, noise_sigma=w.noise * w.c, seed=seed + 1,
                        id_base=w.ppc * w.n[0] * w.n[1] * w.n[2])
    b0 = w.b0()
    if w.box == 3 and w.ndim == 2:
        B = random_phase_dB(w.n, seed + 2, amplitude=float(np.linalg.norm(b0)))
        for c in range(3):
            B[c] += b0[c]
        box.set_fields(np.zeros_like(B), B)
    else:
        box.set_uniform_fields((0.0, 0.0, 0.0), b0)
    return box


def served_ensemble(M, seed=0, full=False, mean_gap_s=0.002):
    """Seeded stream of M independent runs shaped like the served-ensemble
    configuration: shearing, expanding and leaky boxes, 2D and 3D, FP32, with
    s in [0.5, 1.8], expansion rate in [1e-5, 1e-3] omega_p, t_esc in
    [0.5, 4] L/c, Poisson arrivals.  full=True draws the configuration's own
    ranges (2D 32^2..512^2, 3D 32^3..96^3, 8..64 ppc, 200..2000 steps); the
    default draws a bounded sample (2D 32^2..128^2, 3D 16^3..32^3, 8..32 ppc,
    20..100 steps) for a benchmark that must finish in seconds.  Returns a
    list of dicts: arrival time (s) and the run's parameters."""
    r = np.random.default_rng(seed)
    n2 = [32, 64, 128, 256, 512] if full else [32, 48, 64, 96, 128]
    n3 = [32, 48, 64, 96] if full else [16, 24, 32]
    ppc_lo, ppc_hi = (8, 64) if full else (8, 32)
    st_lo, st_hi = (200, 2000) if full else (20, 100)
    t = 0.0
    out = []
    for k in range(M):
        t += r.exponential(mean_gap_s)
        box = int(r.choice([1, 2, 3]))
        ndim = int(r.choice([2, 3]))
        if ndim == 2:
            m = int(r.choice(n2))
            plane = 1 if box == 1 else 0
            n = (m, 1, m) if plane == 1 else (m, m, 1)
            order = 1
        else:
            m = int(r.choice(n3))
            n, plane, order = (m, m, m), 0, 2
        ppc = int(r.integers(ppc_lo, ppc_hi + 1))
        run = dict(arrival_s=t, box=box, ndim=ndim, plane=plane, n=n, order=order, ppc=ppc,
                   steps=int(r.integers(st_lo, st_hi + 1)), c=0.45, skin_depth=5.0, sigma=0.5,
                   s=float(r.uniform(0.5, 1.8)), Omega0_wp=1e-3,
                   rate_wp=float(10 ** r.uniform(-5, -3)), t_esc_Lc=float(r.uniform(0.5, 4.0)),
                   theta={1: 0.1, 2: 0.05, 3: 1.0}[box], seed=int(r.integers(0, 2**31)))
        out.append(run)
    return out


def run_spec_of(run):
    """libpic run spec (pic_run_spec) for one entry of served_ensemble."""
    from . import pic as P

    units = PairUnits(run["c"], run["skin_depth"], run["ppc"])
    wp = units.omega_p
    kw = dict(box=run["box"], nx=run["n"][0], ny=run["n"][1], nz=run["n"][2], ndim=run["ndim"], plane=run["plane"],
              c=run["c"], order=run["order"], precision=P.PIC_FP32, seed=run["seed"])
    b0 = units.b0_from_sigma(run["sigma"])
    B0 = (0.0, 0.0, b0)
    if run["box"] == 1:
        kw.update(s=run["s"], Omega0=run["Omega0_wp"] * wp)
    elif run["box"] == 2:
        kw.update(rate=(0.0, run["rate_wp"] * wp, run["rate_wp"] * wp if run["ndim"] == 3 else 0.0))
        B0 = (b0 / math.sqrt(2.0), b0 / math.sqrt(2.0), 0.0)
    else:
        kw.update(escape_mode=P.PIC_ESC_PROBABILISTIC, p_esc=1.0 / (run["t_esc_Lc"] * run["n"][0] / run["c"]),
                  theta_inj=run["theta"])
    cfg = P.make_config(**kw)
    return P.make_run_spec(cfg, run["steps"], run["ppc"], run["theta"], q=(-units.q, units.q), B0=B0,
                           load_seed=run["seed"])


def ensemble_of_kind(M, box=2, ndim=3, seed=0, sizes=(32, 48, 64), ppc_range=(8, 32)):
    """M runs of one kind (box type, dimensionality: a batchable class of the
    served ensemble) with uneven grids and densities, drawn like
    served_ensemble's entries; used to compare batched and separate
    stepping."""
    r = np.random.default_rng(seed)
    out = []
    for k in range(M):
        m = int(r.choice(sizes))
        if ndim == 2:
            plane = 1 if box == 1 else 0
            n = (m, 1, m) if plane == 1 else (m, m, 1)
            order = 1
        else:
            n, plane, order = (m, m, m), 0, 2
        out.append(dict(arrival_s=0.0, box=box, ndim=ndim, plane=plane, n=n, order=order,
                        ppc=int(r.integers(ppc_range[0], ppc_range[1] + 1)), steps=0, c=0.45, skin_depth=5.0,
                        sigma=0.5, s=float(r.uniform(0.5, 1.8)), Omega0_wp=1e-3,
                        rate_wp=float(10 ** r.uniform(-5, -3)), t_esc_Lc=float(r.uniform(0.5, 4.0)),
                        theta={1: 0.1, 2: 0.05, 3: 1.0}[box], seed=int(r.integers(0, 2**31))))
    return out


def box_of_run(run, device=0, stream=None):
    """A loaded libpic box for one run dict (served_ensemble / ensemble_of_kind)."""
    from . import pic as P

    spec = run_spec_of(run)
    cfg = spec.cfg
    cfg.device = device
    box = P.Box(cfg)
    if stream is not None:
        P.pic_set_stream(box.h, stream)
    for s in range(spec.nspecies):
        box.load_maxwellian(s, spec.q[s], spec.m[s], spec.ppc, spec.theta, seed=spec.load_seed + s,
                            id_base=s * spec.ppc * cfg.nx * cfg.ny * cfg.nz)
    box.set_uniform_fields(tuple(spec.E0), tuple(spec.B0))
    return box

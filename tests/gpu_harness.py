"""Shared helpers of the GPU parity tests: run the same seeded case through
the CPU oracle and through libpic (C ABI via the ctypes binding) and compare
element by element.  Imported by tests only."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle as O
from paper_2602_15939_gb300 import pic as P
from paper_2602_15939_gb300 import workloads as W


@dataclass
class Case:
    name: str
    box: int
    n: tuple
    ndim: int = 3
    plane: int = 0
    order: int = 1
    ppc: int = 4
    uth: float = 0.15
    c: float = 0.45
    step0: int = 0
    s: float = 0.0
    Omega0: float = 0.0
    rate: tuple = (0.0, 0.0, 0.0)
    keb_exact: int = 0
    esc_mode: int = 0
    esc_dims: int = 2
    l_esc: float = 0.0
    p_esc: float = 0.0
    theta_inj: float = 0.0
    fp_iters: int = 4
    seed: int = 1
    b0: tuple = (0.0, 0.0, 0.2)
    tile: tuple = (0, 0, 0)
    q: float = 0.05
    drift: tuple = (0.0, 0.0, 0.0)
    slack: float = 0.0
    variant: int = 0
    masses: tuple = (1.0, 1.0)  # per species (electron, positive species)
    extra: dict = field(default_factory=dict)

    @property
    def ignorable(self):
        if self.ndim == 3:
            return None
        return 2 if self.plane == P.PIC_PLANE_XY else 1

    def oracle_params(self):
        return O.make_params(*self.n, self.c, order=self.order, box=self.box, fp_iters=self.fp_iters,
                             keb_exact=self.keb_exact, esc_mode=self.esc_mode, esc_dims=self.esc_dims,
                             seed=self.seed, s=self.s, Omega0=self.Omega0, rate=self.rate, l_esc=self.l_esc,
                             p_esc=self.p_esc, theta_inj=self.theta_inj)

    def gpu_config(self, fp64: bool):
        return P.make_config(box=self.box, nx=self.n[0], ny=self.n[1], nz=self.n[2], ndim=self.ndim,
                             plane=self.plane, c=self.c, order=self.order,
                             precision=P.PIC_FP64 if fp64 else P.PIC_FP32, fp_iters=self.fp_iters,
                             keb_push=self.keb_exact, escape_mode=self.esc_mode, escape_dims=self.esc_dims,
                             tile=self.tile, seed=self.seed, s=self.s, Omega0=self.Omega0, rate=self.rate,
                             l_esc=self.l_esc, p_esc=self.p_esc, theta_inj=self.theta_inj,
                             capacity_slack=self.slack, kernel_variant=self.variant)


def inputs(case: Case):
    sp = W.uniform_plasma(case.n, case.ppc, case.seed, uth=case.uth, q=case.q, ignorable=case.ignorable,
                          drift=case.drift)
    for d, m in zip(sp, case.masses):
        d["m"] = m  # u is the momentum per unit mass (gamma v): the same spread for every species
    E, B = W.random_fields(case.n, case.seed + 100, b0=case.b0)
    return sp, E, B


def run_oracle(case: Case, nsteps: int):
    sp, E, B = inputs(case)
    st = O.State(case.oracle_params(), E, B, sp, step=case.step0)
    info = st.step(nsteps)
    return st, info


def run_gpu(case: Case, nsteps: int, fp64: bool):
    sp, E, B = inputs(case)
    box = P.Box(case.gpu_config(fp64))
    box.set_fields(E, B)
    for i, d in enumerate(sp):
        box.load(i, d["q"], d["m"], d["x"], d["u"], d["id"])
    box.set_step(case.step0)
    box.step(nsteps)
    diag = box.diagnostics()
    parts = [box.particles(i, want_dr=case.esc_mode == 1) for i in range(len(sp))]
    fields = box.fields()
    box.close()
    return parts, fields, diag


def rel_maxerr(a, b, floor=0.0):
    """max |a - b| over the largest |b|, or over `floor` when that is larger"""
    scale = max(float(np.abs(b).max()), floor)
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())


def current_scale(case):
    """J_ref = |q| c n0: the current of the total density moving at c, the
    natural size of J in a cell; 4 pi J_ref is the field change it drives in
    one step."""
    return abs(case.q) * case.c * 2 * case.ppc


def compare(case: Case, nsteps: int, fp64: bool):
    """Returns a dict of max-norm relative errors (u, E, B, J), the maximum
    absolute position error (cells, periodic-aware) and escape counts."""
    st, info = run_oracle(case, nsteps)
    parts, (E, B, J), diag = run_gpu(case, nsteps, fp64)
    out = {"u": 0.0, "x": 0.0, "dr": 0.0}
    active = [a for a in range(3) if a != case.ignorable]
    n = np.asarray(case.n, dtype=float)
    for d, (x, u, ids, dr) in zip(st.species, parts):
        assert len(ids) == len(d["id"]), "particle count changed"
        og = np.argsort(ids)
        oo = np.argsort(d["id"])
        assert np.array_equal(ids[og], d["id"][oo]), "particle ids differ"
        xg, ug = x[og], u[og]
        xo, uo = d["x"][oo], d["u"][oo]
        dx = xg - xo
        dx -= n * np.round(dx / n)
        out["x"] = max(out["x"], float(np.abs(dx[:, active]).max()))
        out["u"] = max(out["u"], rel_maxerr(ug, uo))
        if dr is not None:
            out["dr"] = max(out["dr"], float(np.abs(dr[og] - d["dr"][oo]).max()))
    jref = 0.0 if fp64 else current_scale(case)
    out["E"] = rel_maxerr(E, st.E, 4 * np.pi * jref)
    out["B"] = rel_maxerr(B, st.B, 4 * np.pi * jref)
    out["J"] = rel_maxerr(J, st.J, jref)
    out["escaped_gpu"] = int(diag.escaped_total)
    out["escaped_oracle"] = int(info["escaped"])
    out["loose"] = int(diag.loose)
    out["error_word"] = int(diag.error_word)
    return out

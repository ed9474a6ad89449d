"""FP64 CPU oracle for the PIC step of arXiv 2602.15939 (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
it.  The product library never calls it, and it shares no code with the CUDA
path.  The arithmetic lives in ``pic_oracle.c`` (plain C, one particle and one
grid point at a time, in the paper's order); this module only compiles it with
gcc and marshals numpy arrays through ctypes.

Conventions (see ``pic_oracle.h``): code units dx = dt = 1; fields are
``[3][nz][ny][nx]`` float64 arrays without guard cells; positions absolute in
cells; momenta u = gamma v in cells/step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_HDR = os.path.join(_HERE, "pic_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BOX_PERIODIC, BOX_SHEAR, BOX_EXPAND, BOX_LEAKY, BOX_SHEAR_EXPAND = 0, 1, 2, 3, 4
ESC_NONE, ESC_DISPLACEMENT, ESC_PROBABILISTIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into a shared library with gcc (no -ffast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("order", C.c_int32), ("box", C.c_int32), ("fp_iters", C.c_int32),
        ("keb_exact", C.c_int32), ("esc_mode", C.c_int32), ("esc_dims", C.c_int32),
        ("seed", C.c_uint32),
        ("c", C.c_double), ("s", C.c_double), ("Omega0", C.c_double),
        ("rate", C.c_double * 3), ("l_esc", C.c_double), ("p_esc", C.c_double),
        ("theta_inj", C.c_double),
    ]


class Fields(C.Structure):
    _fields_ = [("E", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("J", C.POINTER(C.c_double)), ("step", C.c_int64)]


class Species(C.Structure):
    _fields_ = [("n", C.c_int64), ("q", C.c_double), ("m", C.c_double),
                ("x", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)),
                ("id", C.POINTER(C.c_uint32)), ("dr", C.POINTER(C.c_double))]


class StepInfo(C.Structure):
    _fields_ = [("escaped", C.c_int64), ("superluminal", C.c_int64)]


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER(Params)
            sig = {
                "ora_push_boris": (None, [C.c_double, C.c_double, C.c_double, _D, _D, _D]),
                "ora_push_ksb": (None, [C.c_double] * 6 + [_D, _D, _D, _D]),
                "ora_ksb_gamma_bar": (C.c_double, [C.c_double, C.c_double, C.c_double, _D, _D, _D]),
                "ora_push_keb": (None, [C.c_double, C.c_double, C.c_double, _D, _D, _D, _D, C.c_int]),
                "ora_philox4x32_10": (None, [_U32, _U32, _U32]),
                "ora_escape_draw": (C.c_int, [C.c_uint32, C.c_uint32, C.c_int64, C.c_double]),
                "ora_sample_mj": (C.c_int, [C.c_uint32, C.c_uint32, C.c_int64, C.c_double, C.c_double, _D]),
                "ora_shear_shift": (C.c_double, [P, C.c_double]),
                "ora_gather": (None, [P, _D, _D, C.c_double, _D, _D, _D]),
                "ora_deposit_current": (None, [P, _D, C.c_double, C.c_double, _D, _D]),
                "ora_deposit_rho": (None, [P, _D, C.c_double, C.c_double, _D]),
                "ora_ksb_advect_current": (None, [P, _D]),
                "ora_yee_update": (None, [P, _D, _D, _D]),
                "ora_keb_field_update": (None, [P, _D, _D, _D, C.c_double]),
                "ora_ksb_field_solve": (None, [P, _D, _D, _D, C.c_double]),
                "ora_ksb_rhs": (None, [P, _D, _D, _D, C.c_double, _D, _D]),
                "ora_step": (None, [P, C.POINTER(Fields), C.c_int, C.POINTER(Species),
                                    C.POINTER(StepInfo)]),
                "ora_advance_particle": (None, [P, _D, _D, _D, C.c_int64, C.c_double, C.c_double, C.c_uint32,
                                                _D, _D, _D, C.POINTER(StepInfo)]),
                "ora_push_sxe": (None, [C.c_double] * 6 + [_D, _D, _D, _D, _D]),
                "ora_sxe_rhs": (None, [P, _D, _D, _D, C.c_double, _D, _D]),
                "ora_sxe_advect_current": (None, [P, _D, C.c_double]),
                "ora_sxe_field_solve": (None, [P, _D, _D, _D, C.c_double]),
                "ora_set_threads": (None, [C.c_int]),
                "ora_max_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _vec(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3)).copy()


def make_params(nx, ny, nz, c, order=1, box=BOX_PERIODIC, fp_iters=4, keb_exact=0,
                esc_mode=ESC_NONE, esc_dims=2, seed=0, s=0.0, Omega0=0.0,
                rate=(0.0, 0.0, 0.0), l_esc=0.0, p_esc=0.0, theta_inj=0.0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.order, p.box, p.fp_iters, p.keb_exact = order, box, fp_iters, keb_exact
    p.esc_mode, p.esc_dims, p.seed = esc_mode, esc_dims, seed & 0xFFFFFFFF
    p.c, p.s, p.Omega0 = c, s, Omega0
    for a in range(3):
        p.rate[a] = rate[a]
    p.l_esc, p.p_esc, p.theta_inj = l_esc, p_esc, theta_inj
    return p


# ---- single-particle operators ------------------------------------------------

def push_boris(q, m, c, E, B, u):
    uu = _vec(u)
    lib().ora_push_boris(q, m, c, _dp(_vec(E)), _dp(_vec(B)), _dp(uu))
    return uu


def push_ksb(q, m, c, s, Omega0, xc, E, B, u):
    uu = _vec(u)
    gb = C.c_double()
    lib().ora_push_ksb(q, m, c, s, Omega0, xc, _dp(_vec(E)), _dp(_vec(B)), _dp(uu), C.byref(gb))
    return uu, gb.value


def ksb_gamma_bar(c, alpha1, alpha2, um, eps):
    res = C.c_double()
    g = lib().ora_ksb_gamma_bar(c, alpha1, alpha2, _dp(_vec(um)), _dp(_vec(eps)), C.byref(res))
    return g, res.value


def push_keb(q, m, c, Lam, E, B, u, exact=False):
    uu = _vec(u)
    lib().ora_push_keb(q, m, c, _dp(_vec(Lam)), _dp(_vec(E)), _dp(_vec(B)), _dp(uu), int(exact))
    return uu


def push_sxe(q, m, c, s, Omega0, xc, Lam, E, B, u):
    uu = _vec(u)
    gb = C.c_double()
    lib().ora_push_sxe(q, m, c, s, Omega0, xc, _dp(_vec(Lam)), _dp(_vec(E)), _dp(_vec(B)), _dp(uu), C.byref(gb))
    return uu, gb.value


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def escape_draw(pid, seed, step, p):
    return bool(lib().ora_escape_draw(pid & 0xFFFFFFFF, seed & 0xFFFFFFFF, step, p))


def sample_mj(pid, seed, step, theta, c):
    u = np.zeros(3)
    n = lib().ora_sample_mj(pid & 0xFFFFFFFF, seed & 0xFFFFFFFF, step, theta, c, _dp(u))
    return u, n


# ---- grid operators -------------------------------------------------------------

def shear_shift(p: Params, t: float) -> float:
    return lib().ora_shear_shift(C.byref(p), t)


def gather(p: Params, E, B, t, x):
    Ep, Bp = np.zeros(3), np.zeros(3)
    lib().ora_gather(C.byref(p), _dp(E), _dp(B), t, _dp(_vec(x)), _dp(Ep), _dp(Bp))
    return Ep, Bp


def deposit_current(p: Params, J, t, q, x0, x1):
    lib().ora_deposit_current(C.byref(p), _dp(J), t, q, _dp(_vec(x0)), _dp(_vec(x1)))


def deposit_rho(p: Params, rho, t, q, x):
    lib().ora_deposit_rho(C.byref(p), _dp(rho), t, q, _dp(_vec(x)))


def rho_of(p: Params, species_list, t=0.0):
    """Node charge density of all particles; species_list holds (q, x[n,3])."""
    rho = np.zeros((1, p.nz, p.ny, p.nx))
    for q, x in species_list:
        for row in np.asarray(x, dtype=np.float64):
            deposit_rho(p, rho, t, q, row)
    return rho[0]


def ksb_advect_current(p: Params, J):
    lib().ora_ksb_advect_current(C.byref(p), _dp(J))


def yee_update(p: Params, E, B, J):
    lib().ora_yee_update(C.byref(p), _dp(E), _dp(B), _dp(J))


def keb_field_update(p: Params, E, B, J, t):
    lib().ora_keb_field_update(C.byref(p), _dp(E), _dp(B), _dp(J), t)


def ksb_field_solve(p: Params, E, B, J, t):
    lib().ora_ksb_field_solve(C.byref(p), _dp(E), _dp(B), _dp(J), t)


def ksb_rhs(p: Params, E, B, J, t):
    FE, FB = np.zeros_like(E), np.zeros_like(B)
    lib().ora_ksb_rhs(C.byref(p), _dp(E), _dp(B), _dp(J), t, _dp(FE), _dp(FB))
    return FE, FB


def sxe_rhs(p: Params, E, B, J, t):
    FE, FB = np.zeros_like(E), np.zeros_like(B)
    lib().ora_sxe_rhs(C.byref(p), _dp(E), _dp(B), _dp(J), t, _dp(FE), _dp(FB))
    return FE, FB


def sxe_advect_current(p: Params, J, t):
    lib().ora_sxe_advect_current(C.byref(p), _dp(J), t)


def sxe_field_solve(p: Params, E, B, J, t):
    lib().ora_sxe_field_solve(C.byref(p), _dp(E), _dp(B), _dp(J), t)


def advance_particles(p: Params, E, B, step, q, m, ids, x, u, dr=None):
    """Advance a set of particles one step in given fields without depositing
    (gather, push, move, boundary, escape); returns new x, u, dr and counts."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3)).copy()
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 3)).copy()
    dr = np.zeros_like(x) if dr is None else np.ascontiguousarray(np.asarray(dr, dtype=np.float64).reshape(-1, 3)).copy()
    ids = np.asarray(ids, dtype=np.uint32)
    info = StepInfo()
    L = lib()
    for i in range(len(x)):
        L.ora_advance_particle(C.byref(p), _dp(E), _dp(B), None, int(step), q, m, int(ids[i]),
                               x[i].ctypes.data_as(_D), u[i].ctypes.data_as(_D), dr[i].ctypes.data_as(_D),
                               C.byref(info))
    return x, u, dr, {"escaped": info.escaped, "superluminal": info.superluminal}


def set_threads(n: int) -> None:
    """Threads of the particle loop of a step (1, the default, for tests)."""
    lib().ora_set_threads(int(n))


def max_threads() -> int:
    return int(lib().ora_max_threads())


# ---- whole steps ----------------------------------------------------------------

class State:
    """Fields and particles of one box, as float64 numpy arrays owned here."""

    def __init__(self, p: Params, E, B, species, step=0):
        self.p = p
        shape = (3, p.nz, p.ny, p.nx)
        self.E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(shape)).copy()
        self.B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(shape)).copy()
        self.J = np.zeros(shape)
        self.step_index = int(step)
        self.species = []
        for sp in species:
            n = len(sp["x"])
            d = {
                "q": float(sp["q"]), "m": float(sp["m"]),
                "x": np.ascontiguousarray(np.asarray(sp["x"], dtype=np.float64).reshape(n, 3)).copy(),
                "u": np.ascontiguousarray(np.asarray(sp["u"], dtype=np.float64).reshape(n, 3)).copy(),
                "id": np.ascontiguousarray(np.asarray(sp.get("id", np.arange(n)), dtype=np.uint32)).copy(),
            }
            dr = sp.get("dr")
            d["dr"] = (np.zeros((n, 3)) if dr is None
                       else np.ascontiguousarray(np.asarray(dr, dtype=np.float64).reshape(n, 3)).copy())
            self.species.append(d)

    def step(self, nsteps: int = 1):
        f = Fields(_dp(self.E), _dp(self.B), _dp(self.J), self.step_index)
        arr = (Species * len(self.species))()
        for a, d in zip(arr, self.species):
            a.n, a.q, a.m = len(d["x"]), d["q"], d["m"]
            a.x, a.u, a.dr = _dp(d["x"]), _dp(d["u"]), _dp(d["dr"])
            a.id = d["id"].ctypes.data_as(_U32)
        info = StepInfo()
        total = StepInfo()
        for _ in range(nsteps):
            lib().ora_step(C.byref(self.p), C.byref(f), len(self.species), arr, C.byref(info))
            total.escaped += info.escaped
            total.superluminal += info.superluminal
        self.step_index = int(f.step)
        return {"escaped": total.escaped, "superluminal": total.superluminal}

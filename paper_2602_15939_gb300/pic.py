"""ctypes binding of libpic (include/pic.h): the same entry points under the
same names, plus a small ``Box`` convenience wrapper.  Argument marshalling
only -- every step of the PIC path runs in the CUDA kernels of libpic.  The
binding fails loudly (``LibraryMissing``) when the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pic.h")

PIC_OK, PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA, PIC_ERR_TIMEOUT, PIC_ERR_STATE, PIC_ERR_NUMERIC = range(7)
PIC_BOX_PERIODIC, PIC_BOX_SHEAR, PIC_BOX_EXPAND, PIC_BOX_LEAKY, PIC_BOX_SHEAR_EXPAND = range(5)
PIC_PLANE_XY, PIC_PLANE_XZ = 0, 1
PIC_FP32, PIC_FP64 = 0, 1
PIC_KEB_CLOSED_FORM, PIC_KEB_EXACT = 0, 1
PIC_ESC_NONE, PIC_ESC_DISPLACEMENT, PIC_ESC_PROBABILISTIC = 0, 1, 2
PIC_MAX_SPECIES = 4

STATUS_NAMES = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_OOM", 3: "PIC_ERR_CUDA", 4: "PIC_ERR_TIMEOUT",
                5: "PIC_ERR_STATE", 6: "PIC_ERR_NUMERIC"}


class LibraryMissing(RuntimeError):
    pass


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pic_config(C.Structure):
    _fields_ = [
        ("box", C.c_int32), ("ndim", C.c_int32), ("plane", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("shape_order", C.c_int32), ("precision", C.c_int32), ("fp_iters", C.c_int32),
        ("keb_push", C.c_int32), ("escape_mode", C.c_int32), ("escape_dims", C.c_int32),
        ("tile", C.c_int32 * 3), ("device", C.c_int32),
        ("seed", C.c_uint32), ("kernel_variant", C.c_uint32),
        ("c", C.c_double), ("s_shear", C.c_double), ("Omega0", C.c_double),
        ("expand_rate", C.c_double * 3), ("l_esc", C.c_double), ("p_esc", C.c_double),
        ("theta_inj", C.c_double), ("capacity_slack", C.c_double),
    ]


class pic_diag(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("t", C.c_double), ("shear_shift", C.c_double), ("l", C.c_double * 3),
        ("field_energy_E", C.c_double * 3), ("field_energy_B", C.c_double * 3),
        ("kinetic_energy", C.c_double * PIC_MAX_SPECIES), ("count", C.c_int64 * PIC_MAX_SPECIES),
        ("escaped_total", C.c_int64), ("superluminal_total", C.c_int64), ("loose", C.c_int64),
        ("error_word", C.c_int32), ("reserved", C.c_int32),
    ]


class pic_profile(C.Structure):
    _fields_ = [("ms_particle", C.c_double), ("ms_field", C.c_double), ("ms_other", C.c_double),
                ("launches", C.c_int64), ("particle_launches", C.c_int64), ("particle_steps", C.c_int64)]


class pic_run_spec(C.Structure):
    _fields_ = [
        ("cfg", pic_config), ("nspecies", C.c_int32), ("ppc", C.c_int32), ("theta", C.c_double),
        ("q", C.c_double * PIC_MAX_SPECIES), ("m", C.c_double * PIC_MAX_SPECIES), ("drift", C.c_double * 3),
        ("noise_sigma", C.c_double), ("E0", C.c_double * 3), ("B0", C.c_double * 3),
        ("load_seed", C.c_uint32), ("keep_state", C.c_uint32), ("nsteps", C.c_int64),
    ]


class pic_server_info(C.Structure):
    _fields_ = [("queued", C.c_int32), ("active", C.c_int32), ("completed", C.c_int64),
                ("bytes_in_use", C.c_uint64), ("peak_bytes", C.c_uint64), ("peak_active", C.c_int32),
                ("cohorts_formed", C.c_int32)]


_lib = None
_lock = threading.Lock()
_H = C.c_void_p
_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)

_SIGS = {
    "pic_version": (C.c_char_p, []),
    "pic_abi_version": (C.c_int, []),
    "pic_init": (C.c_int, [C.POINTER(pic_config), C.POINTER(_H)]),
    "pic_destroy": (C.c_int, [_H]),
    "pic_last_error": (C.c_char_p, [_H]),
    "pic_set_stream": (C.c_int, [_H, C.c_void_p]),
    "pic_synchronize": (C.c_int, [_H]),
    "pic_load_particles": (C.c_int, [_H, C.c_int, C.c_double, C.c_double, C.c_int64, _D, _D, _U32]),
    "pic_load_maxwellian": (C.c_int, [_H, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, _D,
                                      C.c_double, C.c_uint32, C.c_uint32]),
    "pic_set_fields": (C.c_int, [_H, _D, _D]),
    "pic_set_uniform_fields": (C.c_int, [_H, _D, _D]),
    "pic_step": (C.c_int, [_H, C.c_int]),
    "pic_set_step": (C.c_int, [_H, C.c_int64]),
    "pic_diagnostics": (C.c_int, [_H, C.POINTER(pic_diag)]),
    "pic_get_count": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int64)]),
    "pic_clear_error": (C.c_int, [_H]),
    "pic_get_particles": (C.c_int, [_H, C.c_int, _D, _D, _U32, _D]),
    "pic_get_fields": (C.c_int, [_H, _D, _D, _D]),
    "pic_get_particles_sampled": (C.c_int, [_H, C.c_int, C.c_uint32, C.c_uint32, C.c_int64, _D, _D, _U32, _D,
                                            C.POINTER(C.c_int64)]),
    "pic_set_profiling": (C.c_int, [_H, C.c_int]),
    "pic_get_profile": (C.c_int, [_H, C.POINTER(pic_profile)]),
    "pic_reset_profile": (C.c_int, [_H]),
    "pic_preload_kernels": (C.c_int, [C.c_int32, C.c_int32]),
    "pic_rebalance": (C.c_int, [_H, C.c_int32, C.POINTER(C.c_int32)]),
    "pic_set_capacity_check": (C.c_int, [_H, C.c_int32, C.c_int32]),
    "pic_get_capacity": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pic_set_regroup_interval": (C.c_int, [_H, C.c_int32]),
    "pic_get_regroup_interval": (C.c_int, [_H, C.POINTER(C.c_int32)]),
    "pic_kernel_variant_count": (C.c_int, []),
    "pic_kernel_variant_info": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pic_get_kernel_variant": (C.c_int, [_H, C.POINTER(C.c_int32)]),
    "pic_set_kernel_variant": (C.c_int, [_H, C.c_int32]),
    "pic_take_result": (C.c_int, [_H, C.c_uint64, C.POINTER(_H)]),
    "pic_get_tile": (C.c_int, [_H, C.POINTER(C.c_int32)]),
    "pic_set_tile": (C.c_int, [_H, C.c_int32]),
    "pic_autotune_tile": (C.c_int, [_H, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "pic_autotune_regroup": (C.c_int, [_H, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double)]),
    "pic_batch_create": (C.c_int, [C.POINTER(_H), C.c_int32, C.POINTER(_H)]),
    "pic_batch_step": (C.c_int, [_H, C.c_int32]),
    "pic_batch_set_regroup_interval": (C.c_int, [_H, C.c_int32]),
    "pic_batch_synchronize": (C.c_int, [_H]),
    "pic_batch_destroy": (C.c_int, [_H]),
    "pic_batch_max_boxes_per_launch": (C.c_int32, [C.c_int32]),
    "pic_autotune": (C.c_int, [_H, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "pic_field_energy_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "pic_run_footprint": (C.c_int, [C.POINTER(pic_run_spec), C.POINTER(C.c_uint64)]),
    "pic_admission_count": (C.c_int, [C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_uint64), C.c_int]),
    "pic_server_create": (C.c_int, [C.c_int, C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "pic_submit": (C.c_int, [C.c_void_p, C.POINTER(pic_run_spec), C.POINTER(C.c_uint64)]),
    "pic_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int), C.POINTER(pic_diag), C.POINTER(C.c_double)]),
    "pic_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    "pic_server_stats": (C.c_int, [C.c_void_p, C.POINTER(pic_server_info)]),
    "pic_server_destroy": (C.c_int, [C.c_void_p]),
    "pic_server_set_batching": (C.c_int, [C.c_void_p, C.c_int]),
}


def header_functions(path: str = HEADER):
    """Names of every function the public header declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load libpic.so (built by paper_2602_15939_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LibraryMissing(f"libpic is not built ({LIB_PATH} missing); run paper_2602_15939_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(h, st):
    if st != PIC_OK:
        msg = lib().pic_last_error(h)
        raise PicError(st, msg.decode() if msg else "")


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


# ---- the C entry points, same names ---------------------------------------------

def pic_version() -> str:
    return lib().pic_version().decode()


def pic_abi_version() -> int:
    return lib().pic_abi_version()


def pic_init(cfg: pic_config):
    h = _H()
    st = lib().pic_init(C.byref(cfg), C.byref(h))
    _check(None, st)
    return h


def pic_destroy(h):
    _check(h, lib().pic_destroy(h))


def pic_last_error(h=None) -> str:
    m = lib().pic_last_error(h)
    return m.decode() if m else ""


def pic_set_stream(h, stream: int | None):
    _check(h, lib().pic_set_stream(h, C.c_void_p(stream) if stream else None))


def pic_synchronize(h):
    _check(h, lib().pic_synchronize(h))


def pic_load_particles(h, species, q, m, x, u, ids=None):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    n = len(x)
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        idp = ids.ctypes.data_as(_U32)
    _check(h, lib().pic_load_particles(h, species, q, m, n, _dptr(x), _dptr(u), idp))


def pic_load_maxwellian(h, species, q, m, ppc, theta, drift=(0.0, 0.0, 0.0), noise_sigma=0.0, seed=0, id_base=0):
    d = np.ascontiguousarray(drift, dtype=np.float64)
    _check(h, lib().pic_load_maxwellian(h, species, q, m, ppc, theta, _dptr(d), noise_sigma, seed & 0xFFFFFFFF,
                                        id_base & 0xFFFFFFFF))


def pic_set_fields(h, E, B):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    _check(h, lib().pic_set_fields(h, _dptr(E), _dptr(B)))


def pic_set_uniform_fields(h, E, B):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    _check(h, lib().pic_set_uniform_fields(h, _dptr(E), _dptr(B)))


def pic_set_step(h, step):
    _check(h, lib().pic_set_step(h, step))


def pic_step(h, nsteps=1):
    _check(h, lib().pic_step(h, nsteps))


def pic_diagnostics(h) -> pic_diag:
    d = pic_diag()
    _check(h, lib().pic_diagnostics(h, C.byref(d)))
    return d


def pic_get_count(h, species) -> int:
    n = C.c_int64()
    _check(h, lib().pic_get_count(h, species, C.byref(n)))
    return n.value


def pic_get_particles(h, species, want_dr=False):
    n = pic_get_count(h, species)
    x = np.zeros((n, 3))
    u = np.zeros((n, 3))
    ids = np.zeros(n, dtype=np.uint32)
    dr = np.zeros((n, 3)) if want_dr else None
    _check(h, lib().pic_get_particles(h, species, _dptr(x), _dptr(u), ids.ctypes.data_as(_U32), _dptr(dr)))
    return x, u, ids, dr


def pic_get_particles_sampled(h, species, modulus, remainder, max_out):
    """The particles with id % modulus == remainder (any order): x, u, ids, dr."""
    x = np.zeros((max_out, 3))
    u = np.zeros((max_out, 3))
    ids = np.zeros(max_out, dtype=np.uint32)
    dr = np.zeros((max_out, 3))
    n = C.c_int64()
    _check(h, lib().pic_get_particles_sampled(h, species, modulus, remainder, max_out, _dptr(x), _dptr(u),
                                              ids.ctypes.data_as(_U32), _dptr(dr), C.byref(n)))
    k = min(n.value, max_out)
    return x[:k], u[:k], ids[:k], dr[:k]


def pic_get_fields(h, shape):
    E, B, J = (np.zeros(shape) for _ in range(3))
    _check(h, lib().pic_get_fields(h, _dptr(E), _dptr(B), _dptr(J)))
    return E, B, J


def pic_set_profiling(h, enable=True):
    _check(h, lib().pic_set_profiling(h, int(enable)))


def pic_get_profile(h) -> pic_profile:
    p = pic_profile()
    _check(h, lib().pic_get_profile(h, C.byref(p)))
    return p


def pic_reset_profile(h):
    _check(h, lib().pic_reset_profile(h))


def pic_rebalance(h, force=False) -> bool:
    g = C.c_int32()
    _check(h, lib().pic_rebalance(h, int(force), C.byref(g)))
    return bool(g.value)


def pic_set_capacity_check(h, every=8, block=True):
    _check(h, lib().pic_set_capacity_check(h, every, int(block)))


def pic_get_capacity(h, species: int):
    """(slots per tile, loose-list room, re-layouts so far) of a species."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(h, lib().pic_get_capacity(h, species, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def pic_set_regroup_interval(h, every: int):
    _check(h, lib().pic_set_regroup_interval(h, every))


def pic_get_regroup_interval(h) -> int:
    k = C.c_int32()
    _check(h, lib().pic_get_regroup_interval(h, C.byref(k)))
    return k.value


def pic_preload_kernels(device=0, precision=None):
    _check(None, lib().pic_preload_kernels(device, PIC_FP32 if precision is None else precision))


def pic_kernel_variant_count() -> int:
    return lib().pic_kernel_variant_count()


def pic_kernel_variant_info(k: int):
    """(threads per CTA, stable stayer order 0/1, current-box copies) of
    particle-kernel variant k (1-based)."""
    nt, st, jc = C.c_int32(), C.c_int32(), C.c_int32()
    _check(None, lib().pic_kernel_variant_info(k, C.byref(nt), C.byref(st), C.byref(jc)))
    return nt.value, st.value, jc.value


def pic_get_kernel_variant(h) -> int:
    k = C.c_int32()
    _check(h, lib().pic_get_kernel_variant(h, C.byref(k)))
    return k.value


def pic_set_kernel_variant(h, k: int):
    _check(h, lib().pic_set_kernel_variant(h, k))


def pic_autotune(h, trial_steps: int = 4):
    """Time every fitting particle-kernel variant on live steps and keep the
    fastest: returns (best variant, ms per variant (None where it does not
    fit), steps taken)."""
    n = pic_kernel_variant_count()
    best, taken = C.c_int32(), C.c_int64()
    ms = (C.c_double * n)()
    _check(h, lib().pic_autotune(h, trial_steps, C.byref(best), ms, C.byref(taken)))
    return best.value, [v if v >= 0 else None for v in ms], taken.value


def pic_autotune_regroup(h, candidates=(2, 3, 4, 6), cycles: int = 2):
    """Time whole regroup cycles for each candidate interval and keep the
    fastest: returns (best interval, ms per step per candidate)."""
    n = len(candidates)
    arr = (C.c_int32 * n)(*candidates)
    ms = (C.c_double * n)()
    best = C.c_int32()
    _check(h, lib().pic_autotune_regroup(h, arr, n, cycles, C.byref(best), ms))
    return best.value, list(ms)


def pic_get_tile(h):
    """The particle tile in cells per axis (1 on an ignorable axis)."""
    t = (C.c_int32 * 3)()
    _check(h, lib().pic_get_tile(h, t))
    return tuple(t)


def pic_set_tile(h, side: int):
    """Re-lay the particles out in tiles of `side` cells per axis (2D: 8, 16,
    or 32 in FP32; 3D: 4 or 8)."""
    _check(h, lib().pic_set_tile(h, side))


def pic_autotune_tile(h, trial_steps: int = 4):
    """Time the tile shapes of a box (2D: 8 x 8, 16 x 16 and, FP32, 32 x 32;
    3D: 4^3 and 8^3), each with its best launch variant, and keep the
    fastest: returns (best side, {side: ms per step})."""
    best = C.c_int32()
    ms = (C.c_double * 3)()
    _check(h, lib().pic_autotune_tile(h, trial_steps, C.byref(best), ms))
    sides = (4, 8) if pic_get_tile(h)[2] > 1 and pic_get_tile(h)[1] > 1 else (8, 16, 32)
    return best.value, {s: ms[k] for k, s in enumerate(sides) if ms[k] >= 0}


class Batch:
    """Boxes of one kind stepped together (pic_batch_*): one persistent
    particle kernel per step over all their tiles, graph-replayed."""

    def __init__(self, boxes):
        self.boxes = list(boxes)
        arr = (_H * len(self.boxes))(*[b.h for b in self.boxes])
        out = _H()
        _check(None, lib().pic_batch_create(arr, len(self.boxes), C.byref(out)))
        self.b = out

    def step(self, n=1):
        _check(None, lib().pic_batch_step(self.b, n))

    def set_regroup_interval(self, every: int):
        _check(None, lib().pic_batch_set_regroup_interval(self.b, every))

    def sync(self):
        _check(None, lib().pic_batch_synchronize(self.b))

    def close(self):
        if self.b:
            lib().pic_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_batch_max_boxes_per_launch(precision=None) -> int:
    return lib().pic_batch_max_boxes_per_launch(PIC_FP32 if precision is None else precision)


def pic_field_energy_noalloc(d_field: int, precision: int, n: int, ncomp: int, d_out: int, stream: int | None = None):
    """Allocation-free field energy of a caller-owned device array (raw device
    pointers as integers); see include/pic.h."""
    _check(None, lib().pic_field_energy_noalloc(C.c_void_p(d_field), precision, n, ncomp, C.c_void_p(d_out),
                                                C.c_void_p(stream) if stream else None))


# ---- convenience ------------------------------------------------------------------

def make_config(box=PIC_BOX_PERIODIC, nx=8, ny=8, nz=8, ndim=3, plane=PIC_PLANE_XY, c=0.45, order=1,
                precision=PIC_FP64, fp_iters=4, keb_push=PIC_KEB_CLOSED_FORM, escape_mode=PIC_ESC_NONE,
                escape_dims=2, tile=(0, 0, 0), seed=0, s=0.0, Omega0=0.0, rate=(0.0, 0.0, 0.0), l_esc=0.0,
                p_esc=0.0, theta_inj=0.0, capacity_slack=0.0, device=0, kernel_variant=0) -> pic_config:
    cfg = pic_config()
    cfg.box, cfg.ndim, cfg.plane = box, ndim, plane
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.shape_order, cfg.precision, cfg.fp_iters, cfg.keb_push = order, precision, fp_iters, keb_push
    cfg.escape_mode, cfg.escape_dims = escape_mode, escape_dims
    for a in range(3):
        cfg.tile[a] = tile[a]
        cfg.expand_rate[a] = rate[a]
    cfg.seed = seed & 0xFFFFFFFF
    cfg.c, cfg.s_shear, cfg.Omega0 = c, s, Omega0
    cfg.l_esc, cfg.p_esc, cfg.theta_inj, cfg.capacity_slack = l_esc, p_esc, theta_inj, capacity_slack
    cfg.device = device
    cfg.kernel_variant = kernel_variant
    return cfg


class Box:
    """One simulation box on the current CUDA device (thin owner of a handle)."""

    def __init__(self, cfg: pic_config, handle=None):
        self.cfg = cfg
        self.h = pic_init(cfg) if handle is None else handle
        self.shape = (3, cfg.nz, cfg.ny, cfg.nx)

    @classmethod
    def adopt(cls, handle, cfg: pic_config) -> "Box":
        """Own an existing handle (e.g. a served run's box from pic_take_result)."""
        return cls(cfg, handle=handle)

    def close(self):
        if self.h:
            pic_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, species, q, m, x, u, ids=None):
        pic_load_particles(self.h, species, q, m, x, u, ids)

    def load_maxwellian(self, species, q, m, ppc, theta, drift=(0, 0, 0), noise_sigma=0.0, seed=0, id_base=0):
        pic_load_maxwellian(self.h, species, q, m, ppc, theta, drift, noise_sigma, seed, id_base)

    def set_fields(self, E, B):
        pic_set_fields(self.h, E, B)

    def set_uniform_fields(self, E, B):
        pic_set_uniform_fields(self.h, E, B)

    def set_regroup_interval(self, every: int):
        pic_set_regroup_interval(self.h, every)

    def autotune(self, trial_steps=4):
        """Pick the fastest particle-kernel variant on live steps; see pic_autotune."""
        return pic_autotune(self.h, trial_steps)

    def autotune_regroup(self, candidates=(2, 3, 4, 6), cycles=2):
        """Pick the fastest regroup interval on live steps; see pic_autotune_regroup."""
        return pic_autotune_regroup(self.h, candidates, cycles)

    def tile(self):
        return pic_get_tile(self.h)

    def set_tile(self, side: int):
        pic_set_tile(self.h, side)

    def autotune_tile(self, trial_steps=4):
        """Pick the particle tile shape on live steps; see pic_autotune_tile."""
        return pic_autotune_tile(self.h, trial_steps)

    def step(self, n=1):
        pic_step(self.h, n)

    def set_step(self, step):
        pic_set_step(self.h, step)

    def sync(self):
        pic_synchronize(self.h)

    def diagnostics(self):
        return pic_diagnostics(self.h)

    def particles(self, species, want_dr=False):
        return pic_get_particles(self.h, species, want_dr)

    def fields(self):
        return pic_get_fields(self.h, self.shape)

    def particles_sampled(self, species, modulus, remainder=0, max_out=1 << 20):
        return pic_get_particles_sampled(self.h, species, modulus, remainder, max_out)

    def count(self, species):
        return pic_get_count(self.h, species)

    def clear_error(self):
        _check(self.h, lib().pic_clear_error(self.h))


# ---- serving -------------------------------------------------------------------------

def make_run_spec(cfg: pic_config, nsteps, ppc, theta, q=(-1.0, 1.0), m=(1.0, 1.0), drift=(0.0, 0.0, 0.0),
                  noise_sigma=0.0, E0=(0.0, 0.0, 0.0), B0=(0.0, 0.0, 0.0), load_seed=0,
                  keep_state=False) -> pic_run_spec:
    s = pic_run_spec()
    s.cfg = cfg
    s.nspecies = len(q)
    s.ppc, s.theta = ppc, theta
    for i, (qq, mm) in enumerate(zip(q, m)):
        s.q[i], s.m[i] = qq, mm
    for a in range(3):
        s.drift[a], s.E0[a], s.B0[a] = drift[a], E0[a], B0[a]
    s.noise_sigma, s.load_seed, s.nsteps = noise_sigma, load_seed & 0xFFFFFFFF, nsteps
    s.keep_state = 1 if keep_state else 0
    return s


def pic_run_footprint(spec: pic_run_spec) -> int:
    b = C.c_uint64()
    _check(None, lib().pic_run_footprint(C.byref(spec), C.byref(b)))
    return b.value


def pic_admission_count(budget, in_use, active, max_active, queued_bytes) -> int:
    arr = (C.c_uint64 * max(1, len(queued_bytes)))(*queued_bytes)
    return lib().pic_admission_count(budget, in_use, active, max_active, arr, len(queued_bytes))


class Server:
    """Continuous-batching run server (libpic's pic_server_*)."""

    def __init__(self, device=0, hbm_budget_bytes=64 << 30, max_active=64, steps_per_round=8, min_batch=0):
        h = C.c_void_p()
        _check(None, lib().pic_server_create(device, hbm_budget_bytes, max_active, steps_per_round, C.byref(h)))
        self.h = h
        self._specs = {}
        if min_batch:
            self.set_batching(min_batch)

    def set_batching(self, min_batch: int):
        """Step idle active runs of one kind as batches of at least min_batch
        runs (0: off); see pic_server_set_batching."""
        _check(None, lib().pic_server_set_batching(self.h, min_batch))

    def submit(self, spec: pic_run_spec) -> int:
        t = C.c_uint64()
        _check(None, lib().pic_submit(self.h, C.byref(spec), C.byref(t)))
        self._specs[t.value] = spec
        return t.value

    def poll(self, ticket):
        done = C.c_int()
        d = pic_diag()
        lat = C.c_double()
        _check(None, lib().pic_poll(self.h, ticket, C.byref(done), C.byref(d), C.byref(lat)))
        return (d, lat.value) if done.value else None

    def take(self, ticket) -> "Box":
        """The final box of a run submitted with keep_state (pic_take_result)."""
        h = _H()
        _check(None, lib().pic_take_result(self.h, ticket, C.byref(h)))
        return Box.adopt(h, self._specs[ticket].cfg)

    def wait(self, ticket=0, timeout_s=600.0):
        _check(None, lib().pic_server_wait(self.h, ticket, timeout_s))

    def stats(self) -> pic_server_info:
        s = pic_server_info()
        _check(None, lib().pic_server_stats(self.h, C.byref(s)))
        return s

    def close(self):
        if self.h:
            lib().pic_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

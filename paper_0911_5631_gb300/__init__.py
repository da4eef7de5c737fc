"""GB300-native soft-sphere molecular dynamics (Rapaport, arXiv 0911.5631).

Thin ctypes binding of ``libmd.so`` (the CUDA library built from ``csrc/``;
C ABI in ``include/md.h``).  Every function here only marshals arguments:
all MD arithmetic runs in the library's sm_103a kernels.  Importing the
package never loads the library; the first call does, and raises
``MDLibraryMissing`` if it has not been built -- there is no CPU fallback.

The functions carry the C names (``md_create``, ``md_set_state``,
``md_step``, ``md_measure``, ``md_get_state``, ...); ``Simulation`` wraps a
handle for convenience.  Host arrays are numpy float64 N x 3; the
``*_device`` calls also accept CUDA tensors (anything with ``data_ptr()``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmd.so")

MD_OK = 0
MD_EINVAL = -1
MD_ENOMEM = -2
MD_ECUDA = -3
MD_ESTATE = -4
MD_EOVERFLOW = -5
MD_EUNSTABLE = -6
MD_ENODEV = -7

MD_PREC_MIXED = 0
MD_PREC_FP64 = 1

MD_BUILD_AUTO = 0
MD_BUILD_THREAD = 1
MD_BUILD_WARP = 2
_BUILD = {"auto": MD_BUILD_AUTO, "thread": MD_BUILD_THREAD, "warp": MD_BUILD_WARP}

MD_VARIANT_PLAIN_LOADS = 1
MD_VARIANT_LIST_ROWS = 2
MD_VARIANT_BLOCK64 = 4
MD_VARIANT_BLOCK256 = 8
VARIANTS = {"default": 0, "plain_loads": MD_VARIANT_PLAIN_LOADS, "list_rows": MD_VARIANT_LIST_ROWS,
            "block64": MD_VARIANT_BLOCK64, "block256": MD_VARIANT_BLOCK256}

WCA_RC = 2.0 ** (1.0 / 6.0)


class MDLibraryMissing(RuntimeError):
    pass


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d): %s" % (md_strerror(code), code, msg))
        self.code = code


class md_params(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("reorder_interval", C.c_int32),
        ("cell_list_only", C.c_int32),
        ("even_cells", C.c_int32),
        ("nbr_capacity", C.c_int32),
        ("use_graphs", C.c_int32),
        ("device", C.c_int32),
        ("shell_bins", C.c_int32),
        ("ushift", C.c_double),
        ("stream", C.c_void_p),
        ("build_kernel", C.c_int32),
        ("variant", C.c_int32),
        ("reserved", C.c_int64 * 5),
    ]


class md_plan_t(C.Structure):
    _fields_ = [
        ("G", C.c_int32 * 3),
        ("nbr_capacity", C.c_int32),
        ("n_cells", C.c_int64),
        ("w", C.c_double * 3),
        ("rn", C.c_double),
        ("ushift", C.c_double),
        ("device_bytes", C.c_int64),
    ]


class md_measure_t(C.Structure):
    _fields_ = [
        ("ke", C.c_double),
        ("pe", C.c_double),
        ("virial", C.c_double),
        ("pressure", C.c_double),
        ("temperature", C.c_double),
        ("e_tot_per_atom", C.c_double),
        ("volume", C.c_double),
        ("step", C.c_int64),
        ("rebuilds", C.c_int64),
        ("reorders", C.c_int64),
        ("list_entries", C.c_int64),
        ("max_neighbors", C.c_int32),
        ("max_occupancy", C.c_int32),
        ("nbr_capacity", C.c_int32),
        ("reserved", C.c_int32),
    ]


class md_kernel_stats_t(C.Structure):
    _fields_ = [
        ("launches", C.c_int64),
        ("step_kernel_launches", C.c_int64),
        ("step_kernel_ms", C.c_double),
        ("step_kernel_atoms", C.c_int64),
        ("step_kernel_bytes", C.c_int64),
        ("rebuilds_timed", C.c_int64),
        ("rebuild_ms", C.c_double),
    ]


class md_replica_desc(C.Structure):
    _fields_ = [
        ("box", C.c_double * 3),
        ("n", C.c_int64),
        ("rc", C.c_double),
        ("skin", C.c_double),
        ("dt", C.c_double),
        ("ushift", C.c_double),
        ("reorder_interval", C.c_int32),
        ("nbr_capacity", C.c_int32),
        ("reserved", C.c_int64 * 4),
    ]


# (name, restype, argtypes) of every exported function, in header order.
_H = C.c_void_p
_D3 = C.POINTER(C.c_double)
SIGNATURES = [
    ("md_default_params", None, [C.POINTER(md_params)]),
    ("md_plan", C.c_int, [_D3, C.c_int64, C.c_double, C.c_double, C.c_double, C.POINTER(md_params),
                          C.POINTER(md_plan_t)]),
    ("md_create", C.c_int, [_D3, C.c_int64, C.c_double, C.c_double, C.c_double, C.POINTER(md_params),
                            C.POINTER(_H)]),
    ("md_set_state", C.c_int, [_H, C.c_void_p, C.c_void_p]),
    ("md_set_state_device", C.c_int, [_H, C.c_void_p, C.c_void_p]),
    ("md_rescale", C.c_int, [_H, C.c_double]),
    ("md_step", C.c_int, [_H, C.c_int64]),
    ("md_measure", C.c_int, [_H, C.POINTER(md_measure_t)]),
    ("md_get_state", C.c_int, [_H, C.c_void_p, C.c_void_p]),
    ("md_get_state_device", C.c_int, [_H, C.c_void_p, C.c_void_p]),
    ("md_get_forces", C.c_int, [_H, C.c_void_p]),
    ("md_debug_cells", C.c_int, [_H, C.c_void_p]),
    ("md_debug_neighbors", C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_void_p,
                                     C.c_int64]),
    ("md_get_plan", C.c_int, [_H, C.POINTER(md_plan_t)]),
    ("md_set_profiling", C.c_int, [_H, C.c_int]),
    ("md_kernel_stats", C.c_int, [_H, C.POINTER(md_kernel_stats_t)]),
    ("md_sync", C.c_int, [_H]),
    ("md_destroy", None, [_H]),
    ("md_last_error", C.c_char_p, [_H]),
    ("md_selftest", C.c_int, [C.c_int64, C.POINTER(C.c_int64)]),
    ("md_forces_noalloc", C.c_int, [_D3, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    ("md_ensemble_create", C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(_H)]),
    ("md_ensemble_add", C.c_int, [_H, C.POINTER(md_replica_desc), C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_int32)]),
    ("md_ensemble_remove", C.c_int, [_H, C.c_int32]),
    ("md_ensemble_run", C.c_int, [_H, C.c_int32, C.c_void_p, C.c_void_p]),
    ("md_ensemble_sync", C.c_int, [_H]),
    ("md_ensemble_wait", C.c_int, [_H, C.c_int32]),
    ("md_ensemble_status", C.c_int, [_H, C.c_int32]),
    ("md_ensemble_measure", C.c_int, [_H, C.c_int32, C.POINTER(md_measure_t)]),
    ("md_ensemble_get_state", C.c_int, [_H, C.c_int32, C.c_void_p, C.c_void_p]),
    ("md_ensemble_times", C.c_int, [_H, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("md_ensemble_set_shape", C.c_int, [_H, C.c_int32, C.c_int32, C.c_int32, C.c_int64]),
    ("md_ensemble_autotune", C.c_int, [_H, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]),
    ("md_ensemble_replica_bytes", C.c_int64, [C.POINTER(md_replica_desc)]),
    ("md_ensemble_free_bytes", C.c_int64, [_H]),
    ("md_ensemble_destroy", None, [_H]),
    ("md_ensemble_last_error", C.c_char_p, [_H]),
    ("md_strerror", C.c_char_p, [C.c_int]),
]

MD_NOALLOC_MAX_ATOMS = 65536
MD_NOALLOC_MAX_CELLS = 65536

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libmd (raises MDLibraryMissing if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise MDLibraryMissing(
                    "libmd.so is not built; run `python -c \"import __graft_entry__ as g; g.build()\"`")
            L = C.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _box(box):
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    return b, b.ctypes.data_as(_D3)


def _host3(a, n, writable=False):
    a = np.asarray(a)
    if writable:
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (n, 3)
        return a
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n, 3):
        raise ValueError("expected an (%d, 3) array, got %s" % (n, a.shape))
    return a


def _check(code, h=None):
    if code != MD_OK:
        raise MDError(code, md_last_error(h))
    return code


# ---- C-named functions (argument marshalling only) -------------------------

def md_default_params() -> md_params:
    p = md_params()
    lib().md_default_params(C.byref(p))
    return p


def md_plan(box, n, rc, skin, dt, params: md_params | None = None) -> md_plan_t:
    b, bp = _box(box)
    out = md_plan_t()
    code = lib().md_plan(bp, int(n), float(rc), float(skin), float(dt),
                         C.byref(params) if params is not None else None, C.byref(out))
    _check(code)
    return out


def md_create(box, n, rc, skin, dt, params: md_params | None = None):
    b, bp = _box(box)
    h = C.c_void_p()
    code = lib().md_create(bp, int(n), float(rc), float(skin), float(dt),
                           C.byref(params) if params is not None else None, C.byref(h))
    _check(code)
    return h


def md_set_state(h, pos, vel, n):
    p, v = _host3(pos, n), _host3(vel, n)
    return _check(lib().md_set_state(h, p.ctypes.data, v.ctypes.data), h)


def md_set_state_device(h, pos_ptr: int, vel_ptr: int):
    return _check(lib().md_set_state_device(h, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr)), h)


def md_rescale(h, T):
    return _check(lib().md_rescale(h, float(T)), h)


def md_step(h, nsteps):
    return _check(lib().md_step(h, int(nsteps)), h)


def md_measure(h) -> md_measure_t:
    m = md_measure_t()
    _check(lib().md_measure(h, C.byref(m)), h)
    return m


def md_get_state(h, n):
    pos = np.empty((n, 3))
    vel = np.empty((n, 3))
    _check(lib().md_get_state(h, pos.ctypes.data, vel.ctypes.data), h)
    return pos, vel


def md_get_state_device(h, pos_ptr: int, vel_ptr: int):
    return _check(lib().md_get_state_device(h, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr)), h)


def md_get_forces(h, n):
    f = np.empty((n, 3))
    _check(lib().md_get_forces(h, f.ctypes.data), h)
    return f


def md_debug_cells(h, n):
    c = np.empty(n, dtype=np.int32)
    _check(lib().md_debug_cells(h, c.ctypes.data), h)
    return c


def md_debug_neighbors(h):
    cnt, ent = C.c_int64(), C.c_int64()
    _check(lib().md_debug_neighbors(h, C.byref(cnt), C.byref(ent), None, 0), h)
    pairs = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
    _check(lib().md_debug_neighbors(h, C.byref(cnt), C.byref(ent), pairs.ctypes.data, cnt.value), h)
    return pairs[:cnt.value], ent.value


def md_get_plan(h) -> md_plan_t:
    out = md_plan_t()
    _check(lib().md_get_plan(h, C.byref(out)), h)
    return out


def md_set_profiling(h, on: bool):
    return _check(lib().md_set_profiling(h, int(bool(on))), h)


def md_kernel_stats(h) -> md_kernel_stats_t:
    s = md_kernel_stats_t()
    _check(lib().md_kernel_stats(h, C.byref(s)), h)
    return s


def md_sync(h):
    return _check(lib().md_sync(h), h)


def md_destroy(h):
    if h:
        lib().md_destroy(h)


def md_last_error(h=None) -> str:
    s = lib().md_last_error(h)
    return s.decode() if s else ""


def md_selftest(n=1 << 22):
    f = (C.c_int64 * 4)()
    _check(lib().md_selftest(int(n), f))
    return list(f)


def md_forces_noalloc(box, n, rc, pos_ptr: int, f_ptr: int, pe_vir_ptr: int, ushift=None, stream=None):
    """Forces, U and W of one configuration without any device allocation
    (device pointers in and out; see include/md.h)."""
    b, bp = _box(box)
    code = lib().md_forces_noalloc(bp, int(n), float(rc), math.nan if ushift is None else float(ushift),
                                   C.c_void_p(pos_ptr), C.c_void_p(f_ptr), C.c_void_p(pe_vir_ptr),
                                   None if stream is None else C.c_void_p(int(stream)))
    return _check(code)


def md_strerror(code) -> str:
    try:
        s = lib().md_strerror(int(code))
        return s.decode() if s else ""
    except MDLibraryMissing:
        return "error"


# ---- convenience wrapper ----------------------------------------------------

def _struct_dict(s):
    out = {}
    for name, _ in s._fields_:
        if name.startswith("reserved"):
            continue
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


class Simulation:
    """One simulation handle: ``Simulation(box, n, rc, skin, dt, precision=...)``."""

    def __init__(self, box, n, rc=WCA_RC, skin=0.4, dt=0.005, precision="mixed", reorder_interval=100,
                 cell_list_only=False, even_cells=False, nbr_capacity=0, use_graphs=True, ushift=None,
                 stream=None, device=-1, shell_bins=True, build="auto", variant="default"):
        p = md_default_params()
        p.shell_bins = int(bool(shell_bins))
        p.build_kernel = _BUILD[build] if isinstance(build, str) else int(build)
        p.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        p.precision = MD_PREC_FP64 if precision in ("fp64", MD_PREC_FP64) else MD_PREC_MIXED
        p.reorder_interval = int(reorder_interval)
        p.cell_list_only = int(bool(cell_list_only))
        p.even_cells = int(bool(even_cells))
        p.nbr_capacity = int(nbr_capacity)
        p.use_graphs = int(bool(use_graphs))
        p.ushift = math.nan if ushift is None else float(ushift)
        p.stream = None if stream is None else int(stream)
        p.device = int(device)
        self.params = p
        self.n = int(n)
        self.box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)).copy()
        self.h = md_create(self.box, self.n, rc, skin, dt, p)

    def set_state(self, pos, vel):
        if hasattr(pos, "data_ptr"):
            md_set_state_device(self.h, pos.data_ptr(), vel.data_ptr())
        else:
            md_set_state(self.h, pos, vel, self.n)

    def rescale(self, T):
        md_rescale(self.h, T)

    def step(self, nsteps):
        md_step(self.h, nsteps)

    def measure(self) -> dict:
        return _struct_dict(md_measure(self.h))

    def get_state(self, pos_out=None, vel_out=None):
        if pos_out is not None:
            md_get_state_device(self.h, pos_out.data_ptr(), vel_out.data_ptr())
            return pos_out, vel_out
        return md_get_state(self.h, self.n)

    def forces(self):
        return md_get_forces(self.h, self.n)

    def cells(self):
        return md_debug_cells(self.h, self.n)

    def neighbor_pairs(self):
        return md_debug_neighbors(self.h)

    def plan(self) -> dict:
        return _struct_dict(md_get_plan(self.h))

    def set_profiling(self, on=True):
        md_set_profiling(self.h, on)

    def kernel_stats(self) -> dict:
        return _struct_dict(md_kernel_stats(self.h))

    def sync(self):
        md_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            md_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- ensembles -------------------------------------------------------------

def _ens_check(code, e):
    if code != MD_OK:
        raise MDError(code, lib().md_ensemble_last_error(e).decode())
    return code


def replica_desc(box, n, rc=WCA_RC, skin=0.4, dt=0.005, reorder_interval=100, nbr_capacity=0, ushift=None):
    d = md_replica_desc()
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    for k in range(3):
        d.box[k] = float(b[k])
    d.n = int(n)
    d.rc, d.skin, d.dt = float(rc), float(skin), float(dt)
    d.ushift = float("nan") if ushift is None else float(ushift)
    d.reorder_interval = int(reorder_interval)
    d.nbr_capacity = int(nbr_capacity)
    return d


def md_ensemble_replica_bytes(d: md_replica_desc) -> int:
    return int(lib().md_ensemble_replica_bytes(C.byref(d)))


class Ensemble:
    """Many independent mixed-form replicas in one device arena, advanced
    together by one launch per ``run`` (md_ensemble_* in md.h)."""

    def __init__(self, arena_bytes, max_replicas=4096, device=-1, stream=None):
        h = _H()
        code = lib().md_ensemble_create(int(arena_bytes), int(max_replicas), int(device), stream, C.byref(h))
        if code != MD_OK:
            raise MDError(code, lib().md_ensemble_last_error(None).decode())
        self.e = h
        self.n = {}

    def add(self, pos, vel, box, rc=WCA_RC, skin=0.4, dt=0.005, reorder_interval=100, nbr_capacity=0,
            ushift=None) -> int:
        n = np.asarray(pos).shape[0]
        d = replica_desc(box, n, rc, skin, dt, reorder_interval, nbr_capacity, ushift)
        p = _host3(pos, n)
        v = _host3(vel, n)
        rid = C.c_int32()
        _ens_check(lib().md_ensemble_add(self.e, C.byref(d), p.ctypes.data, v.ctypes.data, C.byref(rid)), self.e)
        self.n[rid.value] = n
        return rid.value

    def remove(self, rid):
        _ens_check(lib().md_ensemble_remove(self.e, int(rid)), self.e)
        self.n.pop(int(rid), None)

    def run(self, ids, nsteps):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        st = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int64), ids.shape))
        _ens_check(lib().md_ensemble_run(self.e, int(ids.size), ids.ctypes.data, st.ctypes.data), self.e)

    def sync(self):
        _ens_check(lib().md_ensemble_sync(self.e), self.e)

    def wait(self, in_flight=1):
        """Blocks until at most `in_flight` queued runs are unfinished."""
        _ens_check(lib().md_ensemble_wait(self.e, int(in_flight)), self.e)

    def status(self, rid) -> int:
        return int(lib().md_ensemble_status(self.e, int(rid)))

    def measure(self, rid) -> dict:
        m = md_measure_t()
        _ens_check(lib().md_ensemble_measure(self.e, int(rid), C.byref(m)), self.e)
        return _struct_dict(m)

    def get_state(self, rid):
        n = self.n[int(rid)]
        pos = np.empty((n, 3))
        vel = np.empty((n, 3))
        _ens_check(lib().md_ensemble_get_state(self.e, int(rid), pos.ctypes.data, vel.ctypes.data), self.e)
        return pos, vel

    def times(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        t0 = np.empty(ids.size)
        t1 = np.empty(ids.size)
        _ens_check(lib().md_ensemble_times(self.e, int(ids.size), ids.ctypes.data, t0.ctypes.data, t1.ctypes.data),
                   self.e)
        return t0, t1

    def set_shape(self, block=0, grid=0, cluster=0, team_atoms=0):
        _ens_check(lib().md_ensemble_set_shape(self.e, int(block), int(grid), int(cluster), int(team_atoms)),
                   self.e)

    def autotune(self, ids, probe_steps=20):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        b = C.c_int32()
        g = C.c_int32()
        _ens_check(lib().md_ensemble_autotune(self.e, int(ids.size), ids.ctypes.data, int(probe_steps), C.byref(b),
                                              C.byref(g)), self.e)
        return b.value, g.value

    def free_bytes(self) -> int:
        return int(lib().md_ensemble_free_bytes(self.e))

    def close(self):
        if getattr(self, "e", None):
            lib().md_ensemble_destroy(self.e)
            self.e = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

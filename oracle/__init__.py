"""FP64 CPU oracle for the soft-sphere MD step (test infrastructure).

This package is the independent reference the CUDA path is checked against.
It is NOT part of the product: only the test suite, the package smoke check
and the benchmark's CPU-baseline arm may import it.  It shares no code with
the CUDA library and never imports it.

The arithmetic lives in ``md_oracle.c`` (plain C, double precision, no FP
contraction); this module compiles it with gcc on first use and wraps it with
ctypes and numpy.  Every function follows a passage of Rapaport,
arXiv 0911.5631:

* ``pair``            -- Eq. (1) plus the soft-sphere shift (Sec. 3.1)
* ``cell_grid``       -- G_d = floor(L_d / r_n) (Sec. 3.1); ``even=True``
                         reproduces the cell counts of Tables 1 and 5
* ``wrap``/``cell_of``-- periodic wrap and cell assignment (Sec. 3.2, Sec. 4.2)
* ``pairs_cells``     -- linked-list cells, half-shell enumeration (Sec. 3.2)
* ``pairs_brute``     -- O(N^2) minimum-image definition of the pair set
* ``forces_cells`` / ``forces_brute`` / ``forces_sampled`` -- forces, U, W
* ``run``             -- the step loop (a)-(f) of Sec. 3.1 with a skin-based
                         neighbour list and the delta/2 rebuild rule

Two builds of the one source: ``liboracle.so`` (plain, single threaded) is
the parity reference every check uses; ``liboracle_omp.so`` (the same code
compiled with OpenMP) only times the oracle on all host cores
(``run(..., threaded=True)``); a CPU test pins it to the plain build.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

CFLAGS = ["-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared"]


def _build_one(path, extra, force):
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False, threaded: bool = True) -> str:
    """Compile md_oracle.c into liboracle.so beside it (gcc, no contraction)
    and, with threaded, also into liboracle_omp.so (-fopenmp)."""
    _build_one(_LIB, [], force)
    if threaded:
        _build_one(_LIB_OMP, ["-fopenmp"], force)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("rc", C.c_double),
        ("skin", C.c_double),
        ("dt", C.c_double),
        ("ushift", C.c_double),
        ("even_cells", C.c_int),
        ("rescale_every", C.c_int),
        ("rescale_until", C.c_int64),
        ("T_target", C.c_double),
    ]


def _load(threaded: bool = False):
    with _lock:
        if threaded in _libs:
            return _libs[threaded]
        lib = C.CDLL(_build_one(_LIB_OMP, ["-fopenmp"], False) if threaded else _build_one(_LIB, [], False))
        lib.orc_threads.restype = C.c_int
        d, i64, i32 = C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32)
        lib.orc_pair.argtypes = [C.c_double, C.c_double, d, d]
        lib.orc_cell_grid.argtypes = [d, C.c_double, C.c_int, C.POINTER(C.c_int)]
        lib.orc_cell_grid.restype = C.c_int
        lib.orc_wrap.argtypes = [i64, d, d]
        lib.orc_cell_of.argtypes = [i64, d, d, C.POINTER(C.c_int), i32]
        lib.orc_pairs_cells.argtypes = [i64, d, d, C.POINTER(C.c_int), C.c_double, i64, i32]
        lib.orc_pairs_cells.restype = i64
        lib.orc_pairs_brute.argtypes = [i64, d, d, C.c_double, i64, i32]
        lib.orc_pairs_brute.restype = i64
        lib.orc_pair_r2.argtypes = [d, d, i64, i64]
        lib.orc_pair_r2.restype = C.c_double
        lib.orc_forces_cells.argtypes = [i64, d, d, C.POINTER(C.c_int), C.c_double, C.c_double, d, d, d]
        lib.orc_forces_cells.restype = C.c_int
        lib.orc_forces_brute.argtypes = [i64, d, d, C.c_double, C.c_double, d, d, d]
        lib.orc_forces_sampled.argtypes = [i64, d, d, C.c_double, C.c_double, i64,
                                           C.POINTER(C.c_int64), d, d]
        lib.orc_neighbors_of.argtypes = [i64, d, d, C.c_double, i64, i64, C.POINTER(C.c_int64)]
        lib.orc_neighbors_of.restype = i64
        lib.orc_run.argtypes = [i64, d, d, C.POINTER(_Params), i64, d, d, d, d,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.orc_run.restype = C.c_int
        _libs[threaded] = lib
        return lib


def threads(threaded: bool = True) -> int:
    """Threads the (threaded) oracle runs on: OMP_NUM_THREADS, else all host
    cores; 1 for the plain build."""
    return int(_load(threaded).orc_threads())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _box(L):
    L = np.asarray(L, dtype=np.float64)
    if L.ndim == 0:
        L = np.full(3, float(L))
    return np.ascontiguousarray(L)


def _pos(p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert p.ndim == 2 and p.shape[1] == 3
    return p


def wca_shift(rc: float) -> float:
    """Shift added to Eq. (1): +epsilon for the soft-sphere cutoff 2^(1/6)
    (Sec. 3.1), none for a plain truncated Lennard-Jones cutoff."""
    return 1.0 if abs(rc - 2.0 ** (1.0 / 6.0)) <= 1e-12 * rc else 0.0


def pair(r2: float, ushift: float = 1.0):
    """(fr, u) for one pair at squared separation r2; force = fr * r_vec."""
    lib = _load()
    fr, u = C.c_double(), C.c_double()
    lib.orc_pair(float(r2), float(ushift), C.byref(fr), C.byref(u))
    return fr.value, u.value


def cell_grid(L, rn: float, even: bool = False):
    """(G, ok): per-dimension cell counts and whether all are >= 3."""
    lib = _load()
    L = _box(L)
    G = (C.c_int * 3)()
    rc = lib.orc_cell_grid(_dp(L), float(rn), int(bool(even)), G)
    return np.array(list(G), dtype=np.int64), rc == 0


def wrap(pos, L):
    lib = _load()
    p = _pos(pos).copy()
    L = _box(L)
    lib.orc_wrap(p.shape[0], _dp(p), _dp(L))
    return p


def cell_of(pos, L, G):
    lib = _load()
    p, L = _pos(pos), _box(L)
    Gc = (C.c_int * 3)(*[int(g) for g in G])
    out = np.empty(p.shape[0], dtype=np.int32)
    lib.orc_cell_of(p.shape[0], _dp(p), _dp(L), Gc, out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def _pairs(fn, *args, n_hint):
    cap = max(1024, n_hint)
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        m = fn(*args, cap, out.ctypes.data_as(C.POINTER(C.c_int32)))
        if m < 0:
            raise ValueError("oracle pair enumeration failed (bad geometry or memory)")
        if m <= cap:
            return out[:m].copy()
        cap = int(m)


def pairs_cells(pos, L, G, rcut, threaded=False):
    """Pairs (i < j) within rcut via the half-shell cell enumeration; the
    positions must already be wrapped into the region."""
    lib = _load(threaded)
    p, L = _pos(pos), _box(L)
    Gc = (C.c_int * 3)(*[int(g) for g in G])
    return _pairs(lib.orc_pairs_cells, p.shape[0], _dp(p), _dp(L), Gc, float(rcut),
                  n_hint=16 * p.shape[0])


def pairs_brute(pos, L, rcut):
    lib = _load()
    p, L = _pos(pos), _box(L)
    return _pairs(lib.orc_pairs_brute, p.shape[0], _dp(p), _dp(L), float(rcut),
                  n_hint=16 * p.shape[0])


def pair_r2(pos, L, i, j):
    lib = _load()
    p, L = _pos(pos), _box(L)
    return lib.orc_pair_r2(_dp(p), _dp(L), int(i), int(j))


def forces_cells(pos, L, G, rc, ushift, threaded=False):
    """(f, U, W) from the cell-list pair set within rc (Newton's third law)."""
    lib = _load(threaded)
    p, L = _pos(pos), _box(L)
    Gc = (C.c_int * 3)(*[int(g) for g in G])
    f = np.empty_like(p)
    U, W = C.c_double(), C.c_double()
    rc_ = lib.orc_forces_cells(p.shape[0], _dp(p), _dp(L), Gc, float(rc), float(ushift), _dp(f),
                               C.byref(U), C.byref(W))
    if rc_:
        raise ValueError("oracle cell forces failed")
    return f, U.value, W.value


def forces_brute(pos, L, rc, ushift):
    lib = _load()
    p, L = _pos(pos), _box(L)
    f = np.empty_like(p)
    U, W = C.c_double(), C.c_double()
    lib.orc_forces_brute(p.shape[0], _dp(p), _dp(L), float(rc), float(ushift), _dp(f),
                         C.byref(U), C.byref(W))
    return f, U.value, W.value


def forces_sampled(pos, L, rc, ushift, idx):
    """Forces and per-atom pair-energy sums of the atoms idx, each by an O(N)
    minimum-image scan (spot checks of large systems)."""
    lib = _load()
    p, L = _pos(pos), _box(L)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = np.empty((idx.size, 3))
    u = np.empty(idx.size)
    lib.orc_forces_sampled(p.shape[0], _dp(p), _dp(L), float(rc), float(ushift), idx.size,
                           idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(f), _dp(u))
    return f, u


def neighbors_of(pos, L, rcut, i):
    lib = _load()
    p, L = _pos(pos), _box(L)
    cap = 256
    while True:
        out = np.empty(cap, dtype=np.int64)
        m = lib.orc_neighbors_of(p.shape[0], _dp(p), _dp(L), float(rcut), int(i), cap,
                                 out.ctypes.data_as(C.POINTER(C.c_int64)))
        if m <= cap:
            return out[:m].copy()
        cap = int(m)


def run(pos, vel, L, rc, skin, dt, nsteps, ushift=None, even_cells=False, rescale_every=0,
        rescale_until=0, T_target=1.0, record=True, threaded=False):
    """Run the reference MD loop.  Returns a dict with the final (wrapped)
    positions, velocities and forces, per-step KE/PE/W arrays (index 0 is the
    initial state), the number of rebuilds after the initial build and the
    summed pair-list length over all builds.  threaded: the OpenMP build
    (timing only; the same pair lists, force sums in another order)."""
    lib = _load(threaded)
    p = _pos(pos).copy()
    v = np.ascontiguousarray(vel, dtype=np.float64).copy()
    assert v.shape == p.shape
    L = _box(L)
    if ushift is None:
        ushift = wca_shift(rc)
    P = _Params()
    P.L[:] = list(L)
    P.rc, P.skin, P.dt, P.ushift = float(rc), float(skin), float(dt), float(ushift)
    P.even_cells = int(bool(even_cells))
    P.rescale_every, P.rescale_until, P.T_target = int(rescale_every), int(rescale_until), float(T_target)
    n = p.shape[0]
    ke = np.empty(nsteps + 1) if record else None
    pe = np.empty(nsteps + 1) if record else None
    vir = np.empty(nsteps + 1) if record else None
    f = np.empty_like(p)
    nreb, psum = C.c_int64(), C.c_int64()
    nul = C.POINTER(C.c_double)()
    rc_ = lib.orc_run(n, _dp(p), _dp(v), C.byref(P), int(nsteps),
                      _dp(ke) if record else nul, _dp(pe) if record else nul,
                      _dp(vir) if record else nul, _dp(f), C.byref(nreb), C.byref(psum))
    if rc_:
        raise ValueError("oracle run failed with code %d" % rc_)
    return {"pos": p, "vel": v, "f": f, "ke": ke, "pe": pe, "vir": vir,
            "nrebuild": nreb.value, "npairs_sum": psum.value}

"""Shared helpers of the GPU parity tests: building and driving a
simulation through the C ABI, and comparing against the oracle."""
import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from paper_0911_5631_gb300 import build as mdbuild
from paper_0911_5631_gb300 import inputs

RC = md.WCA_RC
DT = 0.005

# Tolerances stated for the method: per-atom force relative RMS error of
# 1e-5 for FP32 pair arithmetic and 1e-12 for FP64.
FORCE_TOL = {"mixed": 1e-5, "fp64": 1e-12}


def ensure_built():
    mdbuild.build()
    md.lib()


def state(n, rho, T, seed, jitter=0.0, aspect=(1, 1, 1)):
    pos, vel, L = inputs.wca_state(n, rho, T, seed, jitter_amp=jitter, aspect=aspect)
    return pos, vel, L


def sim(pos, vel, L, skin=0.4, precision="mixed", **kw):
    s = md.Simulation(L, pos.shape[0], RC, skin, DT, precision=precision, **kw)
    s.set_state(pos, vel)
    return s


def rel_rms(a, b):
    d = np.asarray(a) - np.asarray(b)
    den = np.sqrt(np.mean(np.asarray(b) ** 2))
    return float(np.sqrt(np.mean(d * d)) / den) if den > 0 else float(np.sqrt(np.mean(d * d)))


def min_image(d, L):
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    return d - L * np.round(d / L)


def pair_set(pairs):
    return set(map(tuple, np.asarray(pairs).tolist()))


def assert_same_pairs(gpu_pairs, ref_pairs, pos_w, L, rcut, tol=1e-10):
    """Sets must agree except for pairs whose squared distance lies within
    rounding of rcut^2 (both sides decide in FP64 from different but
    mathematically equal expressions)."""
    a, b = pair_set(gpu_pairs), pair_set(ref_pairs)
    diff = a ^ b
    for (i, j) in diff:
        r2 = oracle.pair_r2(pos_w, L, i, j)
        assert abs(r2 - rcut * rcut) < tol, ("pair %d-%d at r2=%.17g differs" % (i, j, r2), len(diff))
    return len(diff)


def oracle_grid(L, rcut):
    G, ok = oracle.cell_grid(L, rcut)
    assert ok
    return G


gpu = pytest.mark.gpu

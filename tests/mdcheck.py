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


def sorted_pairs(pairs):
    """(i, j) rows with i < j, in lexicographic order."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    p = np.sort(p, axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def assert_same_pairs(gpu_pairs, ref_pairs, pos, L, rcut):
    """The two pair sets must be identical.  Both sides decide r^2 < rcut^2
    in FP64 with the same operation sequence on the same coordinates, so no
    difference is allowed; any pair that differs is listed with its
    r^2 - rcut^2 (the reference's minimum-image evaluation) before failing."""
    a, b = sorted_pairs(gpu_pairs), sorted_pairs(ref_pairs)
    if a.shape == b.shape and np.array_equal(a, b):
        return 0
    diff = pair_set(a) ^ pair_set(b)
    only_gpu = pair_set(a) - pair_set(b)
    lines = ["%d-%d (%s) r2 - rcut2 = %.3e" % (i, j, "gpu only" if (i, j) in only_gpu else "oracle only",
                                                oracle.pair_r2(pos, L, i, j) - rcut * rcut)
             for (i, j) in sorted(diff)[:20]]
    raise AssertionError("%d pairs differ:\n%s" % (len(diff), "\n".join(lines)))


def assert_same_cells(gpu_cells, pos, L, G):
    """Stored cells must equal the reference's cell rule on the reported
    positions, element by element; differing atoms are listed with the
    distance of each coordinate to the nearest cell face."""
    ref = oracle.cell_of(pos, L, G)
    bad = np.nonzero(np.asarray(gpu_cells) != ref)[0]
    if bad.size == 0:
        return
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    w = Lv / np.asarray(G)
    u = (np.asarray(pos)[bad] + Lv / 2) / w
    face = np.abs(u - np.round(u)) * w
    lines = ["atom %d gpu %d oracle %d, face distances %s" % (i, gpu_cells[i], ref[i], face[k])
             for k, i in enumerate(bad[:20])]
    raise AssertionError("%d cells differ:\n%s" % (bad.size, "\n".join(lines)))


def trajectory_tol(prec, f_rms, k):
    """(velocity, position) RMS bounds after k steps from the same state: k dt
    times the force error allowed per step, with a factor 10 for growth
    along the segment."""
    fe = FORCE_TOL[prec] * f_rms
    dv = 10.0 * k * DT * fe + (1e-7 if prec == "mixed" else 1e-14)
    return dv, k * DT * dv + 1e-13


def assert_trajectory_matches(p, v, ref, L, prec, k):
    """Positions and velocities after k steps against an oracle.run result
    from the same start, within trajectory_tol."""
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    dv, dx = trajectory_tol(prec, f_rms, k)
    ev = float(np.sqrt(np.mean((v - ref["vel"]) ** 2)))
    ex = float(np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)))
    assert ev <= dv, ("velocity RMS error", ev, dv)
    assert ex <= dx, ("position RMS error", ex, dx)
    return ev, ex


def oracle_grid(L, rcut):
    G, ok = oracle.cell_grid(L, rcut)
    assert ok
    return G


gpu = pytest.mark.gpu

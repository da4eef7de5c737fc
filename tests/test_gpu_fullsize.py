"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times (graphs, reorder every 100 steps): spot checks the oracle
can compute atom by atom, plus properties that hold at any size."""
import numpy as np
import pytest

import oracle
from mdcheck import (DT, FORCE_TOL, RC, assert_same_cells, assert_same_pairs, ensure_built, oracle_grid, rel_rms,
                     sim, state)
from paper_0911_5631_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _sampled_force_check(s, L, prec, nsample=64, seed=0):
    p, v = s.get_state()
    f = s.forces()
    n = p.shape[0]
    idx = np.random.default_rng(seed).choice(n, nsample, replace=False)
    fr, ur = oracle.forces_sampled(p, L, RC, 1.0, idx)
    assert rel_rms(f[idx], fr) <= FORCE_TOL[prec]
    scale = float(np.sqrt(np.mean(fr ** 2)))
    err = np.linalg.norm(f[idx] - fr, axis=1)
    assert np.all(err <= 20 * FORCE_TOL[prec] * (np.linalg.norm(fr, axis=1) + scale))
    return p, v, f


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_one_million_atoms(prec):
    # 1,048,576 atoms: FCC 64^3 x 4, rho 0.8, T 1, skin 0.4, reorder every 100
    cfg = inputs.WORKLOADS["wca_fcc64_n1m"]
    pos, vel, L = state(cfg["n"], cfg["rho"], cfg["T"], cfg["seed"])
    s = sim(pos, vel, L, skin=cfg["skin"], precision=prec, reorder_interval=100)
    s.step(300)
    m = s.measure()
    assert m["step"] == 300 and m["rebuilds"] > 5 and m["reorders"] >= 3
    p, v, f = _sampled_force_check(s, L, prec)
    # momentum: zero at start, conserved up to rounding
    assert np.abs(v.sum(axis=0)).max() < (1e-2 if prec == "mixed" else 1e-8)
    # the next in-trajectory rebuild (incremental re-binning, list rebuilt in
    # place, no reload): every cell and the whole pair set against the
    # reference on the positions of that moment
    G = np.array(s.plan()["G"])
    last = m["rebuilds"]
    for _ in range(40):
        s.step(1)
        if s.measure()["rebuilds"] > last:
            break
    assert s.measure()["rebuilds"] == last + 1
    p, v = s.get_state()
    assert_same_cells(s.cells(), p, L, G)
    pairs, entries = s.neighbor_pairs()
    rn = RC + cfg["skin"]
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    assert entries == 2 * len(pairs)
    assert 11.0 < entries / cfg["n"] < 13.0  # N_p / N_a near 12 for this state
    s.close()


@pytest.mark.parametrize("rho,T", [(1.0, 2.0), (0.6, 0.7)])
def test_eight_million_atoms(rho, T):
    # 8,388,608 atoms: FCC 128^3 x 4, mixed form; at rho 1.0 every
    # nearest-neighbour pair of the start lattice sits exactly on r_c
    n = 8388608
    pos, vel, L = state(n, rho, T, 3)
    s = sim(pos, vel, L, skin=0.4, precision="mixed")
    s.step(60)
    m = s.measure()
    assert m["step"] == 60
    _sampled_force_check(s, L, "mixed", nsample=24)
    s.close()


@pytest.mark.parametrize("rho,T", [(1.0, 2.0), (0.6, 0.7)])
def test_eight_million_energy_drift_and_oracle_segment(rho, T):
    # 8,388,608 atoms (FCC 128^3 x 4), mixed form: total energy per atom over
    # 10^4 steps after 500 steps of melting drifts by less than 1e-4; then an
    # FP64 oracle segment of 5 steps from the GPU's state agrees with the GPU's
    # own 5 steps within the trajectory tolerance
    n = 8388608
    pos, vel, L = state(n, rho, T, 3)
    s = sim(pos, vel, L, skin=0.4, precision="mixed", reorder_interval=100)
    s.step(500)
    e0 = s.measure()["e_tot_per_atom"]
    for _ in range(10):
        s.step(1000)
    m = s.measure()
    assert m["step"] == 10500
    assert abs(m["e_tot_per_atom"] - e0) < 1e-4
    p, v = s.get_state()
    k = 5
    ref = oracle.run(p, v, L, RC, 0.4, DT, k, record=False)
    s.step(k)
    p2, v2 = s.get_state()
    s.close()
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    dv = 10.0 * k * DT * FORCE_TOL["mixed"] * f_rms + 1e-7
    assert np.sqrt(np.mean((v2 - ref["vel"]) ** 2)) <= dv
    d = p2 - ref["pos"]
    d -= np.asarray(L) * np.round(d / np.asarray(L))
    assert np.sqrt(np.mean(d ** 2)) <= k * DT * dv + 1e-12

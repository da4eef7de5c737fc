"""The Lennard-Jones variant (Eq. (1) truncated at r_c, no shift): the
paper's second system, rho = 0.38, T = 1.2, shell 0.8, with the cutoffs of
its comparisons (2.2, 2.5, 3.0).  The kernels are the soft-sphere ones with
another r_c; this checks forces, energy, virial, neighbour sets and short
trajectories against the oracle, and energy conservation."""
import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from mdcheck import DT, FORCE_TOL, assert_same_pairs, ensure_built, min_image, oracle_grid, rel_rms, state

pytestmark = pytest.mark.gpu

RHO, T, SKIN = 0.38, 1.2, 0.8
PRECS = ["mixed", "fp64"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _sim(pos, vel, L, rc, prec, **kw):
    s = md.Simulation(L, pos.shape[0], rc, SKIN, DT, precision=prec, **kw)
    s.set_state(pos, vel)
    return s


@pytest.mark.parametrize("build", ["auto", "warp"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("rc", [2.2, 2.5, 3.0])
def test_lj_forces_pairs_energy(rc, prec, build):
    # with r_c 3 a cell's neighbourhood holds about 560 atoms: the automatic
    # choice is the thread-per-atom build, and the warp build stages the
    # candidates in several batches
    n = 4000
    pos, vel, L = state(n, RHO, T, 61, jitter=0.3)
    s = _sim(pos, vel, L, rc, prec, build=build)
    pw = oracle.wrap(pos, L)
    assert s.plan()["ushift"] == 0.0  # plain truncated LJ
    f_ref, U, W = oracle.forces_cells(pw, L, oracle_grid(L, rc), rc, 0.0)
    f = s.forces()
    assert rel_rms(f, f_ref) <= FORCE_TOL[prec]
    m = s.measure()
    assert m["pe"] == pytest.approx(U, rel=10 * FORCE_TOL[prec])
    assert m["virial"] == pytest.approx(W, rel=10 * FORCE_TOL[prec], abs=1e-9 * abs(U))
    rn = rc + SKIN
    pairs, entries = s.neighbor_pairs()
    p, _ = s.get_state()
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    nbar = 4.0 / 3.0 * np.pi * rn ** 3 * RHO
    assert entries / n == pytest.approx(nbar, rel=0.2)  # about (4/3) pi r_n^3 rho neighbours
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_lj_trajectory_segment(prec):
    rc, k = 2.5, 40
    pos, vel, L = state(2000, RHO, T, 62)
    melt = oracle.run(oracle.wrap(pos, L), vel, L, rc, SKIN, DT, 300, ushift=0.0, record=False)
    pos, vel = melt["pos"], melt["vel"]
    s = _sim(pos, vel, L, rc, prec)
    ref = oracle.run(pos, vel, L, rc, SKIN, DT, k, ushift=0.0)
    s.step(k)
    p, v = s.get_state()
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    fe = FORCE_TOL[prec] * f_rms
    dv = 10.0 * k * DT * fe + (1e-7 if prec == "mixed" else 1e-14)
    assert np.sqrt(np.mean((v - ref["vel"]) ** 2)) <= dv
    assert np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)) <= k * DT * dv + 1e-13
    m = s.measure()
    assert m["ke"] + m["pe"] == pytest.approx(ref["ke"][-1] + ref["pe"][-1], rel=1e-5 if prec == "mixed" else 1e-11)
    s.close()


def test_lj_energy_conservation_mixed():
    # rc = 3: the potential jumps at the cutoff (no shift), so total energy
    # is conserved only up to the crossings; the drift over 4000 steps stays
    # small next to kT
    rc = 3.0
    pos, vel, L = state(13500, RHO, T, 63)
    s = _sim(pos, vel, L, rc, "mixed")
    s.step(500)
    e = []
    for _ in range(35):
        s.step(100)
        m = s.measure()
        e.append(m["e_tot_per_atom"])
    s.close()
    e = np.array(e)
    assert abs(e[-5:].mean() - e[:5].mean()) < 2e-3

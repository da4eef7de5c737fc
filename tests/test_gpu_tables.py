"""The paper's soft-sphere statistics for system S (N_a = 110592 = 48^3,
rho = 0.8, T = 1, dt = 0.005, the even cell grid of its tables), measured on
the GPU under its protocol: 500 steps of equilibration with the velocities
rescaled every 20 steps (Sec. 3.1 (f), Sec. 5), then free dynamics.

Table 5: mean neighbour-list entries per atom N_p/N_a and mean steps
between list updates N_u, for shell thickness delta = 0.4 .. 0.8.
Table 4: block means of e_tot and e_kin over the 1000 steps before step 2000.
The initial state is the paper's (simple cubic lattice, speeds sqrt(3T) in
random directions, Sec. 3.5); the random draw differs from the paper's, so
the comparison is statistical."""
import numpy as np
import pytest

import paper_0911_5631_gb300 as md
from paper_0911_5631_gb300 import inputs
from mdcheck import DT, RC, ensure_built
from conftest import read_golden

pytestmark = pytest.mark.gpu

N_E = 48
N = N_E ** 3
RHO = 0.8


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _run_S(delta, steps=2000, seed=48):
    pos, vel, L = inputs.sc_state(N_E, RHO, 1.0, seed)
    s = md.Simulation(L, N, RC, delta, DT, precision="mixed", reorder_interval=100, even_cells=True)
    s.set_state(pos, vel)
    for _ in range(500 // 20):  # equilibration: rescale every 20 steps
        s.step(20)
        s.rescale(1.0)
    m0 = s.measure()
    e_tot, e_kin, entries, last_reb = [], [], [], m0["rebuilds"]
    for step in range(501, steps + 1):
        s.step(1)
        m = s.measure()
        if m["rebuilds"] != last_reb:
            entries.append(m["list_entries"])
            last_reb = m["rebuilds"]
        if step > steps - 1000:
            e_tot.append(m["e_tot_per_atom"])
            e_kin.append(m["ke"] / N)
    m1 = s.measure()
    plan = s.plan()
    s.close()
    nu = (steps - 500) / max(m1["rebuilds"] - m0["rebuilds"], 1)
    return dict(np_na=float(np.mean(entries)) / N, nu=nu, e_tot=float(np.mean(e_tot)),
                e_kin=float(np.mean(e_kin)), n_cells=plan["n_cells"], n_l=m1["max_occupancy"])


# N_c of Table 5 (the even cell grid); the other columns come from the golden file
N_CELLS = {0.4: 32768, 0.5: 27000, 0.6: 27000, 0.7: 21952, 0.8: 17576}


@pytest.mark.parametrize("delta", sorted(N_CELLS))
def test_table5_neighbour_statistics(delta):
    g = {(k, q): float(v) for k, q, v, _src in read_golden("paper_sp_statistics.txt")}
    key = "delta=%.1f" % delta
    r = _run_S(delta)
    print("delta", delta, r)
    assert r["n_cells"] == N_CELLS[delta]
    assert r["np_na"] == pytest.approx(g[("np_per_atom", key)], rel=0.005)
    assert abs(r["n_l"] - g[("n_l", key)]) <= 1
    # exact displacement test vs the paper's estimate: same or somewhat rarer rebuilds
    assert 0.97 <= r["nu"] / g[("n_u", key)] <= 1.12
    if delta == 0.6:  # Table 4 is system S at the paper's usual delta
        # the oracle under the same protocol gives 2.32625 / 1.50047 at 48^3
        assert r["e_kin"] == pytest.approx(g[("e_kin", "step=2000")], abs=0.002)
        assert r["e_tot"] == pytest.approx(g[("e_tot", "step=2000")], abs=0.003)

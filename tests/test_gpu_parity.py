"""Parity of the CUDA path with the FP64 oracle on seeded inputs, through the
C ABI: cell assignment and neighbour-pair sets (exact), forces, energies and
virial (within the stated tolerances), and short trajectory segments."""
import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from mdcheck import (DT, FORCE_TOL, RC, assert_same_cells, assert_same_pairs, ensure_built, min_image,
                     oracle_grid, rel_rms, sim, state, trajectory_tol)

pytestmark = pytest.mark.gpu

# (n, rho, T, skin, lattice jitter, box aspect, seed): several 256-atom tiles,
# ragged counts, dense/hot and dilute/cold states, a non-cubic box, and a
# 3-cell grid.
CASES = [
    (2048, 0.8, 1.0, 0.4, 0.15, (1, 1, 1), 1),
    (1000, 0.8, 1.0, 0.4, 0.20, (1, 1, 1), 2),
    (4000, 1.0, 2.0, 0.4, 0.08, (1, 1, 1), 3),
    (3001, 0.6, 0.7, 0.3, 0.30, (1.0, 1.4, 0.8), 4),
    (256, 0.8, 1.0, 0.6, 0.20, (1, 1, 1), 5),
]
IDS = ["n2048", "n1000", "n4000_dense", "n3001_rect", "n256_g3"]
PRECS = ["mixed", "fp64"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _setup(case, prec, **kw):
    n, rho, T, skin, jit, aspect, seed = case
    pos, vel, L = state(n, rho, T, seed, jitter=jit, aspect=aspect)
    s = sim(pos, vel, L, skin=skin, precision=prec, **kw)
    return s, pos, vel, L, skin


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_cells_bit_exact(case, prec):
    # the load bins the wrapped input by the reference's rule; the positions
    # the GPU then reports are the wrapped input (an atom whose offset from
    # its cell centre is not exact in FP64 may move by an ulp)
    s, pos, vel, L, skin = _setup(case, prec)
    G = np.array(s.plan()["G"])
    pw = oracle.wrap(pos, L)
    p, _ = s.get_state()
    assert np.abs(p - pw).max() <= 4e-16 * np.max(L)
    assert np.array_equal(s.cells(), oracle.cell_of(pw, L, G))
    assert_same_cells(s.cells(), p, L, G)
    m = s.measure()
    counts = np.bincount(oracle.cell_of(pw, L, G), minlength=int(np.prod(G)))
    assert m["max_occupancy"] == counts.max()
    s.close()


BUILDS = ["warp", "thread"]


@pytest.mark.parametrize("build", BUILDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_neighbor_pairs_match_oracle(case, prec, build):
    # identical sets: the GPU decides the pairs near r_n by the reference's
    # own FP64 expression on the positions it reports
    s, pos, vel, L, skin = _setup(case, prec, build=build)
    p, _ = s.get_state()
    rn = RC + skin
    pairs, entries = s.neighbor_pairs()
    assert entries == 2 * len(pairs)  # full list: every pair in both columns
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    pw = oracle.wrap(pos, L)
    assert_same_pairs(pairs, oracle.pairs_cells(pw, L, oracle_grid(L, rn), rn), pw, L, rn)
    m = s.measure()
    assert m["list_entries"] == entries
    s.close()


def _check_rebuilt_state(s, L, skin, G):
    """Cells and neighbour pairs of the last rebuild against the reference,
    from the positions the GPU reports (the rebuild's own positions when the
    last step rebuilt)."""
    p, _ = s.get_state()
    assert_same_cells(s.cells(), p, L, G)
    rn = RC + skin
    pairs, entries = s.neighbor_pairs()
    assert entries == 2 * len(pairs)
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    return len(pairs)


@pytest.mark.parametrize("build", BUILDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rebuilds_along_trajectory_match_oracle(case, prec, build):
    # The rebuilds of md_step re-bin atoms incrementally (k_bin) and rebuild
    # the lists in place, with periodic reorders; right after every step
    # that rebuilt, the stored cells and the list must be the reference's
    # for the positions of that moment.  No md_set_state in between.
    pos, vel, L, skin = _fluid(case)
    s = sim(pos, vel, L, skin=skin, precision=prec, reorder_interval=15, build=build)
    G = np.array(s.plan()["G"])
    seen, last, steps = 0, s.measure()["rebuilds"], 0
    while seen < 4 and steps < 400:
        s.step(1)
        steps += 1
        m = s.measure()
        if m["rebuilds"] > last:
            last = m["rebuilds"]
            seen += 1
            _check_rebuilt_state(s, L, skin, G)
    assert seen == 4
    assert s.measure()["reorders"] >= 2  # the load's reorder and at least one more
    s.close()


def _clustered_state(seed=7):
    """A dense FCC block (rho 2.1: 42 neighbours within r_n) inside a dilute
    FCC lattice (rho 0.5), both slightly jittered: a low mean density with a
    few atoms whose lists are far longer than the mean."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    def fcc(cells, a):
        g = np.stack(np.meshgrid(*[np.arange(cells)] * 3, indexing="ij"), -1).reshape(-1, 1, 3)
        return ((g + basis[None]) * a).reshape(-1, 3)
    L = np.array([16.0, 16.0, 16.0])
    dilute = fcc(8, 2.0) - 8.0 + 0.5
    a_d = (4 / 2.1) ** (1 / 3)
    dense = fcc(4, a_d) - 2.0 * a_d
    side = 4 * a_d
    keep = np.any(np.abs(dilute + 0.25 * a_d) > side / 2 + 0.8, axis=1)
    pos = np.concatenate([dilute[keep], dense]) + rng.normal(0, 0.01, (keep.sum() + len(dense), 3))
    vel = rng.normal(0, 1.0, pos.shape)
    return pos, vel, L


@pytest.mark.parametrize("prec", PRECS)
def test_thread_build_forms_match_oracle(prec):
    # The thread-per-atom build stages up to 18 candidates per atom; an atom
    # with more is scanned a second time and written unsorted (the dense
    # block of a clustered state).  A workload whose expected list comes
    # near the stage depth takes the direct form, which writes entries as it
    # finds them (skin 1.0: about 32 entries per atom), checked at the load
    # and at in-trajectory rebuilds of a melted state.
    pos, vel, L = _clustered_state()
    s = sim(pos, vel, L, skin=0.4, precision=prec)
    p, _ = s.get_state()
    rn = RC + 0.4
    pairs, entries = s.neighbor_pairs()
    assert entries == 2 * len(pairs)
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    assert s.measure()["max_neighbors"] > 18
    s.close()
    case = (2048, 0.8, 1.0, 1.0, 0.15, (1, 1, 1), 6)
    s, pos, vel, L, skin = _setup(case, prec)
    p, _ = s.get_state()
    rn = RC + skin
    pairs, entries = s.neighbor_pairs()
    assert entries == 2 * len(pairs)
    assert_same_pairs(pairs, oracle.pairs_cells(p, L, oracle_grid(L, rn), rn), p, L, rn)
    s.close()
    pos, vel, L, skin = _fluid(case)
    s = sim(pos, vel, L, skin=skin, precision=prec, reorder_interval=15)
    G = np.array(s.plan()["G"])
    seen, last, steps = 0, s.measure()["rebuilds"], 0
    while seen < 2 and steps < 400:
        s.step(1)
        steps += 1
        if s.measure()["rebuilds"] > last:
            last = s.measure()["rebuilds"]
            seen += 1
            _check_rebuilt_state(s, L, skin, G)
    assert seen == 2
    s.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pair_sets_identical_across_precisions(case):
    a = _setup(case, "mixed")[0]
    b = _setup(case, "fp64")[0]
    pa, pb = a.neighbor_pairs()[0], b.neighbor_pairs()[0]
    assert np.array_equal(pa[np.lexsort(pa.T[::-1])], pb[np.lexsort(pb.T[::-1])])
    a.close()
    b.close()


@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_builds_give_the_same_trajectory(case):
    # The warp-per-cell and thread-per-atom builds store each atom's entries
    # in different orders, with the same pairs and the same shell-bin counts
    # up to rounding; a step reads only entries that cannot interact beyond
    # its shell reach, and the mixed form sums in integers, so the two
    # trajectories are the same bits.
    pos, vel, L, skin = _fluid(case)
    out = []
    for build in BUILDS:
        s = sim(pos, vel, L, skin=skin, precision="mixed", reorder_interval=25, build=build)
        s.step(120)
        out.append(s.get_state() + (s.measure(),))
        s.close()
    (p0, v0, m0), (p1, v1, m1) = out
    assert m0["rebuilds"] == m1["rebuilds"] >= 4
    assert m0["list_entries"] == m1["list_entries"] and m0["max_neighbors"] == m1["max_neighbors"]
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_forces_energy_virial(case, prec):
    s, pos, vel, L, skin = _setup(case, prec)
    pw = oracle.wrap(pos, L)
    f_ref, U, W = oracle.forces_cells(pw, L, oracle_grid(L, RC), RC, 1.0)
    f = s.forces()
    assert np.abs(f_ref).max() > 10.0  # the jitter puts pairs inside r_c
    assert rel_rms(f, f_ref) <= FORCE_TOL[prec]
    m = s.measure()
    tol = FORCE_TOL[prec]
    assert m["pe"] == pytest.approx(U, rel=10 * tol)
    assert m["virial"] == pytest.approx(W, rel=10 * tol)
    ke_ref = 0.5 * np.sum(vel * vel)
    # the mixed form stores velocities in FP32
    assert m["ke"] == pytest.approx(ke_ref, rel=1e-14 if prec == "fp64" else 2e-7)
    n = pos.shape[0]
    V = float(np.prod(L))
    assert m["pressure"] == pytest.approx((2 * m["ke"] + m["virial"]) / (3 * V), rel=1e-14)
    assert m["temperature"] == pytest.approx(2 * m["ke"] / (3 * n), rel=1e-14)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_newton_third_law_in_result(prec):
    s, pos, vel, L, skin = _setup(CASES[0], prec)
    f = s.forces()
    scale = np.abs(f).max()
    # mixed: int64 pair terms cancel exactly; the FP32 conversion of each
    # atom's sum leaves only rounding
    tol = 1e-6 if prec == "mixed" else 1e-12
    assert np.abs(f.sum(axis=0)).max() <= tol * scale * np.sqrt(pos.shape[0])
    s.close()


_trajectory_tol = trajectory_tol


def _fluid(case):
    """A melted state for dynamics: the lattice start run forward by the
    oracle (the jittered lattices above are for static checks only; their
    closest pairs would fling atoms across cells in one step)."""
    n, rho, T, skin, jit, aspect, seed = case
    pos, vel, L = state(n, rho, T, seed, aspect=aspect)
    out = oracle.run(oracle.wrap(pos, L), vel, L, RC, skin, DT, 300, record=False)
    return out["pos"], out["vel"], L, skin


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_trajectory_segment(case, prec):
    k = 40
    pos, vel, L, skin = _fluid(case)
    s = sim(pos, vel, L, skin=skin, precision=prec)
    ref = oracle.run(pos, vel, L, RC, skin, DT, k)
    s.step(k)
    p, v = s.get_state()
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    dv, dx = _trajectory_tol(prec, f_rms, k)
    assert np.sqrt(np.mean((v - ref["vel"]) ** 2)) <= dv
    assert np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)) <= dx
    assert np.all(p >= -np.asarray(L) / 2) and np.all(p < np.asarray(L) / 2)
    m = s.measure()
    assert m["step"] == k
    assert m["rebuilds"] >= 1
    e_gpu = m["ke"] + m["pe"]
    e_ref = ref["ke"][-1] + ref["pe"][-1]
    assert e_gpu == pytest.approx(e_ref, rel=1e-5 if prec == "mixed" else 1e-11)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", [(2916, 0.8, 1.5, 0.8, (1, 1, 1), 11), (3000, 0.95, 1.2, 0.6, (1, 1, 1), 12)],
                         ids=["skin0.8", "rho0.95_skin0.6"])
def test_trajectory_across_shell_bins(case, prec):
    # A step reads only the entries whose distance at the build lies within
    # r_c + 2 (largest displacement so far): a wide skin spreads the list
    # over shell bins of width 0.1; at rho 0.95 with skin 0.6 the lists hold
    # about 21 entries, so atoms with sorted lists and atoms with lists too
    # long to sort (read whole) sit side by side.  Long segments cross
    # several rebuilds.
    n, rho, T, skin, aspect, seed = case
    pos, vel, L = state(n, rho, T, seed, aspect=aspect)
    out = oracle.run(oracle.wrap(pos, L), vel, L, RC, skin, DT, 300, record=False)
    pos, vel = out["pos"], out["vel"]
    k = 60
    s = sim(pos, vel, L, skin=skin, precision=prec)
    ref = oracle.run(pos, vel, L, RC, skin, DT, k)
    pairs, entries = s.neighbor_pairs()
    s.step(k)
    p, v = s.get_state()
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    dv, dx = _trajectory_tol(prec, f_rms, k)
    assert np.sqrt(np.mean((v - ref["vel"]) ** 2)) <= dv
    assert np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)) <= dx
    m = s.measure()
    assert m["rebuilds"] >= 2
    if rho > 0.9:
        assert m["max_neighbors"] > 21 and entries / n < 24  # both kinds of list
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_shell_bins_change_no_force(prec):
    # A step that reads only the entries within r_c + 2 (largest displacement)
    # of their build distance computes the forces of reading every entry.
    # The mixed form sums in integers, so the trajectories agree bit for bit;
    # the FP64 form sums in list order, which the sorting changes.
    pos, vel, L, skin = _fluid(CASES[0])
    k = 200 if prec == "mixed" else 40
    runs = []
    for bins in (True, False):
        s = sim(pos, vel, L, skin=skin, precision=prec, shell_bins=bins)
        s.step(k)
        p, v = s.get_state()
        runs.append((p, v, s.measure()))
        s.close()
    (p1, v1, m1), (p0, v0, m0) = runs
    assert m1["rebuilds"] == m0["rebuilds"] >= 4
    if prec == "mixed":
        assert np.array_equal(p1, p0) and np.array_equal(v1, v0)
    else:
        assert np.abs(v1 - v0).max() < 1e-10
        assert np.abs(min_image(p1 - p0, L)).max() < 1e-11


@pytest.mark.parametrize("prec", PRECS)
def test_cell_list_only_segments(prec):
    # soft-sphere fluid of 2048 atoms (FCC 8^3 x 4) at rho 0.8, T 1, forces
    # straight from the cells every step; compared in 100-step segments, the
    # oracle restarted from the GPU state each time
    n = 2048
    pos, vel, L = state(n, 0.8, 1.0, 1)
    s = sim(pos, vel, L, skin=0.0, precision=prec, cell_list_only=True)
    p, v = oracle.wrap(pos, L), vel
    for seg in range(10):
        ref = oracle.run(p, v, L, RC, 0.0, DT, 100)
        s.step(100)
        p, v = s.get_state()
        f_rms = max(float(np.sqrt(np.mean(ref["f"] ** 2))), 1.0)
        dv, dx = _trajectory_tol(prec, f_rms, 100)
        assert np.sqrt(np.mean((v - ref["vel"]) ** 2)) <= dv, seg
        assert np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)) <= dx, seg
    m = s.measure()
    assert m["step"] == 1000 and m["rebuilds"] == 1000 + 1
    s.close()


def test_tiny_systems():
    # one atom: no partners, zero force; two atoms across the boundary: the
    # closed-form pair force
    L = np.array([6.0, 6.0, 6.0])
    for prec in PRECS:
        s = sim(np.array([[0.1, 0.2, 0.3]]), np.array([[1.0, 0.0, 0.0]]), L, skin=0.4, precision=prec)
        assert np.all(s.forces() == 0.0)
        s.step(10)
        p, v = s.get_state()
        assert p[0, 0] == pytest.approx(0.1 + 10 * DT, abs=1e-6)
        s.close()
        pos = np.array([[-3.0 + 0.45, 0.1, -0.2], [3.0 - 0.45, 0.1, -0.2]])
        s = sim(pos, np.zeros((2, 3)), L, skin=0.4, precision=prec)
        fr, u = oracle.pair(0.81, 1.0)
        f = s.forces()
        assert f[0, 0] == pytest.approx(fr * 0.9, rel=FORCE_TOL[prec] * 10)
        assert f[1, 0] == pytest.approx(-fr * 0.9, rel=FORCE_TOL[prec] * 10)
        assert s.measure()["pe"] == pytest.approx(u, rel=1e-6)
        s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_rescaled_equilibration_segment(prec):
    # step (f): velocities rescaled to T every 20 steps, as the oracle does
    # after its step 20, 40, ..., 100
    k, every, T = 100, 20, 1.3
    pos, vel, L, skin = _fluid(CASES[0])
    s = sim(pos, vel, L, skin=skin, precision=prec)
    ref = oracle.run(pos, vel, L, RC, skin, DT, k, rescale_every=every, rescale_until=k, T_target=T)
    for _ in range(k // every):
        s.step(every)
        s.rescale(T)
        assert 2.0 * s.measure()["ke"] / (3.0 * pos.shape[0]) == pytest.approx(T, rel=1e-6)
    p, v = s.get_state()
    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
    dv, dx = _trajectory_tol(prec, f_rms, k)
    assert np.sqrt(np.mean((v - ref["vel"]) ** 2)) <= dv
    assert np.sqrt(np.mean(min_image(p - ref["pos"], L) ** 2)) <= dx
    s.close()


def test_rescale_rejects_bad_temperature():
    pos, vel, L, skin = _fluid(CASES[1])
    s = sim(pos, vel, L, skin=skin)
    for T in (0.0, -1.0, float("nan")):
        with pytest.raises(md.MDError) as e:
            s.rescale(T)
        assert e.value.code == md.MD_EINVAL
    s.close()

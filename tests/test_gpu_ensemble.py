"""Ensembles (md_ensemble_*): a replica advanced by the per-replica engine
gives bitwise the positions and velocities of md_step from the same state,
its result does not depend on the other replicas in the launch or on the
launch shape, and the arena admits and frees replicas."""
import numpy as np
import pytest

import paper_0911_5631_gb300 as md
import oracle
from mdcheck import DT, RC, assert_trajectory_matches, ensure_built, sim, state

pytestmark = pytest.mark.gpu

ARENA = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _state(n, rho, T, seed):
    return state(n, rho, T, seed, jitter=0.05)


CASES = [  # (n, rho, T, seed, reorder_interval, cluster, team_atoms)
    (500, 0.8, 1.0, 11, 100, 8, 0),
    (2048, 0.6, 0.7, 12, 20, 1, 0),
    (4000, 1.0, 2.0, 13, 0, 4, 1000),   # a team of 4 blocks on a small replica
    (6912, 0.8, 1.5, 14, 7, 2, 1000),
    (10976, 0.7, 1.0, 15, 30, 8, 0),    # above the default team size
]


def _solo(pos, vel, L, steps, reorder):
    s = sim(pos, vel, L, skin=0.4, precision="mixed", reorder_interval=reorder)
    for k in steps:
        s.step(k)
    p, v = s.get_state()
    m = s.measure()
    s.close()
    return p, v, m


def _ens_run(e, rid, steps):
    for k in steps:
        e.run([rid], [k])
    e.sync()
    return e.get_state(rid) + (e.measure(rid),)


@pytest.mark.parametrize("case", CASES)
def test_replica_matches_md_step_bitwise(case):
    n, rho, T, seed, reorder, cluster, team_atoms = case
    pos, vel, L = _state(n, rho, T, seed)
    steps = [37, 1, 64]
    p0, v0, m0 = _solo(pos, vel, L, steps, reorder)
    with md.Ensemble(ARENA) as e:
        e.set_shape(1024 if cluster > 1 else 256, 0, cluster, team_atoms)
        rid = e.add(pos, vel, L, RC, 0.4, DT, reorder_interval=reorder)
        p1, v1, m1 = _ens_run(e, rid, steps)
        assert e.status(rid) == md.MD_OK
    assert np.array_equal(p0, p1)
    assert np.array_equal(v0, v1)
    for k in ("step", "rebuilds", "reorders", "list_entries", "max_neighbors", "max_occupancy"):
        assert m0[k] == m1[k], k
    # both sum KE, PE and W in FP64, in different fixed orders
    for k in ("ke", "pe", "virial"):
        assert abs(m0[k] - m1[k]) <= 1e-12 * abs(m0[k]), (k, m0[k], m1[k])


def test_replicas_match_oracle():
    # Replicas of different N, rho and T, through md_ensemble_run in one
    # launch, each against the FP64 oracle run from the same state: single
    # blocks for the small ones, thread-block clusters of 4 for those of at
    # least 3000 atoms.
    specs = [(256, 0.8, 1.0, 31), (700, 0.6, 0.7, 32), (1500, 1.0, 2.0, 33), (3000, 0.9, 1.2, 34),
             (5324, 0.7, 0.5, 35), (8788, 0.8, 1.5, 36)]
    k = 60
    with md.Ensemble(ARENA) as e:
        e.set_shape(1024, 0, 4, 3000)
        ids, starts = [], []
        for n, rho, T, seed in specs:
            pos, vel, L = _state(n, rho, T, seed)
            ids.append(e.add(pos, vel, L, RC, 0.4, DT, reorder_interval=20))
            starts.append((pos, vel, L))
        e.run(ids, [k] * len(ids))
        e.sync()
        for rid, (pos, vel, L), (n, rho, T, seed) in zip(ids, starts, specs):
            assert e.status(rid) == md.MD_OK
            p, v = e.get_state(rid)
            m = e.measure(rid)
            assert m["step"] == k and m["rebuilds"] >= 1, (n, m["rebuilds"])
            ref = oracle.run(oracle.wrap(pos, L), vel, L, RC, 0.4, DT, k)
            assert_trajectory_matches(p, v, ref, L, "mixed", k)
            e_ref = ref["ke"][-1] + ref["pe"][-1]
            assert m["ke"] + m["pe"] == pytest.approx(e_ref, rel=1e-5), n


def _mix(e, rng, count):
    ids = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(256), np.log(6000))))
        rho = rng.uniform(0.6, 1.0)
        T = rng.uniform(0.5, 2.0)
        pos, vel, L = _state(n, rho, T, 100 + k)
        ids.append(e.add(pos, vel, L, RC, 0.4, DT, reorder_interval=int(rng.integers(0, 60))))
    return ids


def test_result_is_the_same_alone_and_in_the_mix():
    pos, vel, L = _state(3000, 0.85, 1.2, 21)
    with md.Ensemble(ARENA) as e:
        x = e.add(pos, vel, L, RC, 0.4, DT, reorder_interval=50)
        e.run([x], [0])
        e.run([x], [150])
        e.sync()
        alone = e.get_state(x) + (e.measure(x),)
    rng = np.random.default_rng(5)
    with md.Ensemble(ARENA) as e:
        others = _mix(e, rng, 24)
        x = e.add(pos, vel, L, RC, 0.4, DT, reorder_interval=50)
        ids = others + [x]
        e.run(ids, [int(s) for s in rng.integers(0, 200, size=len(others))] + [0])
        e.run(ids, [int(s) for s in rng.integers(1, 300, size=len(others))] + [150])
        e.sync()
        mixed = e.get_state(x) + (e.measure(x),)
        assert all(e.status(i) == md.MD_OK for i in ids)
    assert np.array_equal(alone[0], mixed[0]) and np.array_equal(alone[1], mixed[1])
    assert alone[2] == mixed[2]  # every field, energies included (fixed summation order)


@pytest.mark.parametrize("shape", [(64, 0, 1, 0), (128, 0, 1, 0), (512, 7, 1, 0), (1024, 0, 1, 0),
                                   (1024, 0, 8, 1500), (512, 0, 4, 2500), (256, 16, 2, 1000)])
def test_launch_shape_does_not_change_results(shape):
    ref = None
    for sh in ((256, 0, 1, 0), shape):
        with md.Ensemble(ARENA) as e:
            ids = _mix(e, np.random.default_rng(9), 6)
            e.set_shape(*sh)
            e.run(ids, [40, 80, 120, 10, 0, 60])
            e.sync()
            got = [e.get_state(i) + (e.measure(i),) for i in ids]
        if ref is None:
            ref = got
        else:
            for a, c in zip(ref, got):
                assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
                assert a[2] == c[2]


def test_arena_admission_and_reuse():
    pos, vel, L = _state(4000, 0.8, 1.0, 31)
    need = md.md_ensemble_replica_bytes(md.replica_desc(L, 4000))
    with md.Ensemble(3 * need + need // 2, max_replicas=8) as e:
        ids = [e.add(pos, vel, L) for _ in range(3)]
        with pytest.raises(md.MDError) as err:
            e.add(pos, vel, L)
        assert err.value.code == md.MD_ENOMEM
        e.remove(ids[1])
        again = e.add(pos, vel, L)
        assert again == ids[1]  # the id and the space are reused
        e.run(ids, [20, 20, 20])
        e.sync()
        p = [e.get_state(i)[0] for i in ids]
        assert np.array_equal(p[0], p[1]) and np.array_equal(p[1], p[2])


def test_overflow_stops_only_that_replica():
    pos, vel, L = _state(2048, 0.8, 1.0, 41)
    with md.Ensemble(ARENA) as e:
        good = e.add(pos, vel, L)
        bad = e.add(pos, vel, L, nbr_capacity=4)
        e.run([good, bad], [30, 30])
        e.sync()
        assert e.status(good) == md.MD_OK
        assert e.status(bad) == md.MD_EOVERFLOW
        assert e.measure(good)["step"] == 30


def test_times_and_autotune():
    rng = np.random.default_rng(3)
    with md.Ensemble(ARENA) as e:
        ids = _mix(e, rng, 12)
        b, c = e.autotune(ids, probe_steps=5)
        assert b in (256, 1024) and c in (1, 2, 4, 8)
        e.run(ids, [50] * len(ids))
        t0, t1 = e.times(ids)
        assert np.all(t0 >= 0) and np.all(t1 >= t0)
        for i in ids:
            assert e.measure(i)["step"] == 6 * 5 + 50


@pytest.mark.parametrize("n", [1, 2, 31, 33, 257])
def test_tiny_and_ragged_replicas(n):
    # fewer atoms than a warp, ragged tails, one atom alone in its box
    L = np.array([7.0, 7.5, 8.0])
    rng = np.random.default_rng(n)
    pos = rng.uniform(-L / 2, L / 2, size=(n, 3))
    if n > 1:  # keep the random start free of overlaps: a coarse lattice
        g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
        pos = (g + 0.5) * (L / 7) - L / 2
    vel = rng.normal(size=(n, 3))
    s = sim(pos, vel, L, skin=0.4, precision="mixed")
    s.step(50)
    p0, v0 = s.get_state()
    m0 = s.measure()
    s.close()
    with md.Ensemble(ARENA) as e:
        rid = e.add(pos, vel, L)
        e.run([rid], [50])
        e.sync()
        p1, v1 = e.get_state(rid)
        m1 = e.measure(rid)
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    assert m0["step"] == m1["step"] == 50


def test_load_only_run_measures_the_initial_state():
    pos, vel, L = _state(1500, 0.8, 1.0, 51)
    s = sim(pos, vel, L, skin=0.4, precision="mixed")
    m0 = s.measure()
    s.close()
    with md.Ensemble(ARENA) as e:
        rid = e.add(pos, vel, L)
        with pytest.raises(md.MDError) as err:
            e.measure(rid)  # not loaded yet
        assert err.value.code == md.MD_ESTATE
        e.run([rid], [0])
        m1 = e.measure(rid)
    assert m1["step"] == 0
    for k in ("ke", "pe", "virial"):
        assert m1[k] == pytest.approx(m0[k], rel=1e-12, abs=1e-12)


def test_bad_ids_are_rejected():
    pos, vel, L = _state(500, 0.8, 1.0, 52)
    with md.Ensemble(ARENA) as e:
        rid = e.add(pos, vel, L)
        for ids, steps in (([rid, rid], [1, 1]), ([rid + 7], [1]), ([rid], [-1])):
            with pytest.raises(md.MDError) as err:
                e.run(ids, steps)
            assert err.value.code == md.MD_EINVAL
        e.remove(rid)
        assert e.status(rid) == md.MD_EINVAL  # a removed id is unknown
        with pytest.raises(md.MDError):
            e.measure(rid)

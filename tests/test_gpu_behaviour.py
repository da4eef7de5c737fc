"""Determinism, reordering, capacity growth, error reporting and energy
conservation of the CUDA path (through the C ABI)."""
import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from mdcheck import DT, RC, ensure_built, sim, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _run(prec, steps=300, n=4000, seed=7, **kw):
    pos, vel, L = state(n, 0.8, 1.5, seed, jitter=0.05)
    s = sim(pos, vel, L, skin=0.4, precision=prec, **kw)
    s.step(steps)
    p, v = s.get_state()
    f = s.forces()
    m = s.measure()
    s.close()
    return p, v, f, m


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_run_twice_bitwise(prec):
    a = _run(prec)
    b = _run(prec)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3]["ke"] == b[3]["ke"] and a[3]["pe"] == b[3]["pe"]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graphs_and_stream_launches_agree_bitwise(prec):
    a = _run(prec, use_graphs=True)
    b = _run(prec, use_graphs=False)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_steps_waiting_for_a_rebuild_are_completed(prec):
    # A graph checks for a rebuild before every third step; a step whose
    # rebuild is due in between waits, and md_step runs the waited steps at
    # its end.  A hot fluid with a thin skin rebuilds every few steps, so
    # waits are frequent: every call must still end after exactly its steps,
    # with the trajectory and the rebuilds of stream launches.
    pos, vel, L = state(2048, 0.8, 2.5, 21)
    out = []
    for graphs in (True, False):
        s = sim(pos, vel, L, skin=0.15, precision=prec, use_graphs=graphs)
        done, counts = 0, []
        for k in (37, 1, 64, 5, 100):
            s.step(k)
            done += k
            m = s.measure()
            assert m["step"] == done
            counts.append(m["rebuilds"])
        p, v = s.get_state()
        out.append((p, v, s.forces(), counts))
        s.close()
    assert out[0][3] == out[1][3] and out[0][3][-1] > 40
    for x, y in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(x, y)


def test_mixed_trajectory_independent_of_reordering():
    # int64 force sums make every atom's result independent of storage order
    ref = _run("mixed", reorder_interval=0)
    assert ref[3]["reorders"] == 1  # the initial sort at load
    for interval in (1, 7, 100):
        got = _run("mixed", reorder_interval=interval)
        assert got[3]["reorders"] > 1 or interval == 100
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])


def test_fp64_reordering_changes_only_rounding():
    ref = _run("fp64", reorder_interval=0, steps=100)
    got = _run("fp64", reorder_interval=1, steps=100)
    assert np.abs(got[1] - ref[1]).max() < 1e-11


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_capacity_growth_is_transparent(prec):
    a = _run(prec, nbr_capacity=4, steps=200)
    b = _run(prec, steps=200)
    assert a[3]["nbr_capacity"] > 4
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_integer_conversions_match_hardware():
    # the mixed form converts on the integer pipe; check every routine
    # against the hardware conversion on 2^24 hashed inputs
    assert md.md_selftest(1 << 24) == [0, 0, 0, 0]


def test_step_chunking_is_transparent():
    pos, vel, L = state(2048, 0.8, 1.0, 3, jitter=0.05)
    s1 = sim(pos, vel, L)
    s1.step(100)
    s2 = sim(pos, vel, L)
    for k in (1, 31, 32, 33, 3):
        s2.step(k)
    p1, v1 = s1.get_state()
    p2, v2 = s2.get_state()
    # the last step of a call stores v_n and the next call's first kick
    # repeats exactly the operation the fused kernel would have done
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2)
    assert s1.measure()["step"] == s2.measure()["step"] == 100
    s1.close()
    s2.close()


def test_errors_are_reported():
    pos, vel, L = state(256, 0.8, 1.0, 1)
    s = md.Simulation(L, 256, RC, 0.4, DT)
    with pytest.raises(md.MDError) as e:
        s.step(5)
    assert e.value.code == md.MD_ESTATE
    s.step(0)  # no-op
    with pytest.raises(md.MDError) as e:
        s.set_state(np.full((256, 3), np.nan), vel)
    assert e.value.code == md.MD_EUNSTABLE
    s.close()
    # two atoms far inside the core: reported, not silently wrapped
    L = np.array([6.0, 6.0, 6.0])
    pos = np.array([[0.0, 0.0, 0.0], [0.2, 0.0, 0.0]])
    s = md.Simulation(L, 2, RC, 0.4, DT)
    with pytest.raises(md.MDError) as e:
        s.set_state(pos, np.zeros((2, 3)))
    assert e.value.code == md.MD_EUNSTABLE
    s.close()


def test_state_round_trip_and_device_pointers():
    torch = pytest.importorskip("torch")
    pos, vel, L = state(1372, 0.8, 1.0, 9, jitter=0.05)
    s = sim(pos, vel, L)
    p, v = s.get_state()
    pw = oracle.wrap(pos, L)
    assert np.abs(p - pw).max() < 1e-13
    # FP32 velocity storage: round to nearest, relative error <= 2^-24
    assert np.all(np.abs(v - vel) <= 2.0 ** -24 * np.abs(vel))
    tp = torch.tensor(pos, device="cuda")
    tv = torch.tensor(vel, device="cuda")
    s.set_state(tp, tv)
    op = torch.empty_like(tp)
    ov = torch.empty_like(tv)
    s.get_state(op, ov)
    assert np.abs(op.cpu().numpy() - p).max() == 0.0
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_energy_drift(prec):
    # soft-sphere fluid at rho 0.8, T 1, skin 0.4: |<e_tot> over the last
    # 1000 steps - <e_tot> over steps 1000-2000| per atom after 10^4 steps
    n = 32000
    pos, vel, L = state(n, 0.8, 1.0, 2)
    s = sim(pos, vel, L, precision=prec)
    e = []
    for k in range(1000):
        s.step(10)
        e.append(s.measure()["e_tot_per_atom"])
    e = np.array(e)
    drift = abs(e[-100:].mean() - e[100:200].mean())
    assert drift <= 1e-4
    s.close()


def test_profiled_bytes_count_the_entries_read():
    # In profiling mode the algorithmic bytes of the step kernel are 116 B
    # of per-atom state, the list count (1 B with shell bins, else 4 B) and
    # 4 B for every list entry the step reads.  Without shell bins a step reads the whole list; with them it
    # reads fewer entries, but never fewer than the interacting ones.
    pos, vel, L = state(4000, 0.8, 1.0, 17)
    out = oracle.run(oracle.wrap(pos, L), vel, L, RC, 0.4, DT, 200, record=False)
    res = {}
    for bins in (True, False):
        s = sim(out["pos"], out["vel"], L, skin=0.4, shell_bins=bins, use_graphs=False)
        s.set_profiling(True)
        k0 = s.kernel_stats()
        s.step(60)
        k1 = s.kernel_stats()
        m = s.measure()
        s.close()
        launches = k1["step_kernel_launches"] - k0["step_kernel_launches"]
        base = 116 + (1 if bins else 4)
        reads = ((k1["step_kernel_bytes"] - k0["step_kernel_bytes"]) - base * 4000 * launches) / 4
        assert launches == 60 and reads == int(reads)
        res[bins] = (reads, m)
    reads_on, m_on = res[True]
    reads_off, m_off = res[False]
    assert m_on["rebuilds"] == m_off["rebuilds"]
    # every entry read: between the smallest and largest list of the run
    assert reads_off / 60 <= 1.2 * m_off["list_entries"] and reads_off / 60 >= 0.8 * m_off["list_entries"]
    # the shell bins read fewer, but never fewer than the interacting pairs
    # (about a third of the list for this state)
    assert 0.3 * reads_off < reads_on < reads_off


@pytest.mark.parametrize("variant", ["plain_loads", "list_rows", "block64", "block256"])
def test_ablation_variants_give_the_same_bits(variant):
    # The step-kernel variants of the paper's ablations (texture cache off,
    # W transposed, 64 / 256 threads per block) change where data comes from
    # and how work is split, not what is computed: the mixed-form trajectory
    # across rebuilds and reorders is the default's, bit for bit, and the
    # transposed list holds the same pairs.
    pos, vel, L = state(4000, 0.8, 1.0, 17, jitter=0.05)
    out = []
    for v in ("default", variant):
        s = md.Simulation(L, 4000, RC, 0.4, DT, reorder_interval=30, variant=v)
        s.set_state(pos, vel)
        s.step(150)
        s.step(1)
        out.append(s.get_state() + (s.measure(), s.neighbor_pairs()[0]))
        s.close()
    (p0, v0, m0, n0), (p1, v1, m1, n1) = out
    assert m0["rebuilds"] == m1["rebuilds"] >= 5 and m1["reorders"] >= 4
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    assert np.array_equal(n0[np.lexsort(n0.T[::-1])], n1[np.lexsort(n1.T[::-1])])


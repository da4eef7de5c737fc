"""md_forces_noalloc: forces without any device allocation.

Some callers may not allocate device memory -- code running inside a memory
pool or budget it does not own, or on a path where cudaMalloc/cudaFree must
not run because they synchronise the whole device.  md_forces_noalloc serves
them with a fixed scratch area inside the library.  This test calls it
through the C ABI twice in a row (the second call reuses the scratch the
first one left behind, at the maximum size) and compares each result with
the handle-based entry points (md_set_state + md_get_forces + md_measure,
FP64 form) and with the FP64 oracle, within the FP64 force tolerance used
throughout the tests.  A non-finite position is reported as MD_EUNSTABLE.
It runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from mdcheck import FORCE_TOL, RC, ensure_built, oracle_grid, rel_rms, state

pytestmark = pytest.mark.gpu


def _reference(pos, vel, L):
    s = md.Simulation(L, pos.shape[0], RC, 0.4, 0.005, precision="fp64")
    s.set_state(pos, vel)
    f = s.forces()
    m = s.measure()
    s.close()
    return f, m["pe"], m["virial"]


def _noalloc(torch, pos, L):
    n = pos.shape[0]
    tp = torch.tensor(pos, dtype=torch.float64, device="cuda")
    tf = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    te = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    md.md_forces_noalloc(L, n, RC, tp.data_ptr(), tf.data_ptr(), te.data_ptr())
    torch.cuda.synchronize()
    e = te.cpu().numpy()
    return tf.cpu().numpy(), float(e[0]), float(e[1])


def test_forces_noalloc_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    ensure_built()
    cases = [
        state(2048, 0.8, 1.0, 11, jitter=0.1),
        # the largest accepted size, after a smaller call left its data behind
        state(md.MD_NOALLOC_MAX_ATOMS, 0.8, 1.0, 12, jitter=0.1),
    ]
    for pos, vel, L in cases:
        f_ref, pe_ref, w_ref = _reference(pos, vel, L)
        f, pe, w = _noalloc(torch, pos, L)
        assert np.all(np.isfinite(f))
        assert rel_rms(f, f_ref) <= FORCE_TOL["fp64"]
        assert pe == pytest.approx(pe_ref, rel=10 * FORCE_TOL["fp64"])
        assert w == pytest.approx(w_ref, rel=10 * FORCE_TOL["fp64"])
        # and the FP64 oracle's cell-list forces on the same configuration
        pw = oracle.wrap(pos, L)
        f_orc, u_orc, w_orc = oracle.forces_cells(pw, L, oracle_grid(L, RC), RC, 1.0)
        assert rel_rms(f, f_orc) <= FORCE_TOL["fp64"]
        assert pe == pytest.approx(u_orc, rel=10 * FORCE_TOL["fp64"])
        assert w == pytest.approx(w_orc, rel=10 * FORCE_TOL["fp64"])


def test_forces_noalloc_reports_non_finite_positions():
    torch = pytest.importorskip("torch")
    ensure_built()
    pos, vel, L = state(2048, 0.8, 1.0, 13, jitter=0.1)
    bad = pos.copy()
    bad[77, 1] = np.nan
    bad[1500, 2] = np.inf
    tp = torch.tensor(bad, dtype=torch.float64, device="cuda")
    tf = torch.zeros((2048, 3), dtype=torch.float64, device="cuda")
    te = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_forces_noalloc(L, 2048, RC, tp.data_ptr(), tf.data_ptr(), te.data_ptr())
    assert e.value.code == md.MD_EUNSTABLE
    # the flag does not stick: the next call on finite input succeeds
    f, pe, w = _noalloc(torch, pos, L)
    assert np.all(np.isfinite(f)) and np.isfinite(pe)


def test_forces_noalloc_rejects_sizes_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    ensure_built()
    n = md.MD_NOALLOC_MAX_ATOMS + 1
    L = [45.0, 45.0, 45.0]
    tp = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    tf = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    te = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_forces_noalloc(L, n, RC, tp.data_ptr(), tf.data_ptr(), te.data_ptr())
    assert e.value.code == md.MD_EINVAL
    assert "MD_NOALLOC_MAX_ATOMS" in str(e.value)
    # too many cells for the scratch area
    with pytest.raises(md.MDError) as e:
        md.md_forces_noalloc([80.0, 80.0, 80.0], 100, RC, tp.data_ptr(), tf.data_ptr(), te.data_ptr())
    assert e.value.code == md.MD_EINVAL

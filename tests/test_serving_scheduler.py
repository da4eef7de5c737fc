"""The serving loop's scheduling (host logic only, no GPU): admission in
arrival order by arena space, slices that add up to each request's step
count, retirement, and the latency statistics.  The ensemble engine is
replaced by a host-side stand-in with the same interface, which keeps only
the arena bookkeeping and the step counts; the served results themselves
are checked against md_step on the GPU (test_gpu_serving.py)."""
import numpy as np
import pytest

import paper_0911_5631_gb300 as md
from paper_0911_5631_gb300 import inputs
from paper_0911_5631_gb300.serve import Request, Server


class StandIn:
    """Arena bookkeeping and step counts in the shape of md.Ensemble."""

    def __init__(self, arena_bytes):
        self.arena = arena_bytes
        self.used = 0
        self.reps = {}
        self.next_id = 0
        self.runs = []
        self.peak = 0

    def set_shape(self, *args):
        self.shape = args

    def add(self, pos, vel, box, rc, skin, dt, reorder_interval=100):
        need = md.md_ensemble_replica_bytes(md.replica_desc(box, pos.shape[0], rc, skin, dt, reorder_interval))
        if self.used + need > self.arena:
            raise md.MDError(md.MD_ENOMEM, "arena full")
        rid = self.next_id
        self.next_id += 1
        self.used += need
        self.peak = max(self.peak, self.used)
        self.reps[rid] = {"bytes": need, "steps": 0, "pos": pos.copy(), "vel": vel.copy()}
        return rid

    def run(self, ids, steps):
        assert len(set(ids)) == len(ids)
        self.runs.append(list(zip(ids, steps)))
        for r, k in zip(ids, steps):
            assert k >= 0
            self.reps[r]["steps"] += k

    def sync(self):
        pass

    def wait(self, in_flight=1):
        self.waits = getattr(self, "waits", 0) + 1

    def status(self, rid):
        return md.MD_OK

    def measure(self, rid):
        return {"step": self.reps[rid]["steps"]}

    def get_state(self, rid):
        return self.reps[rid]["pos"], self.reps[rid]["vel"]

    def remove(self, rid):
        self.used -= self.reps.pop(rid)["bytes"]

    def close(self):
        pass


def _requests(count, rate, seed_steps=(50, 400)):
    reqs = []
    for k, (t, n, rho, T, seed, ns) in enumerate(inputs.serving_trace(count, rate=rate, n_min=300, n_max=6000,
                                                                      steps=seed_steps)):
        pos, vel, L = inputs.wca_state(n, rho, T, seed)
        reqs.append(Request(key=k, pos=pos, vel=vel, box=L, nsteps=ns, arrival=t))
    return reqs


def test_every_request_gets_exactly_its_steps_in_slices():
    reqs = _requests(20, rate=2000.0)
    arena = sum(r.bytes() for r in reqs) // 3  # about a third fits at once
    eng = StandIn(arena)
    srv = Server(arena, slice_steps=32, big_atoms=1 << 30, arena_fraction=1.0, ensemble=eng,
                 slice_atom_steps=200_000)
    stats = srv.serve(reqs)
    assert stats["requests"] == 20 and stats["failed"] == 0
    assert stats["atom_steps"] == sum(r.atoms * r.nsteps for r in reqs)
    for r in reqs:
        assert r.measure["step"] == r.nsteps
        assert r.finished >= r.admitted >= r.arrival - 1e-9
        assert r.result is not None and np.array_equal(r.result[0], r.pos)
    assert eng.peak <= arena and eng.used == 0 and not eng.reps
    assert len(eng.runs) == stats["launches"] > 1
    lat = sorted(r.finished - r.arrival for r in reqs)
    assert stats["latency_p50_s"] == pytest.approx(np.percentile(lat, 50))


def test_admission_is_first_come_first_served():
    reqs = _requests(12, rate=5000.0)
    arena = max(r.bytes() for r in reqs) * 2
    eng = StandIn(arena)
    srv = Server(arena, slice_steps=16, big_atoms=1 << 30, arena_fraction=1.0, ensemble=eng,
                 slice_atom_steps=50_000)
    srv.serve(reqs)
    order = sorted(reqs, key=lambda r: r.arrival)
    admitted = [r.admitted for r in order]
    assert admitted == sorted(admitted)  # no request overtakes an earlier arrival
    assert eng.peak <= arena


def test_slices_balance_work_per_block():
    # a slice gives a request about slice_atom_steps / atoms steps (at least
    # slice_steps, at most what it has left)
    reqs = _requests(6, rate=1e6, seed_steps=(2000, 2001))
    eng = StandIn(sum(r.bytes() for r in reqs))
    srv = Server(eng.arena, slice_steps=10, big_atoms=1 << 30, arena_fraction=1.0, ensemble=eng,
                 slice_atom_steps=400_000)
    srv.serve(reqs)
    first = dict(eng.runs[0])
    by_rid = {r.rid: r for r in reqs}
    for rid, k in first.items():
        r = by_rid[rid]
        want = max(10, 400_000 // r.atoms)
        if r.atoms >= srv.team_atoms:
            want = max(1, 400_000 * srv.team_blocks // r.atoms)
        assert k == min(r.nsteps, want)

"""The continuous-batching request loop: requests that arrive while others
run are admitted as space frees up, and each finished request's state is
bitwise the state md_step gives for it alone."""
import numpy as np
import pytest

import paper_0911_5631_gb300 as md
from paper_0911_5631_gb300 import inputs
from paper_0911_5631_gb300.serve import Request, Server
import oracle
from mdcheck import DT, RC, assert_trajectory_matches, ensure_built, sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _requests(count, rate, n_max, steps):
    reqs = []
    for k, (t, n, rho, T, seed, ns) in enumerate(inputs.serving_trace(count, rate=rate, n_min=300, n_max=n_max,
                                                                      steps=steps)):
        pos, vel, L = inputs.wca_state(n, rho, T, seed, jitter_amp=0.05)
        reqs.append(Request(key=k, pos=pos, vel=vel, box=L, nsteps=ns, arrival=t, reorder_interval=40))
    return reqs


def _alone(req):
    s = sim(req.pos, req.vel, req.box, skin=0.4, precision="mixed", reorder_interval=req.reorder_interval)
    s.step(req.nsteps)
    p, v = s.get_state()
    s.close()
    return p, v


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests(12, rate=40.0, n_max=9000, steps=(60, 260))
    budget = sum(r.bytes() for r in reqs) // 2 + (64 << 20)  # not everything fits at once
    srv = Server(budget, slice_steps=48, big_atoms=6000, arena_fraction=0.6)
    try:
        stats = srv.serve(reqs)
    finally:
        srv.close()
    assert stats["requests"] == len(reqs) and stats["failed"] == 0
    assert any(r.atoms >= 6000 for r in reqs) and any(r.atoms < 6000 for r in reqs)  # both routes taken
    assert stats["launches"] > len(reqs) // 2
    for r in reqs:
        assert r.finished >= r.admitted >= r.arrival - 1e-9
        assert r.measure["step"] == r.nsteps
        p, v = _alone(r)
        assert np.array_equal(r.result[0], p), r.key
        assert np.array_equal(r.result[1], v), r.key
    # the smallest request (an ensemble replica) and the largest (its own
    # handle) against the FP64 oracle from the request's start
    for r in (min(reqs, key=lambda q: q.atoms), max(reqs, key=lambda q: q.atoms)):
        ref = oracle.run(oracle.wrap(r.pos, r.box), r.vel, r.box, RC, 0.4, DT, r.nsteps, record=False)
        assert_trajectory_matches(r.result[0], r.result[1], ref, r.box, "mixed", r.nsteps)


def test_admission_waits_for_space():
    reqs = _requests(6, rate=1000.0, n_max=3000, steps=(40, 80))
    one = max(r.bytes() for r in reqs)
    srv = Server(2 * one + (1 << 20), slice_steps=16, big_atoms=1 << 30, arena_fraction=1.0)
    seen = []
    real_step = srv.step

    def step(now):
        out = real_step(now)
        seen.append((len(srv.active), sum(q.bytes() for q in srv.active.values())))
        return out

    srv.step = step
    try:
        stats = srv.serve(reqs)
    finally:
        srv.close()
    assert stats["requests"] == 6 and stats["failed"] == 0
    assert max(b for _, b in seen) <= srv.arena_bytes  # never more than the arena holds
    assert max(c for c, _ in seen) < 6  # so some requests waited for space

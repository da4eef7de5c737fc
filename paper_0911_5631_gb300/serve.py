"""Continuous-batching request loop over an ensemble (md_ensemble_* in md.h).

Requests are independent WCA simulations (N atoms, a state, a number of
steps) that arrive over time.  The loop keeps every admitted simulation's
state resident in one device arena and advances all of them together, one
launch per *slice* of at most ``slice_steps`` steps; a request that arrives
while others are on the GPU is admitted at the next slice boundary as soon
as the arena has room for it (first come, first served), so work of old and
new requests overlaps on the device.  A finished request's state is copied
back and its arena space is freed at the slice boundary where it finishes.

Requests of at least ``big_atoms`` atoms do not go into the ensemble,
whose engine gives a replica one thread block (one SM), or one cluster of
eight blocks when it has 8192 atoms or more: each gets a
single-simulation handle of its own (md_create; device memory counted
against the same budget) driven by a worker thread, so its grid-wide
kernels spread over the SMs the ensemble's launch leaves free, on its own
stream, while the loop keeps slicing the small requests.

Splitting a request's steps into slices does not change its result: each
slice is one md_step-equivalent call and consecutive calls compose bitwise,
and the ensemble engine and md_step give the same bits.  Scheduling is host
logic only (argument marshalling and bookkeeping); every MD operation runs
in the library's kernels.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (MD_ENOMEM, MD_OK, MD_PREC_MIXED, WCA_RC, Ensemble, MDError, Simulation, md_default_params,
               md_ensemble_replica_bytes, md_plan, replica_desc)


@dataclass
class Request:
    key: int
    pos: np.ndarray
    vel: np.ndarray
    box: np.ndarray
    nsteps: int
    arrival: float = 0.0          # seconds after the trace started
    rc: float = WCA_RC
    skin: float = 0.4
    dt: float = 0.005
    reorder_interval: int = 100
    # filled in by the server
    admitted: float | None = None
    finished: float | None = None
    status: int | None = None
    result: tuple | None = None
    measure: dict | None = None
    rid: int = -1
    thread: object = None         # worker of a big request
    solo_need: int = 0
    left: int = 0
    last_launch: int = 0          # ensemble slice that ran the last steps
    atoms: int = field(init=False)

    def __post_init__(self):
        self.atoms = int(np.asarray(self.pos).shape[0])

    def bytes(self) -> int:
        return md_ensemble_replica_bytes(replica_desc(self.box, self.atoms, self.rc, self.skin, self.dt,
                                                      self.reorder_interval))

    def solo_bytes(self) -> int:
        p = md_default_params()
        p.precision = MD_PREC_MIXED
        p.reorder_interval = self.reorder_interval
        return int(md_plan(self.box, self.atoms, self.rc, self.skin, self.dt, p).device_bytes)


class Server:
    """Admits requests by arena space, runs them in slices, retires them."""

    def __init__(self, budget_bytes: int, slice_steps: int = 200, big_atoms: int = 65536, arena_fraction=0.5,
                 max_replicas: int = 4096, device: int = -1, stream=None, keep_results: bool = True,
                 slice_atom_steps: int = 2_000_000, ensemble=None):
        self.arena_bytes = int(budget_bytes * arena_fraction)
        self.solo_budget = int(budget_bytes) - self.arena_bytes
        self.solo_used = 0
        self.device = device
        # `ensemble`: an engine with the Ensemble interface over an arena of
        # arena_bytes (the scheduler's own tests pass a host-side stand-in)
        self.ens = ensemble if ensemble is not None else Ensemble(self.arena_bytes, max_replicas=max_replicas,
                                                                  device=device, stream=stream)
        # big ensemble members run on clusters of team_blocks 1024-thread blocks
        self.team_atoms, self.team_blocks = 8192, 8
        self.ens.set_shape(1024, 0, self.team_blocks, self.team_atoms)
        self.slice_steps = int(slice_steps)
        self.slice_atom_steps = int(slice_atom_steps)
        self.big_atoms = int(big_atoms)
        self.keep_results = keep_results
        self.queue: list[Request] = []
        self.active: dict[int, Request] = {}   # ensemble replicas by id
        self.solo: list[Request] = []           # big requests on their own handles
        self.done: list[Request] = []
        self.launches = 0
        self.atom_steps = 0
        self._lock = threading.Lock()
        self._clock = time.perf_counter
        self._t0 = 0.0

    def close(self):
        for q in list(self.solo):
            if q.thread is not None:
                q.thread.join()
        self.solo = []
        self.ens.close()

    def _run_big(self, req: Request):
        """Worker: the whole request on its own handle (one md_step)."""
        status, meas, result = MD_OK, None, None
        try:
            sim = Simulation(req.box, req.atoms, req.rc, req.skin, req.dt, precision="mixed",
                             reorder_interval=req.reorder_interval, device=self.device)
            try:
                sim.set_state(req.pos, req.vel)
                sim.step(req.nsteps)
                meas = sim.measure()
                if self.keep_results:
                    result = sim.get_state()
            finally:
                sim.close()
        except MDError as e:
            status = e.code
        now = self._clock() - self._t0
        with self._lock:
            req.status, req.measure, req.result = status, meas, result
            req.left = 0
            req.finished = now
            if status == MD_OK:
                self.atom_steps += req.atoms * req.nsteps
            self.launches += 1
            self.solo_used -= req.solo_need
            self.solo.remove(req)
            self.done.append(req)

    # -- request flow -------------------------------------------------------

    def submit(self, req: Request):
        req.left = int(req.nsteps)
        self.queue.append(req)

    def _admit(self, now: float):
        while self.queue:
            req = self.queue[0]
            busy = bool(self.active or self.solo)
            if req.atoms >= self.big_atoms:
                need = req.solo_bytes()
                with self._lock:
                    if self.solo_used + need > self.solo_budget and busy:
                        return  # wait for space (first come, first served)
                    req.solo_need = need
                    self.solo_used += need
                    self.solo.append(req)
                req.thread = threading.Thread(target=self._run_big, args=(req,), daemon=True)
                req.thread.start()
            else:
                try:
                    req.rid = self.ens.add(req.pos, req.vel, req.box, req.rc, req.skin, req.dt,
                                           reorder_interval=req.reorder_interval)
                except MDError as e:
                    if e.code == MD_ENOMEM and busy:
                        return  # wait for space (first come, first served)
                    raise
                self.active[req.rid] = req
            self.queue.pop(0)
            req.admitted = now

    def _retire(self, now: float, finished: int):
        """Retires the requests whose last slice is among the first
        `finished` launches (all finished on the device): the per-replica
        calls below then return without waiting for the slice in flight."""
        for rid in [r for r, q in self.active.items() if q.left == 0 and q.last_launch <= finished]:
            req = self.active.pop(rid)
            req.status = self.ens.status(rid)
            if req.status == MD_OK:
                req.measure = self.ens.measure(rid)
                if self.keep_results:
                    req.result = self.ens.get_state(rid)
            req.finished = now
            self.ens.remove(rid)
            with self._lock:
                self.done.append(req)

    def step(self, now: float) -> bool:
        """One scheduling iteration at time `now`: admit, queue one slice of
        every active request that has steps left.  Returns False when there
        was nothing to run.  Requests whose steps are all queued are retired
        by _retire once their last slice has finished."""
        self._admit(now)
        ids = [r for r, q in self.active.items() if q.left > 0]
        if not ids:
            return False
        # about the same work per block in one slice: small replicas take
        # more steps than big ones (at least slice_steps when they can), so
        # no slice waits long for its largest member
        steps = []
        for r in ids:
            q = self.active[r]
            k = max(self.slice_steps, self.slice_atom_steps // max(q.atoms, 1))
            if q.atoms >= self.team_atoms:
                k = max(1, (self.slice_atom_steps * self.team_blocks) // q.atoms)
            steps.append(min(q.left, k))
        # queue the slice and return at once: the requests that finished in
        # the previous slice are retired while this one runs, and the next
        # iteration waits for the previous slice only (one run in flight
        # behind the newest), so the GPU never idles for the bookkeeping
        self.ens.run(ids, steps)
        with self._lock:
            self.launches += 1
            for r, s in zip(ids, steps):
                q = self.active[r]
                q.left -= s
                if q.left == 0:
                    q.last_launch = self.launches
                self.atom_steps += q.atoms * s
        return True

    def serve(self, requests: list[Request], clock=time.perf_counter) -> dict:
        """Replays a trace in real time: request k becomes visible at
        requests[k].arrival seconds after the start.  Returns summary
        statistics (latency = completion - arrival)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self._clock = clock
        t0 = self._t0 = clock()
        k = 0
        while True:
            with self._lock:
                busy = bool(self.queue or self.active or self.solo)
            if k >= len(pending) and not busy:
                break
            now = clock() - t0
            while k < len(pending) and pending[k].arrival <= now:
                self.submit(pending[k])
                k += 1
            ran = self.step(now)
            if ran:  # the slice before the one just queued has finished
                self.ens.wait(1)
                self._retire(clock() - t0, self.launches - 1)
            else:  # nothing left to queue: finish what runs, then wait for an arrival or a worker
                self.ens.wait(0)
                self._retire(clock() - t0, self.launches)
                now = clock() - t0
                nxt = pending[k].arrival - now if k < len(pending) else 0.002
                time.sleep(max(0.0, min(nxt, 0.002)))
        for q in self.done:
            if q.thread is not None:
                q.thread.join()
        wall = clock() - t0
        lat = np.array([r.finished - r.arrival for r in self.done])
        return {"requests": len(self.done), "wall_s": wall, "launches": self.launches,
                "atom_steps": int(self.atom_steps), "atom_steps_per_s": self.atom_steps / wall if wall > 0 else 0.0,
                "latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "failed": sum(1 for r in self.done if r.status != MD_OK)}

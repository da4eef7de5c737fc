#!/usr/bin/env python3
"""Throughput benchmark of the soft-sphere MD hot path on GB300.

Workload (default): 1,048,576 WCA atoms (FCC 64^3 x 4), rho = 0.8, T = 1.0,
dt = 0.005, neighbour list with skin 0.4, reorder every 100 steps.  The
state is equilibrated untimed, then every benchmark "step" advances 100 MD
steps (one reorder interval: about ten list rebuilds and one reorder) through
md_step.  The metric is atom-steps per second of the mixed-precision form;
the plain FP64 GPU form is timed on the same workload beside it.

One JSON line is printed by rank 0.  Under torchrun every rank runs an
independent replica on its own GPU (the path has no exchange step), timing is
the max over ranks and ``value`` sums the atoms of all ranks.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0911_5631_gb300 import inputs  # noqa: E402

METRIC = "atom-steps/s at 1M WCA atoms (mixed vs FP64 GPU form); ensemble p50/p99 latency"
UNIT = "atom-steps/s"
RC = 2.0 ** (1.0 / 6.0)
DT = 0.005
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="wca_fcc64_n1m")
    ap.add_argument("--chunk", type=int, default=500,
                    help="MD steps per benchmark step (five reorder intervals)")
    ap.add_argument("--equil", type=int, default=1000, help="untimed equilibration MD steps")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble line")
    ap.add_argument("--ens-replicas", type=int, default=inputs.ENSEMBLE["replicas"])
    ap.add_argument("--ens-steps", type=int, default=inputs.ENSEMBLE["steps"])
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-trace lines")
    ap.add_argument("--no-lj", action="store_true", help="skip the Lennard-Jones line")
    ap.add_argument("--drift", action="store_true",
                    help="only the 8M-atom energy-drift runs (10^5 steps at each (rho, T) pairing, FP64 oracle "
                         "segments every 10^4 steps); prints their JSON summary")
    ap.add_argument("--drift-steps", type=int, default=100000)
    ap.add_argument("--drift-every", type=int, default=10000)
    ap.add_argument("--no-ablations", action="store_true",
                    help="skip the ablations (reorder interval, shell bins, kernel variants, builds)")
    ap.add_argument("--serve-requests", type=int, default=500, help="requests per serving trace")
    ap.add_argument("--serve-big-atoms", type=int, default=65536,
                    help="requests of at least this many atoms get a handle of their own")
    ap.add_argument("--serve-sweep", default="0.5,0.7,0.9",
                    help="arrival rates below saturation, as fractions of the rate the lambda=200 trace sustains")
    ap.add_argument("--eager", action="store_true", help="stream launches instead of graphs")
    ap.add_argument("--build", default="auto", choices=["auto", "thread", "warp"],
                    help="neighbour-list build kernel (md_params.build_kernel)")
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="benchmark steps run with per-kernel CUDA events for the roofline")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(units_local, ms_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: units summed over ranks,
    divided by the slowest rank's time.  Returns (units/s, max ms)."""
    if dist is None:
        return units_local / (ms_local / 1e3), ms_local
    import torch
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text):
    """C++ source without comments, whitespace runs collapsed: a comment edit
    leaves the compiled kernels, and so the hash, unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":  # string or character literal, kept whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash():
    """Hash of the kernel source (code only) that the committed ncu
    summaries name in their `kernel_source` line."""
    h = hashlib.sha256()
    for f in ("md_kernels.cuh", "md_common.cuh"):
        with open(os.path.join(ROOT, "paper_0911_5631_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload, precision):
    """Per-launch DRAM bytes (read + write) of the step kernel from the
    committed ncu summary, if that summary was taken on the current kernel
    source (its `kernel_source` line matches); else None."""
    p = os.path.join(ROOT, "profiles", "k_step_%s_%s.md" % (workload, precision))
    if not os.path.exists(p):
        return None
    fields = {}
    with open(p) as fh:
        for line in fh:
            if " = " in line and not line.startswith("|"):
                k, v = line.strip().split(" = ", 1)
                fields[k] = v
    if fields.get("kernel_source") != kernel_source_hash():
        return None
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def _oracle_rate(oracle, pos, vel, L, cfg, threaded, seconds):
    """atom-steps/s of one oracle build on a bounded sample: a 2-step probe
    sizes the sample to about `seconds`, then one run is timed (it includes
    the initial list build).  Returns (value, steps, seconds taken)."""
    n = pos.shape[0]
    t0 = time.perf_counter()
    oracle.run(pos, vel, L, cfg.get("rc", RC), cfg["skin"], DT, 2, record=False, threaded=threaded)
    t1 = time.perf_counter() - t0
    steps = int(max(4, min(2000, seconds / max(t1 / 2, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(pos, vel, L, cfg.get("rc", RC), cfg["skin"], DT, steps, record=False, threaded=threaded)
    t = time.perf_counter() - t0
    return n * steps / t, steps, t


def run_reference(args):
    """Times the FP64 CPU oracle on the host cores (the OpenMP build of the
    oracle source, every core)."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg = inputs.WORKLOADS[args.workload]
    n = cfg["n"]
    pos, vel, L = inputs.wca_state(n, cfg["rho"], cfg["T"], cfg["seed"])
    pos = oracle.wrap(pos, L)
    cores = oracle.threads(True)
    sample = 4  # MD steps per benchmark step, from the lattice start
    for _ in range(args.warmup):
        oracle.run(pos, vel, L, cfg.get("rc", RC), cfg["skin"], DT, sample, record=False, threaded=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(pos, vel, L, cfg.get("rc", RC), cfg["skin"], DT, sample, record=False, threaded=True)
    t = time.perf_counter() - t0
    value = n * sample * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "n_atoms": n, "rho": cfg["rho"],
                                        "T": cfg["T"], "skin": cfg["skin"],
                                        "md_steps_per_bench_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d MD steps of the %d-atom workload from its lattice start per "
                                   "benchmark step, C oracle built with OpenMP on %d threads"
                                   % (sample, n, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(pos, vel, L, cfg, seconds=10.0):
    """The oracle as it stands on the host cores, each build on a bounded
    sample of the equilibrated state: the plain single-threaded build (the
    parity reference) and the OpenMP build of the same source on every
    core.  `value` and `cores` are the all-core figures."""
    import oracle
    n = pos.shape[0]
    p = oracle.wrap(pos, L)
    v1, k1, t1 = _oracle_rate(oracle, p, vel, L, cfg, False, seconds)
    vt, kt, tt = _oracle_rate(oracle, p, vel, L, cfg, True, seconds)
    cores = oracle.threads(True)
    return {"value": vt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d MD steps of the %d-atom equilibrated state (includes the initial list build), "
                      "C oracle built with OpenMP on %d threads, %.1f s" % (kt, n, cores, tt),
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": "%d MD steps, plain single-threaded C oracle, %.1f s" % (k1, t1)}}


def ensemble_bench(md, torch, stream, device, replicas, steps, probe):
    """The batched ensemble: replicas of uneven size and state, loaded into
    one arena, autotuned, then advanced `steps` steps each by one launch.
    Latency = each replica's completion time after the launch began."""
    specs = inputs.ensemble_specs(replicas)
    skin, reorder = inputs.ENSEMBLE["skin"], inputs.ENSEMBLE["reorder_interval"]
    states = [inputs.wca_state(n, rho, T, seed) for (n, rho, T, seed) in specs]
    need = sum(md.md_ensemble_replica_bytes(md.replica_desc(L, p.shape[0], RC, skin, DT, reorder))
               for (p, v, L) in states)
    e = md.Ensemble(int(need * 1.02) + (256 << 20), max_replicas=replicas, device=device,
                    stream=stream.cuda_stream)
    try:
        ids = [e.add(p, v, L, RC, skin, DT, reorder_interval=reorder) for (p, v, L) in states]
        atoms = sum(p.shape[0] for (p, v, L) in states)
        e.run(ids, [0] * len(ids))  # load: wrap, bin, list, forces
        e.sync()
        block, cluster = e.autotune(ids, probe_steps=probe)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e.run(ids, [steps] * len(ids))
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        t0, t1 = e.times(ids)
        bad = [i for i in ids if e.status(i) != md.MD_OK]
        if bad:
            raise RuntimeError("ensemble replicas failed: %s" % bad[:8])
        m = e.measure(ids[0])
        if m["step"] != steps + 6 * probe:
            raise RuntimeError("ensemble replica advanced %d steps" % m["step"])
        return {"workload": "wca_ensemble_%d" % replicas, "replicas": replicas, "atoms": int(atoms),
                "n_range": [inputs.ENSEMBLE["n_min"], inputs.ENSEMBLE["n_max"]], "steps": steps,
                "value": atoms * steps / (ms / 1e3), "unit": UNIT, "ms": ms, "launches": 1,
                "latency_p50_ms": float(np.percentile(t1, 50)), "latency_p99_ms": float(np.percentile(t1, 99)),
                "latency_max_ms": float(np.max(t1)),
                "latency": "completion of each replica after the launch began; all replicas submitted together",
                "block": int(block), "cluster": int(cluster), "autotune_probe_steps": probe}
    finally:
        e.close()


def serving_bench(md, stream, device, count, rate, budget_bytes, slice_steps, big_atoms=65536):
    """Replays a Poisson trace of `count` requests through the
    continuous-batching loop (paper_0911_5631_gb300.serve)."""
    from paper_0911_5631_gb300.serve import Request, Server
    sk = inputs.SERVING["skin"]
    reqs = []
    for k, (t, n, rho, T, seed, ns) in enumerate(inputs.serving_trace(count, rate=rate)):
        pos, vel, L = inputs.wca_state(n, rho, T, seed)
        reqs.append(Request(key=k, pos=pos, vel=vel, box=L, nsteps=ns, arrival=t, skin=sk, dt=DT))
    srv = Server(budget_bytes, slice_steps=slice_steps, device=device, keep_results=False, big_atoms=big_atoms)
    try:
        st = srv.serve(reqs)
    finally:
        srv.close()
    if st["failed"]:
        raise RuntimeError("%d serving requests failed" % st["failed"])
    st.update({"workload": "wca_serving_poisson", "rate_per_s": rate, "requests_offered": count,
               "n_range": [inputs.SERVING["n_min"], inputs.SERVING["n_max"]],
               "steps_range": list(inputs.SERVING["steps"]), "slice_steps": slice_steps,
               "budget_gb": budget_bytes / 1e9, "big_atoms": big_atoms,
               "mean_atom_steps_per_request": float(np.mean([r.atoms * r.nsteps for r in reqs])),
               "offered_atom_steps_per_s": rate * float(np.mean([r.atoms * r.nsteps for r in reqs])),
               "latency": "completion - arrival (s), trace replayed in real time"})
    return st


def lj_bench(md, torch, stream, device, steps, chunk=100):
    """The Lennard-Jones workload (r_c = 3, rho 0.38, T 1.2, shell 0.8, 1M
    atoms, mixed form): atom-steps/s over `steps` benchmark steps of `chunk`
    MD steps after 200 untimed steps."""
    cfg = inputs.WORKLOADS["lj_fcc64_n1m_rc3"]
    n = cfg["n"]
    pos, vel, L = inputs.wca_state(n, cfg["rho"], cfg["T"], cfg["seed"])
    s = md.Simulation(L, n, cfg["rc"], cfg["skin"], DT, precision="mixed", reorder_interval=100,
                      stream=stream.cuda_stream, device=device)
    try:
        s.set_state(pos, vel)
        s.step(200)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        m0 = s.measure()
        e0.record(stream)
        for _ in range(steps):
            s.step(chunk)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        m1 = s.measure()
        if m1["step"] - m0["step"] != steps * chunk:
            raise RuntimeError("LJ run advanced %d steps" % (m1["step"] - m0["step"]))
        return {"workload": "lj_fcc64_n1m_rc3", "n_atoms": n, "rho": cfg["rho"], "T": cfg["T"], "rc": cfg["rc"],
                "skin": cfg["skin"], "value": n * steps * chunk / (ms / 1e3), "unit": UNIT,
                "ms_per_md_step": ms / (steps * chunk), "neighbours_per_atom": m1["list_entries"] / n,
                "rebuilds": m1["rebuilds"] - m0["rebuilds"], "md_steps": steps * chunk}
    finally:
        s.close()


ABLATIONS = [
    # (label, Simulation keyword arguments): the paper's Tables 7 and 8
    # (reorder interval; 0 = never after the load), reading every list entry
    # at every step as the paper does (shell bins off), the texture-cache
    # remark of Sec. 4.4 (plain loads), W transposed, Table 6 (threads per
    # block of the force kernel: 64 and 256 against the default 128), and
    # the warp-cooperative build
    ("reorder_0", {"reorder_interval": 0}),
    ("reorder_20", {"reorder_interval": 20}),
    ("reorder_100 (default)", {"reorder_interval": 100}),
    ("reorder_500", {"reorder_interval": 500}),
    ("shell_bins_off", {"shell_bins": False}),
    ("plain_loads", {"variant": "plain_loads"}),
    ("w_transposed", {"variant": "list_rows"}),
    ("block_64", {"variant": "block64"}),
    ("block_256", {"variant": "block256"}),
    ("warp_build", {"build": "warp"}),
]


def ablations(md, torch, stream, device, pos, vel, L, cfg, chunk=100, steps=5):
    """The paper's ablations on the 1M workload (mixed form), each from the
    equilibrated state: 1000 untimed steps (long enough for the storage
    order to drift from the cell order), then `steps` x `chunk` timed MD
    steps (graphs, CUDA events) and one profiled chunk for the step kernel's
    and the rebuild branch's own times."""
    out = []
    for label, kw in ABLATIONS:
        kw = dict(kw)
        kw.setdefault("reorder_interval", 100)
        s = md.Simulation(L, cfg["n"], cfg.get("rc", RC), cfg["skin"], DT, precision="mixed",
                          stream=stream.cuda_stream, device=device, **kw)
        try:
            s.set_state(pos, vel)
            s.step(1000)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                s.step(chunk)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            s.set_profiling(True)
            k0 = s.kernel_stats()
            s.step(chunk)
            k1 = s.kernel_stats()
            s.set_profiling(False)
            kl = k1["step_kernel_launches"] - k0["step_kernel_launches"]
            rb = k1["rebuilds_timed"] - k0["rebuilds_timed"]
            out.append({"ablation": label, "params": kw,
                        "value": cfg["n"] * chunk * steps / (ms / 1e3), "unit": UNIT,
                        "step_kernel_us": 1e3 * (k1["step_kernel_ms"] - k0["step_kernel_ms"]) / max(kl, 1),
                        "rebuild_us": 1e3 * (k1["rebuild_ms"] - k0["rebuild_ms"]) / rb if rb else None,
                        "reorders": s.measure()["reorders"]})
        finally:
            s.close()
    return out


def run_ours(args):
    import torch
    import paper_0911_5631_gb300 as md

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = inputs.WORKLOADS[args.workload]
    n = cfg["n"]
    pos, vel, L = inputs.wca_state(n, cfg["rho"], cfg["T"], cfg["seed"] + 1000 * rank)
    stream = torch.cuda.Stream()

    def make(precision):
        s = md.Simulation(L, n, cfg.get("rc", RC), cfg["skin"], DT, precision=precision, reorder_interval=100,
                          use_graphs=not args.eager, stream=stream.cuda_stream, device=local, build=args.build)
        s.set_state(pos, vel)
        return s

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(sim, k):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            sim.step(args.chunk)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        barrier()
        return ms

    # ---- mixed form: the headline ----
    sim = make("mixed")
    sim.step(args.equil)
    eq_pos, eq_vel = sim.get_state()
    for _ in range(args.warmup):
        sim.step(args.chunk)
    st0 = sim.kernel_stats()
    m0 = sim.measure()
    clocks = Clocks(local)
    clocks.start()
    ms_local = timed(sim, args.steps)
    clk = clocks.stop()
    m1 = sim.measure()
    st1 = sim.kernel_stats()
    # the timed region must have advanced the simulation by exactly the
    # steps it claims
    done = m1["step"] - m0["step"]
    if done != args.chunk * args.steps:
        raise RuntimeError("timed region advanced %d MD steps, expected %d" % (done, args.chunk * args.steps))
    value, ms = job_throughput(n * args.chunk * args.steps, ms_local, dist, "cuda")
    launches = st1["launches"] - st0["launches"]

    # ---- roofline of the force + integrate kernel (event-timed launches) ----
    sim.set_profiling(True)
    p0 = sim.kernel_stats()
    for _ in range(args.profile_steps):
        sim.step(args.chunk)
    p1 = sim.kernel_stats()
    sim.set_profiling(False)
    kms = p1["step_kernel_ms"] - p0["step_kernel_ms"]
    kl = p1["step_kernel_launches"] - p0["step_kernel_launches"]
    kbytes = p1["step_kernel_bytes"] - p0["step_kernel_bytes"]
    peak, peak_kind = measured_peaks()
    achieved = (kbytes / kl) / (kms / kl / 1e3) / 1e9 if kl and kms > 0 else None
    traffic = ncu_traffic(args.workload, "mixed")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_kind": peak_kind, "kernel": "k_step (force + integrate, mixed)",
                "kernel_ms_per_launch": kms / kl if kl else None,
                "algorithmic_bytes_per_launch": kbytes / kl if kl else None}
    rb = p1["rebuilds_timed"] - p0["rebuilds_timed"]
    rebuild_ms = (p1["rebuild_ms"] - p0["rebuild_ms"]) / rb if rb else None
    list_entries = m1["list_entries"]
    rebuilds = m1["rebuilds"] - m0["rebuilds"]

    # ---- e2e: host buffers through the C ABI, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(eq_pos.copy()).pin_memory()
        hv = torch.from_numpy(eq_vel.copy()).pin_memory()
        op = torch.empty_like(hp).pin_memory()
        ov = torch.empty_like(hv).pin_memory()
        lib = md.lib()
        k_e2e = max(2, args.steps // 4)

        def e2e_step():
            md._check(lib.md_set_state(sim.h, hp.data_ptr(), hv.data_ptr()), sim.h)
            sim.step(args.chunk)
            md._check(lib.md_get_state(sim.h, op.data_ptr(), ov.data_ptr()), sim.h)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        barrier()
        t = time.perf_counter() - t0
        e2e_value, _ = job_throughput(n * args.chunk * k_e2e, 1e3 * t, dist, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(hp.numel() * 8 + hv.numel() * 8),
               "d2h_bytes_per_step": int(op.numel() * 8 + ov.numel() * 8),
               "steps": k_e2e, "what": "md_set_state from pinned host memory, md_step(%d), "
                                        "md_get_state to pinned host memory" % args.chunk}
    sim.close()

    # ---- plain FP64 GPU form on the same workload ----
    fp64 = None
    if not args.no_fp64:
        s64 = make("fp64")
        s64.set_state(eq_pos, eq_vel)
        k64 = max(2, args.steps // 4)
        for _ in range(max(1, args.warmup // 2)):
            s64.step(args.chunk)
        ms64_local = timed(s64, k64)
        s64.set_profiling(True)
        q0 = s64.kernel_stats()
        s64.step(args.chunk)
        q1 = s64.kernel_stats()
        s64.close()
        v64, ms64 = job_throughput(n * args.chunk * k64, ms64_local, dist, "cuda")
        kms64 = q1["step_kernel_ms"] - q0["step_kernel_ms"]
        kl64 = q1["step_kernel_launches"] - q0["step_kernel_launches"]
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                "step_kernel_ms_per_launch": kms64 / kl64 if kl64 else None,
                "mixed_over_fp64": value / v64}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(eq_pos, eq_vel, L, cfg)

    ens = None
    if rank == 0 and not args.no_ensemble:
        ens = ensemble_bench(md, torch, stream, local, args.ens_replicas, args.ens_steps, 10)
    abl = None
    if rank == 0 and not args.no_ablations:
        abl = ablations(md, torch, stream, local, eq_pos, eq_vel, L, cfg)
    lj = None
    if rank == 0 and not args.no_lj:
        lj = lj_bench(md, torch, stream, local, 5)
    serving = None
    if rank == 0 and not args.no_serving:
        # the configured Poisson rate (above saturation: the queue grows and
        # the finite trace drains at the sustained rate), then a sweep below
        # the saturation rate that trace measured
        top = serving_bench(md, stream, local, args.serve_requests, inputs.SERVING["rate"], 40 << 30, 200,
                            args.serve_big_atoms)
        serving = [top]
        lam_sat = top["atom_steps_per_s"] / top["mean_atom_steps_per_request"]
        for f in [float(x) for x in args.serve_sweep.split(",") if x.strip()]:
            st = serving_bench(md, stream, local, args.serve_requests, f * lam_sat, 40 << 30, 200,
                               args.serve_big_atoms)
            st.update({"fraction_of_saturation": f, "saturation_rate_per_s": lam_sat})
            serving.append(st)
    if rank == 0:
        ws_bytes = n * (12 + 24 + 12 + 32 + 4) + list_entries * 4 * 1.3
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair / f64 position / int64 force sum",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_atoms": n, "rho": cfg["rho"], "T": cfg["T"],
                       "skin": cfg["skin"], "dt": DT, "reorder_interval": 100, "precision": "mixed",
                       "md_steps_per_bench_step": args.chunk, "equilibration_steps": args.equil,
                       "graphs": not args.eager,
                       "l2": "no flush: per-step working set %.0f MB > 129 MB L2" % (ws_bytes / 2 ** 20),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "gpu_launches": int(launches),
            "rebuilds_in_timed_region": int(rebuilds),
            "rebuild_ms_per_branch": rebuild_ms,
            "neighbours_per_atom": list_entries / n,
            "roofline": roofline,
            "fp64_form": fp64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "lj": lj,
            "ablations": abl,
            "ensemble": ens,
            "serving": serving,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


DRIFT_WORKLOADS = ["wca_fcc128_n8m_rho0.6_T0.7", "wca_fcc128_n8m_rho0.6_T2.0", "wca_fcc128_n8m_rho1.0_T0.7",
                   "wca_fcc128_n8m_rho1.0_T2.0"]


def drift_runs(args):
    """The 8M-atom mixed-form runs: for each (rho, T) pairing, 500 untimed
    steps from the lattice, then `--drift-steps` steps with the total energy
    per atom sampled every 100 steps; every `--drift-every` steps the FP64
    oracle (all host cores) runs 5 steps from the GPU's state and the GPU's
    own next 5 steps are compared with it (velocity and position RMS
    against the trajectory tolerance of the parity tests).  Drift is
    |<e_tot>_{last 1000 steps} - <e_tot>_{steps 1000-2000}| per atom (block
    means of the samples), beside the largest excursion of e_tot per atom."""
    import torch
    import oracle
    import paper_0911_5631_gb300 as md
    torch.cuda.set_device(0)
    out = []
    k = 5
    for wl in DRIFT_WORKLOADS:
        cfg = inputs.WORKLOADS[wl]
        n = cfg["n"]
        pos, vel, L = inputs.wca_state(n, cfg["rho"], cfg["T"], cfg["seed"])
        s = md.Simulation(L, n, RC, cfg["skin"], DT, precision="mixed", reorder_interval=100, device=0)
        t_wall = time.perf_counter()
        segs, samples = [], []
        try:
            s.set_state(pos, vel)
            s.step(500)
            done = 0
            while done < args.drift_steps:
                if done % args.drift_every == 0:
                    p, v = s.get_state()
                    t0 = time.perf_counter()
                    ref = oracle.run(p, v, L, RC, cfg["skin"], DT, k, record=False, threaded=True)
                    t_orc = time.perf_counter() - t0
                    s.step(k)
                    p2, v2 = s.get_state()
                    f_rms = float(np.sqrt(np.mean(ref["f"] ** 2)))
                    dv_tol = 10.0 * k * DT * 1e-5 * f_rms + 1e-7
                    d = p2 - ref["pos"]
                    d -= np.asarray(L) * np.round(d / np.asarray(L))
                    ev = float(np.sqrt(np.mean((v2 - ref["vel"]) ** 2)))
                    ex = float(np.sqrt(np.mean(d ** 2)))
                    segs.append({"step": done, "vel_rms_err": ev, "vel_tol": dv_tol, "pos_rms_err": ex,
                                 "pos_tol": k * DT * dv_tol + 1e-12, "oracle_s": t_orc,
                                 "ok": ev <= dv_tol and ex <= k * DT * dv_tol + 1e-12})
                    done += k
                s.step(100 - done % 100)
                done += 100 - done % 100
                samples.append((done, s.measure()["e_tot_per_atom"]))
            m = s.measure()
        finally:
            s.close()
        st = np.array([x for x, _ in samples])
        e = np.array([y for _, y in samples])
        early = e[(st > 1000) & (st <= 2000)]
        late = e[st > st[-1] - 1000]
        # the same measure over each window of `--drift-every` steps
        windows = []
        for w0 in range(0, args.drift_steps, args.drift_every):
            a_ = e[(st > w0) & (st <= w0 + 1000)]
            b_ = e[(st > w0 + args.drift_every - 1000) & (st <= w0 + args.drift_every)]
            if a_.size and b_.size:
                windows.append(float(abs(b_.mean() - a_.mean())))
        out.append({"workload": wl, "n_atoms": n, "rho": cfg["rho"], "T": cfg["T"], "steps": int(m["step"]),
                    "window_drift_max_per_atom": max(windows) if windows else None,
                    "rebuilds": int(m["rebuilds"]), "drift_per_atom": float(abs(late.mean() - early.mean())),
                    "max_excursion_per_atom": float(np.max(np.abs(e - e[0]))), "e_tot_first": float(e[0]),
                    "e_tot_last": float(e[-1]), "segments": segs,
                    "segments_ok": all(x["ok"] for x in segs), "wall_s": time.perf_counter() - t_wall})
    print(json.dumps({"drift_runs": out, "oracle_threads": oracle.threads(True)}), flush=True)


def main():
    args = parse()
    if args.drift:
        drift_runs(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

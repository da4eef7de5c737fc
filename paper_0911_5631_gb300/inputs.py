"""Seeded synthetic inputs: lattice starts and Maxwell velocities.

This module only generates input states; it holds none of the MD method's
arithmetic and imports neither the CUDA library nor the oracle, so both
sides of a parity test can be fed the same arrays from here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the xor-shift-multiply finaliser.  Uniform doubles take the top 53
bits; normal deviates use the Box-Muller transform.

Initial states follow the paper's recipe (Sec. 3.5: lattice start, velocity
of given temperature, centre of mass at rest) with an FCC lattice and
Maxwell-distributed velocities in place of the simple cubic lattice and
fixed speed.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for a given seed (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n uniform doubles in (0, 1]."""
    z = splitmix64(seed, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * math.pi * u[1::2]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:n]


def box_for(n: int, rho: float, aspect=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Edge lengths of a box of volume n/rho with the given aspect ratios."""
    a = np.asarray(aspect, dtype=np.float64)
    scale = (n / rho / float(np.prod(a))) ** (1.0 / 3.0)
    return a * scale


def fcc_positions(n: int, L) -> np.ndarray:
    """First n sites of an FCC lattice filling the box, region centred at the
    origin.  With a cubic box and n = 4 k^3 this is the exact k^3-cell FCC
    crystal.  Sites are (i + 1/4 + basis) * a - L/2 in (z, y, x, basis) order."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    vol = float(np.prod(L))
    a0 = (4.0 * vol / max(n, 1)) ** (1.0 / 3.0)
    k = np.maximum(1, np.ceil(L / a0 - 1e-9)).astype(np.int64)
    while 4 * int(np.prod(k)) < n:
        k[np.argmin(k * a0 / L)] += 1
    a = L / k
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(k[2]), np.arange(k[1]), np.arange(k[0]), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + 0.25 + basis[None, :, :]).reshape(-1, 3)
    return (sites[:n] * a - 0.5 * L).copy()


def maxwell_velocities(n: int, T: float, seed: int) -> np.ndarray:
    """Normal velocity components, centre-of-mass motion removed, scaled so
    that sum v^2 = 3 n T exactly (unit mass)."""
    if n == 0:
        return np.zeros((0, 3))
    v = normal(seed, 3 * n).reshape(n, 3)
    v -= v.mean(axis=0)
    s2 = float(np.sum(v * v))
    if s2 > 0:
        v *= math.sqrt(3.0 * n * T / s2)
    return v


def jitter(pos: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """Add independent uniform displacements in [-amp, amp) per component
    (no wrapping: consumers wrap)."""
    u = uniform(seed, pos.size).reshape(pos.shape)
    return pos + amp * (2.0 * u - 1.0)


def wca_state(n: int, rho: float, T: float, seed: int, jitter_amp: float = 0.0,
              aspect=(1.0, 1.0, 1.0)):
    """(pos, vel, L): FCC start in a box of density rho, Maxwell velocities at
    temperature T; optional lattice jitter (in units of length) that breaks
    the perfect crystal so that pairs fall inside the cutoff at t = 0."""
    L = box_for(n, rho, aspect)
    pos = fcc_positions(n, L)
    if jitter_amp > 0.0:
        pos = jitter(pos, jitter_amp, seed ^ 0x5DEECE66D)
    vel = maxwell_velocities(n, T, seed)
    return pos, vel, L


def sc_state(n_e: int, rho: float, T: float, seed: int):
    """(pos, vel, L): the initial state the paper describes -- atoms on a
    simple cubic lattice of edge n_e (n_e^3 atoms, sites (i + 1/2) a - L/2),
    velocities of magnitude sqrt(3 T) in uniformly random directions, then
    the centre-of-mass velocity subtracted."""
    L = box_for(n_e ** 3, rho)
    a = L / n_e
    g = (np.arange(n_e) + 0.5)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel() * a[0], y.ravel() * a[1], z.ravel() * a[2]], axis=1) - L / 2
    u = uniform(seed, 2 * n_e ** 3).reshape(-1, 2)
    cz = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * np.pi * u[:, 1]
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    vel = np.sqrt(3.0 * T) * np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
    vel -= vel.mean(axis=0)
    return pos, vel, L


# Workloads of the soft-sphere benchmark suite, by size and thermodynamic
# state.  rc = 2^(1/6) throughout, dt = 0.005.
WCA_RC = 2.0 ** (1.0 / 6.0)

WORKLOADS = {
    # cell list only (no skin), FP64
    "wca_fcc8_n2048": dict(n=2048, rho=0.8, T=1.0, seed=1, skin=0.0, steps=1000),
    # neighbour list with skin 0.4, reorder every 100 steps
    "wca_fcc64_n1m": dict(n=1048576, rho=0.8, T=1.0, seed=2, skin=0.4, steps=10000),
    # large system, two densities / temperatures
    # (the pairing of density and temperature is not stated: all four)
    "wca_fcc128_n8m_rho0.6_T0.7": dict(n=8388608, rho=0.6, T=0.7, seed=3, skin=0.4, steps=100000),
    "wca_fcc128_n8m_rho0.6_T2.0": dict(n=8388608, rho=0.6, T=2.0, seed=3, skin=0.4, steps=100000),
    "wca_fcc128_n8m_rho1.0_T0.7": dict(n=8388608, rho=1.0, T=0.7, seed=3, skin=0.4, steps=100000),
    "wca_fcc128_n8m_rho1.0_T2.0": dict(n=8388608, rho=1.0, T=2.0, seed=3, skin=0.4, steps=100000),
    # Lennard-Jones system of the paper's comparisons: rho 0.38, T 1.2, shell 0.8
    "lj_fcc64_n1m_rc3": dict(n=1048576, rho=0.38, T=1.2, seed=6, skin=0.8, rc=3.0, steps=6000),
}


# Batched ensemble: independent WCA replicas of uneven size and state.
ENSEMBLE = dict(replicas=512, n_min=256, n_max=32768, rho=(0.6, 1.0), T=(0.5, 2.0), seed=4, skin=0.4,
                steps=2000, reorder_interval=100)


def ensemble_specs(replicas: int = ENSEMBLE["replicas"], seed: int = ENSEMBLE["seed"],
                   n_min: int = ENSEMBLE["n_min"], n_max: int = ENSEMBLE["n_max"]):
    """Per-replica (n, rho, T, seed): n log-uniform in [n_min, n_max], rho and
    T uniform in the ENSEMBLE ranges, all from one seeded SplitMix64 stream."""
    u = uniform(seed, 3 * replicas).reshape(replicas, 3)
    lo, hi = np.log(n_min), np.log(n_max)
    out = []
    for k in range(replicas):
        n = int(np.floor(np.exp(lo + (hi - lo) * u[k, 0])))
        n = min(max(n, n_min), n_max)
        rho = ENSEMBLE["rho"][0] + (ENSEMBLE["rho"][1] - ENSEMBLE["rho"][0]) * u[k, 1]
        T = ENSEMBLE["T"][0] + (ENSEMBLE["T"][1] - ENSEMBLE["T"][0]) * u[k, 2]
        out.append((n, float(rho), float(T), seed * 100003 + k))
    return out


# Serving trace: Poisson arrivals of independent WCA requests.
SERVING = dict(rate=200.0, n_min=500, n_max=200000, steps=(1000, 20000), rho=0.8, T=1.0, seed=5, skin=0.4)


def serving_trace(count: int, rate: float = SERVING["rate"], seed: int = SERVING["seed"],
                  n_min: int = SERVING["n_min"], n_max: int = SERVING["n_max"], steps=SERVING["steps"]):
    """count requests (arrival_s, n, rho, T, seed, nsteps): exponential
    inter-arrival times of mean 1/rate, n log-uniform in [n_min, n_max],
    nsteps uniform in [steps[0], steps[1]], the state (rho, T) of SERVING."""
    u = uniform(seed, 3 * count).reshape(count, 3)
    t = np.cumsum(-np.log(u[:, 0]) / rate)
    lo, hi = np.log(n_min), np.log(n_max)
    out = []
    for k in range(count):
        n = min(max(int(np.floor(np.exp(lo + (hi - lo) * u[k, 1]))), n_min), n_max)
        ns = int(steps[0] + np.floor((steps[1] - steps[0] + 1) * (1.0 - u[k, 2])))
        ns = min(max(ns, steps[0]), steps[1])
        out.append((float(t[k]), n, SERVING["rho"], SERVING["T"], seed * 1000003 + k, ns))
    return out

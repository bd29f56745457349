"""Seeded synthetic particle sets for the Laplace N-body workloads.

This module holds input generation only: no tree, expansion or kernel arithmetic.
Both the FP64 oracle (through the tests) and the CUDA path (through the tests and
bench.py) are fed from here, so the two sides see byte-identical particles.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15), turned into a double in [0, 1) from
its top 53 bits.  Positions and charges are rounded to float32 before either
side sees them.

Distributions (the paper uses "the same model problem" as the GPU Gems 3 all-pairs
chapter and prints no distribution, Section "Improvements of Performance"):
  * uniform cube: x ~ U[0,1)^3, q ~ U[0,1)/N;
  * Plummer sphere: scale radius a = 1 truncated at r = 20, equal masses 1/N.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """n particles uniform in the unit cube, charges uniform in [0, 1)/n.

    Returns float32 (n, 4): x, y, z, q.
    """
    u = uniform01(seed, 4 * n).reshape(n, 4) if n > 0 else np.zeros((0, 4))
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = u[:, :3]
    out[:, 3] = u[:, 3] / max(n, 1)
    return out


PLUMMER_RMAX = 20.0


def plummer(n: int, seed: int, a: float = 1.0, rmax: float = PLUMMER_RMAX) -> np.ndarray:
    """n equal-mass (1/n) particles from a Plummer sphere truncated at rmax.

    Cumulative mass fraction M(r) = r^3 / (a^2 + r^2)^(3/2); a uniform draw
    X in (0, M(rmax)] is inverted to r = a (X^(-2/3) - 1)^(-1/2); the direction
    is uniform on the sphere (cos(theta) ~ U(-1, 1), phi ~ U(0, 2 pi)).
    Returns float32 (n, 4).
    """
    if n == 0:
        return np.zeros((0, 4), dtype=np.float32)
    u = uniform01(seed, 3 * n).reshape(n, 3)
    mmax = rmax**3 / (a * a + rmax * rmax) ** 1.5
    x = (1.0 - u[:, 0]) * mmax  # in (0, mmax]
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    ct = 2.0 * u[:, 1] - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * np.pi * u[:, 2]
    out = np.empty((n, 4), dtype=np.float32)
    out[:, 0] = r * st * np.cos(ph)
    out[:, 1] = r * st * np.sin(ph)
    out[:, 2] = r * ct
    out[:, 3] = 1.0 / n
    return out


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices in [0, n), drawn without replacement (seeded), ascending."""
    k = min(k, n)
    keys = splitmix64(seed ^ 0x5A5A5A5A, n)
    return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int64)


# Seeds: one per named workload so that every consumer draws the same particles.
SEED_BASE = 20260000


def workload(name: str) -> dict:
    """Named workloads (sizes of the paper-derived configurations)."""
    table = {
        # small uniform case checked against the O(N^2) direct sum
        "uniform_4k_p4": dict(n=4096, dist="uniform", p=4, leaf_size=64, seed=SEED_BASE + 0),
        # single large uniform instance, FP32 path
        "uniform_1m_p10": dict(n=1 << 20, dist="uniform", p=10, leaf_size=64, seed=SEED_BASE + 1),
        # same distribution, p and mean leaf occupancy (32) at depth 4: the small profiling case
        "uniform_128k_p10": dict(n=1 << 17, dist="uniform", p=10, leaf_size=64, seed=SEED_BASE + 1),
        # clustered single instance (adaptive octree)
        "plummer_16m_p8": dict(n=1 << 24, dist="plummer", p=8, leaf_size=64, seed=SEED_BASE + 2),
        # same distribution, p and leaf size at 2^21 particles: the small profiling case
        "plummer_2m_p8": dict(n=1 << 21, dist="plummer", p=8, leaf_size=64, seed=SEED_BASE + 2),
    }
    w = dict(table[name], name=name)
    w["tree"] = "adaptive" if w["dist"] == "plummer" else "uniform"
    return w


def make_particles(n: int, dist: str, seed: int) -> np.ndarray:
    if dist == "uniform":
        return uniform_cube(n, seed)
    if dist == "plummer":
        return plummer(n, seed)
    raise ValueError(f"unknown distribution {dist!r}")


def batch_instances(count: int = 512, seed: int = SEED_BASE + 3, n_lo: float = 1e3, n_hi: float = 2e5,
                    orders=(4, 8)) -> list[dict]:
    """Uneven independent instances: N_i = round(exp(U(ln n_lo, ln n_hi))), even i uniform cube,
    odd i Plummer, p_i drawn uniformly from `orders`; instance i uses seed `seed` * 1000 + i."""
    u = uniform01(seed, 2 * count).reshape(count, 2)
    out = []
    for i in range(count):
        n = int(round(float(np.exp(np.log(n_lo) + u[i, 0] * (np.log(n_hi) - np.log(n_lo))))))
        p = int(orders[min(int(u[i, 1] * len(orders)), len(orders) - 1)])
        out.append(dict(n=n, dist="uniform" if i % 2 == 0 else "plummer", p=p, seed=seed * 1000 + i))
    return out


def served_requests(rate: float = 200.0, duration: float = 60.0, seed: int = SEED_BASE + 4, n_lo: float = 1e3,
                    n_hi: float = 1e6, orders=(4, 6, 10)) -> list[dict]:
    """A request stream: Poisson arrivals at `rate` per second over `duration` seconds
    (exponential gaps), N log-uniform in [n_lo, n_hi], uniform cube or Plummer with equal
    probability, p drawn uniformly from `orders`.  Request i is an independent particle set:
    make_particles(n, dist, seed * 1000 + i)."""
    est = int(rate * duration * 1.5 + 64)
    u = uniform01(seed, 4 * est).reshape(est, 4)
    t, out = 0.0, []
    for i in range(est):
        t += -np.log(1.0 - u[i, 0]) / rate
        if t >= duration:
            break
        n = int(round(float(np.exp(np.log(n_lo) + u[i, 1] * (np.log(n_hi) - np.log(n_lo))))))
        out.append(dict(t=t, n=n, dist="uniform" if u[i, 2] < 0.5 else "plummer",
                        p=int(orders[min(int(u[i, 3] * len(orders)), len(orders) - 1)]), seed=seed * 1000 + i))
    return out

"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only draws numbers. Both the
CUDA path and the oracle receive the same draws from here. The generator is
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), mapped to doubles in [0, 1) with the top 53 bits.

Workloads (all synthetic; the paper uses no dataset):
  * bubble grids: the equal-mass scalar bubble on a rectangle of complex x;
  * dressed draws: (a, b, c) with a ~ U[0.5, 2], b ~ U[0, 1], c ~ U[1, 4];
  * sampled subsets of a grid: uniformly drawn flat indices;
  * the serving mix: square grids with side in {32, 64, 128, 256, 512},
    bubble or dressed, D in {3, 4}, node pairs from (256, 64) to (2048, 256),
    FP64 or mixed, exponential inter-arrival times.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)

    def randint(self, n: int) -> int:
        """uniform integer in [0, n)"""
        return int(self.uniform() * n)


def dressed_draws(seed: int, count: int):
    """(a, b, c) triples for the dressed propagator (s + a)/(s^2 + b s + c)."""
    g = SplitMix64(seed)
    out = []
    for _ in range(count):
        a = 0.5 + 1.5 * g.uniform()
        b = 1.0 * g.uniform()
        c = 1.0 + 3.0 * g.uniform()
        out.append((a, b, c))
    return out


def sample_indices(seed: int, population: int, count: int) -> np.ndarray:
    """``count`` distinct flat indices drawn uniformly from range(population),
    returned sorted."""
    g = SplitMix64(seed)
    count = min(count, population)
    chosen = set()
    while len(chosen) < count:
        chosen.add(g.randint(population))
    return np.array(sorted(chosen), dtype=np.int64)


def grid_rect(kind: str):
    """Rectangles of the standard workloads: (re0, re1, im0, im1)."""
    return {
        "small": (-8.0, 4.0, -4.0, 4.0),        # 64 x 64 bubble, dressed 512 x 512, serving
        "production": (-10.0, 5.0, -5.0, 5.0),  # 1024 x 1024 bubble
        "paper": (-5.0, 5.0, -5.0, 5.0),        # the paper's worked example, 128 x 128
    }[kind]


# (n_radial, n_angular) orders of the serving requests
SERVING_NODES = [(256, 64), (512, 128), (1024, 128), (2048, 256)]


def serving_mix(seed: int, count: int, rate_hz: float = 200.0):
    """Request descriptors of the serving workload, in arrival order."""
    g = SplitMix64(seed)
    sides = [32, 64, 128, 256, 512]
    nodes = SERVING_NODES
    masses = [0.5, 1.0, 2.0]
    t = 0.0
    out = []
    for i in range(count):
        t += -np.log(1.0 - g.uniform()) / rate_hz
        side = sides[g.randint(len(sides))]
        if g.uniform() < 0.5:
            m = masses[g.randint(len(masses))]
            prop = {"kind": "scalar", "m2": m * m}
        else:
            a = 0.5 + 1.5 * g.uniform()
            b = 1.0 * g.uniform()
            c = 1.0 + 3.0 * g.uniform()
            prop = {"kind": "dressed", "a": a, "b": b, "c": c}
        dim = 3 if g.uniform() < 0.5 else 4
        nr, na = nodes[g.randint(len(nodes))]
        precision = "fp64" if g.uniform() < 0.5 else "mixed"
        out.append({"id": i, "t_arrival": t, "side": side, "prop": prop, "dim": dim,
                    "n_radial": nr, "n_angular": na, "precision": precision,
                    "mu2": 1.0, "rect": grid_rect("small")})
    return out

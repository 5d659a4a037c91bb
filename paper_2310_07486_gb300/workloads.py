"""Seeded synthetic workloads shared by the tests, the smoke check and the bench.

This module holds shapes, seeds and k ladders only -- none of the method's
arithmetic.  The ladders are uniform in [k_min, k_max] as in the simulation
table of the paper's Methods ("uniformly distributed" k values); the disorder
(J = +-1) is drawn inside each implementation from the seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .qsg import HEATBATH, METROPOLIS, PBC, Shape


def uniform_ladder(k_min: float, k_max: float, n: int) -> np.ndarray:
    if n == 1:
        return np.array([k_min], dtype=np.float64)
    return np.array([k_min + j * (k_max - k_min) / (n - 1) for j in range(n)], dtype=np.float64)


@dataclass
class Workload:
    name: str
    shapes: list
    ladders: list
    seed: int = 1
    sweeps_per_swap: int = 10
    measure_every: int = 10
    total_sweeps: int = 0
    notes: str = ""

    @property
    def spin_updates_per_sweep(self) -> int:
        return sum(s.L * s.L * s.Ltau * s.n_samples * s.n_replicas * s.n_k for s in self.shapes)

    @property
    def words(self) -> int:
        return sum(s.slots * s.L * s.L * s.Ltau for s in self.shapes)


def smallest() -> Workload:
    """One sample, L=6, L_tau=32, k=0.29, 2 replicas, Metropolis, 2000 sweeps,
    correlators every 10 sweeps."""
    return Workload("L6_Lt32_single", [Shape(6, 32, 1, 2, 1, METROPOLIS, PBC)], [np.array([0.29])], seed=1,
                    sweeps_per_swap=10, measure_every=10, total_sweeps=2000)


def mid_scale() -> Workload:
    """64 samples, L=16, L_tau=512, 4 replicas, 24 k in [0.20, 0.40], Metropolis,
    swaps every 10 sweeps (10^5 sweeps in full)."""
    return Workload("L16_Lt512_pt24", [Shape(16, 512, 64, 4, 24, METROPOLIS, PBC)], [uniform_ladder(0.20, 0.40, 24)],
                    seed=2, sweeps_per_swap=10, measure_every=100, total_sweeps=100000)


def largest() -> Workload:
    """128 samples (2 words), L=24, L_tau=2048, 4 replicas, 32 k in [0.22, 0.36],
    heat bath; the elementary step of the paper's Methods is 30 sweeps plus one
    tempering attempt."""
    return Workload("L24_Lt2048_hb", [Shape(24, 2048, 128, 4, 32, HEATBATH, PBC)], [uniform_ladder(0.22, 0.36, 32)],
                    seed=3, sweeps_per_swap=30, measure_every=300)


def ragged() -> Workload:
    """640 samples in five groups (L, L_tau) = (8,128) (12,256) (16,512) (20,1024)
    (24,2048), 128 samples each, 4 replicas, ladders of 16/24/48/56/60 k over the
    ranges of the paper's simulation table (uneven ladders)."""
    rows = [(8, 128, 16, 0.265, 0.305), (12, 256, 24, 0.265, 0.305), (16, 512, 48, 0.265, 0.295986),
            (20, 1024, 56, 0.265, 0.295986), (24, 2048, 60, 0.265, 0.292)]
    shapes = [Shape(L, Lt, 128, 4, K, METROPOLIS, PBC) for (L, Lt, K, a, b) in rows]
    ladders = [uniform_ladder(a, b, K) for (L, Lt, K, a, b) in rows]
    return Workload("ragged_640", shapes, ladders, seed=4, sweeps_per_swap=30, measure_every=300)


ALL = {w().name: w for w in (smallest, mid_scale, largest, ragged)}


def bimodal_couplings(n: int, L: int, seed: int) -> np.ndarray:
    """n samples of J = +-1 with probability 1/2 on the 2 L^2 bonds (the
    paper's bimodal disorder), as host int8 [n][2][L][L] for
    qsg_set_couplings; drawn from numpy's seeded generator."""
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=(n, 2, L, L))).astype(np.int8)


@dataclass
class LadderStudy:
    """Sizes of the learned-ladder study (scaled down from 2000 training runs
    at L = 12..20 and 256 evaluation samples at L = 24, L_tau = 2048):
    training runs at three sizes, evaluation on fresh samples at a larger
    one, a judge capped at 2^max_bin sweeps, several seeds."""
    train_sizes: list = field(default_factory=lambda: [(6, 32), (8, 48), (10, 64)])
    n_train_per_size: int = 640
    eval_size: tuple = (12, 64)
    n_eval: int = 256
    k_min: float = 0.2
    k_max: float = 0.45
    n_k: int = 32
    replicas: int = 4
    sweeps_per_swap: int = 8
    max_bin: int = 14          # bins of sweeps (2^m, 2^(m+1)], m < max_bin
    seed: int = 2024
    seeds: tuple = (2024, 2025, 2026)


def ladder_study() -> LadderStudy:
    return LadderStudy()

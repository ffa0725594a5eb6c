"""Seeded synthetic inputs for the smoothed-cubic random-laser PT simulation.

This module holds input generators only (no part of the Monte Carlo arithmetic): the
quenched couplings, the temperature ladders and the workload definitions.  Both the
CUDA library and the FP64 CPU oracle consume what it produces.

The disorder follows the paper's generative model (arXiv 2511.13508, Sec. II.C): real
couplings J_q i.i.d. Gaussian with zero mean and sigma_J = 1/N (the "sigma_J ~ 1/N"
scaling for p = 4 on the mode-locked graph, read with unit prefactor).  J is produced
in the canonical quadruplet order (lexicographic (a, b, c)), whose length the caller
passes in.  There is no public dataset in the paper: these synthetic samples stand in
for its Table-1 disorder samples.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def geometric_ladder(t_min: float, t_max: float, n: int) -> np.ndarray:
    """T_t = T_min (T_max/T_min)^(t/(n-1)), ascending (index 0 = coldest)."""
    if n == 1:
        return np.array([float(t_min)])
    return t_min * (t_max / t_min) ** (np.arange(n) / (n - 1.0))


def couplings(N: int, n_quads: int, seed: int) -> np.ndarray:
    """J_q ~ N(0, sigma_J^2), sigma_J = 1/N, for the n_quads quadruplets of an N-mode comb."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return rng.standard_normal(int(n_quads)) / float(N)


def random_frequencies(N: int, seed: int) -> np.ndarray:
    """Quenched mode frequencies r_k ~ U[0,1], sorted ascending (Sec. II.C "Quenched random frequencies")."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return np.sort(rng.uniform(0.0, 1.0, size=int(N)))


def sparse_comb_graph(N: int, z: float, seed: int) -> np.ndarray:
    """A sparse mode-locked graph (the finite-connectivity networks of Sec. II.D and Sec. V): round(z N / 4)
    quadruplets of the comb (a<b<c<d with a+d = b+c, term order (a, b, c, d)) drawn uniformly without
    replacement, so every mode holds z of them on average.  A uniform (a, b, c) with d = b + c - a is kept
    when c < d < N, which makes every comb quadruplet equally likely."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    M = int(round(z * N / 4))
    seen, out = set(), []
    while len(out) < M:
        a, b, c = np.sort(rng.choice(N, 3, replace=False))
        d = b + c - a
        if c < d < N and (a, b, c) not in seen:
            seen.add((a, b, c))
            out.append((a, b, c, d))
    out.sort()
    return np.asarray(out, dtype=np.int32).reshape(-1, 4)


def ragged_sizes(n_samples: int, choices=(32, 48, 64, 96, 128), seed: int = 200) -> np.ndarray:
    """Per-sample mode counts drawn uniformly from `choices` (ragged batch workload)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return np.asarray(choices, dtype=np.int32)[rng.integers(0, len(choices), size=int(n_samples))]


@dataclass
class Workload:
    name: str
    Ns: list
    t_min: float
    t_max: float
    n_temps: int
    replicas: int
    seeds: list
    sweeps: int
    swap_every: int = 64
    measure_every: int = 16
    resync_every: int = 64
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def temps(self) -> np.ndarray:
        return geometric_ladder(self.t_min, self.t_max, self.n_temps)

    @property
    def samples(self) -> int:
        return len(self.Ns)

    @property
    def chains(self) -> int:
        return self.samples * self.replicas * self.n_temps


def workloads() -> dict:
    """The five synthetic workloads (comb omega_k = k, sigma_J = 1/N couplings)."""
    ragged = ragged_sizes(96)
    return {
        "n16_fp64": Workload("n16_fp64", [16] * 4, 0.4, 1.6, 8, 2, list(range(1, 5)), 2048,
                             notes="N=16, 8 T in [0.4,1.6], R=2, S=4, FP64"),
        "n64_batched": Workload("n64_batched", [64] * 64, 0.3, 1.6, 32, 2, list(range(101, 165)), 1 << 16,
                                notes="N=64, 32 T in [0.3,1.6], R=2, S=64"),
        "ragged": Workload("ragged", [int(n) for n in ragged], 0.3, 1.6, 24, 2, list(range(201, 297)), 1 << 12,
                           notes="S=96, N ~ U{32,48,64,96,128}, 24 T in [0.3,1.6], R=2"),
        "n256_large": Workload("n256_large", [256] * 16, 0.25, 1.6, 48, 2, list(range(301, 317)), 1 << 14,
                               notes="N=256, S=16, 48 T in [0.25,1.6], R=2, measure every 16"),
        "n64_learned": Workload("n64_learned", [64] * 16, 0.3, 1.6, 32, 2, list(range(401, 417)), 1 << 14,
                                swap_every=64, measure_every=16,
                                notes="N=64, 32 T in [0.3,1.6], S=16, learned global move every 8 sweeps",
                                extra={"global_every": 8, "n_cold": 8, "train_configs": 1 << 14}),
    }

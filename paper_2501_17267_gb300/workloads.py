"""Workload definitions and seeded synthetic inputs.

This module holds no arithmetic of the method.  It names the workloads (lattice
size, instance count, replicas, sweeps, beta range) and draws plain seeded random
arrays (spin configurations, coupling arrays) that the tests and the benchmark
hand to both the CUDA library and the CPU oracle.

The instances themselves are tile-planted lattices (arXiv:2501.17267, Sec. II):
both the library and the oracle generate them from (L, seed, class
probabilities); an instance seed is ``workload_index * 2**32 + instance_index``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

UNIFORM = (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)


@dataclass(frozen=True)
class SAWorkload:
    name: str
    index: int
    L: int
    instances: int
    replicas: int
    sweeps: int
    beta0: float
    beta1: float
    geometric: bool = False
    run_seed: int = 0
    class_prob: tuple = UNIFORM

    def instance_seed(self, k: int) -> int:
        return self.index * 2 ** 32 + k


@dataclass(frozen=True)
class PTWorkload:
    name: str
    index: int
    L: int
    instances: int
    temps: int
    sweeps: int
    beta_min: float
    beta_max: float
    run_seed: int = 0
    class_prob: tuple = UNIFORM

    def instance_seed(self, k: int) -> int:
        return self.index * 2 ** 32 + k


@dataclass(frozen=True)
class BatchedWorkload:
    name: str
    index: int
    instances: int
    L_choices: tuple
    replicas: int
    sweep_choices: tuple
    beta0: float
    beta1: float
    draw_seed: int = 12345
    class_prob: tuple = UNIFORM

    def instance_seed(self, k: int) -> int:
        return self.index * 2 ** 32 + k

    def draw(self):
        """Per-instance (L, sweeps), drawn uniformly from the choices with a fixed seed."""
        rng = np.random.default_rng(self.draw_seed)
        Ls = rng.choice(np.array(self.L_choices), size=self.instances)
        Ss = rng.choice(np.array(self.sweep_choices), size=self.instances)
        return [(int(a), int(b)) for a, b in zip(Ls, Ss)]


@dataclass(frozen=True)
class ServingWorkload:
    name: str
    index: int
    rate_per_s: float
    duration_s: float
    L_choices: tuple
    L_large: int
    large_fraction: float
    sa_replicas: int
    sa_sweeps_per_restart: int
    pt_temps: int
    pt_beta_min: float
    pt_beta_max: float
    sa_sweep_cap: int
    pt_sweep_cap: int
    eps_target: float
    sa_beta0: float = 0.1
    sa_beta1: float = 3.0
    sa_fraction: float = 0.5
    arrival_seed: int = 2024
    class_prob: tuple = UNIFORM

    def instance_seed(self, k: int) -> int:
        return self.index * 2 ** 32 + k

    def stream(self, seconds: float | None = None):
        """The arrival stream over [0, seconds): Poisson arrivals at rate_per_s, each with
        L uniform over L_choices (L_large with probability large_fraction), SA with
        probability sa_fraction else PT, instance seed index*2^32 + k and run seed k for
        the k-th arrival.  Deterministic in arrival_seed."""
        T = self.duration_s if seconds is None else seconds
        rng = np.random.default_rng(self.arrival_seed)
        out, t, k = [], 0.0, 0
        while True:
            t += float(rng.exponential(1.0 / self.rate_per_s))
            if t >= T:
                return out
            big = rng.random() < self.large_fraction
            L = self.L_large if big else int(rng.choice(np.array(self.L_choices)))
            kind = "SA" if rng.random() < self.sa_fraction else "PT"
            out.append({"t": t, "L": L, "kind": kind, "seed": self.instance_seed(k), "run_seed": k})
            k += 1


# L=4, one instance, 8 replicas, 1000 sweeps, beta linear 0.1 -> 3.0, run seed 0
SA_L4 = SAWorkload("sa_L4_R8_S1000", 0, 4, 1, 8, 1000, 0.1, 3.0)
# L=16, one instance, 1024 replicas, 1000 sweeps, beta linear 0.1 -> 3.0
SA_L16 = SAWorkload("sa_L16_R1024_S1000", 1, 16, 1, 1024, 1000, 0.1, 3.0)
# 16 instances at L=64, 32 temperatures geometric 0.2 -> 3.0, 10^4 sweeps
PT_L64 = PTWorkload("pt_L64_I16_K32_S10000", 2, 64, 16, 32, 10000, 0.2, 3.0)
# 512 instances, L uniform in {8,12,16,24,32,48}, 64 replicas, sweeps in {100,1000,10000}
BATCHED = BatchedWorkload("sa_batched_I512_R64", 3, 512, (8, 12, 16, 24, 32, 48), 64,
                          (100, 1000, 10000), 0.1, 3.0)
# Poisson 200 req/s for 60 s, L in {8..64 step 8} plus 1% at L=128, SA/PT 50/50, target
# eps <= 1%; SA: 32 replicas, restarts of 1000 sweeps (beta linear 0.1 -> 3.0); PT: 32
# temperatures geometric 0.2 -> 3.0; cap 1000 sweeps for both (one SA restart): at 2000
# the offered load is about twice what one GPU sweeps
SERVING = ServingWorkload("serve_poisson200", 4, 200.0, 60.0, tuple(range(8, 65, 8)), 128,
                          0.01, 32, 1000, 32, 0.2, 3.0, 1000, 1000, 0.01)

ALL = [SA_L4, SA_L16, PT_L64, BATCHED, SERVING]


def random_spins(seed: int, shape) -> np.ndarray:
    """Uniform +-1 int8 spins."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1).astype(np.int8)


def random_couplings(seed: int, L: int, jmax: int = 2, allow_zero: bool = True) -> np.ndarray:
    """Uniform integer couplings in [-jmax, jmax] (zero optional), shape (L^3, 3)."""
    rng = np.random.default_rng(seed)
    vals = [v for v in range(-jmax, jmax + 1) if allow_zero or v != 0]
    return rng.choice(np.array(vals, dtype=np.int8), size=(L ** 3, 3)).astype(np.int8)

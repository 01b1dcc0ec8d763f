"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds none of the method's arithmetic: it only draws problem
instances (marked bitstrings, iteration counts, phase vectors) from fixed
seeds.  Both the CPU oracle and the CUDA path receive exactly these values.

Marked strings use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): take the low n bits of each
draw and reject duplicates.  Bit l of a string is qubit / MPS site l
(LSB = site 0).

The paper's experiments use M = 1 marked item and k = round(pi/4 sqrt(N))
iterations (Sec. II, Eq. 8); the workloads below follow the configurations
this package is measured on (floor instead of round where stated, which
coincides with round at n = 12 and n = 29).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform_int(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] by rejection (no modulo bias)."""
        span = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            r = self.next()
            if r < limit:
                return lo + r % span


def marked_strings(n: int, M: int, seed: int) -> list[int]:
    """M distinct n-bit strings drawn uniformly from `seed`."""
    if not (1 <= n <= 64):
        raise ValueError("n must be in [1, 64]")
    if not (1 <= M < (1 << n)):
        raise ValueError("M must be in [1, 2^n)")
    g = SplitMix64(seed)
    mask = (1 << n) - 1 if n < 64 else MASK64
    out: list[int] = []
    seen: set[int] = set()
    while len(out) < M:
        w = g.next() & mask
        if w not in seen:
            seen.add(w)
            out.append(w)
    return out


def k_floor(n: int, M: int, cap: int | None = None) -> int:
    """k = floor(pi/4 * sqrt(2^n / M)), optionally capped."""
    k = int(math.floor(math.pi / 4.0 * math.sqrt((2.0 ** n) / M)))
    return min(k, cap) if cap is not None else k


@dataclass
class Instance:
    n: int
    marked: list[int]
    k: int
    chi_max: int
    tol: float = 0.0
    phi: np.ndarray | None = None   # per-iteration oracle phases (None = pi)
    psi: np.ndarray | None = None   # per-iteration diffusion phases (None = pi)
    tag: str = ""

    @property
    def M(self) -> int:
        return len(self.marked)


def plain_instance(n: int, M: int, seed: int, chi_max: int, k: int | None = None,
                   tol: float = 0.0, tag: str = "") -> Instance:
    return Instance(n=n, marked=marked_strings(n, M, seed),
                    k=k_floor(n, M) if k is None else k, chi_max=chi_max, tol=tol, tag=tag)


def config_small() -> Instance:
    """n=12, M=1 (seed 1), k=50, chi_max=4, no truncation."""
    return plain_instance(12, 1, seed=1, chi_max=4, k=50, tag="n12_M1_k50")


def config_n29() -> Instance:
    """n=29, M=1 (seed 3), k=18198, chi_max=4."""
    return plain_instance(29, 1, seed=3, chi_max=4, k=18198, tag="n29_M1_k18198")


def config_multi_marked(k: int = 1000) -> Instance:
    """n=40, M=32 distinct strings (seed 4), chi_max=128, tol=1e-12."""
    return plain_instance(40, 32, seed=4, chi_max=128, k=k, tol=1e-12, tag=f"n40_M32_k{k}")


def config_batched(count: int = 512, seed: int = 5, kcap: int = 4000,
                   n_range=(16, 36), m_range=(1, 16), chi_max: int = 32) -> list[Instance]:
    """`count` instances: n ~ U[16,36], M ~ U[1,16], k_i = min(floor(pi/4 sqrt(2^n/M)), 4000)."""
    g = SplitMix64(seed)
    out = []
    for i in range(count):
        n = g.uniform_int(*n_range)
        M = g.uniform_int(*m_range)
        sub_seed = g.next()
        marked = marked_strings(n, M, sub_seed)
        out.append(Instance(n=n, marked=marked, k=k_floor(n, M, kcap), chi_max=chi_max,
                            tag=f"b{i}"))
    return out


def phase_batch(K: int, B: int, seed: int = 6, mean: float = math.pi, std: float = 0.1):
    """B phase vectors (phi_k, psi_k), k = 1..K, drawn N(mean, std) in float32.

    Returns two float64 arrays of shape (B, K) holding the float32 values.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = rng.normal(mean, std, size=(B, K)).astype(np.float32).astype(np.float64)
    psi = rng.normal(mean, std, size=(B, K)).astype(np.float32).astype(np.float64)
    return phi, psi


def config_differentiable(B: int = 64) -> tuple[Instance, np.ndarray, np.ndarray]:
    """n=20, M=4 (seed 6), K=64 with B trainable phase vectors."""
    inst = plain_instance(20, 4, seed=6, chi_max=8, k=64, tag="n20_M4_K64")
    phi, psi = phase_batch(64, B, seed=6)
    return inst, phi, psi

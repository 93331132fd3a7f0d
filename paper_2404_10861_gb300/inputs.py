"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds none of the method's arithmetic: it only draws starting populations
(uint32 traits and 64-bit surfaces) and run configurations with numpy's own
generators, so that the CUDA path and the CPU oracle can be fed identical
data.  The paper's runs start from founders (every agent identical except
for a random tag); ``founders`` gives that state, ``random_population`` gives
arbitrary states for parity tests that must exercise every bit.
"""
from __future__ import annotations

import numpy as np


def founders(n_agents: int):
    """Founding population: trait 0 and an empty (all-zero) surface."""
    return (np.zeros(n_agents, dtype=np.uint32),
            np.zeros(n_agents, dtype=np.uint64))


def random_population(n_agents: int, seed: int, trait_max: int = 2**32 - 1):
    """Uniform random traits in [0, trait_max] and uniform random surfaces."""
    rng = np.random.default_rng(seed)
    trait = rng.integers(0, trait_max, size=n_agents, dtype=np.uint64,
                         endpoint=True).astype(np.uint32)
    surf = rng.integers(0, 2**64 - 1, size=n_agents, dtype=np.uint64,
                        endpoint=True)
    return trait, surf


def small_trait_population(n_agents: int, seed: int, levels: int = 4):
    """Random surfaces with traits in [0, levels): many fitness ties."""
    rng = np.random.default_rng(seed)
    trait = rng.integers(0, levels, size=n_agents).astype(np.uint32)
    surf = rng.integers(0, 2**64 - 1, size=n_agents, dtype=np.uint64,
                        endpoint=True)
    return trait, surf


def permutation_traits(islands: int, n: int, seed: int):
    """Per island, traits a random permutation of 0..n-1 (all distinct)."""
    rng = np.random.default_rng(seed)
    trait = np.concatenate([rng.permutation(n) for _ in range(islands)]).astype(np.uint32)
    surf = rng.integers(0, 2**64 - 1, size=islands * n, dtype=np.uint64,
                        endpoint=True)
    return trait, surf


def to_words(trait: np.ndarray, surf: np.ndarray, T: int) -> np.ndarray:
    """Pack (trait, surface) into the 4-word record [trait, surf_lo, surf_hi, T]."""
    w = np.empty((len(trait), 4), dtype=np.uint32)
    w[:, 0] = trait
    w[:, 1] = (surf & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    w[:, 2] = (surf >> np.uint64(32)).astype(np.uint32)
    w[:, 3] = np.uint32(T & 0xFFFFFFFF)
    return w


def from_words(words: np.ndarray):
    """Unpack 4-word records into (trait, surface, T)."""
    words = np.asarray(words, dtype=np.uint32).reshape(-1, 4)
    surf = words[:, 1].astype(np.uint64) | (words[:, 2].astype(np.uint64) << np.uint64(32))
    return words[:, 0].copy(), surf, words[:, 3].copy()


# Workloads shaped like the paper's runs (32 agents per island; up to ~16.8M
# agents).  Keys follow the C-ABI configuration fields.
TINY = dict(rows=4, cols=4, n=32, tournament=2, policy="steady", bits=1,
            p_ben=0.0, p_del=0.0, seed=1, generations=2000)
MID = dict(rows=64, cols=64, n=32, tournament=2, bits=2, p_ben=1e-3, p_del=0.0,
           generations=100_000)
WAFER = dict(rows=512, cols=1024, n=32, tournament=2, policy="tilted", bits=1,
             p_ben=1e-3, p_del=0.0, seed=1, generations=1_000_000)

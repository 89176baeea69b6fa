"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle side.

This module holds no arithmetic of the method: only the counter-based
generator (SplitMix64, Steele, Lea & Flood 2014, in its published form) and
helpers that turn it into sequence-id samples, shard choices and initial
weights.  Both the CUDA side and the oracle side receive these values as
inputs; neither derives them itself.
"""
from __future__ import annotations

import numpy as np

SEED = 200805612
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output for counter value(s) x (vectorised, uint64 wrap-around)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sample_ids(N: int, count: int, seed: int = SEED) -> np.ndarray:
    """`count` sequence ids drawn uniformly from [0, 2^N) (with replacement)."""
    c = np.arange(count, dtype=np.uint64) + np.uint64(seed) * np.uint64(0x1000003)
    r = splitmix64(c)
    if N >= 64:
        return r
    return r & np.uint64((1 << N) - 1)


def training_mask(ids: np.ndarray, seed: int = SEED, modulus: int = 10) -> np.ndarray:
    """True for ids in the seeded 1-in-`modulus` training sample: splitmix64(g ^ seed) mod m == 0."""
    ids = np.asarray(ids, dtype=np.uint64)
    return (splitmix64(ids ^ np.uint64(seed)) % np.uint64(modulus)) == 0


def shard_index(j: int, nshards: int = 16, seed: int = SEED) -> int:
    """Shard k_j = splitmix64(seed + j) mod nshards."""
    return int(splitmix64(np.uint64(seed + j)) % np.uint64(nshards))


def init_weights(shape, fan_in: int, seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) float64 weights from SplitMix64."""
    n = int(np.prod(shape))
    r = splitmix64(np.arange(n, dtype=np.uint64) + np.uint64(seed) * np.uint64(0x100000001B3))
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    lim = 1.0 / np.sqrt(fan_in)
    return ((2.0 * u - 1.0) * lim).reshape(shape)

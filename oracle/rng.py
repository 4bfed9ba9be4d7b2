"""SplitMix64 counter-based generator, from its published definition
(G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state advances by the golden gamma
0x9E3779B97F4A7C15 and each output is the state passed through the
two-multiply xor-shift finaliser.

r(seed, stream, i) is output number i+1 of the sequence whose initial state is
mix64(seed * gamma + stream).  The oracle draws the AMG aggregation priorities
(stream 10) and the power-iteration start vector (stream 11) from it.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_PRIORITY = 10
STREAM_POWER = 11


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def rand_u64(seed: int, stream: int, idx) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = mix64(np.uint64(seed) * GAMMA + np.uint64(stream))
        return mix64(key + (idx + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """U in [0, 1): the top 53 bits scaled by 2^-53."""
    r = rand_u64(seed, stream, idx)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def level_index(level: int, i) -> np.ndarray:
    """Counter for entity i of AMG level `level`: level * 2^32 + i."""
    return (np.uint64(level) << np.uint64(32)) + np.asarray(i, dtype=np.uint64)

"""SplitMix64 used as a counter-based generator (Steele, Lea and Flood, OOPSLA 2014).

Value number ``i`` of stream ``seed`` is the (i+1)-th output of a SplitMix64 generator whose
state starts at ``seed``: state_i = seed + (i + 1) * GOLDEN (mod 2^64), then the published
finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31). A double in [-1, 1)
takes the top 53 bits.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, idx):
    """Vectorised SplitMix64 output for counters ``idx`` (uint64 arithmetic mod 2^64)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, idx):
    """Doubles in [-1, 1): (top 53 bits) * 2^-53 * 2 - 1."""
    z = splitmix64(seed, idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0

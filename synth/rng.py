"""Counter-mode SplitMix64 streams (vectorised, numpy uint64 wrap-around)."""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counters):
    """Return value ``counters[i]`` of the SplitMix64 stream started at ``seed``.

    The published generator advances its state by the golden-ratio increment
    and then mixes; value i (0-based) therefore mixes seed + (i+1)*golden.
    """
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, counters):
    """Uniform doubles in [0, 1) from the top 53 bits of each stream value."""
    z = splitmix64(seed, counters)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed, n, offset=0):
    """n standard normal doubles by the Box-Muller transform.

    Pair k uses stream values offset+2k (radius) and offset+2k+1 (angle).
    """
    m = (n + 1) // 2
    k = np.arange(m, dtype=np.uint64) * np.uint64(2) + np.uint64(offset)
    u1 = 1.0 - uniform01(seed, k)          # (0, 1]
    u2 = uniform01(seed, k + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m, dtype=np.float64)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]

"""Counter-based SplitMix64 generator (Steele, Lea & Flood 2014, "Fast splittable
pseudorandom number generators", OOPSLA).

Output i of the stream with key `seed` is mix(seed + (i + 1) * GAMMA), where mix is
the SplitMix64 finaliser.  Being counter-based, any slice of the stream can be
generated without the preceding outputs, so the same draw is reproducible from
any language that implements the published definition.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, n, offset=0):
    """Return outputs offset .. offset+n-1 of the SplitMix64 stream keyed by `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        return _mix(state)


def uniform(seed, n, offset=0):
    """Uniform doubles in [0, 1) with 53 random bits each."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def substream(seed, purpose):
    """Key of an independent stream for one purpose (mesh jitter, patch position, ...)."""
    with np.errstate(over="ignore"):
        k = _mix(np.array([np.uint64(seed) * np.uint64(1000003) + np.uint64(purpose)],
                          dtype=np.uint64))
    return int(k[0])


def normal(seed, n, offset=0):
    """Standard normal deviates by the Box-Muller transform of two uniform streams."""
    u1 = uniform(substream(seed, 1), n, offset)
    u2 = uniform(substream(seed, 2), n, offset)
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

"""splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and the derived uniform / normal draws.

* ``next()`` advances the state by the golden-ratio increment
  0x9E3779B97F4A7C15 and returns the finalised 64-bit word.
* uniform  u = (z >> 11) * 2^-53, in [0, 1).
* normal   Box-Muller: sqrt(-2 ln(1-u1)) * cos(2 pi u2), one normal per pair.

The vectorised ``*_stream`` helpers produce exactly the words a scalar
generator with the same seed would produce, because the k-th output only
depends on seed + (k+1)*increment (the generator is counter based).
"""

import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB


def _finalise(z):
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Scalar splitmix64 generator."""

    def __init__(self, seed):
        self.state = int(seed) & MASK64

    def next_u64(self):
        self.state = (self.state + GOLDEN) & MASK64
        return _finalise(self.state)

    def uniform(self, lo=0.0, hi=1.0):
        u = (self.next_u64() >> 11) * 2.0 ** -53
        return lo + (hi - lo) * u

    def normal(self):
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)

    def randint(self, lo, hi):
        """Uniform integer in [lo, hi] (inclusive) by floor(u * count)."""
        count = hi - lo + 1
        return lo + min(int(self.uniform() * count), count - 1)

    def sign(self):
        return -1.0 if self.uniform() < 0.5 else 1.0


def splitmix64_stream(seed, count):
    """The first ``count`` outputs of SplitMix64(seed), as a uint64 array."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & MASK64) + k * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_stream(seed, count):
    z = splitmix64_stream(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal_stream(seed, count):
    """``count`` standard normals; each uses two consecutive uniforms."""
    u = uniform_stream(seed, 2 * count)
    u1 = u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

"""Counter-based SplitMix64 stream, identical on every platform.

Output i of stream (seed, stream_id) is the SplitMix64 finaliser applied to
``base + (i + 1) * 0x9E3779B97F4A7C15`` where ``base`` mixes the seed and the
stream id (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Everything is uint64 arithmetic modulo 2**64, so the
integers are bit-identical across numpy versions and CPU architectures.  Floats
are derived from the top 53 bits; Gaussian draws use Box-Muller, whose last bits
may differ across libm implementations.

This module holds no solver arithmetic: it only draws random numbers.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A named SplitMix64 stream; ``take(n)`` returns the next n raw uint64."""

    def __init__(self, seed: int, stream_id: int):
        with np.errstate(over="ignore"):
            base = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN
                        + np.uint64(stream_id & 0xFFFFFFFFFFFFFFFF))
        self._base = np.uint64(base)
        self._pos = 0

    def take(self, n: int) -> np.ndarray:
        i = np.arange(self._pos + 1, self._pos + 1 + n, dtype=np.uint64)
        self._pos += n
        with np.errstate(over="ignore"):
            return _mix(self._base + i * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.take(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, n: int, hi: int) -> np.ndarray:
        """n draws in [0, hi) by the multiply-shift map of the top 32 bits."""
        top = (self.take(n) >> np.uint64(32)).astype(np.uint64)
        return ((top * np.uint64(hi)) >> np.uint64(32)).astype(np.int64)

    def permutation(self, n: int) -> np.ndarray:
        """A permutation of range(n): sort by random keys (ties broken by index)."""
        keys = self.take(n)
        return np.lexsort((np.arange(n), keys))

"""SplitMix64 for input generation (Steele, Lea and Flood, OOPSLA 2014).

Value number ``i`` (0-based) of stream ``seed`` is the SplitMix64 output mix
applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64).  Everything is
uint64 numpy arithmetic, which wraps modulo 2^64 without warnings for arrays.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Values start .. start+count-1 of the SplitMix64 stream ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + idx * _GAMMA
        return _mix(z)


class SplitMixStream:
    """Sequential reader over one SplitMix64 stream, refilled in blocks."""

    def __init__(self, seed: int, block: int = 1 << 16):
        self.seed = seed & _MASK64
        self.block = block
        self.pos = 0
        self._buf: list[int] = []
        self._i = 0

    def next_u64(self) -> int:
        if self._i >= len(self._buf):
            self._buf = splitmix64(self.seed, self.pos, self.block).tolist()
            self.pos += self.block
            self._i = 0
        v = self._buf[self._i]
        self._i += 1
        return v

    def below(self, bound: int) -> int:
        """Integer in [0, bound) by a 64x32 multiply-high of the top 32 bits."""
        return ((self.next_u64() >> 32) * bound) >> 32

    def unit(self) -> float:
        """Float in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

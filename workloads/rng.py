"""Seeded counter-free random stream for the synthetic inputs.

SplitMix64 (S. Vigna, "Further scramblings of Marsaglia's xorshift generators",
and the public-domain reference description of splitmix64): a 64-bit Weyl
sequence with increment 0x9E3779B97F4A7C15 followed by two xor-shift-multiply
mixing rounds. Written here from that published definition. Doubles take the
top 53 bits, so every draw is an exact multiple of 2**-53 in [0, 1).

This module holds no arithmetic of the lattice Boltzmann method; it only
produces the random numbers the droplet placement consumes.
"""

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_MUL1 = 0xBF58476D1CE4E5B9
_MUL2 = 0x94D049BB133111EB


class SplitMix64:
    """Deterministic 64-bit stream; ``state`` advances by the golden-ratio Weyl step."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _MUL1) & _MASK
        z = ((z ^ (z >> 27)) * _MUL2) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """A double in [0, 1) from the 53 high bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

"""SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used as a counter-based hash.

Test infrastructure only (see the package docstring).  The CUDA library holds
its own implementation of the same published definition; this module is not
shared with it.

The random initial pivots of TT-cross (Section IV.B: start from random column
sets J) are drawn from ``splitmix64(key)`` with a key that packs the job seed,
the max-call term, the bond k, the attempt number t, the pivot slot b and the
axis j into disjoint bit fields.
"""
MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state x (add the golden gamma, then mix)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def pivot_key(seed: int, term: int, k: int, t: int, b: int, j: int) -> int:
    """Bit fields: term<<52 | k<<40 | t<<24 | b<<12 | j, xor-ed into the seed."""
    assert 0 <= term < 4096 and 0 <= k < 4096 and 0 <= t < 65536
    assert 0 <= b < 4096 and 0 <= j < 4096
    return (seed ^ (term << 52) ^ (k << 40) ^ (t << 24) ^ (b << 12) ^ j) & MASK64

"""SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), counter form.

Output i for a seed s: z = s + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64), then
the published finaliser z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
z *= 0x94D049BB133111EB; z ^= z >> 31.  A double in [0, 1) is (z >> 11) * 2^-53.

Start vectors are uniform(-1, 1) with entry (row i, column c) of an n x b
block drawn at counter i * b + c (the reading of "choose a starting vector",
Algorithm 2 and Algorithm 3).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_block(seed: int, n: int, b: int) -> np.ndarray:
    """n x b block of uniform(-1, 1) doubles from SplitMix64."""
    z = splitmix64(seed, np.arange(n * b, dtype=np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(n, b)

"""Counter-based random numbers shared by every input recipe.

splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser constants are the published ones):
draw i of a stream is mix(key + (i + 1) * GOLDEN) with
key = seed XOR (stream * GOLDEN).  Uniform doubles are (z >> 11) * 2^-53,
which is exact, so any implementation of this definition reproduces the
same bits.  Normals use Box-Muller on consecutive pairs of uniforms,
u1 = 1 - U[2m] in (0, 1], u2 = U[2m + 1], giving r cos(2 pi u2) then
r sin(2 pi u2).

Streams: 1 mesh jitter, 2 right-hand sides, 3 initial candidates,
5 serving arrivals.  (Stream 4 + 16 k is the power-iteration start vector
of level k; the solver draws it itself from this same definition.)

This module holds no arithmetic of the multigrid method.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * GOLDEN)


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit outputs offset .. offset + n - 1 of (seed, stream)."""
    key = stream_key(seed, stream)
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1), exact multiples of 2^-53."""
    z = splitmix64(seed, stream, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller over pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]

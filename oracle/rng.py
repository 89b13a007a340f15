"""Counter-based generator for initial LOBPCG blocks (oracle side; written independently of the CUDA side).

Definition (shared as a specification, not as code):
* mix64(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
  (the splitmix64 output function of Steele, Lea and Flood, OOPSLA 2014), all arithmetic mod 2^64.
* key(seed, stream) = mix64(seed + G * (stream + 1)), G = 0x9E3779B97F4A7C15.
* draw(seed, stream, i) = mix64(key + G * (i + 1)).
* uniform(x) = ((x >> 11) + 0.5) * 2^-53, in (0, 1).
* Element e of a stream is the complex normal from Box-Muller on u1 = uniform(draw(2e)), u2 = uniform(draw(2e+1)):
  sqrt(-2 ln u1) * (cos(2 pi u2) + i sin(2 pi u2)).
* Column j of the initial block of k-point b uses stream = b * 4096 + j.
"""
from __future__ import annotations

import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def draws(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        key = mix64(np.uint64(seed) + G * np.uint64(stream + 1))
        return mix64(key + G * (np.asarray(idx, dtype=np.uint64) + np.uint64(1)))


def uniform(x: np.ndarray) -> np.ndarray:
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def complex_normal(seed: int, stream: int, count: int) -> np.ndarray:
    e = np.arange(count, dtype=np.uint64)
    u1 = uniform(draws(seed, stream, 2 * e))
    u2 = uniform(draws(seed, stream, 2 * e + 1))
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)


def initial_block(seed: int, kidx: int, length: int, m: int) -> np.ndarray:
    """Initial block of shape (length, m) for k-point ``kidx``."""
    return np.stack([complex_normal(seed, kidx * 4096 + j, length) for j in range(m)], axis=1)

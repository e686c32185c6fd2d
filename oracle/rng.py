"""Counter-based bath vectors |v_l> (Sec. 3.1, eq. trace_est; HA[v v^T] = I/d_b).

Test infrastructure only (see ``oracle/__init__``). The CUDA library implements the
same generator independently from the same published definition.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014). Its n-th output for seed s is mix(s + n * GAMMA) with
GAMMA = 0x9E3779B97F4A7C15 and mix the 64-bit finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
Element b of vector l uses counter n = ((l << 40) | b) + 1 (Rademacher) or the two
counters ((l << 40) | 2b) + 1 and ((l << 40) | (2b+1)) + 1 (Gaussian). Values:

* "rademacher": +1/sqrt(d_b) if the top bit of the draw is 0, else -1/sqrt(d_b)
  (unit norm exactly);
* "gauss": Box-Muller cos(2 pi u2) sqrt(-2 ln u1) with u = (draw >> 11 + 0.5) 2^-53,
  then divided by the vector's Euclidean norm (uniform on the sphere);
* "basis": v_l = e_l (needs n_v = d_b; the exhaustive sum is the exact partial trace).
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, counter: int) -> int:
    z = (seed + counter * GAMMA) & MASK
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & MASK
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & MASK
    z ^= z >> 31
    return z


def splitmix64_array(seed: int, counters: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 on uint64 counters (wrapping arithmetic)."""
    c = counters.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + c * np.uint64(GAMMA)
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def bath_vector(d_b: int, l: int, seed: int, dist: str) -> np.ndarray:
    """The l-th bath vector, length d_b, float64."""
    if dist == "basis":
        v = np.zeros(d_b)
        v[l] = 1.0
        return v
    b = np.arange(d_b, dtype=np.uint64)
    base = np.uint64(l) << np.uint64(40)
    if dist == "rademacher":
        z = splitmix64_array(seed, (base | b) + np.uint64(1))
        sign = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
        return sign / np.sqrt(float(d_b))
    if dist == "gauss":
        z1 = splitmix64_array(seed, (base | (b * np.uint64(2))) + np.uint64(1))
        z2 = splitmix64_array(seed, (base | (b * np.uint64(2) + np.uint64(1))) + np.uint64(1))
        u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        u2 = ((z2 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        return g / np.sqrt(np.sum(g * g))
    raise ValueError(f"unknown distribution {dist!r}")


def starting_block(d_s: int, v: np.ndarray) -> np.ndarray:
    """V = I_s (x) |v> as a (d_s*d_b, d_s) matrix: V[i*d_b + b, i] = v[b] (Sec. 3.1)."""
    d_b = v.shape[0]
    out = np.zeros((d_s * d_b, d_s))
    for i in range(d_s):
        out[i * d_b:(i + 1) * d_b, i] = v
    return out

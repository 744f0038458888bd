"""Seeded synthetic inputs: Ising instances (J, h) and packed initial spin states.

This module holds no arithmetic of the search method. It only turns counter-based
random draws into coupling values and spin bits, so that the CPU oracle and the
CUDA path are fed the very same bytes.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). Value number ``c`` (0-based) of the stream whose
state starts at ``key`` is ``mix(key + (c + 1) * 0x9E3779B97F4A7C15)`` with the
published 64-bit finaliser ``mix``. Every draw is addressed by (key, counter), so any
subset can be regenerated independently.

Gaussian draws use the Box-Muller transform. Its logarithm and cosine are evaluated
here with plain IEEE-754 additions, multiplications and divisions (series with a fixed
evaluation order), never with the platform's libm, so the same seed yields the same bits
on x86-64 and on AArch64.

Coupling ensembles (the paper's H0 of Eq. (1); i<j couplings, zero diagonal):
  * ``gaussian``  J_ij, h_i ~ N(0, 1)
  * ``uniform``   J_ij, h_i ~ U[-1/2, 1/2], the paper's ensemble (Sec. IV)
  * ``pm1``       J_ij uniform in {-1, +1}, h_i uniform in {-1, 0, +1}
Real-valued draws are rounded to the nearest multiple of 2**-GRID_BITS (2**-32 ~ 2.3e-10).
With |J| < 8 and N <= 2048 every partial sum of an energy is then an exact FP64 number,
so energies do not depend on summation order.

State bits follow the paper's encoding (Eq. (4)): bit i of psi is sigma_i, sigma_i = 1
meaning s_i = -1. A state of N spins is W = ceil(N / 64) little-endian uint64 words;
bit i lives in word i // 64 at position i % 64. Unused high bits are zero.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
GRID_BITS = 32

# stream tags (second-level keys)
TAG_J = 1
TAG_H = 2
TAG_STATE = 3


def words(n: int) -> int:
    """Number of uint64 words holding an n-spin state."""
    return (n + 63) // 64


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(key, counter) -> np.ndarray:
    """Value number ``counter`` of the SplitMix64 stream whose state starts at ``key``."""
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        return _mix(np.uint64(key) + (c + np.uint64(1)) * GOLDEN)


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Derive a stream key from a seed and a tuple of integer tags."""
    k = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF), 0)
    for t in tags:
        k = splitmix64(k ^ np.uint64(t & 0xFFFFFFFFFFFFFFFF), 0)
    return np.uint64(k)


def uniform01(key, counter) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2**-53."""
    x = splitmix64(key, counter)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


_LN2 = 0.6931471805599453
_SQRT_HALF = 0.7071067811865476
_HALF_PI = 1.5707963267948966


def _log_unit(x: np.ndarray) -> np.ndarray:
    """Natural log for x in (0, 1] from IEEE + - * / only (atanh series)."""
    m, e = np.frexp(x)                    # exact: x = m * 2**e, m in [0.5, 1)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)             # |t| <= 0.1716
    t2 = t * t
    s = np.full_like(t, 1.0 / 25.0)
    for k in range(23, 0, -2):
        s = s * t2 + 1.0 / k
    return 2.0 * t * s + e * _LN2


_COS_C = [((-1.0) ** m) / float(math.factorial(2 * m)) for m in range(13)]
_SIN_C = [((-1.0) ** m) / float(math.factorial(2 * m + 1)) for m in range(13)]


def _cos_2pi(u: np.ndarray) -> np.ndarray:
    """cos(2*pi*u) for u in [0, 1) from IEEE + - * only (quadrant split + Taylor to x**25)."""
    v = u * 4.0                            # exact
    q = np.floor(v)
    x = (v - q) * _HALF_PI                 # in [0, pi/2)
    x2 = x * x
    c = np.zeros_like(x)
    s = np.zeros_like(x)
    for m in range(12, -1, -1):
        c = c * x2 + _COS_C[m]
        s = s * x2 + _SIN_C[m]
    s = s * x
    q = q.astype(np.int64) & 3
    return np.select([q == 0, q == 1, q == 2], [c, -s, -c], default=s)


def gaussian(key, counter) -> np.ndarray:
    """N(0, 1) doubles; Gaussian number n uses draws 2n and 2n+1 (Box-Muller, cosine branch)."""
    c = np.asarray(counter, dtype=np.uint64)
    x1 = splitmix64(key, c * np.uint64(2))
    x2 = splitmix64(key, c * np.uint64(2) + np.uint64(1))
    u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53    # (0, 1]
    u2 = (x2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53            # [0, 1)
    return np.sqrt(-2.0 * _log_unit(u1)) * _cos_2pi(u2)


def to_grid(x: np.ndarray, bits: int = GRID_BITS) -> np.ndarray:
    """Round to the nearest multiple of 2**-bits (ties to even); exact for |x| < 2**(52-bits)."""
    return np.rint(x * 2.0 ** bits) * 2.0 ** -bits


def _upper_pairs(n: int):
    iu, ju = np.triu_indices(n, 1)        # lexicographic (i, j), i < j
    return iu, ju


def instance(ensemble: str, n: int, seed: int, inst: int = 0, grid_bits: int | None = GRID_BITS):
    """One Ising instance: (J, h) with J symmetric (n x n, zero diagonal) and h (n,), FP64.

    Draw number k of the coupling stream is the k-th pair (i, j), i < j, in lexicographic order.
    grid_bits=None keeps the real-valued draws as they come (full FP64 values, not on a grid).
    """
    def rnd(x):
        return x if grid_bits is None else to_grid(x, grid_bits)

    kj = stream_key(seed, inst, TAG_J)
    kh = stream_key(seed, inst, TAG_H)
    iu, ju = _upper_pairs(n)
    cnt = np.arange(iu.size, dtype=np.uint64)
    hc = np.arange(n, dtype=np.uint64)
    if ensemble == "gaussian":
        vals = rnd(gaussian(kj, cnt))
        h = rnd(gaussian(kh, hc))
    elif ensemble == "uniform":
        vals = rnd(uniform01(kj, cnt)) - 0.5
        h = rnd(uniform01(kh, hc)) - 0.5
    elif ensemble == "pm1":
        vals = np.where((splitmix64(kj, cnt) >> np.uint64(63)) == 1, -1.0, 1.0)
        h = np.floor(uniform01(kh, hc) * 3.0) - 1.0
    else:
        raise ValueError(f"unknown ensemble {ensemble!r}")
    J = np.zeros((n, n), dtype=np.float64)
    J[iu, ju] = vals
    J[ju, iu] = vals
    return J, h.astype(np.float64)


def random_states(n: int, count: int, seed: int, inst: int = 0) -> np.ndarray:
    """``count`` uniformly random n-spin states (each bit an independent fair draw), packed
    as a (count, words(n)) uint64 array: the role of rand_between(0, 2**N - 1)."""
    k = stream_key(seed, inst, TAG_STATE)
    cnt = np.arange(count * n, dtype=np.uint64)
    sig = (splitmix64(k, cnt) >> np.uint64(63)).astype(np.uint8).reshape(count, n)
    return pack_bits(sig)


def pack_bits(sigma: np.ndarray) -> np.ndarray:
    """(count, n) array of 0/1 sigma values -> (count, words(n)) uint64, bit i = sigma_i."""
    sigma = np.atleast_2d(np.asarray(sigma, dtype=np.uint64))
    count, n = sigma.shape
    w = words(n)
    out = np.zeros((count, w), dtype=np.uint64)
    for i in range(n):
        out[:, i // 64] |= sigma[:, i] << np.uint64(i % 64)
    return out


def unpack_bits(packed: np.ndarray, n: int) -> np.ndarray:
    """(count, words(n)) uint64 -> (count, n) uint8 sigma values."""
    packed = np.atleast_2d(np.asarray(packed, dtype=np.uint64))
    out = np.zeros((packed.shape[0], n), dtype=np.uint8)
    for i in range(n):
        out[:, i] = ((packed[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)).astype(np.uint8)
    return out

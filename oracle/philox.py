"""Philox-4x32-10 counter-based generator and the two random draws of CoFEM (oracle side).

TEST INFRASTRUCTURE ONLY: this package is the plain CPU reference that the CUDA path is
checked against.  Only tests, the smoke check and the benchmark's CPU-baseline leg may
import it; the library never does.

Philox-4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11, Sec. 5): a 4x32-bit counter and a 2x32-bit key;
each of the 10 rounds multiplies counter words 0 and 2 by the two Philox multipliers,
swaps and xors the high halves with the other words and the round key, and the key is
advanced by the two Weyl constants between rounds.

Two draws of the method use it, both keyed by the 64-bit seed (low word, high word):

* Alg. 2, first step -- alpha_c ~ Uniform(0, 1): for (c, d) the counter is
  (d >> 2, c, 0, 2); output word d & 3, taken as w, gives ((w >> 9) + 1/2) * 2^-23, which
  lies strictly inside (0, 1) and is exact in FP32.
* Alg. 2 (probe sampling) and Eq. 4 -- Rademacher probe p_{t,c,k} of EM iteration e:
  for coordinate d the counter is (d >> 7, k, t*C + c, (e << 4) | 1); bit d & 31 of output
  word (d >> 5) & 3 selects the sign, 0 giving +1 and 1 giving -1.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF

TAG_PROBE = 1
TAG_ALPHA = 2


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox-4x32-10.  All arguments are integer arrays (or ints) holding
    32-bit values; returns four uint64 arrays holding the 32-bit output words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & np.uint64(_MASK) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & np.uint64(_MASK)
    k1 = np.asarray(k1, dtype=np.uint64) & np.uint64(_MASK)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    mask, s32 = np.uint64(_MASK), np.uint64(32)
    for rnd in range(10):
        p0 = m0 * c0          # 32 x 32 -> 64 bit, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(PHILOX_W0)) & mask
            k1 = (k1 + np.uint64(PHILOX_W1)) & mask
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & _MASK, (seed >> 32) & _MASK


def alpha_init(seed: int, C: int, D: int) -> np.ndarray:
    """Alg. 2 initialisation: alpha_c ~ Uniform(0, 1) for every cluster, as float64 [C, D]."""
    k0, k1 = _key(seed)
    d = np.arange(D, dtype=np.uint64)
    out = np.empty((C, D), dtype=np.float64)
    for c in range(C):
        w = philox4x32_10(d >> np.uint64(2), c, 0, TAG_ALPHA, k0, k1)
        word = np.choose((d & np.uint64(3)).astype(np.int64), w)
        out[c] = ((word >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
    return out


def probes(seed: int, em_iter: int, t: int, c: int, C: int, K: int, D: int) -> np.ndarray:
    """Rademacher probes p_{t,c,1..K} of EM iteration em_iter, as float64 [K, D] of +-1."""
    k0, k1 = _key(seed)
    d = np.arange(D, dtype=np.uint64)
    out = np.empty((K, D), dtype=np.float64)
    c3 = ((int(em_iter) << 4) | TAG_PROBE) & _MASK
    for k in range(K):
        w = philox4x32_10(d >> np.uint64(7), k, t * C + c, c3, k0, k1)
        word = np.choose(((d >> np.uint64(5)) & np.uint64(3)).astype(np.int64), w)
        bit = (word >> (d & np.uint64(31))) & np.uint64(1)
        out[k] = 1.0 - 2.0 * bit.astype(np.float64)
    return out

"""Projection matrix A for sign random projection (Eq. 4).  TEST INFRASTRUCTURE ONLY.

Eq. 4 needs projection vectors a with i.i.d. standard normal entries; the paper
names no generator.  This oracle and the CUDA library each implement, from the
published definitions and independently of each other:

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): 10 rounds; each round multiplies counter words 0 and 2 by
  the two 64-bit multipliers, XORs the high halves with the other words and the
  round key, and the key advances by the two Weyl constants between rounds.
* Box-Muller: z = sqrt(-2 ln u1) * cos(2 pi u2), with u = (w >> 12 + 1/2) * 2^-52
  taken from output words 0 and 1 (exact in FP64, strictly inside (0, 1)).
* the drawn z rounded once, to nearest-even, to bfloat16 precision (8
  significant bits), stored as an exact double.

Entry A[r, b] (row r in [0, d], the extra row r = d multiplying the SIMPLE-LSH
tail component; column b in [0, L)) uses counter (r, b, 0, 0) and key (seed, 0).
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(ctr, key):
    """One Philox4x64-10 block: four 64-bit counter words, two key words."""
    c0, c1, c2, c3 = (int(v) & MASK64 for v in ctr)
    k0, k1 = (int(v) & MASK64 for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64,
                          (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
    return c0, c1, c2, c3


def unit_open(w: int) -> float:
    """Map a 64-bit word to (0, 1): ((w >> 12) + 1/2) * 2^-52, exact in FP64."""
    return ((w >> 12) + 0.5) * 2.0 ** -52


def box_muller(w0: int, w1: int) -> float:
    u1, u2 = unit_open(w0), unit_open(w1)
    return math.sqrt(-2.0 * math.log(u1)) * math.cos((2.0 * math.pi) * u2)


def round_bf16(z: float) -> float:
    """Round a double to the nearest bfloat16 value (ties to even), in one step."""
    if z == 0.0:
        return 0.0
    mant, ex = math.frexp(z)            # z = mant * 2^ex, 0.5 <= |mant| < 1
    q = round(mant * 256.0)             # 8 significant bits; round() is half-even
    return math.ldexp(float(q), ex - 8)


def projections(seed: int, d: int, L: int) -> np.ndarray:
    """A with shape (d + 1, L): bfloat16-valued N(0, 1) entries as float64."""
    A = np.empty((d + 1, L), dtype=np.float64)
    key = (seed & MASK64, 0)
    for r in range(d + 1):
        for b in range(L):
            w = philox4x64_10((r, b, 0, 0), key)
            A[r, b] = round_bf16(box_muller(w[0], w[1]))
    return A

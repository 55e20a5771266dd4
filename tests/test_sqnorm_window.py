"""The integer-window arithmetic of the squared-norm kernels (s_x = sum_k x_k^2,
exact, rounded once to FP64; Algorithm 1's ranking key), emulated with Python
integers and checked against math.fsum (correctly rounded) on rows with wide
exponent ranges, zeros, subnormals and rows built next to a rounding tie.

Per row: W0 = top + bitlen(d) + 1 - 128 under the largest square; every value
x = M 2^E gives T = (M 2^8)^2 = M^2 2^16 and t = 2 max(e, 1) - 316 - W0 (e the
biased exponent); t in [32, 64) takes the fast form (three 32-bit funnel shifts
into words 1..3), anything else the general form with clamped 64-bit shifts and
the bits below the window noted; the 128-bit sum is rounded to nearest even
unless the noted bits could decide it (the exact slow path)."""
import math
import struct

import numpy as np

M32, M64 = (1 << 32) - 1, (1 << 64) - 1


def _bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _shl(a, s):
    return 0 if s >= 64 else (a << s) & M64


def _shr(a, s):
    return 0 if s >= 64 else a >> s


def _funnel(lo, hi, s):  # high word of (hi:lo) << (s mod 32)
    return ((((hi << 32) | lo) << (s & 31)) >> 32) & M32


def window_sum(xs):
    """(value, path) with path 'zero', 'fast' or 'slow' (value None on the slow path)."""
    d = len(xs)
    amax = max(abs(x) for x in xs)
    if amax == 0.0:
        return 0.0, "zero"
    if amax < 2.0 ** -126:
        return None, "slow"
    u = _bits(amax)
    e, f = (u >> 23) & 0xFF, u & 0x7FFFFF
    M2m, E2m = (f | 0x800000) ** 2, 2 * (e - 150)
    W0 = E2m + M2m.bit_length() + d.bit_length() + 1 - 128
    tbase = -300 - W0 - 16
    thr1 = ((max((33 - tbase) >> 1, 1) << 23) - 1) & M32
    acc, dropped = 0, 0
    for x in xs:
        u = _bits(x)
        mag = u & 0x7FFFFFFF
        e = (u >> 23) & 0xFF
        M8 = ((u << 8) & M32) | (0x80000000 if e else 0)
        T = M8 * M8
        if ((mag - 1) & M32) < thr1:
            t = 2 * max(e, 1) + tbase
            assert t < 64
            tp, tn = max(t, 0), max(-t, 0)
            acc += _shr(_shl(T, tp), tn) + (_shr(T, 64 - tp) << 64)
            dropped |= T & ~_shl(M64, tn) & M64
        else:
            sh = 2 * e + tbase - 32
            assert e == 0 or 0 <= sh < 32
            T0, T1 = T & M32, T >> 32
            acc += (_funnel(0, T0, sh) << 32) + (_funnel(T0, T1, sh) << 64) + (_funnel(T1, 0, sh) << 96)
    assert acc < 1 << 128
    pos = acc.bit_length() - 1
    cut = pos - 52
    mant, rem, half = acc >> cut, acc & ((1 << cut) - 1), 1 << (cut - 1)
    if rem > half:
        up = True
    elif rem == half:
        up = bool(dropped) or bool(mant & 1)
    else:
        if dropped and half - rem <= d:
            return None, "slow"
        up = False
    ex = W0 + pos
    if up:
        mant += 1
        if mant == 1 << 53:
            mant >>= 1
            ex += 1
    return math.ldexp(mant, ex - 52), "fast"


def _tie_row(t, d):
    """1 + 2^-53 - 2^W0 inside the window, plus t squares of 2^(W0 - 2) below it."""
    W0 = 1 + d.bit_length() + 1 - 128
    row = [1.0, 11863283 * 2.0 ** -50]
    rem = 4817239 * 2 ** (-100 - W0) - 1
    while rem > 0:
        j = max(0, (rem.bit_length() - 46) // 2)
        M = min(math.isqrt(rem // 4 ** j), 2 ** 24 - 1)
        row.append(M * 2.0 ** (j + W0 // 2))
        rem -= M * M * 4 ** j
    row += [2.0 ** ((W0 - 2) // 2)] * t
    return np.array(row + [0.0] * (d - len(row)), dtype=np.float32)


def _exact(xs):
    return math.fsum(float(x) * float(x) for x in xs)


def test_random_rows_round_exactly():
    rng = np.random.default_rng(5)
    paths = set()
    for it in range(1200):
        d = int(rng.integers(1, 80))
        x = rng.standard_normal(d)
        kind = it % 4
        if kind == 1:
            x *= 2.0 ** rng.integers(-60, 60, d)
        elif kind == 2:
            x *= 2.0 ** rng.integers(-140, -100, d)
        elif kind == 3:
            x[rng.random(d) < 0.5] = 0.0
        xs = [float(v) for v in x.astype(np.float32)]
        got, path = window_sum(xs)
        paths.add(path)
        if got is not None:
            assert got == _exact(xs), (it, got, _exact(xs))
    assert {"fast", "slow"} <= paths


def test_tie_rows_take_the_slow_path_only_when_the_dropped_bits_decide():
    for d in (15, 32, 200, 512):
        for t in (0, 3, 4, 5, 9):
            row = [float(v) for v in _tie_row(t, d)]
            got, path = window_sum(row)
            assert path == ("fast" if t == 0 else "slow"), (d, t, path)
            if got is not None:
                assert got == _exact(row) == 1.0
        assert _exact([float(v) for v in _tie_row(5, d)]) == 1.0 + 2.0 ** -52

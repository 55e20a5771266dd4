"""Constants written into the CUDA sources are checked against exact values
(no GPU needed): the double-double Taylor coefficients 1/i! and pi used for the
correctly rounded cosines of the bucket order (Eq. 12)."""
import math
import os
import re
from decimal import Decimal, getcontext
from fractions import Fraction

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD_CU = os.path.join(ROOT, "paper_1809_08782_gb300", "csrc", "build.cu")


def _hexf(t: str) -> float:
    return float.fromhex(t.strip())


def test_inverse_factorial_table():
    src = open(BUILD_CU).read()
    body = src[src.index("kInvFact[30] = {"):]
    body = body[:body.index("};")]
    pairs = re.findall(r"\{\s*([-0-9a-fx.p+]+),\s*([-0-9a-fx.p+]+)\s*\}", body)
    assert len(pairs) == 30
    for i, (hi, lo) in enumerate(pairs):
        exact = Fraction(1, math.factorial(i))
        h, l = _hexf(hi), _hexf(lo)
        assert h == float(exact)                       # hi is 1/i! rounded to nearest
        err = abs(Fraction(h) + Fraction(l) - exact)
        assert err <= exact * Fraction(1, 2 ** 104)


def _pi_decimal(prec=60):
    getcontext().prec = prec + 10

    def atan_inv(x):
        x2, term, total, k = x * x, Decimal(1) / x, Decimal(1) / x, 1
        while True:
            term /= x2
            t = term / (2 * k + 1)
            if abs(t) < Decimal(10) ** -(prec + 5):
                return total
            total = total - t if k % 2 else total + t
            k += 1
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def test_pi_double_double():
    src = open(BUILD_CU).read()
    m = re.search(r"const dd pi = \{([0-9.e+-]+), ([0-9.e+-]+)\};", src)
    assert m, "pi constant not found"
    hi, lo = float(m.group(1)), float(m.group(2))
    pi = _pi_decimal()
    assert hi == math.pi
    assert lo == float(pi - Decimal(hi))
    assert abs(Decimal(hi) + Decimal(lo) - pi) < Decimal(2) ** -105

"""The error bounds that let the GPU decide a code bit or a score from a cheaper
evaluation than the canonical FP64 sum, checked by emulating that evaluation in
IEEE float32 (numpy, round to nearest) against the exactly rounded sum.

* FP32 tier (Eq. 4 bits and the re-rank intervals): any summation order of the
  fp32 products is within (d + 2) 2^-22 sum|x_k a_k| of the exact dot product;
  here the lane-strided order with a 5-level tree.
* Compensated tier (Ogita, Rump, Oishi, "Accurate sum and dot product", 2005):
  TwoProduct and TwoSum per lane, lane-strided, then TwoSum down a 5-level tree;
  |hi + lo - x^T a| <= u^2 (2m + 10)(m + 6) sum|x_k a_k|, u = 2^-24, m terms per lane.

Inputs mix random vectors, vectors made orthogonal in float64 (heavy
cancellation) and wide exponent ranges."""
import math

import numpy as np

F = np.float32


def two_sum(a, b):
    s = (a + b).astype(F)
    bb = (s - a).astype(F)
    t = ((a - (s - bb).astype(F)).astype(F) + (b - bb).astype(F)).astype(F)
    return s, t


def emulate(x, a):
    """x, a: (trials, d) float32.  Returns (plain fp32 sum, dot2 hi, dot2 lo), each in
    the lane-strided order of 32 lanes and a 5-level xor tree."""
    T, d = x.shape
    plain = np.zeros((T, 32), F)
    sh = np.zeros((T, 32), F)
    sl = np.zeros((T, 32), F)
    for k0 in range(0, d, 32):
        xs = np.zeros((T, 32), F)
        as_ = np.zeros((T, 32), F)
        w = min(32, d - k0)
        xs[:, :w] = x[:, k0:k0 + w]
        as_[:, :w] = a[:, k0:k0 + w]
        # plain: fma(x, a, acc), one rounding of the exact x a + acc
        plain = (xs.astype(np.float64) * as_.astype(np.float64) + plain.astype(np.float64)).astype(F)
        pr = (xs * as_).astype(F)
        er = (xs.astype(np.float64) * as_.astype(np.float64) - pr.astype(np.float64)).astype(F)
        s2, t = two_sum(sh, pr)
        sh = s2
        sl = ((sl + t).astype(F) + er).astype(F)
    lanes = np.arange(32)
    for o in (16, 8, 4, 2, 1):
        plain = (plain + plain[:, lanes ^ o]).astype(F)
        oh, ol = sh[:, lanes ^ o], sl[:, lanes ^ o]
        s2, t = two_sum(sh, oh)
        sh = s2
        sl = ((sl + ol).astype(F) + t).astype(F)
    return plain[:, 0], sh[:, 0], sl[:, 0]


def exact(x, a):
    return np.array([math.fsum((x[i].astype(np.float64) * a[i].astype(np.float64)).tolist())
                     for i in range(x.shape[0])])


def cases(d, seed):
    rng = np.random.default_rng(seed)
    T = 400
    x = rng.standard_normal((T, d))
    a = rng.standard_normal((T, d))
    # a third made orthogonal to x in float64 (the rounding to fp32 leaves a tiny dot)
    k = T // 3
    a[:k] -= (np.sum(a[:k] * x[:k], 1) / np.sum(x[:k] * x[:k], 1))[:, None] * x[:k]
    # a third with exponents spread over 2^-30 .. 2^30
    x[k:2 * k] *= 2.0 ** rng.integers(-30, 30, (k, d))
    return x.astype(F), a.astype(F)


def test_fp32_tier_bound():
    for d, seed in ((300, 1), (40, 2), (1000, 3), (7, 4)):
        x, a = cases(d, seed)
        plain, _, _ = emulate(x, a)
        S = exact(x, a)
        sabs = np.sum(np.abs(x.astype(np.float64) * a.astype(np.float64)), 1)
        err = np.abs(plain.astype(np.float64) - S)
        assert np.all(err <= (d + 2) * 2.0 ** -22 * sabs), (d, float(np.max(err / sabs)))
        # the first-order bound d 2^-24 itself holds with room: the 4x is margin
        assert np.all(err <= d * 2.0 ** -24 * sabs * 1.01)


def test_compensated_tier_bound():
    u = 2.0 ** -24
    for d, seed in ((300, 5), (40, 6), (1000, 7), (7, 8)):
        x, a = cases(d, seed)
        _, hi, lo = emulate(x, a)
        S = exact(x, a)
        sabs = np.sum(np.abs(x.astype(np.float64) * a.astype(np.float64)), 1)
        m = -(-d // 32)
        got = hi.astype(np.float64) + lo.astype(np.float64)   # exact in float64 here
        err = np.abs(got - S)
        bound = u * u * (2 * m + 10) * (m + 6) * sabs
        assert np.all(err <= bound + 2.0 ** -52 * np.abs(S)), (d, float(np.max(err / sabs)))


def test_compensated_tier_is_much_tighter_than_fp32():
    """The point of the tier: on cancellation-heavy inputs its error is orders of
    magnitude below the FP32 sum's."""
    x, a = cases(300, 9)
    plain, hi, lo = emulate(x, a)
    S = exact(x, a)
    e32 = np.abs(plain.astype(np.float64) - S)
    e2 = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - S)
    assert np.median(e2[e32 > 0] / e32[e32 > 0]) < 1e-4


def _bf16(v):
    """Round float32 to bfloat16 (nearest, ties to even), back as float32."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=F)).to(torch.bfloat16).to(torch.float32).numpy()


def _tc_factor(q, d, fp32_items):
    """a_q of the tensor-core score interval e = a_q ||x|| (query_bound_kernel):
    D = ||q - bf16(q)||, Q = ||q||, rx = 2^-8 for fp32 items entered as bf16."""
    D = math.sqrt(math.fsum(float(r) ** 2 for r in (q - _bf16(q)).astype(np.float64)))
    Q = math.sqrt(math.fsum(float(v) ** 2 for v in q.astype(np.float64)))
    rx = 2.0 ** -8 if fp32_items else 0.0
    K = 16 * -(-d // 16)
    return (D + rx * (Q + D) + (K + 8) * 2.0 ** -20 * (Q + D) * (1 + rx) + (d + 2) * 2.0 ** -53 * Q) * (1 + 2.0 ** -20)


def test_tensor_core_score_interval_bound():
    """bf16 operands (query always, items when stored as fp32) and FP32 accumulation,
    emulated in two orders (sequential, and 16-wide partial sums as the K = 16 MMA
    steps add them): the FP64 score lies within a_q ||x||.  Random, cancelling and
    worst-case rounding inputs (every coordinate just below or above a bf16
    rounding midpoint, so the two roundings err by up to 2^-8 each, aligned)."""
    rng = np.random.default_rng(11)
    for d in (7, 64, 129, 300):
        q = rng.standard_normal((60, d)).astype(F)
        x = rng.standard_normal((60, d)).astype(F)
        # worst case: q and x just below the midpoint 1 + 2^-8 (both round down)
        q[:10] = F(1 + 2 ** -8 - 2 ** -20)
        x[:10] = F(1 + 2 ** -8 - 2 ** -20)
        # cancellation: x orthogonal to q in float64
        x[10:20] -= (np.sum(x[10:20] * q[10:20], 1) / np.sum(q[10:20] ** 2, 1))[:, None] * q[10:20]
        for fp32_items in (True, False):
            xs = x if fp32_items else _bf16(x)
            qt, xt = _bf16(q), _bf16(xs)
            S = exact(q, xs)
            prods = (qt.astype(np.float64) * xt.astype(np.float64)).astype(F)   # exact in fp32
            seq = np.zeros(q.shape[0], F)
            for k in range(d):
                seq = (seq + prods[:, k]).astype(F)
            chunk = np.zeros(q.shape[0], F)
            for k0 in range(0, d, 16):
                part = np.zeros(q.shape[0], F)
                for k in range(k0, min(d, k0 + 16)):
                    part = (part + prods[:, k]).astype(F)
                chunk = (chunk + part).astype(F)
            xn = np.sqrt(np.sum(xs.astype(np.float64) ** 2, 1))
            for s in (seq, chunk):
                err = np.abs(s.astype(np.float64) - S)
                bound = np.array([_tc_factor(q[i], d, fp32_items) for i in range(q.shape[0])]) * xn
                assert np.all(err <= bound), (d, fp32_items, float(np.max(err / bound)))
            if fp32_items:
                # 2^-9 per rounding (half the unit roundoff) does not hold here
                Qn = np.sqrt(np.sum(q.astype(np.float64) ** 2, 1))
                half = ((1 + 2.0 ** -9) ** 2 - 1) * Qn * xn
                assert np.any(np.abs(seq.astype(np.float64) - S) > half)

"""Pins for the CPU oracle: each test ties the oracle to something other than
itself (a value worked by hand, a closed form, an invariant, an independent
library routine or brute force), so that a dropped term, a wrong sign or index,
or a transposed operand in the oracle fails at least one of them."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, nrlsh as O, philox, simple_lsh
from paper_1809_08782_gb300 import workloads as W


def rand_items(n, d, seed, sigma=0.8):
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((n, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    return (dirs * rng.lognormal(0.0, sigma, n)[:, None]).astype(np.float32).astype(np.float64)


def rand_queries(nq, d, seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((nq, d))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------- generator

def _numpy_philox_block(ctr, key):
    """numpy's Philox4x64-10 advances the 256-bit counter before each block."""
    c = [int(v) for v in ctr]
    for i in range(4):                       # counter - 1 with borrow
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1
    g = np.random.Philox(key=np.array(key, dtype=np.uint64),
                        counter=np.array(c, dtype=np.uint64))
    return tuple(int(v) for v in g.random_raw(4))


@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((5, 7, 0, 0), (3000, 0)),
    ((300, 63, 0, 0), (0xFFFFFFFFFFFFFFFF, 0)),
    ((1, 2, 3, 4), (0x0123456789ABCDEF, 0xFEDCBA9876543210)),
])
def test_philox_matches_numpy_bit_generator(ctr, key):
    assert philox.philox4x64_10(ctr, key) == _numpy_philox_block(ctr, key)


def test_round_bf16_ties_and_torch():
    import torch
    assert philox.round_bf16(1.0 + 2.0 ** -8) == 1.0                   # tie -> even
    assert philox.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie -> even
    assert philox.round_bf16(-(1.0 + 2.0 ** -8 + 2.0 ** -30)) == -(1.0 + 2.0 ** -7)
    rng = np.random.default_rng(1)
    v32 = rng.standard_normal(2000).astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    ours = np.array([philox.round_bf16(float(x)) for x in v32])
    assert np.array_equal(ours, ref)


def test_projection_entries_are_standard_normal():
    from scipy import stats
    A = philox.projections(seed=11, d=199, L=64)
    z = A.ravel()
    assert z.size == 200 * 64
    assert np.all([philox.round_bf16(float(v)) == v for v in z[:500]])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # rows and columns are distinct streams
    assert not np.array_equal(A[0], A[1]) and not np.array_equal(A[:, 0], A[:, 1])
    assert np.array_equal(A, philox.projections(seed=11, d=199, L=64))
    assert not np.array_equal(A, philox.projections(seed=12, d=199, L=64))


# -------------------------------------------------------------- Algorithm 1

def test_sq_norms_are_the_exact_sum_rounded_once():
    """Against exact rational arithmetic (Fraction sums, converted by Python's
    correctly rounded int/int division), integer rows, and order independence."""
    X = rand_items(60, 37, 3)
    s = O.sq_norms(X)
    for i in range(60):
        exact = sum((Fraction(float(v)) ** 2 for v in X[i]), Fraction(0))
        assert s[i] == float(exact)
    rng = np.random.default_rng(4)
    for i in range(0, 60, 7):
        perm = rng.permutation(37)
        assert O.sq_norms(X[i:i + 1, perm])[0] == s[i]
    Xi = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0], [-4.0, 0.5, 0.25]])
    assert list(O.sq_norms(Xi)) == [14.0, 0.0, 16.3125]


def squares_near_a_tie(t: int):
    """A row whose exact ||x||^2 is 1 + 2^-53 - 2^-106 + t 2^-108: the in-range
    part sits one 2^-106 unit below the half-way point between 1 and 1 + 2^-52,
    and t squares of 2^-54 (2^-108 each) decide the rounding: t < 4 rounds down,
    t = 4 is an exact tie (to even, 1.0), t > 4 rounds up.  The terms:
    (11863283 2^-50)^2 = 2^-53 - 4817239 2^-100, and 17558, 141, 7, 1 times
    2^-53 squared make up 4817239 2^-100 - 2^-106 exactly."""
    row = [1.0, 11863283 * 2.0 ** -50, 17558 * 2.0 ** -53, 141 * 2.0 ** -53,
           7 * 2.0 ** -53, 1 * 2.0 ** -53] + [2.0 ** -54] * t
    return np.array(row, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("t,expected", [(0, 1.0), (3, 1.0), (4, 1.0), (5, 1.0 + 2.0 ** -52),
                                        (9, 1.0 + 2.0 ** -52)])
def test_sq_norms_ties_and_far_below_terms(t, expected):
    row = squares_near_a_tie(t)
    exact = sum((Fraction(float(v)) ** 2 for v in row), Fraction(0))
    assert exact == 1 + Fraction(1, 2 ** 53) - Fraction(1, 2 ** 106) + t * Fraction(1, 2 ** 108)
    assert O.sq_norms(row[None, :])[0] == expected == float(exact)
    rng = np.random.default_rng(t)
    assert O.sq_norms(row[None, rng.permutation(row.size)])[0] == expected


@pytest.mark.parametrize("n,m", [(1, 1), (7, 3), (10, 10), (33, 4), (64, 5)])
def test_partition_against_bruteforce(n, m):
    rng = np.random.default_rng(n * 100 + m)
    s = rng.integers(0, 5, n).astype(np.float64)      # many ties
    sub, U2, bounds, _ = O.partition(s, m)
    ranked = sorted(range(n), key=lambda i: (s[i], i))
    for r, i in enumerate(ranked):
        j = max(jj for jj in range(m) if (jj * n) // m <= r)
        assert sub[i] == j
    sizes = np.bincount(sub, minlength=m)
    assert sizes.min() >= 1 and sizes.max() - sizes.min() <= 1
    for j in range(m):
        assert U2[j] == max(s[i] for i in range(n) if sub[i] == j)
    assert np.all(np.diff(U2) >= 0)


def test_partition_rejects_bad_m():
    with pytest.raises(ValueError):
        O.partition(np.ones(3), 4)
    with pytest.raises(ValueError):
        O.partition(np.ones(3), 0)


# ---------------------------------------- uniform norm ranges (Section 5)

@pytest.mark.parametrize("lo,top,m", [(0, 64, 8), (5, 32, 4), (3, 16, 16), (0, 8, 1)])
def test_uniform_partition_exact_dyadic_norms(lo, top, m):
    """Integer norms lo..lo+top with a power-of-two width: every FP64 step is
    exact, so j = min(m-1, floor((nu - lo) m / top)) in integers."""
    nu = np.arange(lo, lo + top + 1, dtype=np.float64)
    rng = np.random.default_rng(lo + top + m)
    perm = rng.permutation(nu.size)
    s = (nu * nu)[perm]
    sub, U2, bounds = O.partition_uniform(s, m)
    for i, p in enumerate(perm):
        v = int(nu[p]) - lo
        assert sub[i] == min(m - 1, (v * m) // top)
    for j in range(m):
        members = s[sub == j]
        assert U2[j] == (members.max() if members.size else 0.0)
    assert bounds == [0] + np.cumsum(np.bincount(sub, minlength=m)).tolist()


def test_uniform_partition_matches_numpy_histogram():
    """Bin counts equal numpy.histogram's equal-width bins over [min, max] (last
    bin closed), away from bin edges where the two roundings may differ."""
    rng = np.random.default_rng(11)
    for trial in range(5):
        nu = rng.lognormal(0.0, 0.8, 5000)
        s = nu * nu
        nu = np.sqrt(s)
        m = [4, 16, 32, 64, 100][trial]
        edges = np.linspace(nu.min(), nu.max(), m + 1)
        gap = np.min(np.abs(nu[:, None] - edges[None, 1:-1]))
        if gap < 1e-9 * nu.max():
            continue
        sub, _, _ = O.partition_uniform(s, m)
        counts, _ = np.histogram(nu, bins=m, range=(nu.min(), nu.max()))
        assert np.array_equal(np.bincount(sub, minlength=m), counts)


def test_uniform_partition_against_exact_rationals():
    """j from exact rational arithmetic on the same nu values agrees wherever the
    exact t = (nu - nu_min) m / w is not within 1e-9 of an integer."""
    rng = np.random.default_rng(12)
    s = rng.lognormal(0.0, 1.0, 400) ** 2
    m = 12
    sub, _, _ = O.partition_uniform(s, m)
    nu = np.sqrt(s)
    lo, hi = Fraction(float(nu.min())), Fraction(float(nu.max()))
    checked = 0
    for i in range(s.size):
        t = (Fraction(float(nu[i])) - lo) * m / (hi - lo)
        if abs(t - round(t)) < Fraction(1, 10**9):
            continue
        assert sub[i] == min(m - 1, math.floor(t))
        checked += 1
    assert checked > 390


def test_uniform_partition_invariants_and_degenerate_cases():
    rng = np.random.default_rng(13)
    s = np.concatenate([rng.uniform(0.5, 1.0, 300), rng.uniform(9.0, 16.0, 300)])  # a gap
    sub, U2, bounds = O.partition_uniform(s, 10)
    order = np.argsort(s, kind="stable")
    assert np.all(np.diff(sub[order]) >= 0)                  # contiguous in ||x||
    assert sub[np.argmin(s)] == 0 and sub[np.argmax(s)] == 9
    sizes = np.bincount(sub, minlength=10)
    assert (sizes == 0).any()                                 # the gap leaves empty ranges
    assert np.all(U2[sizes == 0] == 0.0)
    assert bounds[-1] == s.size
    # equal norms: everything in S_0
    sub, U2, _ = O.partition_uniform(np.full(50, 2.25), 8)
    assert np.all(sub == 0) and U2[0] == 2.25 and np.all(U2[1:] == 0.0)
    # m = 1 is the percentile partition with m = 1
    s = rng.uniform(0, 4, 40)
    a, Ua, _ = O.partition_uniform(s, 1)
    b, Ub, _, _ = O.partition(s, 1)
    assert np.array_equal(a, b) and np.array_equal(Ua, Ub)
    # zero vectors alongside non-zero ones sit in S_0
    s = np.concatenate([np.zeros(5), rng.uniform(1, 2, 20)])
    sub, _, _ = O.partition_uniform(s, 4)
    assert np.all(sub[:5] == 0)


def test_uniform_index_full_budget_returns_exact_mips():
    X = rand_items(60, 7, 31)
    idx = O.build(X, 6, 12, seed=5, eps=0.2, partition_scheme="uniform")
    assert idx.bounds[-1] == 60
    Q = rand_queries(6, 7, 32)
    ids, _ = O.query(idx, Q, 4, B=60)
    for i in range(6):
        assert np.array_equal(ids[i], exact.exact_topk(X, Q[i], 4))


# ------------------------------------------------------------- Eq. 8 and 4

def test_simple_lsh_transform_invariants():
    X = rand_items(300, 16, 5, sigma=1.0)
    Q = rand_queries(5, 16, 6)
    s = O.sq_norms(X)
    sub, U2, _, _ = O.partition(s, 8)
    for j in range(8):
        members = np.flatnonzero(sub == j)
        U = math.sqrt(U2[j])
        P = simple_lsh.transform_items(X[members], U)
        assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-12, rtol=0)
        top = members[np.argmax(s[members])]
        assert simple_lsh.transform_items(X[[top]], U)[0, -1] == pytest.approx(0.0, abs=1e-7)
        PQ = simple_lsh.transform_queries(Q)
        assert np.allclose(PQ @ P.T, (Q @ X[members].T) / U, atol=1e-13, rtol=0)


def test_scale_free_codes_equal_sign_of_transformed_projection():
    X = rand_items(500, 24, 7, sigma=1.0)
    A = philox.projections(seed=5, d=24, L=32)
    idx = O.build(X, 8, 32, seed=5, eps=0.1)
    assert np.array_equal(idx.A, A)
    bits = np.zeros((500, 32), dtype=bool)
    for j in range(8):
        members = np.flatnonzero(idx.sub == j)
        P = simple_lsh.transform_items(X[members], math.sqrt(idx.U2[j]))
        bits[members] = simple_lsh.srp_bits(P, A)
    assert np.array_equal(O.pack_bits(bits), idx.codes)
    # a wrongly oriented A (columns as rows) would not even have the right shape
    assert idx.A.shape == (25, 32)


def test_tail_component_and_zero_subdataset():
    s = np.array([0.0, 0.0, 4.0, 9.0])
    sub, U2, _, _ = O.partition(s, 2)
    tau = O.tail_component(s, sub, U2)
    assert list(U2) == [0.0, 9.0]
    assert list(tau) == [1.0, 1.0, math.sqrt(5.0), 0.0]


def test_collision_rate_is_one_minus_theta_over_pi():
    """Eq. 4: P[h_a(x) = h_a(y)] = 1 - theta/pi for sign random projection."""
    d, L = 12, 64
    rng = np.random.default_rng(21)
    for theta in (0.3, 1.2, 2.5):
        u = rng.standard_normal(d); u /= np.linalg.norm(u)
        w = rng.standard_normal(d); w -= (w @ u) * u; w /= np.linalg.norm(w)
        y = math.cos(theta) * u + math.sin(theta) * w
        V = np.stack([u, y])
        same = 0
        trials = 0
        for seed in range(10_000, 10_000 + 160):
            A = philox.projections(seed, d - 1, L)       # (d, L): rows for all d coordinates
            b = simple_lsh.srp_bits(V, A)
            same += int((b[0] == b[1]).sum())
            trials += L
        p = 1 - theta / math.pi
        sigma = math.sqrt(p * (1 - p) / trials)
        assert abs(same / trials - p) < 5 * sigma, (theta, same / trials, p)


def test_collision_rate_within_subdataset():
    """Section 3.3: for x in S_j and a unit query, one bit collides with probability
    1 - arccos(q^T x / U_j) / pi."""
    d, L, m = 10, 64, 4
    X = rand_items(40, d, 31, sigma=1.0)
    q = rand_queries(1, d, 32)
    s = O.sq_norms(X)
    sub, U2, _, _ = O.partition(s, m)
    picks = [int(np.flatnonzero(sub == j)[0]) for j in range(m)]
    same = np.zeros(len(picks))
    trials = 0
    for seed in range(160):
        idx = O.build(X, m, L, seed=seed, eps=0.1)
        cq = int(O.query_codes(q, idx.A)[0])
        for t, i in enumerate(picks):
            same[t] += L - int(np.bitwise_count(np.uint64(int(idx.codes[i]) ^ cq)))
        trials += L
    for t, i in enumerate(picks):
        c = float(q[0] @ X[i]) / math.sqrt(U2[sub[i]])
        p = 1 - math.acos(c) / math.pi
        sigma = math.sqrt(p * (1 - p) / trials)
        assert abs(same[t] / trials - p) < 5 * sigma


# ------------------------------------------------------------------ Eq. 12

def test_cos_class_values():
    for L in (1, 2, 16, 17, 32, 64):
        for eps in (1e-9, 0.1, 0.3, 0.5):
            for l in range(L + 1):
                c = O.cos_class(L, l, eps)
                ref = math.cos(math.pi * (1 - eps) * (L - l) / L)
                assert abs(c - ref) <= 4e-16 + 2 * abs(ref) * 2.0 ** -52
    assert O.cos_class(2, 0, 0.5) == 0.0              # pi/2 exactly
    assert O.cos_class(64, 0, 0.5) == 0.0
    assert O.cos_class(48, 16, 0.5) == 0.5           # pi/3 exactly
    assert O.cos_class(32, 32, 0.1) == 1.0
    assert O.cos_class(4, 2, 0.5) == pytest.approx(math.sqrt(0.5), abs=0, rel=2.0 ** -52)


def _cos_correctly_rounded(L, l, eps):
    """cos(pi (1 - eps)(L - l) / L) correctly rounded to FP64 (Eq. 12's c_l): mpmath
    at 200 bits, then the exact binary value of that result rounded once through
    a Fraction (Python's int division rounds to nearest); 0 exactly at pi/2."""
    import mpmath
    from fractions import Fraction
    fe = Fraction(eps)
    if 2 * (1 - fe) * (L - l) == L:
        return 0.0, True
    with mpmath.workprec(200):
        v = mpmath.cos(mpmath.pi * (1 - mpmath.mpf(eps)) * (L - l) / L)
        sign, man, exp, _ = v._mpf_                 # v = (-1)^sign man 2^exp exactly
        exact = (-1) ** sign * Fraction(int(man)) * Fraction(2) ** int(exp)
        r = float(exact)
        # unambiguous: the 200-bit value is far from the midpoint between doubles
        lo_nb, hi_nb = math.nextafter(r, -math.inf), math.nextafter(r, math.inf)
        mid = min(abs(exact - (Fraction(r) + Fraction(lo_nb)) / 2),
                  abs(exact - (Fraction(r) + Fraction(hi_nb)) / 2))
        ok = mid > abs(exact) * Fraction(2) ** -150 + Fraction(2) ** -1000
    return r, ok


def test_cos_class_is_correctly_rounded():
    """c_l against an independent 200-bit evaluation rounded once, for the code
    lengths and eps values the tests and presets use (eps as its float32 value,
    which is what the C ABI receives), every l."""
    pytest.importorskip("mpmath")
    import numpy as _np
    for L in (1, 2, 8, 16, 17, 24, 32, 48, 63, 64):
        for e in (1e-9, 0.1, 0.2, 0.3, 0.5, 0.9):
            eps = float(_np.float32(e))
            for l in range(L + 1):
                want, ok = _cos_correctly_rounded(L, l, eps)
                assert ok
                assert O.cos_class(L, l, eps) == want, (L, l, eps)


def test_negative_region_matches_paper_bound():
    """cos < 0 exactly when l < L [1/2 - eps / (2 (1 - eps))] (Section 3.3)."""
    for L, eps in ((32, 0.1), (64, 0.2), (16, 0.3)):
        bound = L * (0.5 - eps / (2 * (1 - eps)))
        for l in range(L + 1):
            assert (O.cos_class(L, l, eps) < 0) == (l < bound - 1e-12)


def test_bucket_order_monotone_in_l_and_ties():
    U2 = np.array([0.0, 0.25, 1.0, 1.0, 4.0])
    for eps in (1e-9, 0.1, 0.5, 0.9):
        table, shat, c = O.class_table(U2, 16, eps)
        assert np.all(np.diff(c) > 0)
        pos = {jl: t for t, jl in enumerate(table)}
        for j in range(5):
            for l in range(16):
                assert pos[(j, l + 1)] < pos[(j, l)]       # larger l probed first
        assert pos[(3, 16)] < pos[(2, 16)]                 # equal U: larger j first
        assert len(set(table)) == 5 * 17
        vals = [shat[j, l] for j, l in table]
        assert all(a >= b for a, b in zip(vals, vals[1:]))


# --------------------------------------------------------- query probing

def small_index(n=400, d=16, m=8, L=16, eps=0.2, seed=9, sigma=1.0):
    X = rand_items(n, d, seed, sigma)
    return X, O.build(X, m, L, seed=seed + 1, eps=eps)


def test_threshold_walk_equals_sorted_definition():
    X, idx = small_index()
    Q = rand_queries(6, 16, 99)
    cq = O.query_codes(Q, idx.A)
    for i in range(6):
        H = O.histogram(idx, int(cq[i]))
        assert H.sum() == idx.n
        for B in (1, 7, 50, 399, 400, 1000):
            lam, js, ls, r, full = O.threshold(idx, H, B)
            l = O.matches(idx, int(cq[i]))
            sel = l >= np.array(lam)[idx.sub]
            bnd = np.flatnonzero((idx.sub == js) & (l == ls))[:r]
            walk = np.union1d(np.flatnonzero(sel), bnd)
            direct = np.sort(O.candidates(idx, int(cq[i]), B))
            assert np.array_equal(walk, direct)
            assert direct.size == min(B, idx.n) and sel.sum() == full
            rep = O.candidates_reported(idx, int(cq[i]), B)
            assert np.array_equal(np.sort(rep), direct)


def test_prefix_property_and_whole_class():
    X, idx = small_index()
    q = rand_queries(1, 16, 5)
    cq = int(O.query_codes(q, idx.A)[0])
    prev = set()
    for B in (1, 2, 5, 20, 80, 200, 400):
        cur = set(O.candidates(idx, cq, B).tolist())
        assert prev <= cur
        prev = cur
        whole = set(O.candidates(idx, cq, B, whole_class=True).tolist())
        assert cur <= whole
        H = O.histogram(idx, cq)
        lam, js, ls, r, full = O.threshold(idx, H, B)
        assert len(whole) == full + H[js, ls]


def test_single_subdataset_reduces_to_simple_lsh():
    X, idx = small_index(n=300, m=1, L=24, eps=0.1, seed=13)
    Q = rand_queries(5, 16, 77)
    cq = O.query_codes(Q, idx.A)
    for i in range(5):
        for B in (10, 60, 150):
            ours = np.sort(O.candidates(idx, int(cq[i]), B))
            theirs = np.sort(simple_lsh.candidates(X, Q[i], idx.A, B))
            assert np.array_equal(ours, theirs)


def test_equal_norms_reduce_to_plain_srp():
    rng = np.random.default_rng(4)
    base = rng.standard_normal(12).astype(np.float32).astype(np.float64)
    signs = rng.choice([-1.0, 1.0], size=(64, 12))
    X = signs * base[None, :]
    idx = O.build(X, 4, 32, seed=8, eps=0.1)
    assert np.all(idx.tau == 0.0)
    bits = simple_lsh.srp_bits(X, idx.A[:12])
    assert np.array_equal(O.pack_bits(bits), idx.codes)


def test_full_budget_returns_exact_mips():
    X, idx = small_index(n=48, d=6, m=4, L=8, seed=17)
    Q = rand_queries(8, 6, 18)
    ids, sc = O.query(idx, Q, 5, B=48)
    for i in range(8):
        assert np.array_equal(ids[i], exact.exact_topk(X, Q[i], 5))
        ex = exact.exact_scores(X[ids[i]], Q[i])
        for v, e in zip(sc[i], ex):
            assert abs(float(v) - float(e)) <= 2.0 ** -23 * abs(float(e)) + 1e-30


def test_scores_fp64_sequential_against_fractions():
    X = rand_items(30, 40, 23)
    q = rand_queries(1, 40, 24)[0]
    s = O.scores_fp64(X, q)
    ex = exact.exact_scores(X, q)
    bound = 40 * 2.0 ** -53 * np.abs(X * q[None, :]).sum(axis=1)
    assert np.all(np.abs(s - np.array([float(e) for e in ex])) <= bound)


def test_topk_ties_and_padding():
    ids, sc = O.topk(np.array([5, 3, 9, 1]), np.array([1.0, 2.0, 2.0, 1.0]), 6)
    assert list(ids) == [3, 9, 1, 5, -1, -1]
    assert sc[4] == -np.inf


def test_range_lsh_probes_fewer_items_than_simple_lsh():
    """Figure 2 / Section 5: on long-tailed norms norm-ranging LSH reaches a given
    recall with fewer probed items than SIMPLE-LSH (qualitative, synthetic data)."""
    X = rand_items(3000, 24, 41, sigma=1.0)
    Q = rand_queries(60, 24, 42)
    truth = exact.brute_topk_fp64(X, Q, 10)
    idx = O.build(X, 16, 32, seed=43, eps=0.3)
    B = 150
    ids, _ = O.query(idx, Q, 10, B)
    rec_range = exact.recall_at_k(ids, truth)
    simp = [simple_lsh.candidates(X, Q[i], idx.A, B) for i in range(60)]
    found = []
    for i in range(60):
        sc = O.scores_fp64(X[simp[i]], Q[i])
        found.append(O.topk(simp[i].astype(np.int64), sc, 10)[0])
    rec_simple = exact.recall_at_k(np.array(found), truth)
    assert rec_range > rec_simple + 0.1, (rec_range, rec_simple)


# ---------------------------------------------------------------- golden

def test_hand_worked_example(golden_dir):
    with open(os.path.join(golden_dir, "tiny_example.json")) as f:
        g = json.load(f)
    X = np.array(g["items"])
    A = np.array(g["A"])
    idx = O.build(X, g["m"], g["L"], seed=0, eps=g["eps"], A=A)
    assert list(idx.sub) == g["sub_of_id"]
    assert list(idx.U2) == g["U2"]
    assert list(idx.tau) == g["tau"]
    assert [int(c) for c in idx.codes] == g["codes"]
    _, _, c = O.class_table(idx.U2, g["L"], g["eps"])
    assert c[0] == 0.0 and c[2] == 1.0
    assert c[1] == pytest.approx(g["c"][1], rel=2.0 ** -52)
    assert [list(t) for t in idx.table] == g["probe_order"]
    q = np.array([g["query"]])
    cq = int(O.query_codes(q, A)[0])
    assert cq == g["query_code"]
    assert list(O.matches(idx, cq)) == g["matches"]
    H = O.histogram(idx, cq)
    assert H.tolist() == g["histogram"]
    for case in g["budget_cases"]:
        lam, js, ls, r, full = O.threshold(idx, H, case["B"])
        assert lam == case["lam"] and [js, ls] == case["boundary"]
        assert r == case["r"] and full == case["full"]
        rep = O.candidates_reported(idx, cq, case["B"])
        assert list(rep) == case["candidates_reported"]
        ids, sc = O.query(idx, q, case["topk_k"], case["B"])
        assert list(ids[0]) == case["topk_ids"]
        assert [float(v) for v in sc[0]] == [float(v) for v in case["topk_scores"]]


def test_workload_generator_shapes_and_determinism():
    w = W.make_workload("small-n10k-d64", n=500, nq=20)
    assert w.items.shape == (500, 64) and w.items.dtype == np.float32
    assert w.queries.shape == (20, 64)
    assert np.allclose(np.linalg.norm(w.queries, axis=1), 1.0, atol=1e-6)
    part = W.gen_items(500, 64, w.item_seed, w.norm_dist, w.norm_param, "f32",
                       rows=slice(100, 300), chunk=64)
    assert np.array_equal(part, w.items[100:300])
    wb = W.make_workload("imagenet-n2340373-d150", n=300, nq=4)
    assert wb.items.dtype == np.uint16
    x = W.items_to_f64(wb.items, "bf16")
    assert np.all(np.linalg.norm(x, axis=1) >= 0.99)      # Pareto norms are >= 1


def test_query_code_bits_on_the_hyperplanes_are_exact_signs():
    """Eq. 4 on P(q) = [q; 0] at and next to a_b^T q = 0: queries whose in-order
    partial sums are exact, so the canonical FP64 sum has the sign of the exact
    rational value, [0 >= 0] = 1 included."""
    d, L = 40, 32
    A = philox.projections(9, d, L)
    rng = np.random.default_rng(11)
    for b in (0, 5, 31):
        for r in (0.0, 2.0 ** -60, 2.0 ** -42, 2.0 ** -30):
            for sign in (1.0, -1.0):
                k1, k2, k3 = sorted(rng.choice(d, 3, replace=False))
                q = np.zeros(d)
                q[k1], q[k2] = A[k2, b], -A[k1, b]
                scale = np.linalg.norm(q) * np.linalg.norm(A[:d, b])
                q[k3] = np.float32(sign * r * scale / A[k3, b])
                exact_val = sum(Fraction(float(q[k])) * Fraction(float(A[k, b])) for k in range(d))
                bit = (int(O.query_codes(q[None, :], A)[0]) >> b) & 1
                assert bit == int(exact_val >= 0), (b, r, sign)
                if r == 0.0:
                    assert exact_val == 0 and bit == 1

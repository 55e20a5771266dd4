"""Pins of the multi-table single-probe oracle (Algorithm 2 with T tables of
L/T bits each) against the multi-probe oracle's histograms, a pure-Python
restatement with integer bit operations, the collision law of Eq. 4 per table,
and Algorithm 2's per-sub-dataset structure."""
import math

import numpy as np
import pytest

from oracle import multitable as MT, nrlsh as O, philox


def rand_items(n, d, seed, sigma=1.0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return (x * rng.lognormal(0, sigma, n)[:, None]).astype(np.float32).astype(np.float64)


def rand_queries(nq, d, seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((nq, d))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def small():
    X = rand_items(500, 12, 1)
    return X, O.build(X, 8, 16, seed=2, eps=0.2)


def test_one_table_is_the_exact_match_class(small):
    X, idx = small
    for q in rand_queries(10, 12, 3):
        cq = int(O.query_codes(q[None, :], idx.A)[0])
        cand = MT.candidates(idx, cq, 1)
        H = O.histogram(idx, cq)
        assert cand.size == H[:, idx.L].sum()
        assert set(cand.tolist()) == set(np.flatnonzero(O.matches(idx, cq) == idx.L).tolist())


def test_one_bit_tables_are_any_identical_bit(small):
    X, idx = small
    for q in rand_queries(10, 12, 4):
        cq = int(O.query_codes(q[None, :], idx.A)[0])
        cand = MT.candidates(idx, cq, idx.L)
        assert set(cand.tolist()) == set(np.flatnonzero(O.matches(idx, cq) >= 1).tolist())


@pytest.mark.parametrize("T", [1, 2, 4, 8, 16])
def test_against_integer_bit_loops(small, T):
    """Independent restatement: Python integers, shifts and masks, one table at a
    time; candidates in (sub-dataset, id) order."""
    X, idx = small
    Lt = idx.L // T
    for q in rand_queries(6, 12, 5 + T):
        cq = int(O.query_codes(q[None, :], idx.A)[0])
        hits = []
        for i in range(idx.n):
            cx = int(idx.codes[i])
            if any(((cx >> (t * Lt)) & ((1 << Lt) - 1)) == ((cq >> (t * Lt)) & ((1 << Lt) - 1))
                   for t in range(T)):
                hits.append((int(idx.sub[i]), i))
        assert MT.candidates(idx, cq, T).tolist() == [i for _, i in sorted(hits)]


def test_table_collision_rate_is_p_to_the_table_length():
    """Eq. 4 per table: all L_t bits of a table agree with probability
    (1 - theta/pi)^L_t for two directions at angle theta (independent columns)."""
    d, L, Lt = 12, 64, 4
    rng = np.random.default_rng(31)
    for theta in (0.4, 1.0):
        u = rng.standard_normal(d); u /= np.linalg.norm(u)
        w = rng.standard_normal(d); w -= (w @ u) * u; w /= np.linalg.norm(w)
        y = math.cos(theta) * u + math.sin(theta) * w
        same = trials = 0
        for seed in range(20_000, 20_000 + 400):
            A = philox.projections(seed, d - 1, L)
            codes = O.pack_bits(np.stack([u, y]) @ A >= 0.0)
            f = MT.table_fields(codes, L // Lt, L)
            same += int((f[0] == f[1]).sum())
            trials += L // Lt
        p = (1 - theta / math.pi) ** Lt
        sigma = math.sqrt(p * (1 - p) / trials)
        assert abs(same / trials - p) < 5 * sigma, (theta, same / trials, p)


def test_answer_is_the_best_of_the_subdataset_answers(small):
    """Algorithm 2: the top-1 of the union is the best x*_j over the sub-datasets."""
    X, idx = small
    Q = rand_queries(12, 12, 7)
    ids, _, probed = MT.query(idx, Q, 1, 4)
    cqs = O.query_codes(Q, idx.A)
    for i in range(12):
        best = [b for b in MT.per_subdataset_best(idx, Q[i], int(cqs[i]), 4) if b is not None]
        if not best:
            assert probed[i] == 0 and ids[i, 0] == -1
            continue
        sc = O.scores_fp64(X[best], Q[i])
        top, _ = O.topk(np.array(best), sc, 1)
        assert ids[i, 0] == top[0]


def test_cap_truncates_in_storage_order_and_reports_the_full_count(small):
    X, idx = small
    Q = rand_queries(8, 12, 9)
    ids_full, _, probed = MT.query(idx, Q, 5, 16)
    ids_cap, sc_cap, probed_cap = MT.query(idx, Q, 5, 16, cap=20)
    assert np.array_equal(probed, probed_cap)
    cqs = O.query_codes(Q, idx.A)
    for i in range(8):
        cand = MT.candidates(idx, int(cqs[i]), 16)[:20]
        ref_ids, ref_sc = O.topk(cand, O.scores_fp64(X[cand], Q[i]), 5)
        assert np.array_equal(ids_cap[i], ref_ids) and np.array_equal(sc_cap[i], ref_sc)
        if probed[i] <= 20:
            assert np.array_equal(ids_cap[i], ids_full[i])


def test_more_tables_probe_more_and_recall_more():
    X = rand_items(3000, 16, 11)
    idx = O.build(X, 16, 64, seed=12, eps=0.2)
    Q = rand_queries(40, 16, 13)
    from oracle import exact
    truth = [set(exact.exact_topk(X, q, 10).tolist()) for q in Q]
    prev_probed, prev_rec = -1.0, -1.0
    for T in (1, 2, 4, 8):            # tables of 64 / T bits: fewer bits, more tables
        ids, _, probed = MT.query(idx, Q, 10, T)
        rec = np.mean([len(set(ids[i].tolist()) & truth[i]) / 10 for i in range(40)])
        assert probed.mean() >= prev_probed and rec >= prev_rec - 1e-12
        prev_probed, prev_rec = probed.mean(), rec


def test_bad_table_count():
    with pytest.raises(ValueError):
        MT.table_fields(np.zeros(3, np.uint64), 3, 16)
    with pytest.raises(ValueError):
        MT.table_fields(np.zeros(3, np.uint64), 0, 16)

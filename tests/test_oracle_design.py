"""Pins for oracle.design: Thm 2.2 optimality, eq. 3.10, eq. 4.2 optimality, apportionment."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic as S


def _design_inputs(seed=0, m=9, n=40, p=7, K=5):
    off = S.block_offsets_uneven(n, K, 4, 12, seed=seed)
    M, N = S.scaled_gaussian(m, n, p, off, 1.0, seed=seed + 1)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    return off, M, N, x, y, st, f


def _variance(x, y, p, off, ck, f):
    # summed variance of Remark 2.2 with real c_k
    return oracle.expected_sq_error_alg2(x, y, p, off, ck, f)


def test_probabilities_sum_to_one():
    off, M, N, x, y, st, f = _design_inputs()
    for p in (oracle.p_col_opt(st["w"], st["a"], off), oracle.p_col_uniform(off)):
        for a, b in zip(off[:-1], off[1:]):
            assert abs(p[a:b].sum() - 1.0) < 1e-14
    for p in (oracle.p_blk_prodnorm(f), oracle.p_blk_normprod(st["mf"], st["nf"])):
        assert abs(p.sum() - 1.0) < 1e-14 and np.all(p >= 0)


def test_eq_1_4_equals_product_of_block_norms():
    off, M, N, x, y, st, f = _design_inputs(seed=3)
    nm = np.array([np.linalg.norm(M[:, a:b]) for a, b in zip(off[:-1], off[1:])])
    nn = np.array([np.linalg.norm(N[a:b, :]) for a, b in zip(off[:-1], off[1:])])
    np.testing.assert_allclose(oracle.p_blk_normprod(st["mf"], st["nf"]), nm * nn / np.sum(nm * nn), rtol=1e-13)
    fr = np.array([np.linalg.norm(M[:, a:b] @ N[a:b, :]) for a, b in zip(off[:-1], off[1:])])
    np.testing.assert_allclose(oracle.p_blk_prodnorm(f), fr / fr.sum(), rtol=1e-12)


def test_zero_block_gets_uniform_probabilities():
    off = np.array([0, 3, 6])
    M = np.ones((2, 6))
    M[:, 3:] = 0.0
    N = np.ones((6, 2))
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    np.testing.assert_allclose(p[3:], 1.0 / 3)


def test_eq_3_8_minimises_summed_variance_for_any_block_sizes():
    # Thm 2.2, first inequality: for fixed c_k, p_{k_i} proportional to w_i is optimal
    off, M, N, x, y, st, f = _design_inputs(seed=4)
    rng = np.random.default_rng(0)
    ck = rng.uniform(1.0, 5.0, size=len(off) - 1)
    p_opt = oracle.p_col_opt(st["w"], st["a"], off)
    v_opt = _variance(x, y, p_opt, off, ck, f)
    for _ in range(200):
        q = p_opt * np.exp(0.3 * rng.standard_normal(len(p_opt)))
        for a, b in zip(off[:-1], off[1:]):
            q[a:b] /= q[a:b].sum()
        assert _variance(x, y, q, off, ck, f) >= v_opt * (1 - 1e-12)
    # the uniform choice is never better
    assert _variance(x, y, oracle.p_col_uniform(off), off, ck, f) >= v_opt


def test_eq_3_9_minimises_and_attains_eq_3_10():
    # Thm 2.2 second inequality and Remark 2.3
    off, M, N, x, y, st, f = _design_inputs(seed=5)
    c = 17.0
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = oracle.real_block_sizes(oracle.g_opt(st["a"], f), c)
    v_opt = _variance(x, y, p, off, ck, f)
    np.testing.assert_allclose(v_opt, oracle.optimal_value_eq310(st["a"], f, c), rtol=1e-11)
    rng = np.random.default_rng(1)
    for _ in range(300):
        d = ck * np.exp(0.4 * rng.standard_normal(len(ck)))
        d *= c / d.sum()
        assert _variance(x, y, p, off, d, f) >= v_opt * (1 - 1e-12)
    # eq. 4.2 and c/K are feasible but not better
    for g in (oracle.g_hat(st["a"]), oracle.g_equal(len(ck))):
        assert _variance(x, y, p, off, oracle.real_block_sizes(g, c), f) >= v_opt * (1 - 1e-12)


def test_eq_4_2_minimises_the_upper_bound_4_1():
    # the bound drops the -f_k/c_k term: sum_k (1/c_k) sum_i x_i y_i / p_{k_i} = sum_k a_k^2 / c_k
    off, M, N, x, y, st, f = _design_inputs(seed=6)
    c = 11.0
    p = oracle.p_col_opt(st["w"], st["a"], off)
    zero = np.zeros(len(off) - 1)
    ch = oracle.real_block_sizes(oracle.g_hat(st["a"]), c)
    u_opt = _variance(x, y, p, off, ch, zero)
    np.testing.assert_allclose(u_opt, st["a"].sum() ** 2 / c, rtol=1e-12)
    rng = np.random.default_rng(2)
    for _ in range(300):
        d = ch * np.exp(0.4 * rng.standard_normal(len(ch)))
        d *= c / d.sum()
        assert _variance(x, y, p, off, d, zero) >= u_opt * (1 - 1e-12)


def test_g_weights_and_fallback():
    a = np.array([3.0, 4.0, 0.0])
    f = np.array([5.0, 16.0, 0.0])
    np.testing.assert_allclose(oracle.g_opt(a, f), [2.0, 0.0, 0.0])
    np.testing.assert_allclose(oracle.g_tilde(a, np.array([13.0, 16.0, 1.0])), [2.0, 0.0, 1.0])
    np.testing.assert_allclose(oracle.g_hat(a), a)
    # every block rank-one aligned: g = 0 everywhere -> a_k; a = 0 too -> n_k
    np.testing.assert_allclose(oracle.g_with_fallback(np.zeros(3), a, [2, 2, 2]), a)
    np.testing.assert_allclose(oracle.g_with_fallback(np.zeros(3), np.zeros(3), [2, 5, 1]), [2, 5, 1])


# ---------------------------------------------------------------- apportionment

def _dhondt(g, nk, c):
    """Highest averages with exact rationals: a first draw for every block, cap n_k, ties -> smaller k."""
    K = len(g)
    s = [1] * K
    G = [Fraction(float(v)) for v in g]
    for _ in range(c - K):
        best, bk = None, None
        for k in range(K):
            if s[k] >= nk[k]:
                continue
            qv = G[k] / (s[k] + 1)
            if best is None or qv > best:
                best, bk = qv, k
        s[bk] += 1
    return np.array(s)


def test_apportion_hand_example():
    # c g / sum g = 7 * [0.6, 0.3, 0.1] = [4.2, 2.1, 0.7] -> [4, 2, 1]
    assert list(oracle.apportion([6.0, 3.0, 1.0], [4, 4, 4], 7)) == [4, 2, 1]
    # exact ties go to the smaller index: seats (1,1,1) then 1/2 = 1/2 = 1/2
    assert list(oracle.apportion([1.0, 1.0, 1.0], [3, 3, 3], 5)) == [2, 2, 1]
    # the cap binds: block 0 wants 9 of 10 but holds only 3
    assert list(oracle.apportion([100.0, 1.0, 1.0], [3, 10, 10], 10)) == [3, 4, 3]


def test_apportion_matches_exact_highest_averages():
    rng = np.random.default_rng(7)
    for trial in range(120):
        K = int(rng.integers(1, 12))
        nk = rng.integers(1, 9, size=K)
        n = int(nk.sum())
        c = int(rng.integers(K, n + 1))
        g = rng.lognormal(0.0, 1.5, size=K)
        if trial % 5 == 0:
            g[rng.random(K) < 0.3] = 0.0
            if not np.any(g > 0):
                g[0] = 1.0
        ck = oracle.apportion(g, nk, c)
        assert ck.sum() == c and np.all(ck >= 1) and np.all(ck <= nk)
        np.testing.assert_array_equal(ck, _dhondt(g, nk, c))


def test_apportion_extremes_and_errors():
    nk = np.array([3, 5, 2])
    assert list(oracle.apportion([1.0, 2.0, 3.0], nk, 3)) == [1, 1, 1]
    assert list(oracle.apportion([1.0, 2.0, 3.0], nk, 10)) == [3, 5, 2]
    assert list(oracle.apportion([0.0, 2.0, 0.0], nk, 10)) == [3, 5, 2]
    with pytest.raises(oracle.InfeasibleBudget):
        oracle.apportion([1.0, 1.0, 1.0], nk, 2)
    with pytest.raises(oracle.InfeasibleBudget):
        oracle.apportion([1.0, 1.0, 1.0], nk, 11)
    with pytest.raises(ValueError):
        oracle.apportion([1.0, np.nan, 1.0], nk, 5)


def test_apportion_tracks_real_sizes():
    # unclamped, a divisor method meets lower quota: c_k >= floor(c g_k / sum g),
    # and c_k <= lam* g_k + 1 with lam* < (c + K) / sum g
    rng = np.random.default_rng(8)
    K = 64
    g = rng.uniform(1.0, 2.0, size=K)
    nk = np.full(K, 1000)
    c = 3000
    ck = oracle.apportion(g, nk, c)
    real = oracle.real_block_sizes(g, c)
    assert np.all(ck >= np.floor(real))
    assert np.all(ck <= (c + K) * g / g.sum() + 1.0)


def test_apportion_is_house_monotone():
    """A divisor method never takes a draw away from a block when the budget grows: c_k(c + 1) >=
    c_k(c) for every block, one block gaining exactly one, over every budget from K to n (weights with
    ties, zeros and blocks that reach their cap n_k).  A wrong bisection bound, a remainder handed to
    blocks that do not grow at the next lambda, or a cap applied after the remainder would break it."""
    rng = np.random.default_rng(21)
    for trial in range(6):
        K = 7
        nk = rng.integers(1, 9, size=K)
        g = rng.choice([0.0, 0.5, 1.0, 1.0, 2.5, 7.0], size=K)
        if trial == 0:
            g[:] = 1.0  # all tied
        prev = oracle.apportion(g, nk, K)
        assert np.all(prev == 1)
        for c in range(K + 1, int(nk.sum()) + 1):
            cur = oracle.apportion(g, nk, c)
            assert cur.sum() == c and np.all(cur <= nk), (trial, c)
            d = cur - prev
            assert np.all(d >= 0) and d.sum() == 1, (trial, c, prev, cur)
            prev = cur
        assert np.array_equal(prev, nk)

"""Pins for oracle.estimator: exact enumeration of all sampling outcomes, special cases,
Monte Carlo against the closed form, the bounds of Thm 2.3 / Thm 3.2."""
import itertools

import numpy as np
import pytest

import oracle
import synthetic as S


def _enumerate_alg2(M, N, off, p, ck):
    """Every outcome of Alg. 2 with its probability: returns E[CD] and E||MN - CD||^2."""
    MN = M @ N
    per_block = []
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        outcomes = []
        for draw in itertools.product(range(a, b), repeat=int(ck[k])):
            pr = np.prod([p[i] for i in draw])
            if pr == 0:
                continue
            est = sum(np.outer(M[:, i], N[i, :]) / (ck[k] * p[i]) for i in draw)
            outcomes.append((pr, est))
        per_block.append(outcomes)
    mean = np.zeros_like(MN)
    sq = 0.0
    for combo in itertools.product(*per_block):
        pr = np.prod([c[0] for c in combo])
        CD = sum(c[1] for c in combo)
        mean += pr * CD
        sq += pr * np.sum((MN - CD) ** 2)
    return mean, sq


def _tiny(seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((3, 5))
    N = rng.standard_normal((5, 2))
    off = np.array([0, 2, 5])
    return M, N, off


@pytest.mark.parametrize("kind", ["opt", "random"])
def test_alg2_unbiased_and_exact_error_by_enumeration(kind):
    # Lemma 2.1 (E[CD] = MN) and Remark 2.2 (sum of variances = E||MN - CD||^2)
    M, N, off = _tiny(1)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    if kind == "opt":
        p = oracle.p_col_opt(st["w"], st["a"], off)
    else:
        p = S.random_probabilities(off, seed=2)
    ck = np.array([2, 2])
    mean, sq = _enumerate_alg2(M, N, off, p, ck)
    np.testing.assert_allclose(mean, M @ N, rtol=1e-12, atol=1e-12)
    f = oracle.block_frob_sq(M, N, off)
    np.testing.assert_allclose(oracle.expected_sq_error_alg2(x, y, p, off, ck, f), sq, rtol=1e-11)


def test_block_sampling_unbiased_and_exact_error_by_enumeration():
    M, N, off = _tiny(3)
    f = oracle.block_frob_sq(M, N, off)
    MN = M @ N
    for pblk in (oracle.p_blk_prodnorm(f), np.array([0.3, 0.7])):
        c = 3
        mean = np.zeros_like(MN)
        sq = 0.0
        for draw in itertools.product(range(2), repeat=c):
            pr = np.prod(pblk[list(draw)])
            CD = oracle.sampled_product_blocks(M, N, off, np.array(draw), 1.0 / (c * pblk[list(draw)]))
            mean += pr * CD
            sq += pr * np.sum((MN - CD) ** 2)
        np.testing.assert_allclose(mean, MN, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(oracle.expected_sq_error_blocks(f, pblk, c, np.sum(MN ** 2)), sq, rtol=1e-11)


def test_every_index_once_with_unit_scale_is_exact():
    # eq. 2.3: MN = sum_k sum_i M^{k(i)} N_{k(i)}
    rng = np.random.default_rng(4)
    M = rng.standard_normal((6, 9))
    N = rng.standard_normal((9, 4))
    CD = oracle.sampled_product_columns(M, N, np.arange(9), np.ones(9))
    np.testing.assert_allclose(CD, M @ N, rtol=1e-13, atol=1e-13)
    off = np.array([0, 4, 9])
    CD = oracle.sampled_product_blocks(M, N, off, np.array([0, 1]), np.ones(2))
    np.testing.assert_allclose(CD, M @ N, rtol=1e-13, atol=1e-13)


def test_unit_blocks_reproduce_the_product():
    # n_k = 1 for all k and c = n: one draw per block with p = 1 and scale 1
    rng = np.random.default_rng(5)
    M = rng.standard_normal((4, 6))
    N = rng.standard_normal((6, 3))
    off = np.arange(7)
    for method in ("OPL", "ONC", "UU"):
        r = oracle.run_method(M, N, off, method, 6, seed=1)
        np.testing.assert_array_equal(r["ck"], np.ones(6))
        np.testing.assert_allclose(r["CD"], M @ N, rtol=1e-13, atol=1e-13)
        assert oracle.expected_sq_error_alg2(r["x"], r["y"], r["p"], off, r["ck"], oracle.block_frob_sq(M, N, off)) == pytest.approx(0.0, abs=1e-12)


def test_single_block_is_algorithm_1():
    # K = 1: p_i = ||M^(i)|| ||N_(i)|| / sum (eq. 1.1) and C^(t) = M^(i_t) / sqrt(c p_{i_t}) (Alg. 1)
    rng = np.random.default_rng(6)
    M = rng.standard_normal((5, 8))
    N = rng.standard_normal((8, 4))
    off = np.array([0, 8])
    r = oracle.run_method(M, N, off, "ONC", 6, seed=2)
    w = np.linalg.norm(M, axis=0) * np.linalg.norm(N, axis=1)
    np.testing.assert_allclose(r["p"], w / w.sum(), rtol=1e-13)
    assert list(r["ck"]) == [6]
    C = M[:, r["idx"]] / np.sqrt(6 * r["p"][r["idx"]])
    D = N[r["idx"], :] / np.sqrt(6 * r["p"][r["idx"]])[:, None]
    np.testing.assert_allclose(r["CD"], C @ D, rtol=1e-12)


def test_rank_one_aligned_block_has_zero_variance():
    # v_k = 1 (M^k and N_k rank one and aligned) -> g_k = 0 -> one draw, zero error in that block
    rng = np.random.default_rng(7)
    u, r_ = rng.standard_normal(4), rng.standard_normal(3)
    v = np.abs(rng.standard_normal(3)) + 0.1
    M = np.zeros((4, 6))
    N = np.zeros((6, 3))
    M[:, :3] = np.outer(u, v)
    N[:3, :] = np.outer(v, r_)
    M[:, 3:] = rng.standard_normal((4, 3))
    N[3:, :] = rng.standard_normal((3, 3))
    off = np.array([0, 3, 6])
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    g = oracle.g_opt(st["a"], f)
    assert g[0] < 1e-6 * st["a"][0]
    p = oracle.p_col_opt(st["w"], st["a"], off)
    # every draw from block 0 reproduces M^0 N_0 exactly
    for i in range(3):
        np.testing.assert_allclose(np.outer(M[:, i], N[i, :]) / p[i], M[:, :3] @ N[:3, :], rtol=1e-12)


def test_monte_carlo_matches_closed_form_small_config():
    """1000 seeds of the small FP64 configuration (256x4096x256, K=64, c=16 blocks -> L=1024)."""
    off = S.block_offsets_equal(4096, 64)
    M, N = S.scaled_gaussian(256, 4096, 256, off, 1.0, seed=1)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    nk = np.diff(off)
    L = oracle.equal_budget(16, 4096, 64)
    assert L == 1024
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = oracle.apportion(oracle.g_opt(st["a"], f), nk, L)
    E = oracle.expected_sq_error_alg2(x, y, p, off, ck, f)
    MN = M @ N
    errs = np.empty(1000)
    for s in range(1000):
        idx, scale = oracle.sample_alg2(p, off, ck, seed=s, sid=0)
        errs[s] = np.sum((MN - oracle.sampled_product_columns(M, N, idx, scale)) ** 2)
    se = errs.std(ddof=1) / np.sqrt(len(errs))
    assert abs(errs.mean() - E) < 4 * se, (errs.mean(), E, se)
    # the RMS relative error sits at the closed form's value
    assert np.sqrt(errs.mean()) <= 1.05 * np.sqrt(E)


def test_bounds_eq_3_11_and_4_3():
    off = S.block_offsets_equal(240, 6)
    M, N = S.scaled_gaussian(12, 240, 10, off, 1.0, seed=8)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    c = 40.0
    mf2, nf2 = np.sum(M ** 2), np.sum(N ** 2)
    v_opt = oracle.expected_sq_error_alg2(x, y, p, off, oracle.real_block_sizes(oracle.g_opt(st["a"], f), c), f)
    assert v_opt <= oracle.bound_eq311(st["a"], f, mf2, nf2, c) * (1 + 1e-12)
    v_hat = oracle.expected_sq_error_alg2(x, y, p, off, oracle.real_block_sizes(oracle.g_hat(st["a"]), c), f)
    assert v_hat <= oracle.bound_eq43(st["a"], f, mf2, nf2, c) * (1 + 1e-12)


def test_pilot_estimate_expectation_by_enumeration():
    # Alg. 3 step 1: E||C^{0k} D_{0k}||^2 = ||M^k N_k||^2 + E||M^k N_k - C^{0k} D_{0k}||^2
    M, N, off = _tiny(9)
    p0 = oracle.p_col_uniform(off)
    x, y = oracle.col_row_sq_norms(M, N)
    f = oracle.block_frob_sq(M, N, off)
    c0p = 2
    for k in range(2):
        a, b = off[k], off[k + 1]
        mean_sq = 0.0
        for draw in itertools.product(range(a, b), repeat=c0p):
            pr = np.prod(p0[list(draw)])
            P = sum(np.outer(M[:, i], N[i, :]) / (c0p * p0[i]) for i in draw)
            mean_sq += pr * np.sum(P ** 2)
        var = (np.sum(x[a:b] * y[a:b] / p0[a:b]) - f[k]) / c0p
        np.testing.assert_allclose(mean_sq, f[k] + var, rtol=1e-11)
    # and the oracle's pilot uses exactly c0' draws per block with scale 1/(c0' p0)
    fhat, idx, scale = oracle.pilot_frob_sq(M, N, off, p0, c0p, seed=4, sid=1)
    for k in range(2):
        sl = slice(2 * k, 2 * k + 2)
        assert np.all((idx[sl] >= off[k]) & (idx[sl] < off[k + 1]))
        P = oracle.sampled_product_columns(M, N, idx[sl], scale[sl])
        np.testing.assert_allclose(fhat[k], np.sum(P ** 2), rtol=1e-13)


def test_methods_run_and_respect_budget():
    off = S.block_offsets_uneven(400, 10, 20, 60, seed=1)
    M, N = S.scaled_gaussian(20, 400, 15, off, 1.5, seed=2)
    for method in oracle.METHODS:
        c = 80 if method not in ("SSM", "WU") else 4
        r = oracle.run_method(M, N, off, method, c, seed=3, c0=40)
        assert len(r["idx"]) == c
        if "ck" in r:
            assert r["ck"].sum() == c and np.all(r["ck"] >= 1) and np.all(r["ck"] <= np.diff(off))


def test_repeated_draws_are_one_term_each():
    """eq. 3.2 with repeats: every draw of index i carries the same scale 1/(c_k p_i), so the sum over
    the draws equals the sum over the distinct indices with weight multiplicity x scale (the form
    the apply computes); the same for block draws (1/(c p_k))."""
    off = S.block_offsets_uneven(600, 8, 40, 110, seed=3)
    M, N = S.scaled_gaussian(20, 600, 14, off, 1.0, seed=4)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = oracle.apportion(oracle.g_hat(st["a"]), np.diff(off), 300)
    idx, scale = oracle.sample_alg2(p, off, ck, 5, 0)
    ui, inv, cnt = np.unique(idx, return_inverse=True, return_counts=True)
    assert cnt.max() > 1
    us = np.zeros(len(ui))
    us[inv] = scale
    assert np.all(us[inv] == scale)  # one scale per index
    a = oracle.sampled_product_columns(M, N, idx, scale)
    b = oracle.sampled_product_columns(M, N, ui, cnt * us)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())
    pblk = oracle.p_blk_normprod(st["mf"], st["nf"])
    kidx, ks = oracle.sample_blocks(pblk, 20, 6, 0)
    uk, kinv, kcnt = np.unique(kidx, return_inverse=True, return_counts=True)
    assert kcnt.max() > 1
    uks = np.zeros(len(uk))
    uks[kinv] = ks
    a = oracle.sampled_product_blocks(M, N, off, kidx, ks)
    b = oracle.sampled_product_blocks(M, N, off, uk, kcnt * uks)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_block_draws_carry_their_scale():
    """The block sampler's draws through the estimator of eq. 1.2 / 1.4: (i) when every block but one
    has M^k N_k = 0, eq. 1.2 puts all mass on that block and any c draws reproduce MN exactly (zero
    variance); (ii) over many seeds the mean of the sampled products approaches MN (Lemma 2.1) for
    eq. 1.2 and eq. 1.4 probabilities, within five standard errors of the closed-form variance."""
    rng = np.random.default_rng(17)
    m, n, p, K = 6, 12, 5, 3
    off = np.array([0, 4, 9, 12])
    M = rng.standard_normal((m, n))
    N = rng.standard_normal((n, p))
    M1 = M.copy()
    M1[:, :4] = 0.0
    M1[:, 9:] = 0.0  # only block 1 carries the product
    f1 = oracle.block_frob_sq(M1, N, off)
    pblk = oracle.p_blk_prodnorm(f1)
    assert pblk[1] == 1.0
    for c in (1, 4, 7):
        idx, scale = oracle.sample_blocks(pblk, c, seed=5, sid=0)
        assert np.all(idx == 1)
        np.testing.assert_allclose(oracle.sampled_product_blocks(M1, N, off, idx, scale), M1 @ N, rtol=1e-13,
                                   atol=1e-13)
    MN = M @ N
    f = oracle.block_frob_sq(M, N, off)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    c, seeds = 3, 3000
    for pb in (oracle.p_blk_prodnorm(f), oracle.p_blk_normprod(st["mf"], st["nf"])):
        acc = np.zeros_like(MN)
        for sd in range(seeds):
            idx, scale = oracle.sample_blocks(pb, c, seed=sd, sid=0)
            acc += oracle.sampled_product_blocks(M, N, off, idx, scale)
        var = oracle.expected_sq_error_blocks(f, pb, c, float(np.sum(MN ** 2)))  # summed over entries
        err = np.sqrt(np.sum((acc / seeds - MN) ** 2))
        assert err <= 5.0 * np.sqrt(var / seeds), (err, np.sqrt(var / seeds))

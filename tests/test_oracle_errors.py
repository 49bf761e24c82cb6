"""Pins for oracle.errors: the per-entry variance of eq. 3.7 and its one-sample estimate against
exact enumeration of every sampling outcome, the whole-matrix report against Remark 2.2, the
bounds of Thm 3.3 / Thm 4.2, the special case of Remark 4.4 and the ordering of Remark 4.6."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic as S


def _tiny(seed, m=3, p=2):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((m, 5))
    N = rng.standard_normal((5, p))
    off = np.array([0, 2, 5])
    return M, N, off


def _all_entries(m, p):
    return np.array([(h, f) for h in range(m) for f in range(p)], dtype=np.int64)


def _alg2_outcomes(off, p, ck):
    """Every outcome of Alg. 2 (draws of all blocks, in block order) with its probability."""
    per_block = []
    for k in range(len(off) - 1):
        per_block.append([(np.prod([p[i] for i in d]), d) for d in
                          itertools.product(range(off[k], off[k + 1]), repeat=int(ck[k]))])
    for combo in itertools.product(*per_block):
        pr = np.prod([c[0] for c in combo])
        if pr == 0:
            continue
        idx = np.concatenate([np.array(c[1], dtype=np.int64) for c in combo])
        ckd = np.concatenate([np.full(int(ck[k]), ck[k]) for k in range(len(ck))])
        yield pr, idx, 1.0 / (ckd * p[idx])


@pytest.mark.parametrize("kind", ["opt", "random"])
def test_entry_variance_is_the_exact_variance_by_enumeration(kind):
    # Lemma 3.1: E[(CD)_hf] = (MN)_hf (eq. 3.6) and Var[(CD)_hf] = eq. 3.7, over all 108 outcomes
    M, N, off = _tiny(11)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off) if kind == "opt" else S.random_probabilities(off, seed=12)
    ck = np.array([2, 3])
    ent = _all_entries(3, 2)
    mean = np.zeros((3, 2))
    second = np.zeros((3, 2))
    for pr, idx, scale in _alg2_outcomes(off, p, ck):
        CD = oracle.sampled_product_columns(M, N, idx, scale)
        mean += pr * CD
        second += pr * CD * CD
    var = second - mean * mean
    np.testing.assert_allclose(mean, M @ N, rtol=1e-12, atol=1e-12)
    got = oracle.entry_variance_columns(M, N, off, p, ck, ent)
    np.testing.assert_allclose(got, var[ent[:, 0], ent[:, 1]], rtol=1e-10, atol=1e-13)


def test_entry_variances_sum_to_the_expected_squared_error():
    # Remark 2.2: sum over all entries of sigma^2 = E||MN - CD||_F^2
    off = S.block_offsets_uneven(96, 6, 4, 30, seed=3)
    M, N = S.scaled_gaussian(7, 96, 5, off, 1.0, seed=4)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.array([3, 1, 4, 2, 5, 2])
    f = oracle.block_frob_sq(M, N, off)
    total = oracle.entry_variance_columns(M, N, off, p, ck, _all_entries(7, 5)).sum()
    np.testing.assert_allclose(total, oracle.expected_sq_error_alg2(x, y, p, off, ck, f), rtol=1e-11)


def test_entry_estimate_is_unbiased_by_enumeration():
    # E[one-sample estimate] = sigma^2 exactly when every c_k >= 2; the value part is (CD)_hf
    M, N, off = _tiny(13)
    p = S.random_probabilities(off, seed=14)
    ck = np.array([2, 3])
    ent = _all_entries(3, 2)
    e_s2 = np.zeros(len(ent))
    for pr, idx, scale in _alg2_outcomes(off, p, ck):
        cd, s2, unest = oracle.entry_estimate_columns(M, N, off, ck, idx, scale, ent)
        assert unest == 0
        CD = oracle.sampled_product_columns(M, N, idx, scale)
        np.testing.assert_allclose(cd, CD[ent[:, 0], ent[:, 1]], rtol=1e-12, atol=1e-12)
        e_s2 += pr * s2
    np.testing.assert_allclose(e_s2, oracle.entry_variance_columns(M, N, off, p, ck, ent), rtol=1e-10, atol=1e-13)


def test_entry_estimate_counts_single_draw_blocks():
    M, N, off = _tiny(15)
    p = S.random_probabilities(off, seed=16)
    ck = np.array([1, 3])
    idx = np.array([1, 2, 4, 4])
    scale = 1.0 / (np.array([1, 3, 3, 3]) * p[idx])
    cd, s2, unest = oracle.entry_estimate_columns(M, N, off, ck, idx, scale, [(0, 0), (2, 1)])
    assert unest == 1
    # block 0 adds its value but no variance: the estimate equals the one of block 1 alone
    _, s2_b1, _ = oracle.entry_estimate_columns(M[:, 2:], N[2:, :], off[1:] - 2, ck[1:], idx[1:] - 2, scale[1:],
                                                [(0, 0), (2, 1)])
    np.testing.assert_allclose(s2, s2_b1, rtol=1e-14)


def test_block_draws_variance_and_estimate_by_enumeration():
    # c i.i.d. block draws: exact variance and the unbiasedness of the one-sample estimate
    rng = np.random.default_rng(17)
    M = rng.standard_normal((2, 6))
    N = rng.standard_normal((6, 3))
    off = np.array([0, 1, 3, 6])
    ent = _all_entries(2, 3)
    for pblk in (np.array([0.2, 0.5, 0.3]), np.array([0.0, 0.6, 0.4])):
        c = 3
        mean = np.zeros((2, 3))
        second = np.zeros((2, 3))
        e_s2 = np.zeros(len(ent))
        for draw in itertools.product(range(3), repeat=c):
            kidx = np.array(draw)
            pr = np.prod(pblk[kidx])
            if pr == 0:
                continue
            scale = 1.0 / (c * pblk[kidx])
            CD = oracle.sampled_product_blocks(M, N, off, kidx, scale)
            mean += pr * CD
            second += pr * CD * CD
            cd, s2 = oracle.entry_estimate_blocks(M, N, off, kidx, scale, ent)
            np.testing.assert_allclose(cd, CD[ent[:, 0], ent[:, 1]], rtol=1e-12, atol=1e-12)
            e_s2 += pr * s2
        var = (second - mean * mean)[ent[:, 0], ent[:, 1]]
        got = oracle.entry_variance_blocks(M, N, off, pblk, c, ent)
        np.testing.assert_allclose(got, var, rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(e_s2, var, rtol=1e-10, atol=1e-13)


def test_report_matches_remark_2_2_and_the_bounds():
    off = S.block_offsets_equal(240, 6)
    M, N = S.scaled_gaussian(12, 240, 10, off, 1.0, seed=8)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    c = 40
    for g, bound in ((oracle.g_opt(st["a"], f), "eq311"), (oracle.g_hat(st["a"]), "eq43")):
        ck = oracle.real_block_sizes(g, c)  # the real-valued c_k the theorems take
        r = oracle.error_report(x, y, p, off, ck, st["a"], f, st["mf"], st["nf"], c, 0.05)
        assert abs(r["beta"] - 1.0) < 1e-12  # eq. 3.8 probabilities
        np.testing.assert_allclose(r["expected_sq_error"], oracle.expected_sq_error_alg2(x, y, p, off, ck, f),
                                   rtol=1e-12)
        np.testing.assert_allclose(r["m_fro2"] * r["n_fro2"], np.sum(M ** 2) * np.sum(N ** 2), rtol=1e-12)
        assert r["expected_sq_error"] <= r[bound] * (1 + 1e-12)  # Thm 3.3 / Thm 4.2
        assert r["eq312"] >= r["eq311"] and r["eq44"] >= r["eq43"]
        if bound == "eq311":  # eq. 3.10 is the value at the eq. 3.9 sizes
            np.testing.assert_allclose(r["eq310"], r["expected_sq_error"], rtol=1e-11)
    np.testing.assert_allclose(r["eq311"], oracle.bound_eq311(st["a"], f, np.sum(M ** 2), np.sum(N ** 2), c),
                               rtol=1e-12)


def test_report_beta_of_uniform_probabilities():
    # one block with sqrt(x_i y_i) = (2, 1, 1): p* = (1/2, 1/4, 1/4); uniform p = 1/3 gives beta = 2/3
    x = np.array([4.0, 1.0, 1.0])
    y = np.ones(3)
    off = np.array([0, 3])
    r = oracle.error_report(x, y, np.full(3, 1 / 3), off, np.array([2]), np.array([4.0]), None, [6.0], [3.0], 2,
                            0.1)
    assert r["beta"] == pytest.approx(2 / 3, rel=1e-15)
    assert math.isnan(r["eq311"])  # needs f


def test_report_equal_v_special_case_remark_4_4():
    # every block a scaled copy of one block: all v_k equal, theta_1 = theta_2 = theta.  With
    # beta = 1: phi^2 = theta (Thm 3.3), phihat^2 = theta (Thm 4.2), and the probability bounds of
    # eq. 3.12 and eq. 4.4 coincide (Remark 4.4).
    rng = np.random.default_rng(21)
    U = rng.standard_normal((6, 4))
    V = rng.standard_normal((4, 5))
    scales = np.array([0.5, 2.0, 3.0])
    M = np.concatenate([s * U for s in scales], axis=1)
    N = np.concatenate([s * V for s in scales], axis=0)
    off = np.array([0, 4, 8, 12])
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.array([3, 3, 4])
    r = oracle.error_report(x, y, p, off, ck, st["a"], f, st["mf"], st["nf"], 10, 0.05)
    theta = 1.0 - f[0] / st["a"][0] ** 2
    assert r["theta1"] == pytest.approx(theta, rel=1e-12) and r["theta2"] == pytest.approx(theta, rel=1e-12)
    assert r["phi"] ** 2 == pytest.approx(theta, rel=1e-10)
    assert r["phihat"] ** 2 == pytest.approx(theta, rel=1e-10)
    assert r["eq312"] == pytest.approx(r["eq44"], rel=1e-10)
    # the pilot form with exact pilot values (f^ = f) reduces to Thm 3.3
    r2 = oracle.error_report(x, y, p, off, ck, st["a"], f, st["mf"], st["nf"], 10, 0.05, fhat=f)
    assert r2["eq48"] == pytest.approx(r2["eq311"], rel=1e-12) and r2["eq49"] == pytest.approx(r2["eq312"], rel=1e-12)


def test_interval_coverage_monte_carlo():
    # Thm 3.1: with many draws per block the interval (CD)_hf +- 1.96 sigma-hat covers (MN)_hf
    # about 95% of the time (the one-sample sigma-hat in place of sigma)
    off = S.block_offsets_equal(64, 4)
    M, N = S.scaled_gaussian(4, 64, 3, off, 0.5, seed=31)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.array([40, 40, 40, 40])
    ent = _all_entries(4, 3)
    MN = (M @ N)[ent[:, 0], ent[:, 1]]
    hits = 0
    total = 0
    for seed in range(150):
        idx, scale = oracle.sample_alg2(p, off, ck, seed, 0)
        cd, s2, _ = oracle.entry_estimate_columns(M, N, off, ck, idx, scale, ent)
        hits += int(np.sum(np.abs(cd - MN) <= 1.96 * np.sqrt(s2)))
        total += len(ent)
    assert 0.90 <= hits / total <= 0.98, hits / total


def test_report_probability_bounds_orderings():
    # Thm 3.3: eta = phi + (theta2/theta1)^{1/2} (8/beta log 1/delta)^{1/2} with theta1 <= theta2, so the
    # second term is at least the bare (8/beta log 1/delta)^{1/2} of Thm 4.2, with equality only when
    # theta1 = theta2.  Remark 4.6: with pilot values theta2hat > 1 >= theta1hat and 1 - theta2 small,
    # the Thm 4.4 bound (eq. 4.9) is weaker than the Thm 4.2 one (eq. 4.4).
    off = S.block_offsets_equal(320, 8)
    M, N = S.scaled_gaussian(16, 320, 12, off, 1.0, seed=41)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.full(8, 10)
    delta = 0.05
    fhat = f.copy()
    fhat[0] = 2.5 * st["a"][0] ** 2  # |1 - fhat/a^2| = 1.5 > 1
    r = oracle.error_report(x, y, p, off, ck, st["a"], f, st["mf"], st["nf"], 80, delta, fhat=fhat)
    bare = math.sqrt(8.0 / r["beta"] * math.log(1.0 / delta))
    assert r["theta1"] < r["theta2"] <= 1.0
    assert r["eta312"] - r["phi"] > bare * (1 + 1e-12)
    assert r["eta44"] - r["phihat"] == pytest.approx(bare, rel=1e-14)
    assert 1.0 - r["theta2"] < 0.2 and r["theta2hat"] > 1.0 >= r["theta1hat"]
    assert r["eq49"] > r["eq44"]


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "error_report_thm33_thm44.json")


def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_report_hand_worked_example_theta1_ne_theta2_beta_below_one():
    """Every report field against values simplified by hand from Remark 2.2, eq. 3.10, Thm 3.3,
    Thm 4.2 and Thm 4.4 (tests/golden/error_report_thm33_thm44.json): theta_1 = 0.25 != theta_2 = 0.64,
    beta = 0.5 and theta-hat = (0.5, 0.6), so every term of phi and phi-tilde carries weight.  A
    slip such as swapping theta_1 beta and theta_2 theta_1 beta in phi (phi^2 = 1.7125 instead of
    1.4875), or theta-hat_2 for theta_2 in phi-tilde, moves a field far outside the tolerance."""
    fx = _golden()
    i = fx["inputs"]
    r = oracle.error_report(i["x"], i["y"], i["p"], i["offsets"], i["ck"], i["a"], i["f"], i["mf"], i["nf"], i["c"],
                            math.exp(-1.0), fhat=i["fhat"])
    for name, e in fx["expected"].items():
        assert r[name] == pytest.approx(e["value"], rel=1e-13, abs=0.0), name


def test_report_hand_worked_example_discriminates():
    """The example separates the readings a slip would produce: the pinned phi^2 and phi-tilde^2
    differ from the swapped-term and hatted-theta_2 variants by far more than the tolerance."""
    ex = _golden()["expected"]
    assert abs(ex["phi"]["value"] ** 2 - 1.4875) < 1e-14
    assert abs(1.7125 - 1.4875) > 0.2  # theta_1 beta and theta_2 theta_1 beta swapped
    assert abs(ex["phitilde"]["value"] ** 2 * math.sqrt(0.3) - 0.51) < 1e-14
    assert abs(0.50 - 0.51) > 1e-3  # theta-hat_2 in place of theta_2

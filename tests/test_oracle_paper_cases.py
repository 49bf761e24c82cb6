"""The oracle on the inputs of the paper's experiments (Sec. 4): Case I / Case II generators and
the qualitative findings the text states, from the exact closed-form expected errors (Lemma 2.1
applied to Alg. 2 and to block sampling), at a reduced n so that the CPU suite stays fast.

Block sampling (SSM, eq. 1.4) is compared at the same contraction budget: c outer products for
Alg. 2 and round(c K / n) whole blocks for SSM.
"""
import numpy as np
import pytest

import oracle
import synthetic as S

M_ROWS, P_COLS = 26, 28  # m and p of Sec. 4


def _design_errors(M, N, off, c):
    """Relative RMS errors sqrt(E||MN - CD||_F^2) / ||MN||_F of OPL, ONC, UU and SSM."""
    K = len(off) - 1
    n = int(off[-1])
    nk = np.diff(off)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    mn2 = float(np.sum((M @ N) ** 2))
    p_opt = oracle.p_col_opt(st["w"], st["a"], off)
    out = {}
    for name, g, p in (("OPL", oracle.g_opt(st["a"], f), p_opt), ("ONC", oracle.g_hat(st["a"]), p_opt),
                       ("UU", oracle.g_equal(K), oracle.p_col_uniform(off))):
        ck = oracle.apportion(oracle.g_with_fallback(g, st["a"], nk), nk, c)
        out[name] = np.sqrt(oracle.expected_sq_error_alg2(x, y, p, off, ck, f) / mn2)
    cb = max(1, int(round(c * K / n)))
    out["SSM"] = np.sqrt(oracle.expected_sq_error_blocks(f, oracle.p_blk_normprod(st["mf"], st["nf"]), cb, mn2) / mn2)
    return out


def test_case_generators_follow_sec4():
    """Case I columns of M are N(0, S1) with S1 = 0.7^|i-j| and rows of N are N(0, S2) with
    S2 = 2 x 0.7^|i-j|; Case II has location one and heavy (t_1) tails."""
    n = 200000
    M, N = S.paper_case(8, n, 6, case=1, seed=3)
    S1 = 0.7 ** np.abs(np.subtract.outer(np.arange(8), np.arange(8)))
    S2 = 2.0 * 0.7 ** np.abs(np.subtract.outer(np.arange(6), np.arange(6)))
    np.testing.assert_allclose(M @ M.T / n, S1, atol=0.02)
    np.testing.assert_allclose(N.T @ N / n, S2, atol=0.04)
    M2, N2 = S.paper_case(8, n, 6, case=2, seed=3)
    assert abs(np.median(M2) - 1.0) < 0.02 and abs(np.median(N2) - 1.0) < 0.02  # location vector of ones
    assert np.max(np.abs(M2)) > 1e3  # one degree of freedom: no finite variance


@pytest.mark.parametrize("K,c", [(10, 2000), (10, 10000), (100, 2000)])
def test_case2_opl_and_onc_beat_ssm(K, c):
    """Case II: OPL and ONC are more accurate than SSM (the first two experiments); OPL, the
    A-optimal design, is at least as accurate as ONC."""
    n = 20000
    M, N = S.paper_case(M_ROWS, n, P_COLS, case=2, seed=2)
    e = _design_errors(M, N, S.block_offsets_equal(n, K), c)
    assert e["OPL"] < 0.5 * e["SSM"] and e["ONC"] < 0.5 * e["SSM"], e
    assert e["OPL"] <= e["ONC"] * (1 + 1e-9), e


@pytest.mark.parametrize("K,c", [(10, 2000), (100, 2000)])
def test_case1_methods_similar(K, c):
    """Case I: the four methods have similar accuracy."""
    n = 20000
    M, N = S.paper_case(M_ROWS, n, P_COLS, case=1, seed=2)
    e = _design_errors(M, N, S.block_offsets_equal(n, K), c)
    v = np.array(list(e.values()))
    assert v.max() / v.min() < 1.3, e


def test_onmcnr_approaches_opl_as_pilot_grows():
    """Alg. 3 (ONMCNR): with a pilot of many draws per block, f^_k approaches f_k and c~_k the
    A-optimal c_k, so the expected error approaches OPL's (the fifth experiment)."""
    n, K, c = 20000, 10, 2000
    M, N = S.paper_case(M_ROWS, n, P_COLS, case=2, seed=2)
    off = S.block_offsets_equal(n, K)
    nk = np.diff(off)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    mn2 = float(np.sum((M @ N) ** 2))
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck_opt = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], f), st["a"], nk), nk, c)
    e_opl = oracle.expected_sq_error_alg2(x, y, p, off, ck_opt, f) / mn2
    ratios = []
    for per in (5, 50, 1000):
        fh, _, _ = oracle.pilot_frob_sq(M, N, off, p, per, seed=1, sid=oracle.stream_id(0, oracle.PURPOSE_PILOT))
        ck = oracle.apportion(oracle.g_with_fallback(oracle.g_tilde(st["a"], fh), st["a"], nk), nk, c)
        ratios.append(oracle.expected_sq_error_alg2(x, y, p, off, ck, f) / mn2 / e_opl)
    # OPL's c_k minimise the variance over real block sizes; integer roundings may differ a little
    assert all(r >= 0.99 for r in ratios), ratios
    assert ratios[-1] < 1.05, ratios

"""Pins for oracle.stats: library norms, rank-one closed forms, the trace identity."""
import numpy as np
import pytest

import oracle
import synthetic as S


def _rank_one(m, n, p, seed):
    rng = np.random.default_rng(seed)
    u, v = rng.standard_normal(m), rng.standard_normal(n)
    q, r = rng.standard_normal(n), rng.standard_normal(p)
    return np.outer(u, v), np.outer(q, r), (u, v, q, r)


def test_sq_norms_against_library_norms():
    # non-square shapes so a transposed operand would fail
    rng = np.random.default_rng(0)
    M = rng.standard_normal((7, 11))
    N = rng.standard_normal((11, 5))
    x, y = oracle.col_row_sq_norms(M, N)
    np.testing.assert_allclose(x, np.linalg.norm(M, axis=0) ** 2, rtol=1e-14)
    np.testing.assert_allclose(y, np.linalg.norm(N, axis=1) ** 2, rtol=1e-14)
    with pytest.raises(ValueError):
        oracle.col_row_sq_norms(M, N.T)


def test_fp32_inputs_are_squared_exactly():
    # an FP32 value squared in FP64 is exact: compare with Python's exact rationals
    from fractions import Fraction
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 4)).astype(np.float32)
    N = rng.standard_normal((4, 2)).astype(np.float32)
    x, _ = oracle.col_row_sq_norms(M, N)
    for i in range(4):
        exact = sum(Fraction(float(v)) ** 2 for v in M[:, i])
        assert abs(Fraction(x[i]) - exact) <= exact * Fraction(1, 2 ** 50)


def test_rank_one_closed_forms():
    # M = u v^T, N = q r^T:  x_i = |u|^2 v_i^2, y_i = q_i^2 |r|^2,
    # a_k = |u||r| sum_k |v_i q_i|, f_k = |u|^2 |r|^2 (v_k . q_k)^2
    m, n, p = 6, 12, 5
    M, N, (u, v, q, r) = _rank_one(m, n, p, 3)
    off = np.array([0, 3, 7, 12])
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    nu, nr = np.linalg.norm(u), np.linalg.norm(r)
    np.testing.assert_allclose(x, nu ** 2 * v ** 2, rtol=1e-13)
    np.testing.assert_allclose(y, q ** 2 * nr ** 2, rtol=1e-13)
    for k in range(3):
        sl = slice(off[k], off[k + 1])
        np.testing.assert_allclose(st["a"][k], nu * nr * np.abs(v[sl] * q[sl]).sum(), rtol=1e-13)
        np.testing.assert_allclose(st["s"][k], nu ** 2 * nr ** 2 * np.sum((v[sl] * q[sl]) ** 2), rtol=1e-13)
        np.testing.assert_allclose(st["mf"][k], nu ** 2 * np.sum(v[sl] ** 2), rtol=1e-13)
        np.testing.assert_allclose(st["nf"][k], nr ** 2 * np.sum(q[sl] ** 2), rtol=1e-13)
    f = oracle.block_frob_sq(M, N, off)
    for k in range(3):
        sl = slice(off[k], off[k + 1])
        np.testing.assert_allclose(f[k], nu ** 2 * nr ** 2 * np.dot(v[sl], q[sl]) ** 2, rtol=1e-12)
    # eq. 3.8 probabilities of a rank-one pair: |v_i q_i| / sum_k |v q|
    p = oracle.p_col_opt(st["w"], st["a"], off)
    for k in range(3):
        sl = slice(off[k], off[k + 1])
        np.testing.assert_allclose(p[sl], np.abs(v[sl] * q[sl]) / np.abs(v[sl] * q[sl]).sum(), rtol=1e-13)


def test_block_frob_two_formulas_and_library_norm():
    off = S.block_offsets_uneven(96, 6, 8, 24, seed=5)
    M, N = S.scaled_gaussian(13, 96, 9, off, 1.0, seed=6)
    f1 = oracle.block_frob_sq(M, N, off)
    f2 = oracle.block_frob_sq_gram(M, N, off)
    f3 = np.array([np.linalg.norm(M[:, a:b] @ N[a:b, :], "fro") ** 2 for a, b in zip(off[:-1], off[1:])])
    np.testing.assert_allclose(f1, f2, rtol=1e-12)
    np.testing.assert_allclose(f1, f3, rtol=1e-12)
    # blocks add up to the whole product only through cross terms: sum f_k != ||MN||^2 in general,
    # but with orthogonal blocks (disjoint row supports of M^k) they do
    Mo = np.zeros_like(M)
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        Mo[k::6, a:b] = M[k::6, a:b]
    fo = oracle.block_frob_sq(Mo, N, off)
    np.testing.assert_allclose(fo.sum(), np.linalg.norm(Mo @ N) ** 2, rtol=1e-12)


def test_a_squared_dominates_f():
    # (sum_i ||M^{k(i)}|| ||N_{k(i)}||)^2 >= ||M^k N_k||_F^2 (proof of Thm 2.2)
    off = S.block_offsets_equal(64, 8)
    M, N = S.scaled_gaussian(10, 64, 12, off, 1.5, seed=2)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    assert np.all(st["a"] ** 2 >= f * (1 - 1e-14))
    # and f >= s_k is false in general; s_k is the diagonal of the Gram inner product
    assert np.all(st["s"] <= st["a"] ** 2 * (1 + 1e-14))


def test_offsets_validation():
    with pytest.raises(ValueError):
        oracle.check_offsets([0, 3, 3, 8], 8)
    with pytest.raises(ValueError):
        oracle.check_offsets([1, 3, 8], 8)
    assert list(oracle.check_offsets([0, 3, 8], 8)) == [0, 3, 8]

"""Pins for the adjoint of the sampled product: finite differences, the exact-sum gradient,
and the Monte Carlo mean of sampled gradients."""
import numpy as np

import oracle
import synthetic as S


def test_adjoint_finite_differences_64x512x64():
    # loss <R, CD(M, N)> with the sample frozen; K = 8 blocks of 64, c = 2 blocks -> L = 128
    off = S.block_offsets_equal(512, 8)
    M, N = S.scaled_gaussian(64, 512, 64, off, 1.0, seed=11)
    rng = np.random.default_rng(12)
    R = rng.standard_normal((64, 64))
    r = oracle.run_method(M, N, off, "ONC", oracle.equal_budget(2, 512, 8), seed=5)
    idx, scale = r["idx"], r["scale"]
    dM, dN = oracle.adjoint_columns(M, N, idx, scale, R)

    def loss(Mv, Nv):
        return np.sum(R * oracle.sampled_product_columns(Mv, Nv, idx, scale))

    h = 1e-6
    for (i, j) in [(0, int(idx[0])), (5, int(idx[3])), (63, int(idx[-1])), (7, int(np.setdiff1d(np.arange(512), idx)[0]))]:
        Mp, Mm = M.copy(), M.copy()
        Mp[i, j] += h
        Mm[i, j] -= h
        fd = (loss(Mp, N) - loss(Mm, N)) / (2 * h)
        assert abs(fd - dM[i, j]) <= 1e-6 * max(1.0, abs(dM[i, j]))
    for (i, j) in [(int(idx[1]), 0), (int(idx[7]), 33), (int(np.setdiff1d(np.arange(512), idx)[1]), 2)]:
        Np, Nm = N.copy(), N.copy()
        Np[i, j] += h
        Nm[i, j] -= h
        fd = (loss(M, Np) - loss(M, Nm)) / (2 * h)
        assert abs(fd - dN[i, j]) <= 1e-6 * max(1.0, abs(dN[i, j]))


def test_adjoint_all_indices_once_is_exact_gradient():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((6, 10))
    N = rng.standard_normal((10, 5))
    G = rng.standard_normal((6, 5))
    dM, dN = oracle.adjoint_columns(M, N, np.arange(10), np.ones(10), G)
    np.testing.assert_allclose(dM, G @ N.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(dN, M.T @ G, rtol=1e-13, atol=1e-13)
    off = np.array([0, 3, 10])
    dM, dN = oracle.adjoint_blocks(M, N, off, np.array([0, 1]), np.ones(2), G)
    np.testing.assert_allclose(dM, G @ N.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(dN, M.T @ G, rtol=1e-13, atol=1e-13)


def test_sampled_gradient_is_unbiased():
    # E[dM] = G N^T and E[dN] = M^T G because E[CD] = MN is linear in the outer products
    off = S.block_offsets_equal(24, 3)
    M, N = S.scaled_gaussian(5, 24, 4, off, 0.5, seed=2)
    G = np.random.default_rng(3).standard_normal((5, 4))
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.array([4, 4, 4])
    R = 4000
    acc_M = np.zeros_like(M)
    acc_N = np.zeros_like(N)
    sq_M = np.zeros_like(M)
    for s in range(R):
        idx, scale = oracle.sample_alg2(p, off, ck, seed=s, sid=0)
        dM, dN = oracle.adjoint_columns(M, N, idx, scale, G)
        acc_M += dM
        acc_N += dN
        sq_M += dM ** 2
    mean_M = acc_M / R
    sd_M = np.sqrt(np.maximum(sq_M / R - mean_M ** 2, 0) / R)
    z = np.abs(mean_M - G @ N.T) / np.maximum(sd_M, 1e-12)
    assert np.max(z) < 5.0
    np.testing.assert_allclose(acc_N / R, M.T @ G, rtol=0.15, atol=0.15 * np.abs(M.T @ G).max())


def test_block_adjoint_matches_column_adjoint_on_expanded_sample():
    off = np.array([0, 2, 5, 9])
    rng = np.random.default_rng(4)
    M = rng.standard_normal((3, 9))
    N = rng.standard_normal((9, 4))
    G = rng.standard_normal((3, 4))
    kidx = np.array([2, 0, 2])
    scale = np.array([0.5, 2.0, 0.5])
    dMb, dNb = oracle.adjoint_blocks(M, N, off, kidx, scale, G)
    cols = np.concatenate([np.arange(off[k], off[k + 1]) for k in kidx])
    sc = np.concatenate([np.full(off[k + 1] - off[k], s) for k, s in zip(kidx, scale)])
    dMc, dNc = oracle.adjoint_columns(M, N, cols, sc, G)
    np.testing.assert_allclose(dMb, dMc, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(dNb, dNc, rtol=1e-13, atol=1e-13)

"""The seeded input generators give the shapes and structure the input recipe states: block sizes
inside their range and summing to n, the batched products' shape grid, block scales shared by M's
column block and N's row block, probabilities that sum to one per segment with the requested zeros,
and identical output for identical seeds."""
import numpy as np

import synthetic as S


def test_uneven_offsets_stay_in_range_and_sum_to_n():
    for seed in range(20):
        rng = np.random.default_rng(seed)
        K = int(rng.integers(1, 200))
        lo, hi = 16, 128
        n = int(rng.integers(K * lo, K * hi + 1))
        off = S.block_offsets_uneven(n, K, lo, hi, seed=seed)
        nk = np.diff(off)
        assert off[0] == 0 and off[-1] == n and len(off) == K + 1
        assert nk.min() >= lo and nk.max() <= hi
        np.testing.assert_array_equal(off, S.block_offsets_uneven(n, K, lo, hi, seed=seed))


def test_equal_offsets():
    off = S.block_offsets_equal(4096, 64)
    assert np.all(np.diff(off) == 64) and off[-1] == 4096


def test_batched_products_grid():
    shapes = S.batched_products(64, seed=5)
    assert len(shapes) == 64
    for sh in shapes:
        assert sh["m"] % 128 == 0 and 128 <= sh["m"] <= 2048
        assert sh["p"] % 128 == 0 and 128 <= sh["p"] <= 2048
        assert sh["n"] % 4096 == 0 and 4096 <= sh["n"] <= 65536
        nk = np.diff(sh["offsets"])
        assert sh["offsets"][-1] == sh["n"] and nk.min() >= 32 and nk.max() <= 128
    again = S.batched_products(64, seed=5)
    assert all(a["m"] == b["m"] and a["n"] == b["n"] and a["p"] == b["p"] for a, b in zip(shapes, again))


def test_scaled_gaussian_shares_block_scales():
    off = S.block_offsets_equal(256, 4)
    M, N = S.scaled_gaussian(400, 256, 300, off, 1.5, seed=9)
    assert M.shape == (400, 256) and N.shape == (256, 300)
    # per block, the RMS of M's columns over the RMS of N's rows is about one (the same s_k on both)
    for k in range(4):
        a, b = off[k], off[k + 1]
        ratio = np.sqrt(np.mean(M[:, a:b] ** 2) / np.mean(N[a:b, :] ** 2))
        assert 0.9 < ratio < 1.1
    M2, N2 = S.scaled_gaussian(400, 256, 300, off, 1.5, seed=9)
    np.testing.assert_array_equal(M, M2)
    np.testing.assert_array_equal(N, N2)


def test_random_probabilities_per_segment():
    off = S.block_offsets_uneven(1000, 10, 50, 150, seed=3)
    p = S.random_probabilities(off, seed=4, zero_frac=0.2)
    for k in range(10):
        seg = p[off[k]:off[k + 1]]
        assert abs(seg.sum() - 1.0) < 1e-12 and seg.min() >= 0.0 and seg.max() > 0.0
    assert np.mean(p == 0.0) > 0.05

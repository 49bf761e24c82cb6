"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no norms, probabilities, block sizes, sampling or
products).  Every generator is deterministic in its seed.

Workload recipes (shapes follow the numerical experiments of Sec. 4 of
Niu & Li, "Optimal Sampling Algorithms for Block Matrix Multiplication", and
the scaled synthetic configurations built on them):

* ``block_offsets_equal(n, K)``: n_k = n/K (the equal blocks of Sec. 4).
* ``block_offsets_uneven(n, K, lo, hi, seed)``: K i.i.d. sizes uniform in
  {lo..hi}, then single-unit moves on random blocks (kept inside [lo, hi])
  until the sizes sum to n.
* ``scaled_gaussian``: entries N(0,1) times a per-block scale
  s_k ~ LogNormal(0, sigma); the same s_k multiplies column block k of M and
  row block k of N, so block norms are strongly non-uniform.
* ``low_rank_plus_noise``: rank-r Gaussian factors plus a small Gaussian noise.
* ``paper_case``: Case I (Gaussian columns/rows with covariance 0.7^|i-j|) and
  Case II (multivariate t with one degree of freedom, location 1) of Sec. 4.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "block_offsets_equal",
    "block_offsets_uneven",
    "scaled_gaussian",
    "scaled_gaussian_torch",
    "low_rank_plus_noise",
    "paper_case",
    "random_probabilities",
]


def block_offsets_equal(n: int, K: int) -> np.ndarray:
    """Offsets [K+1] of K equal contraction blocks (n must be divisible by K)."""
    if n % K:
        raise ValueError("n must be divisible by K for equal blocks")
    return np.arange(K + 1, dtype=np.int64) * (n // K)


def block_offsets_uneven(n: int, K: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Offsets [K+1] of K blocks with sizes in [lo, hi] summing to n.

    Sizes start i.i.d. uniform on {lo..hi}; random blocks then gain or lose one
    unit (never leaving [lo, hi]) until the total is n.
    """
    if not (K * lo <= n <= K * hi):
        raise ValueError("n is not reachable with K blocks of size in [lo, hi]")
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=K).astype(np.int64)
    total = int(sizes.sum())
    while total != n:
        k = int(rng.integers(0, K))
        if total > n and sizes[k] > lo:
            sizes[k] -= 1
            total -= 1
        elif total < n and sizes[k] < hi:
            sizes[k] += 1
            total += 1
    off = np.zeros(K + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def batched_products(count: int, seed: int):
    """Shapes of the batched workload: m, p uniform on {128..2048 step 128}, n uniform on
    {4096..65536 step 4096}, K = n / 64 blocks with sizes in [32, 128] summing to n.
    Returns a list of dicts (m, n, p, offsets)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(1, 17)) * 128
        p = int(rng.integers(1, 17)) * 128
        n = int(rng.integers(1, 17)) * 4096
        K = n // 64
        out.append(dict(m=m, n=n, p=p, offsets=block_offsets_uneven(n, K, 32, 128, seed=seed * 100003 + i)))
    return out


def _block_scales(K: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return rng.lognormal(mean=0.0, sigma=sigma, size=K)


def scaled_gaussian(m: int, n: int, p: int, offsets: np.ndarray, sigma: float, seed: int,
                    dtype=np.float64):
    """M (m x n) and N (n x p), entries N(0,1) * s_k with s_k ~ LogNormal(0, sigma).

    Column block k of M and row block k of N share s_k.  Returned as C-ordered
    numpy arrays of ``dtype`` (float64 or float32).
    """
    rng = np.random.default_rng(seed)
    K = len(offsets) - 1
    s = _block_scales(K, sigma, rng)
    col_scale = np.repeat(s, np.diff(offsets))
    M = rng.standard_normal((m, n)) * col_scale[None, :]
    N = rng.standard_normal((n, p)) * col_scale[:, None]
    return np.ascontiguousarray(M, dtype=dtype), np.ascontiguousarray(N, dtype=dtype)


def scaled_gaussian_torch(m: int, n: int, p: int, offsets: np.ndarray, sigma: float, seed: int,
                          dtype=None, device="cuda", m_layout="row"):
    """Device-side version of :func:`scaled_gaussian` for large workloads.

    Uses a seeded ``torch.Generator`` on ``device``.  ``m_layout='col'`` returns M
    stored column-major (a row-major n x m buffer holding M transposed).
    Returns (M_storage, N, scales) as torch tensors.
    """
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    K = len(offsets) - 1
    rng = np.random.default_rng(seed)
    s = _block_scales(K, sigma, rng)
    col_scale = torch.from_numpy(np.repeat(s, np.diff(offsets))).to(device=device, dtype=torch.float32)
    if m_layout == "row":
        M = torch.randn(m, n, generator=g, device=device, dtype=torch.float32)
        M.mul_(col_scale[None, :])
    else:
        M = torch.randn(n, m, generator=g, device=device, dtype=torch.float32)
        M.mul_(col_scale[:, None])
    N = torch.randn(n, p, generator=g, device=device, dtype=torch.float32)
    N.mul_(col_scale[:, None])
    return M.to(dtype), N.to(dtype), s


def low_rank_plus_noise(rows: int, cols: int, rank: int, noise: float, seed: int, dtype=np.float64):
    """A = F G / sqrt(rank) + noise * Z with F, G, Z standard Gaussian."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((rows, rank))
    G = rng.standard_normal((rank, cols))
    A = F @ G / np.sqrt(rank) + noise * rng.standard_normal((rows, cols))
    return np.ascontiguousarray(A, dtype=dtype)


def _ar_cov(d: int, scale: float) -> np.ndarray:
    i = np.arange(d)
    return scale * 0.7 ** np.abs(i[:, None] - i[None, :])


def paper_case(m: int, n: int, p: int, case: int, seed: int):
    """Case I / Case II inputs of Sec. 4 (columns of M are m-vectors, rows of N are p-vectors).

    Case I: M^(i) ~ N(0, S1), N_(i) ~ N(0, S2) with S1 = 0.7^|i-j|, S2 = 2 * 0.7^|i-j|.
    Case II: multivariate t with one degree of freedom, location vector of ones,
    scale S1 (resp. S2): x = 1 + z / sqrt(g), z ~ N(0, S), g ~ chi^2_1.
    """
    rng = np.random.default_rng(seed)
    L1 = np.linalg.cholesky(_ar_cov(m, 1.0))
    L2 = np.linalg.cholesky(_ar_cov(p, 2.0))
    Zm = rng.standard_normal((n, m)) @ L1.T  # row i = column i of M
    Zn = rng.standard_normal((n, p)) @ L2.T
    if case == 1:
        return np.ascontiguousarray(Zm.T), np.ascontiguousarray(Zn)
    if case == 2:
        gm = rng.chisquare(1.0, size=(n, 1))
        gn = rng.chisquare(1.0, size=(n, 1))
        return np.ascontiguousarray((1.0 + Zm / np.sqrt(gm)).T), np.ascontiguousarray(1.0 + Zn / np.sqrt(gn))
    raise ValueError("case must be 1 or 2")


def random_probabilities(offsets: np.ndarray, seed: int, zero_frac: float = 0.0) -> np.ndarray:
    """A random probability vector that sums to one inside every segment of ``offsets``.

    ``zero_frac`` of the entries are forced to zero (never the whole segment).
    Used to feed identical probabilities to both samplers.
    """
    rng = np.random.default_rng(seed)
    n = int(offsets[-1])
    w = rng.random(n) ** 3
    if zero_frac > 0:
        w[rng.random(n) < zero_frac] = 0.0
    p = np.zeros(n)
    for k in range(len(offsets) - 1):
        a, b = int(offsets[k]), int(offsets[k + 1])
        seg = w[a:b].copy()
        if seg.sum() == 0:
            seg[rng.integers(0, b - a)] = 1.0
        p[a:b] = seg / seg.sum()
    return p

"""Sampling probabilities and block sizes (oracle; test infrastructure only).

Probabilities
  p_col_opt       eq. 3.8   p_{k_i} = ||M^{k(i)}|| ||N_{k(i)}|| / a_k
  p_col_uniform   Table 2   p_{k_i} = 1/n_k (UU, and the ONU pilot)
  p_blk_prodnorm  eq. 1.2   p_k = ||M^k N_k||_F / sum_j ||M^j N_j||_F
  p_blk_normprod  eq. 1.4   p_k = ||M^k||_F ||N_k||_F / sum_j (...)   (SSM)

Block-size weights g_k (real block size c * g_k / sum_j g_j)
  g_opt    eq. 3.9  sqrt(a_k^2 - f_k)
  g_hat    eq. 4.2  a_k
  g_tilde  eq. 4.7  sqrt(|a_k^2 - fhat_k|)
  g_equal  Table 2  1 (UU: c/K)

Readings where the paper is silent
  * a block with a_k = 0 (every outer product zero) gets uniform p;
  * all g_k = 0 falls back to g_k = a_k, then to g_k = n_k;
  * integers: Alg. 2 needs c_k in Z+, 1 <= c_k <= n_k, sum c_k = c.  The
    real sizes are turned into integers by :func:`apportion` (a highest-averages
    rule with a first draw guaranteed and a cap of n_k, see its docstring).
"""
from __future__ import annotations

import struct

import numpy as np

__all__ = [
    "p_col_opt", "p_col_uniform", "p_blk_prodnorm", "p_blk_normprod",
    "g_opt", "g_hat", "g_tilde", "g_equal", "g_with_fallback",
    "real_block_sizes", "apportion", "InfeasibleBudget", "INF_BITS",
]

INF_BITS = 0x7FF0000000000000


class InfeasibleBudget(ValueError):
    """c outside [K, n]: Alg. 2 cannot give every block 1 <= c_k <= n_k draws."""


def _segments(offsets):
    off = np.asarray(offsets, dtype=np.int64)
    return off, np.diff(off)


def p_col_opt(w, a, offsets) -> np.ndarray:
    """eq. 3.8: p_{k_i} = w_i / a_k with w_i = ||M^{k(i)}||_2 ||N_{k(i)}||_2.

    A block with a_k = 0 contributes exactly zero whatever is drawn; it gets
    uniform probabilities so the draws stay well defined.
    """
    off, nk = _segments(offsets)
    w = np.asarray(w, dtype=np.float64)
    p = np.empty_like(w)
    for k in range(len(nk)):
        lo, hi = off[k], off[k + 1]
        if a[k] > 0:
            p[lo:hi] = w[lo:hi] / a[k]
        else:
            p[lo:hi] = 1.0 / nk[k]
    return p


def p_col_uniform(offsets) -> np.ndarray:
    """Table 2 (UU, ONU pilot): p_{k_i} = 1/n_k."""
    off, nk = _segments(offsets)
    return np.repeat(1.0 / nk.astype(np.float64), nk)


def _normalise(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    t = v.sum()
    if t > 0:
        return v / t
    return np.full(len(v), 1.0 / len(v))


def p_blk_prodnorm(f) -> np.ndarray:
    """eq. 1.2 (Wu): p_k proportional to ||M^k N_k||_F = sqrt(f_k)."""
    return _normalise(np.sqrt(np.asarray(f, dtype=np.float64)))


def p_blk_normprod(mf, nf) -> np.ndarray:
    """eq. 1.4 (SSM): p_k proportional to ||M^k||_F ||N_k||_F = sqrt(mf_k nf_k)."""
    return _normalise(np.sqrt(np.asarray(mf, dtype=np.float64) * np.asarray(nf, dtype=np.float64)))


def g_opt(a, f) -> np.ndarray:
    """eq. 3.9 numerator: ((sum_i ||M^{k(i)}|| ||N_{k(i)}||)^2 - ||M^k N_k||_F^2)^{1/2}.

    The bracket is >= 0 mathematically (proof of Thm 2.2); the clamp at zero
    only absorbs rounding.
    """
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(np.maximum(a * a - np.asarray(f, dtype=np.float64), 0.0))


def g_hat(a) -> np.ndarray:
    """eq. 4.2 numerator: a_k."""
    return np.asarray(a, dtype=np.float64).copy()


def g_tilde(a, fhat) -> np.ndarray:
    """eq. 4.7 numerator: |a_k^2 - ||C^{0k} D_{0k}||_F^2|^{1/2}."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(np.abs(a * a - np.asarray(fhat, dtype=np.float64)))


def g_equal(K: int) -> np.ndarray:
    """Table 2 (UU): c_k = c/K, i.e. equal weights."""
    return np.ones(K)


def g_with_fallback(g, a, nk) -> np.ndarray:
    """Weights of eq. 3.9 / 4.2 / 4.7 for the block sizes; all-zero weights fall back to a_k, then
    to n_k (reading: the paper is silent on a product whose weights all vanish)."""
    g = np.asarray(g, dtype=np.float64)
    if np.any(g > 0):
        return g
    a = np.asarray(a, dtype=np.float64)
    if np.any(a > 0):
        return a.copy()
    return np.asarray(nk, dtype=np.float64)


def real_block_sizes(g, c) -> np.ndarray:
    """Real-valued c * g_k / sum_j g_j (eq. 3.9, 4.2, 4.7)."""
    g = np.asarray(g, dtype=np.float64)
    return c * g / g.sum()


def _bits_to_double(u: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def _counts(lam: float, g: np.ndarray, nk: np.ndarray) -> np.ndarray:
    """clamp(floor(lam * g_k), 1, n_k); a zero weight always counts one draw."""
    with np.errstate(invalid="ignore", over="ignore"):
        v = np.floor(np.float64(lam) * g)
    v = np.where(g > 0, v, 1.0)
    v = np.minimum(np.maximum(v, 1.0), nk.astype(np.float64))
    return v.astype(np.int64)


def apportion(g, nk, c: int) -> np.ndarray:
    """Integer block sizes c_k with 1 <= c_k <= n_k and sum c_k = c (Alg. 2 input).

    Rule (the paper gives only the real values c g_k / sum g_j):
      1. lam* = the largest FP64 value lam >= 0 (+inf allowed) with
         F(lam) = sum_k clamp(floor(lam * g_k), 1, n_k) <= c, found exactly by
         bisection over the IEEE bit patterns (F is monotone in lam);
      2. c_k = clamp(floor(lam* g_k), 1, n_k);
      3. the r = c - sum c_k remaining draws go, one each and in increasing k,
         to the blocks whose count grows at the next representable lam; if
         lam* = +inf they fill the remaining capacity n_k - c_k in increasing k.
    With exact arithmetic this is the highest-averages (D'Hondt) method with a
    guaranteed first draw and a cap of n_k; unclamped it tracks c g_k/sum g_j.
    """
    g = np.asarray(g, dtype=np.float64)
    nk = np.asarray(nk, dtype=np.int64)
    K = len(g)
    n = int(nk.sum())
    if not (K <= c <= n):
        raise InfeasibleBudget(f"need K <= c <= n, got K={K}, c={c}, n={n}")
    if np.any(~np.isfinite(g)) or np.any(g < 0):
        raise ValueError("block-size weights must be finite and non-negative")

    def F(u: int) -> int:
        return int(_counts(_bits_to_double(u), g, nk).sum())

    lo, hi = 0, INF_BITS
    if F(hi) <= c:
        ustar = hi
    else:
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if F(mid) <= c:
                lo = mid
            else:
                hi = mid
        ustar = lo
    ck = _counts(_bits_to_double(ustar), g, nk)
    r = c - int(ck.sum())
    if r > 0:
        if ustar < INF_BITS:
            grow = np.nonzero(_counts(_bits_to_double(ustar + 1), g, nk) > ck)[0]
            assert len(grow) > r
            ck[grow[:r]] += 1
        else:
            for k in range(K):
                add = min(r, int(nk[k] - ck[k]))
                ck[k] += add
                r -= add
    return ck

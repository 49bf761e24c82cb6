"""Statistics the sampling design needs (oracle; test infrastructure only).

Notation (Sec. 2, eq. 2.3): M is m x n, N is n x p; the contraction index
i = 1..n is split into K consecutive blocks, block k holding n_k indices
[offsets[k], offsets[k+1]).  M^{k(i)} is column i of block k of M and
N_{k(i)} the matching row of N.
"""
from __future__ import annotations

import numpy as np

__all__ = ["col_row_sq_norms", "block_stats", "block_frob_sq", "block_frob_sq_gram", "check_offsets"]


def check_offsets(offsets, n: int) -> np.ndarray:
    """Validate block offsets: offsets[0]=0 < offsets[1] < ... < offsets[K] = n (eq. 2.3)."""
    off = np.asarray(offsets, dtype=np.int64)
    if off.ndim != 1 or len(off) < 2 or off[0] != 0 or off[-1] != n or np.any(np.diff(off) <= 0):
        raise ValueError("offsets must start at 0, end at n and strictly increase")
    return off


def col_row_sq_norms(M, N):
    """x_i = ||M^{(i)}||_2^2 and y_i = ||N_{(i)}||_2^2 for i = 1..n.

    These are the squared factors of the probabilities eq. 1.1 / eq. 3.8.
    Squares are formed in FP64 (exact for FP32 inputs) and summed in FP64.
    """
    M64 = np.asarray(M, dtype=np.float64)
    N64 = np.asarray(N, dtype=np.float64)
    if M64.shape[1] != N64.shape[0]:
        raise ValueError("inner dimensions differ")
    # sum over the rows of M for every column; transpose copy so numpy sums a
    # contiguous axis (pairwise summation)
    x = np.ascontiguousarray((M64 * M64).T).sum(axis=1)
    y = (N64 * N64).sum(axis=1)
    return x, y


def block_stats(x, y, offsets):
    """Per-block statistics built from x_i and y_i.

    a_k  = sum_{i in k} ||M^{k(i)}|| ||N_{k(i)}||      (denominator of eq. 3.8)
    s_k  = sum_{i in k} ||M^{k(i)}||^2 ||N_{k(i)}||^2  (Remark 2.2 first term with eq. 3.8)
    mf_k = ||M^k||_F^2, nf_k = ||N_k||_F^2            (eq. 1.4)
    The column weight is w_i = sqrt(x_i * y_i).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    K = len(off) - 1
    xy = x * y
    w = np.sqrt(xy)
    a = np.empty(K)
    s = np.empty(K)
    mf = np.empty(K)
    nf = np.empty(K)
    for k in range(K):
        lo, hi = off[k], off[k + 1]
        a[k] = w[lo:hi].sum()
        s[k] = xy[lo:hi].sum()
        mf[k] = x[lo:hi].sum()
        nf[k] = y[lo:hi].sum()
    return {"w": w, "a": a, "s": s, "mf": mf, "nf": nf}


def block_frob_sq(M, N, offsets) -> np.ndarray:
    """f_k = ||M^k N_k||_F^2 by forming each block product (eq. 1.2, eq. 3.9)."""
    M64 = np.asarray(M, dtype=np.float64)
    N64 = np.asarray(N, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    K = len(off) - 1
    f = np.empty(K)
    for k in range(K):
        P = M64[:, off[k]:off[k + 1]] @ N64[off[k]:off[k + 1], :]
        f[k] = np.sum(P * P)
    return f


def block_frob_sq_gram(M, N, offsets) -> np.ndarray:
    """f_k = ||M^k N_k||_F^2 (eq. 1.2, eq. 3.9) through the trace identity ||A B||_F^2 = <A^T A, B B^T>_F.

    Not in the paper; a second formula for the same quantity, used to pin
    :func:`block_frob_sq` and as the definition the GPU's Gram form follows.
    """
    M64 = np.asarray(M, dtype=np.float64)
    N64 = np.asarray(N, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    K = len(off) - 1
    f = np.empty(K)
    for k in range(K):
        A = M64[:, off[k]:off[k + 1]]
        B = N64[off[k]:off[k + 1], :]
        f[k] = np.sum((A.T @ A) * (B @ B.T))
    return f

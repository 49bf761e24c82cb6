"""Estimators, closed-form errors, bounds and the adjoint (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np

from .stats import col_row_sq_norms, block_stats, block_frob_sq
from .design import (p_col_opt, p_col_uniform, p_blk_prodnorm, p_blk_normprod, g_opt, g_hat,
                     g_tilde, g_equal, g_with_fallback, apportion)
from .sampler import sample_alg2, sample_blocks, sample_segments, stream_id, PURPOSE_MAIN, PURPOSE_PILOT

__all__ = [
    "METHODS", "exact_product", "sampled_product_columns", "sampled_product_blocks",
    "expected_sq_error_alg2", "expected_sq_error_blocks", "optimal_value_eq310",
    "bound_eq311", "bound_eq43", "pilot_frob_sq", "equal_budget", "run_method",
    "adjoint_columns", "adjoint_blocks",
]

# Table 2 presets plus the two block-sampling baselines of Sec. 1.
METHODS = ("OPL", "ONC", "ONU", "ONMCNR", "UU", "SSM", "WU")


def exact_product(M, N) -> np.ndarray:
    """MN = sum_k M^k N_k (eq. 2.3), FP64."""
    return np.asarray(M, dtype=np.float64) @ np.asarray(N, dtype=np.float64)


def sampled_product_columns(M, N, idx, scale) -> np.ndarray:
    """CD with C^{(t)} = M^{(i_t)} sqrt(scale_t), D_{(t)} = N_{(i_t)} sqrt(scale_t).

    Alg. 1 step 1(b) / Alg. 2 step 4 / eq. 3.3 with scale_t = 1/(c_k p_{k_{i_t}}).
    """
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    r = np.sqrt(np.asarray(scale, dtype=np.float64))
    C = M[:, idx] * r[None, :]
    D = N[idx, :] * r[:, None]
    return C @ D


def sampled_product_blocks(M, N, offsets, kidx, scale) -> np.ndarray:
    """sum_t M^{k_t} N_{k_t} / (c p_{k_t}) -- the block-sampling estimator (eq. 1.2/1.4 methods)."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    cols = np.concatenate([np.arange(off[k], off[k + 1]) for k in kidx]) if len(kidx) else np.zeros(0, np.int64)
    r = np.concatenate([np.full(off[k + 1] - off[k], np.sqrt(s)) for k, s in zip(kidx, scale)]) if len(kidx) else np.zeros(0)
    return (M[:, cols] * r[None, :]) @ (N[cols, :] * r[:, None])


def expected_sq_error_alg2(x, y, p, offsets, ck, f) -> float:
    """E||MN - CD||_F^2 for Alg. 2 (Remark 2.2, summing eq. 3.7 over all entries):

    sum_k (1/c_k) ( sum_{i in k} x_i y_i / p_{k_i} - f_k ).
    Terms with p_{k_i} = 0 must have x_i y_i = 0 (else the estimator is biased).
    """
    off = np.asarray(offsets, dtype=np.int64)
    xy = np.asarray(x, dtype=np.float64) * np.asarray(y, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    if np.any((p == 0) & (xy > 0)):
        raise ValueError("zero probability on a non-zero outer product")
    q = np.where(p > 0, xy / np.where(p > 0, p, 1.0), 0.0)
    total = 0.0
    for k in range(len(off) - 1):
        total += (q[off[k]:off[k + 1]].sum() - f[k]) / ck[k]
    return float(total)


def expected_sq_error_blocks(f, pblk, c: int, mn_fro2: float) -> float:
    """E||MN - CD||_F^2 for c i.i.d. block draws: (1/c)(sum_k f_k / p_k - ||MN||_F^2).

    Lemma 2.1 applied with whole blocks as the sampled terms.
    """
    f = np.asarray(f, dtype=np.float64)
    pblk = np.asarray(pblk, dtype=np.float64)
    if np.any((pblk == 0) & (f > 0)):
        raise ValueError("zero probability on a non-zero block product")
    q = np.where(pblk > 0, f / np.where(pblk > 0, pblk, 1.0), 0.0)
    return float((q.sum() - mn_fro2) / c)


def optimal_value_eq310(a, f, c) -> float:
    """eq. 3.10: (1/c) [sum_k (1 - v_k^2)^{1/2} a_k]^2 with v_k = ||M^k N_k||_F / a_k."""
    a = np.asarray(a, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    v = np.where(a > 0, np.sqrt(f) / np.where(a > 0, a, 1.0), 0.0)
    return float(np.sum(np.sqrt(np.maximum(1.0 - v * v, 0.0)) * a) ** 2 / c)


def _thetas(a, f):
    a = np.asarray(a, dtype=np.float64)
    v2 = np.asarray(f, dtype=np.float64) / (a * a)
    one_minus = 1.0 - v2
    return float(one_minus.min()), float(one_minus.max())


def bound_eq311(a, f, m_fro2, n_fro2, c, beta=1.0) -> float:
    """eq. 3.11: phi^2 / (beta c) ||M||_F^2 ||N||_F^2 (Thm 2.3), theta from the data."""
    t1, t2 = _thetas(a, f)
    phi = np.sqrt(t2 - t1 * beta + t2 * t1 * beta) / (t2 * t1) ** 0.25
    return float(phi ** 2 / (beta * c) * m_fro2 * n_fro2)


def bound_eq43(a, f, m_fro2, n_fro2, c, beta=1.0) -> float:
    """eq. 4.3: hat-phi^2 / (beta c) ||M||_F^2 ||N||_F^2 with hat-phi = (1 - beta(1 - theta_2))^{1/2}."""
    _, t2 = _thetas(a, f)
    phi = np.sqrt(1.0 - beta * (1.0 - t2))
    return float(phi ** 2 / (beta * c) * m_fro2 * n_fro2)


def pilot_frob_sq(M, N, offsets, p0, c0_per_block: int, seed: int, sid: int):
    """Alg. 3 step 1: ||C^{0k} D_{0k}||_F^2 from c0' = [c0/K] draws per block with p0.

    C^{0k} D_{0k} = sum_t M^{k(i_t)} N_{k(i_t)} / (c0' p0_{k_{i_t}}) (Alg. 1 on block k).
    Returns (fhat [K], idx, scale).
    """
    off = np.asarray(offsets, dtype=np.int64)
    K = len(off) - 1
    counts = np.full(K, int(c0_per_block), dtype=np.int64)
    idx = sample_segments(p0, off, counts, seed, sid)
    scale = 1.0 / (np.float64(c0_per_block) * np.asarray(p0, dtype=np.float64)[idx])
    fhat = np.empty(K)
    for k in range(K):
        sl = slice(k * c0_per_block, (k + 1) * c0_per_block)
        P = sampled_product_columns(M, N, idx[sl], scale[sl])
        fhat[k] = np.sum(P * P)
    return fhat, idx, scale


def equal_budget(c_blocks: int, n: int, K: int) -> int:
    """Outer-product budget matching c whole blocks of eq. 1.2 / 1.4: L = round(c n / K) (reading R3:
    Alg. 2 and block sampling compared at the same contraction budget)."""
    return int(np.floor(c_blocks * n / K + 0.5))


def run_method(M, N, offsets, method: str, c: int, seed: int, replicate: int = 0, c0: int | None = None):
    """One approximate product by a Table 2 method or a block-sampling baseline.

    ``c`` counts outer products for Alg. 2/3 methods and blocks for SSM/WU.
    Returns a dict with the design (p, ck), the sample (idx, scale) and CD.
    """
    off = np.asarray(offsets, dtype=np.int64)
    nk = np.diff(off)
    K = len(nk)
    x, y = col_row_sq_norms(M, N)
    st = block_stats(x, y, off)
    sid = stream_id(replicate, PURPOSE_MAIN)
    out = {"x": x, "y": y, **st}
    if method in ("SSM", "WU"):
        if method == "SSM":
            pblk = p_blk_normprod(st["mf"], st["nf"])
        else:
            out["f"] = block_frob_sq(M, N, off)
            pblk = p_blk_prodnorm(out["f"])
        idx, scale = sample_blocks(pblk, c, seed, sid)
        out.update(p=pblk, idx=idx, scale=scale, CD=sampled_product_blocks(M, N, off, idx, scale))
        return out
    if method == "UU":
        p = p_col_uniform(off)
        g = g_equal(K)
    else:
        p = p_col_opt(st["w"], st["a"], off)
        if method == "OPL":
            out["f"] = block_frob_sq(M, N, off)
            g = g_opt(st["a"], out["f"])
        elif method == "ONC":
            g = g_hat(st["a"])
        elif method in ("ONU", "ONMCNR"):
            if c0 is None:
                raise ValueError("two-step methods need c0")
            p0 = p_col_uniform(off) if method == "ONU" else p
            c0p = max(1, c0 // K)
            fhat, pidx, pscale = pilot_frob_sq(M, N, off, p0, c0p, seed, stream_id(replicate, PURPOSE_PILOT))
            out.update(fhat=fhat, pilot_idx=pidx, pilot_scale=pscale, p0=p0)
            g = g_tilde(st["a"], fhat)
        else:
            raise ValueError(f"unknown method {method}")
    g = g_with_fallback(g, st["a"], nk)
    ck = apportion(g, nk, c)
    idx, scale = sample_alg2(p, off, ck, seed, sid)
    out.update(p=p, g=g, ck=ck, idx=idx, scale=scale, CD=sampled_product_columns(M, N, idx, scale))
    return out


def adjoint_columns(M, N, idx, scale, G):
    """Gradients of <G, CD> with the sample frozen (p treated as constant), CD the estimator of
    eq. 3.3 (the adjoint is not in the paper; it is the derivative of that sum of outer products):

    dM^{(i_t)} += scale_t G N_{(i_t)}^T,  dN_{(i_t)} += scale_t M^{(i_t)T} G.
    """
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    dM = np.zeros_like(M)
    dN = np.zeros_like(N)
    for t, i in enumerate(idx):
        dM[:, i] += scale[t] * (G @ N[i, :])
        dN[i, :] += scale[t] * (M[:, i] @ G)
    return dM, dN


def adjoint_blocks(M, N, offsets, kidx, scale, G):
    """Block-sampling adjoint (the derivative of the eq. 1.2 / 1.4 estimator's sum of block products,
    sample frozen): dM^{k_t} += scale_t G N_{k_t}^T, dN_{k_t} += scale_t M^{k_t T} G."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    dM = np.zeros_like(M)
    dN = np.zeros_like(N)
    for t, k in enumerate(kidx):
        sl = slice(off[k], off[k + 1])
        dM[:, sl] += scale[t] * (G @ N[sl, :].T)
        dN[sl, :] += scale[t] * (M[:, sl].T @ G)
    return dM, dN

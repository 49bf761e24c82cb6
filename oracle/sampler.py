"""I.i.d. sampling with replacement (oracle; test infrastructure only).

Alg. 1 step 1(a) draws i_t with Pr(i_t = s) = p_s, independently and with
replacement.  The paper does not say how; this implementation fixes a reproducible
convention so the CPU and GPU samplers can be compared index for index:

* Random bits: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11).  key = (seed_lo, seed_hi),
  counter = (t_lo, t_hi, sid_lo, sid_hi) where t is the global draw number and
  sid the stream id; r = (x1 << 32) | x0 is the 64-bit uniform.
* Fixed-point CDF: W_j = floor(p_j * 2^62) as an unsigned integer, S_j the
  inclusive prefix sum inside the segment, T = S_last.  The draw is the
  smallest j with S_j > floor(r * T / 2^64).  Pr(j) = W_j / T up to 2^-64, and
  W_j / T differs from p_j by at most about n_seg * 2^-62.
* Segments: Alg. 2 draws c_k indices from each block k (eq. 3.2), segment by
  segment, draw numbers running on across segments; block sampling (eq. 1.2,
  1.4) uses one segment of length K.
* Stream id: (replicate << 8) | purpose with purpose MAIN = 0, PILOT = 1.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "PURPOSE_MAIN", "PURPOSE_PILOT", "stream_id", "philox4x32_10", "uniform64",
    "fixed_point_weights", "inverse_cdf", "sample_segments", "sample_alg2", "sample_blocks",
]

PURPOSE_MAIN = 0
PURPOSE_PILOT = 1

_M32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)


def stream_id(replicate: int, purpose: int) -> int:
    """Counter words 2-3 of the draws: (replicate << 8) | purpose, so that the main draws of Alg. 1
    step 1(a) and the pilot draws of Alg. 3 step 1 never share random bits (a convention of this
    implementation; the paper does not say how draws are made)."""
    return (int(replicate) << 8) | int(purpose)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words (held in uint64): the random bits behind
    Alg. 1 step 1(a)'s draws, from the generator's published definition (Salmon et al., SC'11).

    Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit products);
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is
    bumped by the Weyl constants (W0, W1).
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _M32 for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    for _ in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _PHILOX_W0) & _M32
        k1 = (k1 + _PHILOX_W1) & _M32
    return c0, c1, c2, c3


def uniform64(seed: int, sid: int, t) -> np.ndarray:
    """The 64-bit uniform of draw number(s) t of Alg. 1 step 1(a): (x1 << 32) | x0."""
    t = np.asarray(t, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    sid = int(sid) & 0xFFFFFFFFFFFFFFFF
    x0, x1, _, _ = philox4x32_10(t & _M32, t >> np.uint64(32),
                                 np.uint64(sid & 0xFFFFFFFF), np.uint64(sid >> 32),
                                 np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))
    return (x1 << np.uint64(32)) | x0


def fixed_point_weights(p) -> np.ndarray:
    """W_j = floor(p_j * 2^62) (exact: scaling by a power of two, then floor): the probabilities of
    eq. 3.8 / 1.2 / 1.4 as integer weights for Alg. 1 step 1(a)'s inverse-CDF draw."""
    p = np.asarray(p, dtype=np.float64)
    if np.any(~np.isfinite(p)) or np.any(p < 0) or np.any(p > 1):
        raise ValueError("probabilities must be finite and in [0, 1]")
    return np.floor(np.ldexp(p, 62)).astype(np.uint64)


def inverse_cdf(S: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Smallest j with S_j > floor(r * T / 2^64), T = S[-1] (exact 128-bit product): one draw of
    Alg. 1 step 1(a), Pr(j) = W_j / T."""
    T = int(S[-1])
    target = np.array([(int(ri) * T) >> 64 for ri in r], dtype=np.uint64)
    return np.searchsorted(S, target, side="right").astype(np.int64)


def sample_segments(p, seg_offsets, counts, seed: int, sid: int) -> np.ndarray:
    """Draw counts[s] indices from segment s of p (global indices into p), i.i.d. with replacement
    inside each segment (Alg. 1 step 1(a); per block for Alg. 2, eq. 3.2)."""
    seg_offsets = np.asarray(seg_offsets, dtype=np.int64)
    counts = np.asarray(counts, dtype=np.int64)
    W = fixed_point_weights(p)
    out = np.empty(int(counts.sum()), dtype=np.int64)
    t = 0
    for s in range(len(counts)):
        lo, hi = int(seg_offsets[s]), int(seg_offsets[s + 1])
        cnt = int(counts[s])
        if cnt == 0:
            continue
        S = np.cumsum(W[lo:hi], dtype=np.uint64)
        if int(S[-1]) == 0:
            raise ValueError(f"segment {s} has zero probability mass")
        r = uniform64(seed, sid, np.arange(t, t + cnt, dtype=np.uint64))
        out[t:t + cnt] = lo + inverse_cdf(S, r)
        t += cnt
    return out


def sample_alg2(p, offsets, ck, seed: int, sid: int):
    """Alg. 2: c_k draws inside block k; scale_t = 1 / (c_k p_{k_{i_t}}) (eq. 3.2)."""
    idx = sample_segments(p, offsets, ck, seed, sid)
    ck = np.asarray(ck, dtype=np.int64)
    ck_of_draw = np.repeat(ck, ck).astype(np.float64)
    scale = 1.0 / (ck_of_draw * np.asarray(p, dtype=np.float64)[idx])
    return idx, scale


def sample_blocks(pblk, c: int, seed: int, sid: int):
    """Block sampling (eq. 1.2 / 1.4): c draws over K blocks; scale_t = 1 / (c p_{k_t})."""
    pblk = np.asarray(pblk, dtype=np.float64)
    idx = sample_segments(pblk, [0, len(pblk)], [c], seed, sid)
    scale = 1.0 / (np.float64(c) * pblk[idx])
    return idx, scale

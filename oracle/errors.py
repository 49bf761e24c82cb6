"""Error bars of the sampled product (oracle; test infrastructure only).

Per entry (h, f) of CD:
  * the exact variance of Lemma 3.1, eq. 3.7 (the sigma^2 of Thm 3.1): for Alg. 2
      sum_k (1/c_k) [ sum_{i in k} M_hi^2 N_if^2 / p_i - ((M^k N_k)_hf)^2 ],
    and, for c i.i.d. whole-block draws (Alg. 1 with blocks as the sampled terms),
      (1/c) [ sum_k ((M^k N_k)_hf)^2 / p_k - ((MN)_hf)^2 ];
  * a one-sample estimate of that variance from the draws themselves: the draws of block k are
    c_k i.i.d. terms Z_t = scale_t M_{h,i_t} N_{i_t,f} whose sum is block k's part of (CD)_hf, so
    c_k times their unbiased sample variance estimates block k's variance.  Blocks with c_k = 1 carry
    no such information and are counted, not estimated.  With the entry's value this gives the
    normal interval (CD)_hf +- z sigma of Thm 3.1.

For the whole matrix (Remark 2.2, Thm 3.3, Thm 4.2, Thm 4.4): E||MN - CD||_F^2, eq. 3.10, the
bounds of eq. 3.11 / 3.12 (c_k of eq. 3.9), eq. 4.3 / 4.4 (c_k of eq. 4.2) and eq. 4.8 / 4.9
(Alg. 3, pilot estimates f^_k), with theta_1, theta_2, beta read off the data.

Readings (the paper states these quantities for its own estimator only):
  * terms with p_i = 0 are never drawn; the variance is that of the estimator as run, i.e. those
    terms are left out of both sums (eq. 3.7 unchanged whenever every p_i > 0);
  * beta = min(1, min_i p_i / p*_i) over the columns with p*_i > 0, p* the eq. 3.8 probabilities;
  * theta_1, theta_2 = min, max over blocks with a_k > 0 of 1 - v_k^2 = 1 - f_k / a_k^2, and the
    hatted ones of |1 - f^_k / a_k^2| (Thm 4.3).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "entry_variance_columns", "entry_variance_blocks", "entry_estimate_columns", "entry_estimate_blocks",
    "error_report", "REPORT_FIELDS",
]


def _entries(entries):
    e = np.asarray(entries, dtype=np.int64).reshape(-1, 2)
    return e[:, 0], e[:, 1]


def entry_variance_columns(M, N, offsets, p, ck, entries) -> np.ndarray:
    """Var[(CD)_hf] of Alg. 2 for each listed (h, f): Lemma 3.1, eq. 3.7."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    hs, fs = _entries(entries)
    out = np.zeros(len(hs))
    for e, (h, f) in enumerate(zip(hs, fs)):
        total = 0.0
        for k in range(len(off) - 1):
            s = 0.0
            dot = 0.0
            for i in range(off[k], off[k + 1]):
                if p[i] > 0.0:
                    t = M[h, i] * N[i, f]
                    s += t * t / p[i]
                    dot += t
            total += (s - dot * dot) / ck[k]
        out[e] = total
    return out


def entry_variance_blocks(M, N, offsets, pblk, c: int, entries) -> np.ndarray:
    """Var[(CD)_hf] for c i.i.d. block draws with probabilities pblk (Lemma 2.1 with blocks as terms)."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    pblk = np.asarray(pblk, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    hs, fs = _entries(entries)
    out = np.zeros(len(hs))
    for e, (h, f) in enumerate(zip(hs, fs)):
        s = 0.0
        mean = 0.0
        for k in range(len(off) - 1):
            if pblk[k] > 0.0:
                d = float(M[h, off[k]:off[k + 1]] @ N[off[k]:off[k + 1], f])
                s += d * d / pblk[k]
                mean += d
        out[e] = (s - mean * mean) / c
    return out


def entry_estimate_columns(M, N, offsets, ck, idx, scale, entries):
    """(CD)_hf and the one-sample variance estimate sum_{k: c_k >= 2} c_k/(c_k - 1) sum_t (Z_t - Zbar_k)^2
    from Alg. 2's draws (block k's draws at positions [sum_{j<k} c_j, sum_{j<=k} c_j)): the plug-in
    estimate of eq. 3.7's per-entry variance behind Thm 3.1's normal interval.
    Returns (cd, s2, blocks with c_k = 1)."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    scale = np.asarray(scale, dtype=np.float64)
    ck = np.asarray(ck, dtype=np.int64)
    start = np.concatenate([[0], np.cumsum(ck)])
    hs, fs = _entries(entries)
    cd = np.zeros(len(hs))
    s2 = np.zeros(len(hs))
    for e, (h, f) in enumerate(zip(hs, fs)):
        for k in range(len(ck)):
            z = [scale[t] * M[h, idx[t]] * N[idx[t], f] for t in range(start[k], start[k + 1])]
            cd[e] += sum(z)
            if len(z) >= 2:
                zbar = sum(z) / len(z)
                s2[e] += len(z) / (len(z) - 1) * sum((v - zbar) ** 2 for v in z)
    return cd, s2, int(np.sum(ck == 1))


def entry_estimate_blocks(M, N, offsets, kidx, scale, entries):
    """(CD)_hf and c/(c - 1) sum_t (Z_t - Zbar)^2 with Z_t = scale_t (M^{k_t} N_{k_t})_hf, for c
    i.i.d. block draws (scale_t = 1/(c p_{k_t}), eq. 1.2 / 1.4): the same plug-in variance estimate
    for block sampling, whose terms are i.i.d. (Lemma 2.1's setting with one segment)."""
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    kidx = np.asarray(kidx, dtype=np.int64)
    scale = np.asarray(scale, dtype=np.float64)
    hs, fs = _entries(entries)
    c = len(kidx)
    cd = np.zeros(len(hs))
    s2 = np.zeros(len(hs))
    for e, (h, f) in enumerate(zip(hs, fs)):
        z = [scale[t] * float(M[h, off[k]:off[k + 1]] @ N[off[k]:off[k + 1], f]) for t, k in enumerate(kidx)]
        cd[e] = sum(z)
        if c >= 2:
            zbar = sum(z) / c
            s2[e] = c / (c - 1) * sum((v - zbar) ** 2 for v in z)
    return cd, s2


REPORT_FIELDS = (
    "expected_sq_error",  # Remark 2.2: sum_k (1/c_k)(sum_{i in k} x_i y_i / p_i - f_k)
    "eq310",              # (1/c) [sum_k (1 - v_k^2)^{1/2} a_k]^2
    "theta1", "theta2",   # min, max of 1 - v_k^2
    "beta",               # min(1, min_i p_i / p*_i)
    "m_fro2", "n_fro2",   # ||M||_F^2, ||N||_F^2
    "phi", "eq311",       # Thm 3.3
    "eta312", "eq312",    # Thm 3.3 with delta
    "phihat", "eq43",     # Thm 4.2
    "eta44", "eq44",      # Thm 4.2 with delta
    "theta1hat", "theta2hat", "phitilde", "eq48", "eta49", "eq49",  # Thm 4.4 (pilot f^_k)
)


def error_report(x, y, p, offsets, ck, a, f, mf, nf, c: int, delta: float, fhat=None) -> dict:
    """The quantities of REPORT_FIELDS (NaN where f or fhat is missing): Remark 2.2's expected squared
    error, eq. 3.10 and Thm 3.3's bounds (eq. 3.11 / 3.12), Thm 4.2's (eq. 4.3 / 4.4) and, with the
    pilot's fhat, Thm 4.4's (eq. 4.8 / 4.9)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    nan = float("nan")
    r = dict.fromkeys(REPORT_FIELDS, nan)
    r["m_fro2"] = float(np.sum(mf))
    r["n_fro2"] = float(np.sum(nf))
    prod = r["m_fro2"] * r["n_fro2"]
    # beta against the eq. 3.8 probabilities
    beta = 1.0
    for k in range(len(off) - 1):
        if a[k] > 0.0:
            for i in range(off[k], off[k + 1]):
                pstar = math.sqrt(x[i] * y[i]) / a[k]
                if pstar > 0.0:
                    beta = min(beta, p[i] / pstar)
    r["beta"] = beta
    log_term = math.sqrt(8.0 / beta * math.log(1.0 / delta))
    pos = a > 0.0
    if f is not None:
        f = np.asarray(f, dtype=np.float64)
        total = 0.0
        for k in range(len(off) - 1):
            q = 0.0
            for i in range(off[k], off[k + 1]):
                if p[i] > 0.0:
                    q += x[i] * y[i] / p[i]
            total += (q - f[k]) / ck[k]
        r["expected_sq_error"] = total
        r["eq310"] = float(np.sum(np.sqrt(np.maximum(a * a - f, 0.0)))) ** 2 / c
        one_minus = 1.0 - f[pos] / (a[pos] * a[pos])
        t1, t2 = float(one_minus.min()), float(one_minus.max())
        r["theta1"], r["theta2"] = t1, t2
        phi = math.sqrt(t2 - t1 * beta + t2 * t1 * beta) / (t2 * t1) ** 0.25 if t1 > 0.0 else math.inf
        r["phi"] = phi
        r["eq311"] = phi * phi / (beta * c) * prod
        eta = phi + math.sqrt(t2 / t1) * log_term if t1 > 0.0 else math.inf
        r["eta312"] = eta
        r["eq312"] = eta * eta / (beta * c) * prod
        phihat = math.sqrt(1.0 - beta * (1.0 - t2))
        r["phihat"] = phihat
        r["eq43"] = phihat * phihat / (beta * c) * prod
        r["eta44"] = phihat + log_term
        r["eq44"] = r["eta44"] ** 2 / (beta * c) * prod
        if fhat is not None:
            fh = np.asarray(fhat, dtype=np.float64)
            th = np.abs(1.0 - fh[pos] / (a[pos] * a[pos]))
            h1, h2 = float(th.min()), float(th.max())
            r["theta1hat"], r["theta2hat"] = h1, h2
            phit = math.sqrt(h2 - h1 * beta + t2 * h1 * beta) / (h2 * h1) ** 0.25 if h1 > 0.0 else math.inf
            r["phitilde"] = phit
            r["eq48"] = phit * phit / (beta * c) * prod
            r["eta49"] = phit + math.sqrt(h2 / h1) * log_term if h1 > 0.0 else math.inf
            r["eq49"] = r["eta49"] ** 2 / (beta * c) * prod
    return r

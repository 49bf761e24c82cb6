"""A CPU model of the block-size search that the CUDA kernel runs: a geometric first bracket
(32 candidates lam0 2^(w-8), lam0 = c / sum g), 32-way rounds over the IEEE bit patterns in the
bracket, and the exact endgame that locates every step of F in (lo, hi] (the smallest bit pattern
u with RN(u g_k) >= j, from RN(j / g_k) and single-pattern steps) and reads lam* off by rank.

The model is checked against the definition of lam* -- the largest FP64 bit pattern u with
F(u) = sum_k clamp(floor(u g_k), 1, n_k) <= c, i.e. F(lam*) <= c < F(lam* + 1) -- and against the
oracle's c_k, on random weights spanning many binades, zero weights and budgets from K to n; and the
endgame's step search is checked to end within two steps, as the kernel's bound of eight assumes."""
import struct

import numpy as np
import pytest

import oracle

INF = 0x7FF0000000000000


def lam(u):
    return struct.unpack("<d", struct.pack("<Q", int(u)))[0]


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def counts(u, g, nk):
    with np.errstate(invalid="ignore", over="ignore"):
        v = np.floor(np.float64(lam(u)) * g)
    v = np.where(g > 0, v, 1.0)
    return np.minimum(np.maximum(v, 1.0), nk).astype(np.int64)


def F(u, g, nk):
    return int(counts(u, g, nk).sum())


def breakpoint(gk, j):
    """Smallest pattern u with RN(u gk) >= j, and the number of single-pattern steps taken."""
    u = bits(np.float64(j) / np.float64(gk))
    steps = 0
    if np.float64(lam(u)) * gk >= j:
        while u > 0 and np.float64(lam(u - 1)) * gk >= j:
            u -= 1
            steps += 1
    else:
        while not (np.float64(lam(u)) * gk >= j):
            u += 1
            steps += 1
    return u, steps


def search(g, nk, c, stats):
    if F(INF, g, nk) <= c:
        return INF
    lo, hi = 0, INF
    lam0 = np.float64(c) / np.float64(np.sum(g.astype(np.float32), dtype=np.float32))
    b0 = bits(lam0)
    e0 = (b0 >> 52) & 0x7FF
    if np.isfinite(lam0) and lam0 > 0 and e0 >= 1:
        def geo(w):
            e = e0 + (w - 8)
            return INF if e >= 2047 else (0 if e <= 0 else b0 + ((w - 8) << 52))
        ok = [F(geo(w), g, nk) <= c for w in range(32)]
        t = sum(ok) - 1
        assert ok == [True] * (t + 1) + [False] * (31 - t)  # monotone: a prefix
        lo = geo(t) if t >= 0 else 0
        hi = geo(t + 1) if t < 31 else INF
    while hi - lo > 1:
        clo, chi = counts(lo, g, nk), counts(hi, g, nk)
        act = np.nonzero(clo != chi)[0]
        nbrk = int((chi - clo).sum())
        if 0 < nbrk <= 256:
            brk = []
            for k in act:
                for j in range(int(clo[k]) + 1, int(chi[k]) + 1):
                    u, st = breakpoint(g[k], j)
                    stats["max_steps"] = max(stats["max_steps"], st)
                    brk.append(u)
            brk.sort()
            r = c - int(clo.sum())
            stats["endgames"] += 1
            return brk[r] - 1
        d = hi - lo
        cand = [lo + (d >> 5) * w + (((d & 31) * w) >> 5) for w in range(32)]
        ok = [True] + [F(u, g, nk) <= c for u in cand[1:]]
        t = sum(ok) - 1
        lo, hi = cand[t], (cand[t + 1] if t < 31 else hi)
    return lo


def remainder(ustar, g, nk, c):
    ck = counts(ustar, g, nk)
    r = c - int(ck.sum())
    if r > 0 and ustar < INF:
        grow = np.nonzero(counts(ustar + 1, g, nk) > ck)[0]
        ck[grow[:r]] += 1
    elif r > 0:
        for k in range(len(g)):
            add = min(r, int(nk[k] - ck[k]))
            ck[k] += add
            r -= add
    return ck


@pytest.mark.parametrize("sigma", [0.5, 2.0, 6.0])
def test_search_model_finds_lambda_star(sigma):
    rng = np.random.default_rng(int(sigma * 10))
    stats = {"max_steps": 0, "endgames": 0}
    for case in range(60):
        K = int(rng.integers(1, 300))
        nk = rng.integers(1, 130, size=K)
        n = int(nk.sum())
        g = np.exp(rng.normal(0.0, sigma, size=K)) * 10.0 ** rng.integers(-30, 30)
        if case % 7 == 3:
            g[rng.random(K) < 0.3] = 0.0
        for c in (K, int(rng.integers(K, n + 1)), n):
            u = search(g, nk, c, stats)
            assert F(u, g, nk) <= c
            assert u == INF or F(u + 1, g, nk) > c
            np.testing.assert_array_equal(remainder(u, g, nk, c), oracle.apportion(g, nk, c))
    assert stats["endgames"] > 0
    assert stats["max_steps"] <= 2


def test_breakpoint_steps_are_bounded():
    # RN(j / g) is within a few units in the last place of the breakpoint for any j and g
    rng = np.random.default_rng(5)
    worst = 0
    for _ in range(20000):
        g = np.float64(np.exp(rng.normal(0, 20)))
        j = int(rng.integers(2, 1 << 20))
        u, st = breakpoint(g, j)
        assert np.float64(lam(u)) * g >= j and not (np.float64(lam(u - 1)) * g >= j)
        worst = max(worst, st)
    assert worst <= 2

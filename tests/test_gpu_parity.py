"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances, derived from the arithmetic of each step:
  statistics, probabilities   1e-12 relative (FP64-accurate sums on both sides)
  exact f_k (trace identity)  1e-10 relative (FP64-accurate dot products, cancellation in
                              the off-diagonal terms)
  block sizes, sample indices bit-exact given identical FP64 inputs
  sampled product             |CD_gpu - CD| <= tol * sum_t scale_t |M_{h,i_t}| |N_{i_t,f}| with
                              tol = 2^-7 + L 2^-22 (BF16: two operand roundings of 2^-8 plus
                              FP32 accumulation), 2^-14 + L 2^-22 (split BF16: hi+lo keeps
                              ~16 bits, lo*lo dropped), 1e-13 + L 2^-52 (FP64)
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests._gpu_util import as_layout, host, product_bound, rel_err, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bmm():
    import paper_2105_04940_gb300 as P
    P.build()
    P._abi.load()
    assert torch.cuda.is_available()
    return P


def _problem(m, n, p, K, seed, dtype=np.float64, lo=None, hi=None, sigma=1.0):
    if lo is None:
        off = S.block_offsets_equal(n, K)
    else:
        off = S.block_offsets_uneven(n, K, lo, hi, seed=seed)
    M, N = S.scaled_gaussian(m, n, p, off, sigma, seed=seed + 1, dtype=np.float64)
    if dtype == "bf16":
        Mt, Nt = to_dev(M, torch.bfloat16), to_dev(N, torch.bfloat16)
        M, N = host(Mt.double()), host(Nt.double())
    else:
        Mt, Nt = to_dev(M.astype(dtype)), to_dev(N.astype(dtype))
        M, N = M.astype(dtype).astype(np.float64), N.astype(dtype).astype(np.float64)
    return off, M, N, Mt, Nt


def _tol(mode, L):
    if mode == "bf16":
        return 2.0 ** -7 + L * 2.0 ** -22
    if mode == "split_bf16":
        return 2.0 ** -14 + L * 2.0 ** -22
    return 1e-13 + L * 2.0 ** -52


# ---------------------------------------------------------------- statistics and probabilities
@pytest.mark.parametrize("dtype", [np.float64, np.float32, "bf16"])
@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "col"), ("row", "col")])
def test_stats_and_probs(bmm, dtype, layouts):
    off, M, N, Mt, Nt = _problem(203, 3001, 157, 37, seed=3, dtype=dtype, lo=40, hi=120)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    prob = bmm.prepare(Mt, Nt, off, max_draws=500)
    p = torch.empty(3001, dtype=torch.float64, device=Mt.device)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_NONE, p, prob.st, prob.ws)
    bmm.check_status(prob)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    assert rel_err(host(prob.st["x"]), x) < 1e-12
    assert rel_err(host(prob.st["y"]), y) < 1e-12
    for k in ("a", "s", "mf", "nf"):
        assert rel_err(host(prob.st[k]), st[k]) < 1e-12, k
    assert rel_err(host(p), oracle.p_col_opt(st["w"], st["a"], off)) < 1e-12
    # block probabilities of eq. 1.4 and uniform ones, reusing the statistics
    pb = torch.empty(37, dtype=torch.float64, device=Mt.device)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_BLK_NORMPROD, bmm._abi.F_NONE | bmm._abi.REUSE_STATS, pb, prob.st, prob.ws)
    assert rel_err(host(pb), oracle.p_blk_normprod(st["mf"], st["nf"])) < 1e-12
    bmm.bmm_probs(None, None, prob.B, bmm._abi.P_COL_UNIFORM, bmm._abi.F_NONE, p, None, prob.ws)
    np.testing.assert_array_equal(host(p), oracle.p_col_uniform(off))
    bmm.check_status(prob)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_exact_block_frobenius(bmm, dtype):
    off, M, N, Mt, Nt = _problem(150, 1400, 90, 20, seed=5, dtype=dtype, lo=20, hi=110)
    prob = bmm.prepare(Mt, Nt, off, max_draws=300)
    pb = torch.empty(20, dtype=torch.float64, device=Mt.device)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_BLK_PRODNORM, bmm._abi.F_EXACT, pb, prob.st, prob.ws)
    bmm.check_status(prob)
    f = oracle.block_frob_sq(M, N, off)
    assert rel_err(host(prob.st["f"]), f) < 1e-10
    assert rel_err(host(pb), oracle.p_blk_prodnorm(f)) < 1e-10


def _tf32_gram_bound(M, N, off, m, p, round_in=2.0 ** -9):
    """Error scale of the off-diagonal trace from tensor-core Grams: tau * sum_{i != j} (|M|^T|M| |G_N| + |G_M| |N||N|^T)
    with tau = round_in + len * 2^-23 (FP32 accumulation); round_in = 2^-9 for TF32 (both factors
    rounded), 0 for BF16 inputs (their products are exact in FP32)."""
    out = []
    for a_, b_ in zip(off[:-1], off[1:]):
        A, B = M[:, a_:b_], N[a_:b_, :]
        GM, GN = A.T @ A, B @ B.T
        AM, AN = np.abs(A).T @ np.abs(A), np.abs(B) @ np.abs(B).T
        tM, tN = round_in + m * 2.0 ** -23, round_in + p * 2.0 ** -23
        E = tM * AM * np.abs(GN) + tN * np.abs(GM) * AN + tM * tN * AM * AN
        np.fill_diagonal(E, 0.0)
        out.append(E.sum())
    return np.array(out)


@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "col"), ("row", "col"), ("col", "row")])
@pytest.mark.parametrize("p", [264, 261])
@pytest.mark.parametrize("dtype", [np.float32, "bf16"])
def test_fused_statistics_and_tensor_core_f(bmm, layouts, p, dtype):
    """One pass for x, y, a_k, s_k, ||M^k||_F^2, ||N_k||_F^2 and f_k = s_k + tensor-core off-diagonal trace.

    Leading dimensions that are multiples of 16 bytes run the fused tensor-core pass (TF32 Grams for
    FP32, BF16 for BF16); others (p = 261, m = 300 for BF16) take the exact fallback."""
    m, n = 300, 6000
    off, M, N, Mt, Nt = _problem(m, n, p, 60, seed=41, dtype=dtype, lo=16, hi=128)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    prob = bmm.prepare(Mt, Nt, off, max_draws=100)
    pv = torch.empty(n, dtype=torch.float64, device=Mt.device)
    launches = bmm._abi.bmm_launch_count()
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_TC, pv, prob.st, prob.ws)
    bmm.check_status(prob)
    # the fused pass is one kernel after the window pass (plus the probabilities); odd leading
    # dimensions fall back
    ld_m = n if layouts[0] == "row" else m
    ld_n = p if layouts[1] == "row" else n
    align = 4 if dtype is np.float32 else 8
    fused = ld_m % align == 0 and ld_n % align == 0
    assert (bmm._abi.bmm_launch_count() - launches == 3) == fused
    assert bmm._abi.bmm_f_tc_supported(Mt, Nt, prob.B) == fused  # the query names the path that ran
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    assert rel_err(host(prob.st["x"]), x) < 1e-12
    assert rel_err(host(prob.st["y"]), y) < 1e-12
    for k in ("a", "s", "mf", "nf"):
        assert rel_err(host(prob.st[k]), st[k]) < 1e-12, k
    assert rel_err(host(pv), oracle.p_col_opt(st["w"], st["a"], off)) < 1e-12
    f = oracle.block_frob_sq(M, N, off)
    bound = _tf32_gram_bound(M, N, off, m, p, round_in=2.0 ** -9 if dtype is np.float32 else 0.0)
    err = np.abs(host(prob.st["f"]) - f)
    assert np.all(err <= bound + 1e-12 * f), np.max(err / (bound + 1e-300))
    # the statistics-reusing form computes f only, from the given s_k
    prob.st["f"].zero_()
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_BLK_PRODNORM, bmm._abi.F_TC | bmm._abi.REUSE_STATS, None, prob.st, prob.ws)
    bmm.check_status(prob)
    err = np.abs(host(prob.st["f"]) - f)
    assert np.all(err <= bound + 1e-12 * f)


@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "col"), ("row", "col"), ("col", "row")])
@pytest.mark.parametrize("dtype", [np.float32, "bf16"])
def test_fused_statistics_offsets_wide_and_low_rank_blocks(bmm, layouts, dtype):
    """Blocks at every offset mod 4 (FP32) or mod 8 (BF16): strided tiles start at the 16-byte
    boundary below the block; the widest blocks (FP32: 127 at offset 3 and 128 at offset 1;
    BF16: 128 at offset 7) exceed the 128 operand rows of an in-place strided tile, 126 at offset 2
    fills them exactly; tiny blocks; and one rank-one block (off-diagonal trace as large as the
    diagonal)."""
    rng = np.random.default_rng(3)
    if dtype is np.float32:
        sizes = np.array([3, 127, 126, 128, 1, 128, 5, 77, 16, 100, 34, 3])  # n = 748: every ld % 4 == 0
        low_rank = 7
    else:
        sizes = np.array([7, 128, 1, 127, 2, 126, 128, 5, 77, 16, 100, 34, 1])  # n = 752: every ld % 8 == 0
        low_rank = 8
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n, m, p = int(off[-1]), 96, 152
    M = rng.standard_normal((m, n)).astype(np.float32)
    N = rng.standard_normal((n, p)).astype(np.float32)
    u, v = rng.standard_normal(m), rng.standard_normal(p)
    w = rng.standard_normal(sizes[low_rank])
    M[:, off[low_rank]:off[low_rank + 1]] = np.outer(u, w)
    N[off[low_rank]:off[low_rank + 1], :] = np.outer(w, v)
    tdt = torch.float32 if dtype is np.float32 else torch.bfloat16
    Mt = as_layout(to_dev(M, tdt), layouts[0])
    Nt = as_layout(to_dev(N, tdt), layouts[1])
    M, N = host(Mt.double()), host(Nt.double())
    prob = bmm.prepare(Mt, Nt, off, max_draws=50)
    launches = bmm._abi.bmm_launch_count()
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_TC, None, prob.st, prob.ws)
    bmm.check_status(prob)
    assert bmm._abi.bmm_launch_count() - launches == 2  # the window pass and the fused pass (no p requested)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    assert rel_err(host(prob.st["x"]), x) < 1e-12
    assert rel_err(host(prob.st["y"]), y) < 1e-12
    for k in ("a", "s", "mf", "nf"):
        assert rel_err(host(prob.st[k]), st[k]) < 1e-12, k
    f = oracle.block_frob_sq(M, N, off)
    err = np.abs(host(prob.st["f"]) - f)
    round_in = 2.0 ** -9 if dtype is np.float32 else 0.0
    assert np.all(err <= _tf32_gram_bound(M, N, off, m, p, round_in) + 1e-12 * f)
    # the Gram-only form (statistics reused) gives the same f
    f_fused = host(prob.st["f"]).copy()
    prob.st["f"].zero_()
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_BLK_PRODNORM, bmm._abi.F_TC | bmm._abi.REUSE_STATS, None, prob.st, prob.ws)
    bmm.check_status(prob)
    assert np.array_equal(host(prob.st["f"]), f_fused)


@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "row")])
@pytest.mark.parametrize("dtype", [np.float32, "bf16"])
def test_fused_statistics_packed_small_blocks(bmm, layouts, dtype):
    """Consecutive small blocks share one 128-vector MMA tile (a window): 5000 blocks of 1..8
    vectors, more than two passes of the window search, with wide blocks (121..128 vectors) that
    stay alone.  Per-block statistics and f_k as the oracle, in the fused and Gram-only forms."""
    rng = np.random.default_rng(11)
    sizes = rng.integers(1, 9, size=5000)
    sizes[rng.choice(5000, size=12, replace=False)] = rng.integers(121, 129, size=12)
    align = 4 if dtype is np.float32 else 8
    sizes[-1] += (-int(sizes.sum())) % align  # row-major M needs ld = n aligned to 16 bytes
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n, m, p = int(off[-1]), 40, 72
    M = rng.standard_normal((m, n)).astype(np.float32)
    N = rng.standard_normal((n, p)).astype(np.float32)
    tdt = torch.float32 if dtype is np.float32 else torch.bfloat16
    Mt = as_layout(to_dev(M, tdt), layouts[0])
    Nt = as_layout(to_dev(N, tdt), layouts[1])
    M, N = host(Mt.double()), host(Nt.double())
    prob = bmm.prepare(Mt, Nt, off, max_draws=50)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_TC, None, prob.st, prob.ws)
    bmm.check_status(prob)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    assert rel_err(host(prob.st["x"]), x) < 1e-12
    assert rel_err(host(prob.st["y"]), y) < 1e-12
    for k in ("a", "s", "mf", "nf"):
        assert rel_err(host(prob.st[k]), st[k]) < 1e-12, k
    f = oracle.block_frob_sq(M, N, off)
    round_in = 2.0 ** -9 if dtype is np.float32 else 0.0
    bound = _tf32_gram_bound(M, N, off, m, p, round_in)
    assert np.all(np.abs(host(prob.st["f"]) - f) <= bound + 1e-12 * f)
    f_fused = host(prob.st["f"]).copy()
    prob.st["f"].zero_()
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_BLK_PRODNORM, bmm._abi.F_TC | bmm._abi.REUSE_STATS, None, prob.st, prob.ws)
    bmm.check_status(prob)
    assert np.array_equal(host(prob.st["f"]), f_fused)


# ---------------------------------------------------------------- block sizes (identical inputs)
@pytest.mark.parametrize("kind", ["opt", "hat", "equal"])
@pytest.mark.parametrize("K", [300, 3000])
def test_blocksizes_bit_exact(bmm, kind, K):
    """Bit-exact against the oracle given the same FP64 inputs; K = 300 keeps every block in the
    kernel's shared-memory lists (FP32-decided counts with FP64 fallback), K = 3000 does not."""
    rng = np.random.default_rng(9)
    nk = rng.integers(1, 200 if K <= 300 else 40, size=K)
    off = np.concatenate([[0], np.cumsum(nk)]).astype(np.int64)
    n = int(off[-1])
    a = rng.lognormal(0, 2, size=K)
    f = a * a * rng.uniform(0, 1, size=K)
    f[::17] = a[::17] ** 2  # rank-one aligned blocks: g = 0
    dev = torch.device("cuda:0")
    st = {k: torch.zeros(K if k not in ("x", "y") else n, dtype=torch.float64, device=dev)
          for k in ("x", "y", "a", "s", "mf", "nf", "f")}
    st["a"].copy_(torch.from_numpy(a))
    st["f"].copy_(torch.from_numpy(f))
    off_dev = torch.as_tensor(off, device=dev)
    B = bmm._abi.blocks(off_dev, n, int(nk.max()))
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
    ck = torch.empty(K, dtype=torch.int64, device=dev)
    g = torch.empty(K, dtype=torch.float64, device=dev)
    ckind = {"opt": bmm._abi.CK_OPT, "hat": bmm._abi.CK_HAT, "equal": bmm._abi.CK_EQUAL}[kind]
    gw = {"opt": oracle.g_opt(a, f), "hat": oracle.g_hat(a), "equal": oracle.g_equal(K)}[kind]
    for c in (K, K + 1, 2 * K + 7, n // 3, n - 1, n):
        bmm.bmm_blocksizes(None, None, B, st, ckind, c, None, None, 0, ck, g, None, ws)
        assert bmm.bmm_read_device_status(ws) == 0
        want = oracle.apportion(oracle.g_with_fallback(gw, a, nk), nk, c)
        np.testing.assert_array_equal(host(ck), want, err_msg=f"c={c}")
        np.testing.assert_array_equal(host(g), oracle.g_with_fallback(gw, a, nk))
    with pytest.raises(bmm.BmmError):
        bmm.bmm_blocksizes(None, None, B, st, ckind, K - 1, None, None, 0, ck, g, None, ws)


# ---------------------------------------------------------------- sampler (identical p)
@pytest.mark.parametrize("seed", [0, 1, 2 ** 40 + 5])
def test_sampler_bit_exact_columns(bmm, seed):
    off = S.block_offsets_uneven(5000, 40, 20, 400, seed=seed % 97)
    p = S.random_probabilities(off, seed=seed % 89, zero_frac=0.2)
    K = 40
    nk = np.diff(off)
    ck = oracle.apportion(oracle.g_hat(np.ones(K)), nk, 1500)
    sid = oracle.stream_id(3, oracle.PURPOSE_MAIN)
    want_idx, want_scale = oracle.sample_alg2(p, off, ck, seed, sid)
    dev = torch.device("cuda:0")
    off_dev = torch.as_tensor(off, device=dev)
    B = bmm._abi.blocks(off_dev, 5000, int(nk.max()))
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
    idx = torch.empty(1500, dtype=torch.int32, device=dev)
    scale = torch.empty(1500, dtype=torch.float64, device=dev)
    bmm.bmm_sample(to_dev(p), bmm._abi.UNIT_COLUMN, B, to_dev(ck), 1500, seed, sid, idx, scale, ws)
    assert bmm.bmm_read_device_status(ws) == 0
    np.testing.assert_array_equal(host(idx), want_idx)
    np.testing.assert_array_equal(host(scale), want_scale)


def test_sampler_bit_exact_blocks_and_long_segment(bmm):
    dev = torch.device("cuda:0")
    ws = torch.zeros(1 << 22, dtype=torch.uint8, device=dev)
    # one segment longer than a scan tile (K = 1: Alg. 1)
    n = 70000
    off = np.array([0, n])
    p = S.random_probabilities(off, seed=4, zero_frac=0.5)
    off_dev = torch.as_tensor(off, device=dev)  # kept alive: the struct holds only its address
    B = bmm._abi.blocks(off_dev, n, n)
    idx = torch.empty(3000, dtype=torch.int32, device=dev)
    scale = torch.empty(3000, dtype=torch.float64, device=dev)
    bmm.bmm_sample(to_dev(p), bmm._abi.UNIT_COLUMN, B, to_dev(np.array([3000])), 3000, 77, 0, idx, scale, ws)
    wi, wsc = oracle.sample_alg2(p, off, np.array([3000]), 77, 0)
    np.testing.assert_array_equal(host(idx), wi)
    np.testing.assert_array_equal(host(scale), wsc)
    # block sampling over K blocks
    off = S.block_offsets_uneven(20000, 2500, 4, 12, seed=1)
    pb = S.random_probabilities(np.array([0, 2500]), seed=2, zero_frac=0.3)
    off_dev = torch.as_tensor(off, device=dev)
    B = bmm._abi.blocks(off_dev, 20000, 12)
    idx = torch.empty(700, dtype=torch.int32, device=dev)
    scale = torch.empty(700, dtype=torch.float64, device=dev)
    bmm.bmm_sample(to_dev(pb), bmm._abi.UNIT_BLOCK, B, None, 700, 5, 1, idx, scale, ws)
    assert bmm.bmm_read_device_status(ws) == 0
    wi, wsc = oracle.sample_blocks(pb, 700, 5, 1)
    np.testing.assert_array_equal(host(idx), wi)
    np.testing.assert_array_equal(host(scale), wsc)


# ---------------------------------------------------------------- sampled product
@pytest.mark.parametrize("mode", ["f64", "bf16", "split_bf16"])
@pytest.mark.parametrize("shape", [(300, 2000, 520), (70, 1200, 100)])
@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "row")])
def test_apply_columns(bmm, mode, shape, layouts):
    m, n, p = shape
    off, M, N, Mt, Nt = _problem(m, n, p, 25, seed=11, dtype=np.float32, lo=20, hi=140)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    L = 517
    prob = bmm.prepare(Mt, Nt, off, max_draws=L)
    r = bmm.run(prob, "ONC", L, seed=4, gemm_mode=bmm.MODES[mode])
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    want = oracle.sampled_product_columns(M, N, idx, scale)
    bound = product_bound(M, N, idx, scale)
    got = host(r["out"]).astype(np.float64)
    assert np.all(np.abs(got - want) <= _tol(mode, L) * bound + 1e-300), np.max(np.abs(got - want) / bound)


def _e4m3_bound(M, N, cols, w, L):
    """Element-wise error bound of the e4m3 sampled product.  Per drawn index j (column c_j of M, row
    c_j of N, weight w_j): a = M[:, c_j] sqrt(w_j), b = N[c_j, :] sqrt(w_j); the kernel scales a by
    2^(e_j + gA) and b by 2^(gB - e_j) (e_j balances max|a| and max|b|, gA and gB bring each operand's
    largest value to at most 448) and rounds to e4m3: |q(x) - x| <= 2^-4 |x| in the normal range, or
    2^-10 in scaled units below it.  The exponents are recomputed here in FP64; the subnormal terms
    carry a factor 4 for an exponent one off from the kernel's."""
    u = 2.0 ** -4
    sw = np.sqrt(np.asarray(w, dtype=np.float64))
    Aa = np.abs(M[:, cols]) * sw[None, :]
    Bb = np.abs(N[cols, :]) * sw[:, None]
    al, be = Aa.max(axis=0), Bb.max(axis=1)
    e = np.zeros(len(cols))
    pos = (al > 0) & (be > 0)
    e[pos] = np.clip(np.rint(0.5 * np.log2(be[pos] / al[pos])), -60, 60)
    gA = int(np.floor(np.log2(448.0 / np.max(al * 2.0 ** e)))) if np.any(al > 0) else 0
    gB = int(np.floor(np.log2(448.0 / np.max(be * 2.0 ** -e)))) if np.any(be > 0) else 0
    da = 4 * 2.0 ** -10 * 2.0 ** -(e + gA)
    db = 4 * 2.0 ** -10 * 2.0 ** -(gB - e)
    AB = Aa @ Bb
    bound = (2 * u + u * u + 1.2 * L * 2.0 ** -23) * AB
    bound += (1 + u) * ((da @ Bb)[None, :] + (Aa @ db)[:, None]) + np.sum(da * db)
    return bound


@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "row"), ("row", "col")])
@pytest.mark.parametrize("shape", [(300, 2000, 520), (70, 1200, 100)])
def test_apply_columns_e4m3(bmm, shape, layouts):
    """FP8 e4m3 operands with per-outer-product balancing scales and per-operand powers of two."""
    m, n, p = shape
    off, M, N, Mt, Nt = _problem(m, n, p, 25, seed=11, dtype=np.float32, lo=20, hi=140)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    L = 517
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=bmm._abi.GEMM_E4M3)
    r = bmm.run(prob, "ONC", L, seed=4, gemm_mode=bmm._abi.GEMM_E4M3)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    want = oracle.sampled_product_columns(M, N, idx, scale)
    got = host(r["out"]).astype(np.float64)
    bound = _e4m3_bound(M, N, idx, scale, L)
    assert np.all(np.abs(got - want) <= bound + 1e-300), np.max(np.abs(got - want) / bound)
    assert np.linalg.norm(got - want) <= 0.1 * np.linalg.norm(want)


def test_apply_blocks_e4m3(bmm):
    off, M, N, Mt, Nt = _problem(260, 3000, 300, 50, seed=12, dtype=np.float32, lo=10, hi=110)
    prob = bmm.prepare(Mt, Nt, off, max_draws=9, unit=bmm._abi.UNIT_BLOCK, gemm_mode=bmm._abi.GEMM_E4M3)
    r = bmm.run(prob, "SSM", 9, seed=2, gemm_mode=bmm._abi.GEMM_E4M3)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    want = oracle.sampled_product_blocks(M, N, off, idx, scale)
    cols = np.concatenate([np.arange(off[k], off[k + 1]) for k in idx])
    w = np.concatenate([np.full(off[k + 1] - off[k], sc) for k, sc in zip(idx, scale)])
    got = host(r["out"]).astype(np.float64)
    bound = _e4m3_bound(M, N, cols, w, len(cols))
    assert np.all(np.abs(got - want) <= bound + 1e-300), np.max(np.abs(got - want) / bound)


@pytest.mark.parametrize("mode", ["f64", "bf16"])
def test_apply_blocks(bmm, mode):
    off, M, N, Mt, Nt = _problem(260, 3000, 300, 50, seed=12, dtype=np.float32, lo=10, hi=110)
    prob = bmm.prepare(Mt, Nt, off, max_draws=9, unit=bmm._abi.UNIT_BLOCK)
    r = bmm.run(prob, "SSM", 9, seed=2, gemm_mode=bmm.MODES[mode])
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    want = oracle.sampled_product_blocks(M, N, off, idx, scale)
    bound = product_bound(M, N, idx, scale, off, unit="block")
    L = int(sum(off[k + 1] - off[k] for k in idx))
    got = host(r["out"]).astype(np.float64)
    assert np.all(np.abs(got - want) <= _tol(mode, L) * bound + 1e-300)


def test_apply_accumulate_and_empty(bmm):
    off, M, N, Mt, Nt = _problem(64, 256, 64, 4, seed=13, dtype=np.float64)
    prob = bmm.prepare(Mt, Nt, off, max_draws=16)
    out = torch.ones(64, 64, dtype=torch.float64, device=Mt.device)
    idx = to_dev(np.arange(0, 256, 16).astype(np.int32))
    scale = to_dev(np.full(16, 2.0))
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, idx, scale, 16, bmm._abi.GEMM_F64, out, True, prob.ws)
    want = 1.0 + 2.0 * M[:, ::16] @ N[::16, :]
    np.testing.assert_allclose(host(out), want, rtol=1e-12, atol=1e-12)
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, idx, scale, 0, bmm._abi.GEMM_F64, out, False, prob.ws)
    assert np.all(host(out) == 0.0)


def test_every_index_once_reproduces_product(bmm):
    off, M, N, Mt, Nt = _problem(200, 640, 180, 10, seed=14, dtype=np.float64)
    prob = bmm.prepare(Mt, Nt, off, max_draws=640)
    out = torch.empty(200, 180, dtype=torch.float64, device=Mt.device)
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, to_dev(np.arange(640, dtype=np.int32)),
                  to_dev(np.ones(640)), 640, bmm._abi.GEMM_F64, out, False, prob.ws)
    np.testing.assert_allclose(host(out), M @ N, rtol=1e-12, atol=1e-10)


# ---------------------------------------------------------------- methods end to end
@pytest.mark.parametrize("method", ["OPL", "ONC", "ONU", "ONMCNR", "UU", "SSM", "WU"])
def test_methods_match_oracle(bmm, method):
    off = S.block_offsets_equal(4096, 64)
    M, N = S.scaled_gaussian(256, 4096, 256, off, 1.0, seed=1)
    Mt, Nt = to_dev(M), to_dev(N)
    c = 16 if method in ("SSM", "WU") else 1024
    prob = bmm.prepare(Mt, Nt, off, max_draws=1024, unit=bmm._abi.UNIT_BLOCK if method in ("SSM", "WU") else 0)
    r = bmm.run(prob, method, c, seed=7, c0=256, gemm_mode=bmm._abi.GEMM_F64)
    bmm.check_status(prob)
    o = oracle.run_method(M, N, off, method, c, seed=7, c0=256)
    assert rel_err(host(r["p"]), o["p"]) < 1e-12
    if "ck" in o:
        np.testing.assert_array_equal(host(r["ck"]), o["ck"])
    if "fhat" in o:
        assert rel_err(host(r["fhat"]), o["fhat"]) < 1e-10
    np.testing.assert_array_equal(host(r["idx"]), o["idx"])
    np.testing.assert_allclose(host(r["scale"]), o["scale"], rtol=1e-12)
    np.testing.assert_allclose(host(r["out"]), o["CD"], rtol=1e-10, atol=1e-10 * np.abs(o["CD"]).max())


def test_tilde_block_sizes_from_pilot(bmm):
    off = S.block_offsets_uneven(3000, 30, 40, 160, seed=2)
    M, N = S.scaled_gaussian(120, 3000, 90, off, 1.5, seed=3)
    Mt, Nt = to_dev(M), to_dev(N)
    prob = bmm.prepare(Mt, Nt, off, max_draws=2000)
    r = bmm.run(prob, "ONU", 600, seed=3, c0=30 * 40, gemm_mode=bmm._abi.GEMM_F64)
    bmm.check_status(prob)
    fhat, pidx, pscale, _ = None, host(r["pilot_idx"]), host(r["pilot_scale"]), None
    fh_or, idx_or, sc_or = oracle.pilot_frob_sq(M, N, off, oracle.p_col_uniform(off), 40, seed=3,
                                                sid=oracle.stream_id(0, oracle.PURPOSE_PILOT))
    np.testing.assert_array_equal(pidx, idx_or)
    np.testing.assert_array_equal(pscale, sc_or)
    assert rel_err(host(r["fhat"]), fh_or) < 1e-10
    # the integer decision, given the GPU's own fhat, is the oracle's
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    g = oracle.g_tilde(host(prob.st["a"]), host(r["fhat"]))
    np.testing.assert_array_equal(host(r["ck"]), oracle.apportion(oracle.g_with_fallback(g, st["a"], np.diff(off)), np.diff(off), 600))


@pytest.mark.parametrize("per", [1, 3, 4, 8, 9])
@pytest.mark.parametrize("dtype,layout", [(np.float32, "row"), (np.float32, "col"), ("bf16", "row"), (np.float64, "row")])
def test_pilot_fhat_small_and_tiled(bmm, per, dtype, layout):
    """Alg. 3 pilot f^_k with 1..8 draws per block (the one-CTA-per-block kernel, rounded up to
    1, 2, 4 or 8 vectors) and 9 (the tiled kernel), every storage order of M and element type."""
    off, M, N, Mt, Nt = _problem(300, 2200, 170, 20, seed=31, dtype=dtype, lo=40, hi=180)
    Mt = as_layout(Mt, layout)
    K = len(off) - 1
    prob = bmm.prepare(Mt, Nt, off, max_draws=800)
    r = bmm.run(prob, "ONU", 400, seed=5, c0=per * K, gemm_mode=bmm._abi.GEMM_F64)
    bmm.check_status(prob)
    fh_or, idx_or, sc_or = oracle.pilot_frob_sq(M, N, off, oracle.p_col_uniform(off), per, seed=5,
                                                sid=oracle.stream_id(0, oracle.PURPOSE_PILOT))
    np.testing.assert_array_equal(host(r["pilot_idx"]), idx_or)
    np.testing.assert_array_equal(host(r["pilot_scale"]), sc_or)
    assert rel_err(host(r["fhat"]), fh_or) < 1e-10


@pytest.mark.parametrize("dtype", [np.float64, np.float32, "bf16"])
@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "col")])
def test_exact_f_direct_form_large_blocks(bmm, dtype, layouts):
    """Exact f_k = ||M^k N_k||_F^2 for blocks of thousands of vectors with small m, p (the shape of
    the paper's experiments): the direct m x p product per block (FP64 sums over slices of the
    block) replaces the Gram form, whose n_k^2 pair tiles it would not take."""
    m, p, n, K = 26, 28, 20000, 4
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=51, dtype=dtype, lo=2000, hi=8000)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    prob = bmm.prepare(Mt, Nt, off, max_draws=2000)
    pv = torch.empty(n, dtype=torch.float64, device=Mt.device)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_EXACT, pv, prob.st, prob.ws)
    bmm.check_status(prob)
    assert rel_err(host(prob.st["f"]), oracle.block_frob_sq(M, N, off)) < 1e-10
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    assert rel_err(host(pv), oracle.p_col_opt(st["w"], st["a"], off)) < 1e-12


@pytest.mark.parametrize("per", [40, 500])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pilot_fhat_direct_form(bmm, per, dtype):
    """Alg. 3 pilots of 40 and 500 draws per block with m = 26, p = 28: f^_k through the direct
    product of the drawn, rescaled outer products, against the oracle."""
    m, p, n, K = 26, 28, 12000, 6
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=53, dtype=dtype, lo=1000, hi=3000)
    prob = bmm.prepare(Mt, Nt, off, max_draws=per * K)
    r = bmm.run(prob, "ONMCNR", 3 * K, seed=9, c0=per * K, gemm_mode=bmm._abi.GEMM_F64)
    bmm.check_status(prob)
    fh_or, idx_or, sc_or = oracle.pilot_frob_sq(M, N, off, host(r["p0"]), per, seed=9,
                                                sid=oracle.stream_id(0, oracle.PURPOSE_PILOT))
    np.testing.assert_array_equal(host(r["pilot_idx"]), idx_or)
    assert rel_err(host(r["fhat"]), fh_or) < 1e-10


@pytest.mark.parametrize("L", [5000, 20011])
def test_f64_product_split_k(bmm, L):
    """FP64 sampled product of a 26 x 28 output (one 64 x 64 tile) with thousands of drawn columns:
    the K range is split over CTAs and the partial tiles summed in split order; against the
    oracle's FP64 product of the same draws, and identical on a second call."""
    m, p, n, K = 26, 28, 30000, 10
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=57, dtype=np.float64)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L)
    r = bmm.run(prob, "ONC", L, seed=4, gemm_mode=bmm._abi.GEMM_F64)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    want = oracle.sampled_product_columns(M, N, idx, scale)
    bound = product_bound(M, N, idx, scale)
    assert np.all(np.abs(host(r["out"]) - want) <= _tol("f64", L) * bound + 1e-300)
    first = host(r["out"]).copy()
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, r["idx"], r["scale"], L, bmm._abi.GEMM_F64, r["out"], False,
                  prob.ws)
    np.testing.assert_array_equal(host(r["out"]), first)


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("mode", ["f64", "bf16"])
@pytest.mark.parametrize("unit", ["column", "block"])
def test_backward(bmm, mode, unit):
    off, M, N, Mt, Nt = _problem(136, 1500, 200, 15, seed=21, dtype=np.float32 if mode == "bf16" else np.float64,
                                 lo=40, hi=160)
    method, c = ("ONC", 400) if unit == "column" else ("SSM", 6)
    gm = bmm.MODES[mode]
    prob = bmm.prepare(Mt, Nt, off, max_draws=c, unit=bmm._abi.UNIT_BLOCK if unit == "block" else 0)
    r = bmm.run(prob, method, c, seed=8, gemm_mode=gm)
    G = np.random.default_rng(5).standard_normal((136, 200))
    gdt = torch.float64 if mode == "f64" else torch.float32
    Gt = to_dev(G.astype(np.float64 if mode == "f64" else np.float32))
    dM = torch.full(Mt.shape, 7.0, dtype=gdt, device=Mt.device)
    dN = torch.full(Nt.shape, 7.0, dtype=gdt, device=Mt.device)
    bmm.bmm_backward(Gt, Mt, Nt, prob.B, r["unit"], r["p"], r["ck"], c, 8, r["sid"], gm, dM, dN, False, prob.ws)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    Gd = host(Gt).astype(np.float64)
    if unit == "column":
        wM, wN = oracle.adjoint_columns(M, N, idx, scale, Gd)
    else:
        wM, wN = oracle.adjoint_blocks(M, N, off, idx, scale, Gd)
    tol = 1e-11 if mode == "f64" else 2.0 ** -7 + 300 * 2.0 ** -22
    # error scale: the same sums with absolute values
    if unit == "column":
        bM, bN = oracle.adjoint_columns(np.abs(M), np.abs(N), idx, scale, np.abs(Gd))
    else:
        bM, bN = oracle.adjoint_blocks(np.abs(M), np.abs(N), off, idx, scale, np.abs(Gd))
    assert np.all(np.abs(host(dM) - wM) <= tol * bM + 1e-300)
    assert np.all(np.abs(host(dN) - wN) <= tol * bN + 1e-300)
    # accumulate=1 adds onto the existing gradient
    dM2 = torch.ones_like(dM)
    bmm.bmm_backward(Gt, Mt, Nt, prob.B, r["unit"], r["p"], r["ck"], c, 8, r["sid"], gm, dM2, None, True, prob.ws)
    np.testing.assert_allclose(host(dM2) - 1.0, host(dM), rtol=1e-6 if mode == "bf16" else 1e-13,
                               atol=1e-6 * np.abs(host(dM)).max())


@pytest.mark.parametrize("unit", ["column", "block"])
@pytest.mark.parametrize("layout", ["row", "col"])
def test_backward_bf16_gradients(bmm, unit, layout):
    """BF16 inputs, BF16 mode: gradients written as BF16 equal the FP32 gradients rounded to BF16,
    bit for bit (every touched element is rounded once); untouched ones are zero; both storage
    orders of the gradient."""
    off, M, N, Mt, Nt = _problem(136, 1500, 200, 15, seed=23, dtype="bf16", lo=40, hi=160)
    method, c = ("ONC", 400) if unit == "column" else ("SSM", 6)
    gm = bmm._abi.GEMM_BF16
    prob = bmm.prepare(Mt, Nt, off, max_draws=c, unit=bmm._abi.UNIT_BLOCK if unit == "block" else 0)
    r = bmm.run(prob, method, c, seed=8, gemm_mode=gm)
    Gt = to_dev(np.random.default_rng(6).standard_normal((136, 200)).astype(np.float32))
    args = (Gt, Mt, Nt, prob.B, r["unit"], r["p"], r["ck"], c, 8, r["sid"], gm)
    dM32 = torch.empty(Mt.shape, dtype=torch.float32, device=Mt.device)
    dN32 = torch.empty(Nt.shape, dtype=torch.float32, device=Mt.device)
    bmm.bmm_backward(*args, dM32, dN32, False, prob.ws)
    dM16 = as_layout(torch.full(Mt.shape, 3.0, dtype=torch.bfloat16, device=Mt.device), layout)
    dN16 = as_layout(torch.full(Nt.shape, 3.0, dtype=torch.bfloat16, device=Mt.device), layout)
    bmm.bmm_backward(*args, dM16, dN16, False, prob.ws)
    bmm.check_status(prob)
    np.testing.assert_array_equal(host(dM16.float()), host(dM32.to(torch.bfloat16).float()))
    np.testing.assert_array_equal(host(dN16.float()), host(dN32.to(torch.bfloat16).float()))


def test_autograd_function(bmm):
    off = S.block_offsets_equal(512, 8)
    M, N = S.scaled_gaussian(64, 512, 64, off, 1.0, seed=11)
    Mt = to_dev(M).requires_grad_(True)
    Nt = to_dev(N).requires_grad_(True)
    out = bmm.sampled_matmul(Mt, Nt, off, method="ONC", c=128, seed=5, mode="f64")
    R = to_dev(np.random.default_rng(12).standard_normal((64, 64)))
    (out * R).sum().backward()
    r = oracle.run_method(M, N, off, "ONC", 128, seed=5)
    wM, wN = oracle.adjoint_columns(M, N, r["idx"], r["scale"], host(R))
    np.testing.assert_allclose(host(Mt.grad), wM, rtol=1e-10, atol=1e-10 * np.abs(wM).max())
    np.testing.assert_allclose(host(Nt.grad), wN, rtol=1e-10, atol=1e-10 * np.abs(wN).max())


# ---------------------------------------------------------------- device-detected conditions
def test_device_status_conditions(bmm):
    off, M, N, Mt, Nt = _problem(32, 128, 16, 4, seed=30, dtype=np.float64)
    Mt[3, 5] = float("nan")
    prob = bmm.prepare(Mt, Nt, off, max_draws=32)
    p = torch.empty(128, dtype=torch.float64, device=Mt.device)
    bmm.bmm_probs(Mt, Nt, prob.B, bmm._abi.P_COL_OPT, bmm._abi.F_NONE, p, prob.st, prob.ws)
    assert bmm.bmm_read_device_status(prob.ws) == bmm._abi.ERR_NONFINITE
    bmm.bmm_clear_device_status(prob.ws)
    assert bmm.bmm_read_device_status(prob.ws) == 0
    # a probability segment without mass
    pz = torch.zeros(128, dtype=torch.float64, device=Mt.device)
    ck = to_dev(np.full(4, 2, dtype=np.int64))
    idx = torch.empty(8, dtype=torch.int32, device=Mt.device)
    sc = torch.empty(8, dtype=torch.float64, device=Mt.device)
    bmm.bmm_sample(pz, bmm._abi.UNIT_COLUMN, prob.B, ck, 8, 1, 0, idx, sc, prob.ws)
    assert bmm.bmm_read_device_status(prob.ws) == bmm._abi.ERR_ARG
    bmm.bmm_clear_device_status(prob.ws)
    # c_k that do not add up to c
    bmm.bmm_sample(to_dev(oracle.p_col_uniform(off)), bmm._abi.UNIT_COLUMN, prob.B, ck, 7, 1, 0, idx, sc, prob.ws)
    assert bmm.bmm_read_device_status(prob.ws) == bmm._abi.ERR_INFEASIBLE
    bmm.bmm_clear_device_status(prob.ws)
    # offsets that are not increasing (validated on the device, nothing read out of range)
    bad = to_dev(np.array([0, 40, 30, 90, 128], dtype=np.int64))
    Bbad = bmm._abi.blocks(bad, 128, 60)
    Mt[3, 5] = 0.0
    bmm.bmm_probs(Mt, Nt, Bbad, bmm._abi.P_COL_OPT, bmm._abi.F_NONE, p, prob.st, prob.ws)
    assert bmm.bmm_read_device_status(prob.ws) == bmm._abi.ERR_SHAPE
    bmm.bmm_clear_device_status(prob.ws)
    # host-side rejections
    with pytest.raises(bmm.BmmError) as e:
        bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, idx, sc, 8, bmm._abi.GEMM_BF16,
                      torch.empty(32, 16, dtype=torch.float64, device=Mt.device), False, prob.ws)
    assert e.value.code == bmm._abi.ERR_DTYPE
    with pytest.raises(bmm.BmmError) as e:
        bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, idx, sc, 8, bmm._abi.GEMM_F64,
                      torch.empty(32, 16, dtype=torch.float64, device=Mt.device), False, prob.ws[:100])
    assert e.value.code == bmm._abi.ERR_WORKSPACE


def test_mlp_forward_backward_matches_oracle_chain(bmm):
    """Differentiation configuration at small size: y_l = GELU(y_{l-1} W_l) with every product sampled
    (ONC, K = 8 blocks of 64, c = 2 blocks -> L = 128), forward and backward in FP64 through the
    autograd function, against the same chain built from the oracle's sample and adjoint."""
    import math
    rng = np.random.default_rng(17)
    m, n = 64, 512
    off = S.block_offsets_equal(n, 8)
    L = bmm.equal_budget(2, n, 8)
    X = rng.standard_normal((m, n))
    Ws = [rng.standard_normal((n, n)) / math.sqrt(n) for _ in range(4)]
    R = rng.standard_normal((m, n))

    def gelu(z):
        return 0.5 * z * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))

    def dgelu(z):
        return 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)

    # oracle chain
    h, pre, samples = X, [], []
    for l, W in enumerate(Ws):
        r = oracle.run_method(h, W, off, "ONC", L, seed=100 + l)
        pre.append((h, r["CD"]))
        samples.append((r["idx"], r["scale"]))
        h = gelu(r["CD"])
    G = R.copy()
    dWs = [None] * 4
    for l in range(3, -1, -1):
        hin, z = pre[l]
        G = G * dgelu(z)
        dh, dW = oracle.adjoint_columns(hin, Ws[l], samples[l][0], samples[l][1], G)
        dWs[l], G = dW, dh
    # GPU chain through SampledMatmul
    Xt = to_dev(X).requires_grad_(True)
    Wt = [to_dev(W).requires_grad_(True) for W in Ws]
    h = Xt
    for l, W in enumerate(Wt):
        h = torch.nn.functional.gelu(bmm.sampled_matmul(h, W, off, method="ONC", c=L, seed=100 + l, mode="f64"))
    (h * to_dev(R)).sum().backward()
    np.testing.assert_allclose(host(Xt.grad), G, rtol=1e-8, atol=1e-8 * np.abs(G).max())
    for l in range(4):
        np.testing.assert_allclose(host(Wt[l].grad), dWs[l], rtol=1e-8, atol=1e-8 * np.abs(dWs[l]).max())


def test_batched_uneven_products_and_graph_replay(bmm):
    """Uneven products (both GEMM tile widths) through bmm_apply_batched, then the same sequence
    captured as one CUDA graph and replayed: identical outputs, each within the BF16 bound."""
    rng = np.random.default_rng(23)
    probs, host_inputs, cs = [], [], []
    for i in range(9):
        m = int(rng.integers(1, 5)) * 128 - (17 if i % 3 == 0 else 0)
        p = int(rng.choice([96, 200, 384, 520]))
        n = int(rng.integers(2, 5)) * 1024
        K = n // 64
        off = S.block_offsets_uneven(n, K, 32, 100, seed=100 + i)
        M, N = S.scaled_gaussian(m, n, p, off, 1.0, seed=200 + i, dtype=np.float32)
        Mt, Nt = to_dev(M), to_dev(N)
        c = bmm.equal_budget(max(1, K // 8), n, K)
        probs.append(bmm.prepare(Mt, Nt, off, max_draws=c, gemm_mode=bmm._abi.GEMM_BF16))
        host_inputs.append((M.astype(np.float64), N.astype(np.float64), off))
        cs.append(c)
    seeds = list(range(50, 59))
    res = bmm.run_batched(probs, "ONC", cs, seeds, gemm_mode=bmm._abi.GEMM_BF16)
    for pr in probs:
        bmm.check_status(pr)
    eager = [host(r["out"]).astype(np.float64) for r in res]
    for (M, N, off), r, c, got in zip(host_inputs, res, cs, eager):
        idx, scale = host(r["idx"]), host(r["scale"])
        want = oracle.sampled_product_columns(M, N, idx, scale)
        assert np.all(np.abs(got - want) <= _tol("bf16", c) * product_bound(M, N, idx, scale) + 1e-300)
    # one graph: design, draws and the batched product of all nine
    side = [torch.cuda.Stream() for _ in range(3)]
    outs = [torch.empty_like(r["out"]) for r in res]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gres = bmm.run_batched(probs, "ONC", cs, seeds, gemm_mode=bmm._abi.GEMM_BF16, outs=outs, streams=side)
    g.replay()
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    for a_, b_ in zip(eager, outs):
        np.testing.assert_array_equal(host(b_).astype(np.float64), a_)


@pytest.mark.parametrize("layout", ["row", "col"])
def test_overlapped_apply_large_product(bmm, layout):
    """A column-sampled BF16 product with m p >= 2^24 and >= 4096 draws runs in two row halves, the
    second half's gathers overlapping the first half's GEMM on a side stream: within the BF16
    bound of the oracle's product of the same draws, bit-identical to the unsplit grouped path
    (bmm_apply_batched) and repeatable, and accumulate adds onto the output."""
    m, n, p, K = 4096, 8192, 4096, 128
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=73, dtype=np.float32, lo=32, hi=96)
    Mt = as_layout(Mt, layout)
    L = 5000
    prob = bmm.prepare(Mt, Nt, off, max_draws=L)
    r = bmm.run(prob, "ONC", L, seed=2, gemm_mode=bmm._abi.GEMM_BF16)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]), host(r["scale"])
    got = host(r["out"]).astype(np.float64)
    rows = np.random.default_rng(1).choice(m, size=96, replace=False)  # oracle rows (a full product is slow)
    want = oracle.sampled_product_columns(M[rows], N, idx, scale)
    bound = product_bound(M[rows], N, idx, scale)
    assert np.all(np.abs(got[rows] - want) <= _tol("bf16", L) * bound + 1e-300)
    out2 = torch.empty_like(r["out"])
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, r["idx"], r["scale"], L, bmm._abi.GEMM_BF16, out2, False,
                  prob.ws)
    np.testing.assert_array_equal(host(out2), host(r["out"]))
    out3 = torch.empty_like(r["out"])
    bmm.bmm_apply_batched([Mt], [Nt], [prob.B], bmm._abi.UNIT_COLUMN, [r["idx"]], [r["scale"]], [L],
                          bmm._abi.GEMM_BF16, [out3], False, [prob.ws])
    np.testing.assert_array_equal(host(out3), host(r["out"]))
    bmm.bmm_apply(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, r["idx"], r["scale"], L, bmm._abi.GEMM_BF16, out2, True,
                  prob.ws)
    bmm.check_status(prob)
    np.testing.assert_allclose(host(out2)[rows], 2 * got[rows], rtol=2e-6, atol=1e-6 * np.abs(got).max())


@pytest.mark.parametrize("bn", [128, 256, 512, 1024])
@pytest.mark.parametrize("m,L", [(64, 37), (333, 700), (1000, 130)])
def test_apply_equals_grouped_apply(bmm, bn, m, L):
    """bmm_apply against the grouped path (bmm_apply_batched, whose gathers and GEMM are table-driven
    launches over products): the same product bit for bit for every tile width, with fewer rows
    than one 128-row tile, ragged tiles, fewer draws than one 64-column unit, and with
    accumulate."""
    A = bmm._abi
    n, p, K = 2400, 270, 30
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=m + L, dtype=np.float32, lo=40, hi=120)
    assert Mt.stride(1) == 1 and Mt.dtype == torch.float32
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "ONC", L, seed=6, gemm_mode=A.GEMM_BF16, compute_product=False)
    A.bmm_autotune_clear()
    A.bmm_autotune_set(m, p, L, A.GEMM_BF16, bn, 8)
    base = torch.from_numpy(np.random.default_rng(m).standard_normal((m, p)).astype(np.float32)).to(Mt.device)
    for accumulate in (False, True):
        fused, sep = base.clone(), base.clone()
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, A.GEMM_BF16, fused, accumulate, prob.ws)
        A.bmm_apply_batched([Mt], [Nt], [prob.B], A.UNIT_COLUMN, [r["idx"]], [r["scale"]], [L], A.GEMM_BF16, [sep],
                            accumulate, [prob.ws])
        bmm.check_status(prob)
        np.testing.assert_array_equal(host(fused), host(sep), err_msg=f"accumulate={accumulate}")
    A.bmm_autotune_clear()


def test_apply_reports_a_bad_index(bmm):
    """A draw index outside M's columns: bmm_apply and the grouped path both record BMM_ERR_ARG on the
    device and use zeros for that column, so their outputs still agree."""
    A = bmm._abi
    m, n, p, K, L = 300, 2000, 200, 25, 400
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=91, dtype=np.float32, lo=40, hi=120)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "ONC", L, seed=3, gemm_mode=A.GEMM_BF16, compute_product=False)
    idx = r["idx"].clone()
    idx[17] = n + 5
    outs = []
    for single in (True, False):
        out = torch.empty(m, p, dtype=torch.float32, device=Mt.device)
        A.bmm_clear_device_status(prob.ws)
        if single:
            A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, idx, r["scale"], L, A.GEMM_BF16, out, False, prob.ws)
        else:
            A.bmm_apply_batched([Mt], [Nt], [prob.B], A.UNIT_COLUMN, [idx], [r["scale"]], [L], A.GEMM_BF16, [out],
                                False, [prob.ws])
        assert A.bmm_read_device_status(prob.ws) == A.ERR_ARG
        outs.append(host(out))
    A.bmm_clear_device_status(prob.ws)
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("layout", ["row", "col"])
def test_apply_parts_equal_one_apply(bmm, layout):
    """bmm_apply_part's parts -- REDUCE, then GATHER_B and GATHER_A in either order, then the GEMMs --
    in any row split (multiples of 128, the last ending at m) and on one or two streams, give
    bmm_apply's product bit for bit, with and without accumulate.  The parts run in a workspace of
    their own whose scratch starts as 0xFF bytes, so nothing left by bmm_apply's own reduction can
    stand in for REDUCE."""
    m, n, p, K, L = 700, 3000, 300, 40, 900
    off, M, N, Mt, Nt = _problem(m, n, p, K, seed=81, dtype=np.float32, lo=40, hi=110)
    Mt = as_layout(Mt, layout)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=bmm._abi.GEMM_BF16)
    r = bmm.run(prob, "ONC", L, seed=4, gemm_mode=bmm._abi.GEMM_BF16, compute_product=False)
    A = bmm._abi
    want = torch.empty(m, p, dtype=torch.float32, device=Mt.device)
    A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, A.GEMM_BF16, want, False, prob.ws)
    parts = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=bmm._abi.GEMM_BF16)
    for split, b_first in (([0, m], True), ([0, 128, m], False), ([0, 384, 512, m], True)):
        parts.ws[256:].fill_(255)
        got = torch.full((m, p), float("nan"), dtype=torch.float32, device=Mt.device)
        A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, got, False, A.APPLY_REDUCE, 0, 0, parts.ws)
        if b_first:
            A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, got, False, A.APPLY_GATHER_B, 0, 0, parts.ws)
        for lo, hi in zip(split[:-1], split[1:]):
            A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, got, False, A.APPLY_GATHER_A, lo, hi, parts.ws)
        if not b_first:
            A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, got, False, A.APPLY_GATHER_B, 0, 0, parts.ws)
        for lo, hi in zip(split[:-1], split[1:]):
            A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, got, False, A.APPLY_GEMM, lo, hi, parts.ws)
        bmm.check_status(parts)
        np.testing.assert_array_equal(host(got), host(want), err_msg=str(split))
    # accumulate: out += CD, rows split across a second stream
    acc = want.clone()
    side = torch.cuda.Stream()
    A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, acc, True, A.APPLY_REDUCE, 0, 0, prob.ws)
    A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, acc, True, A.APPLY_GATHER_B, 0, 0, prob.ws)
    A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, acc, True, A.APPLY_GATHER_A, 0, m, prob.ws)
    side.wait_stream(torch.cuda.current_stream())
    A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, acc, True, A.APPLY_GEMM, 0, 256, prob.ws, side)
    A.bmm_apply_part(Mt, Nt, prob.B, r["idx"], r["scale"], L, acc, True, A.APPLY_GEMM, 256, m, prob.ws)
    torch.cuda.current_stream().wait_stream(side)
    bmm.check_status(prob)
    twice = torch.empty_like(want)
    A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, A.GEMM_BF16, twice, False, prob.ws)
    A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, A.GEMM_BF16, twice, True, prob.ws)
    np.testing.assert_array_equal(host(acc), host(twice))


@pytest.mark.parametrize("dtype", [np.float32, "bf16"])
@pytest.mark.parametrize("mode", ["bf16", "split_bf16"])
@pytest.mark.parametrize("layout", ["row", "col"])
def test_apply_batched_equals_single_products(bmm, dtype, mode, layout):
    """bmm_apply_batched gathers the operands of all its column-sampled products in grouped
    launches (one grid over a table of products): every product must equal bmm_apply's for that
    product alone, bit for bit, for FP32 and BF16 inputs, both storage orders of M and ragged m, p, L."""
    rng = np.random.default_rng(29)
    gm = bmm.MODES[mode]
    probs, cs, samples = [], [], []
    for i in range(5):
        m = int(rng.integers(40, 300))
        p = int(rng.choice([64, 136, 300]))
        n = int(rng.integers(2, 4)) * 1024
        K = n // 64
        off, M, N, Mt, Nt = _problem(m, n, p, K, seed=300 + i, dtype=dtype, lo=32, hi=100)
        Mt = as_layout(Mt, layout)
        c = bmm.equal_budget(max(1, K // 8), n, K) + (17 if i % 2 else 0)
        pr = bmm.prepare(Mt, Nt, off, max_draws=c, gemm_mode=gm)
        r = bmm.run(pr, "ONC", c, seed=70 + i, compute_product=False)
        probs.append(pr)
        cs.append(c)
        samples.append((r["idx"], r["scale"]))
    single = []
    for pr, c, (idx, scale) in zip(probs, cs, samples):
        out = torch.empty(pr.M.shape[0], pr.N.shape[1], dtype=torch.float32, device=pr.M.device)
        bmm.bmm_apply(pr.M, pr.N, pr.B, bmm._abi.UNIT_COLUMN, idx, scale, c, gm, out, False, pr.ws)
        bmm.check_status(pr)
        single.append(host(out))
    outs = [torch.full((pr.M.shape[0], pr.N.shape[1]), float("nan"), dtype=torch.float32, device=pr.M.device)
            for pr in probs]
    bmm.bmm_apply_batched([pr.M for pr in probs], [pr.N for pr in probs], [pr.B for pr in probs],
                          bmm._abi.UNIT_COLUMN, [s_[0] for s_ in samples], [s_[1] for s_ in samples], cs, gm, outs,
                          False, [pr.ws for pr in probs])
    for pr in probs:
        bmm.check_status(pr)
    for a_, b_ in zip(single, outs):
        np.testing.assert_array_equal(host(b_), a_)


def test_probs_batched_grouped_norm_pass(bmm):
    """bmm_probs_batched without f_k runs the norm pass of all FP32 / BF16 products in grouped
    launches (vector sets of every product in one grid, then the per-block sums): x_i, y_i, a_k,
    s_k, ||M^k||_F^2, ||N_k||_F^2 and p within 1e-12 of the oracle, for both element types, all
    storage orders, ragged and odd sizes, more products than one table holds, and an FP64 product
    that takes the single-product path."""
    rng = np.random.default_rng(37)
    A = bmm._abi
    cases = []
    for i in range(600):  # more jobs than one table of the grouped launch holds
        dt = torch.float64 if i == 5 else (torch.float32 if i % 3 else torch.bfloat16)
        m = int(rng.choice([1, 7, 64, 200, 301]))
        p = int(rng.choice([1, 24, 128, 136]))
        n = int(rng.integers(1, 6)) * 128 + (int(rng.integers(0, 8)) if i % 5 == 0 else 0)
        K = max(1, n // 64)
        off = S.block_offsets_uneven(n, K, 1, 2 * n // K + 1, seed=500 + i)
        M, N = S.scaled_gaussian(m, n, p, off, 1.5, seed=600 + i, dtype=np.float64)
        Mt = as_layout(to_dev(M, dt), "col" if i % 4 == 1 else "row")
        Nt = as_layout(to_dev(N, dt), "col" if i % 4 == 2 else "row")
        cases.append((Mt, Nt, off, host(Mt.double()), host(Nt.double())))
    probs = [bmm.prepare(Mt, Nt, off, max_draws=16) for Mt, Nt, off, _, _ in cases]
    ps = [torch.empty(pr.n, dtype=torch.float64, device=pr.M.device) for pr in probs]
    A.bmm_probs_batched([pr.M for pr in probs], [pr.N for pr in probs], [pr.B for pr in probs], A.P_COL_OPT,
                        A.F_NONE, ps, [pr.st for pr in probs], [pr.ws for pr in probs])
    for pr in probs:
        bmm.check_status(pr)
    for (Mt, Nt, off, M, N), pr, pv in zip(cases, probs, ps):
        x, y = oracle.col_row_sq_norms(M, N)
        st = oracle.block_stats(x, y, off)
        assert rel_err(host(pr.st["x"]), x) < 1e-12
        assert rel_err(host(pr.st["y"]), y) < 1e-12
        for k in ("a", "s", "mf", "nf"):
            assert rel_err(host(pr.st[k]), st[k]) < 1e-12, k
        assert rel_err(host(pv), oracle.p_col_opt(st["w"], st["a"], off)) < 1e-12


@pytest.mark.parametrize("reuse", [False, True])
def test_probs_batched_matches_single_products(bmm, reuse):
    """bmm_probs_batched over products of both element types, all storage orders and one that the
    tensor-core pass does not take (odd leading dimension): every output equals bmm_probs's for
    that product alone, bit for bit (each block is computed the same way in a grouped launch), and
    a grouped launch spans several tables (25 products > one kernel-parameter table)."""
    rng = np.random.default_rng(31)
    A = bmm._abi
    cases = []
    for i in range(25):
        dt = torch.float32 if i % 3 else torch.bfloat16
        m = int(rng.choice([64, 96, 200])) + (3 if i == 7 else 0)  # product 7: odd ld when column-major
        p = int(rng.choice([64, 128, 136]))
        n = int(rng.integers(2, 6)) * 512
        K = n // 64
        off = S.block_offsets_uneven(n, K, 16, 128, seed=300 + i)
        M, N = S.scaled_gaussian(m, n, p, off, 1.0, seed=400 + i, dtype=np.float32)
        Mt = as_layout(to_dev(M, dt), "col" if i % 4 == 1 else "row")
        Nt = as_layout(to_dev(N, dt), "col" if i % 4 == 2 else "row")
        cases.append((Mt, Nt, off))

    def fresh():
        return [bmm.prepare(Mt, Nt, off, max_draws=64) for Mt, Nt, off in cases]

    single, batch = fresh(), fresh()
    ps_single = [torch.empty(pr.n, dtype=torch.float64, device=pr.M.device) for pr in single]
    ps_batch = [torch.empty(pr.n, dtype=torch.float64, device=pr.M.device) for pr in batch]
    for pr, pv in zip(single, ps_single):
        if reuse:
            bmm.bmm_probs(pr.M, pr.N, pr.B, A.P_COL_OPT, A.F_NONE, pv, pr.st, pr.ws)
            bmm.bmm_probs(pr.M, pr.N, pr.B, A.P_COL_OPT, A.F_TC | A.REUSE_STATS, None, pr.st, pr.ws)
        else:
            bmm.bmm_probs(pr.M, pr.N, pr.B, A.P_COL_OPT, A.F_TC, pv, pr.st, pr.ws)
    if reuse:
        for pr, pv in zip(batch, ps_batch):
            bmm.bmm_probs(pr.M, pr.N, pr.B, A.P_COL_OPT, A.F_NONE, pv, pr.st, pr.ws)
        A.bmm_probs_batched([pr.M for pr in batch], [pr.N for pr in batch], [pr.B for pr in batch], A.P_COL_OPT,
                            A.F_TC | A.REUSE_STATS, None, [pr.st for pr in batch], [pr.ws for pr in batch])
    else:
        A.bmm_probs_batched([pr.M for pr in batch], [pr.N for pr in batch], [pr.B for pr in batch], A.P_COL_OPT,
                            A.F_TC, ps_batch, [pr.st for pr in batch], [pr.ws for pr in batch])
    torch.cuda.synchronize()
    for a_, b_, pa, pb in zip(single, batch, ps_single, ps_batch):
        bmm.check_status(a_)
        bmm.check_status(b_)
        for key in ("x", "y", "a", "s", "mf", "nf", "f"):
            np.testing.assert_array_equal(host(a_.st[key]), host(b_.st[key]), err_msg=key)
        np.testing.assert_array_equal(host(pa), host(pb))


@pytest.mark.parametrize("ckind", ["opt", "hat", "equal"])
def test_blocksizes_batched_equals_single_products(bmm, ckind):
    """bmm_blocksizes_batched over 430 products (two launches of the grouped kernel) gives every
    product's c_k and g_k bit for bit as bmm_blocksizes alone, and the c_k equal the oracle's
    apportionment of the same weights."""
    A = bmm._abi
    kind = {"opt": A.CK_OPT, "hat": A.CK_HAT, "equal": A.CK_EQUAL}[ckind]
    rng = np.random.default_rng(211)
    dev = torch.device("cuda", 0)
    Bs, sts, cs, wss, offs, hosts = [], [], [], [], [], []
    for i in range(430):
        K = int(rng.integers(1, 40))
        n = K * int(rng.integers(2, 30)) + int(rng.integers(0, 5))
        off = S.block_offsets_uneven(n, K, 1, 2 * n // K + 1, seed=300 + i)
        a = np.exp(rng.normal(0, 1.5, K)) * 10
        f = a * a * rng.uniform(0, 0.9, K)
        c = int(rng.integers(K, n + 1))
        off_dev = to_dev(off.astype(np.int64))
        offs.append(off_dev)
        Bs.append(A.Blocks(K, n, int(np.max(np.diff(off))), off_dev.data_ptr()))
        st = {k: None for k in ("x", "y", "s", "mf", "nf")}
        st["a"], st["f"] = to_dev(a), to_dev(f)
        sts.append(st)
        cs.append(c)
        wss.append(torch.zeros(1 << 16, dtype=torch.uint8, device=dev))
        hosts.append((off, a, f, c))
    cks = [torch.empty(B.K, dtype=torch.int64, device=dev) for B in Bs]
    gs = [torch.empty(B.K, dtype=torch.float64, device=dev) for B in Bs]
    A.bmm_blocksizes_batched(Bs, sts if kind != A.CK_EQUAL else None, kind, cs, cks, gs, wss)
    for i in (0, 1, 199, 399, 400, 429):
        ck1 = torch.empty_like(cks[i])
        g1 = torch.empty_like(gs[i])
        A.bmm_blocksizes(None, None, Bs[i], sts[i], kind, cs[i], None, None, 0, ck1, g1, None, wss[i])
        assert torch.equal(ck1, cks[i]) and torch.equal(g1, gs[i]), i
    for i in range(0, 430, 37):
        off, a, f, c = hosts[i]
        nk = np.diff(off)
        g = {"opt": oracle.g_opt(a, f), "hat": oracle.g_hat(a), "equal": oracle.g_equal(len(nk))}[ckind]
        np.testing.assert_array_equal(host(cks[i]), oracle.apportion(oracle.g_with_fallback(g, a, nk), nk, c))
    for w in wss:
        assert A.bmm_read_device_status(w) == A.OK
    with pytest.raises(bmm.BmmError):  # c below K is refused on the host, before any launch
        A.bmm_blocksizes_batched(Bs[:2], sts[:2], A.CK_HAT, [Bs[0].K - 1 if Bs[0].K > 1 else 0, cs[1]], cks[:2],
                                 None, wss[:2])


@pytest.mark.parametrize("case", ["all_aligned", "all_zero", "one_heavy"])
def test_blocksizes_degenerate_weights(bmm, case):
    """Block sizes when every eq. 3.9 weight is zero (every block rank-one aligned: fall back to
    a_k), when every statistic is zero (fall back to n_k), and when one block's weight dwarfs the
    rest by 2^80 (the geometric bracket and the exact endgame at the ends of the FP64 range):
    bit-exact against the oracle for c from K to n."""
    rng = np.random.default_rng(17)
    K = 257
    nk = rng.integers(1, 60, size=K)
    off = np.concatenate([[0], np.cumsum(nk)]).astype(np.int64)
    n = int(off[-1])
    a = rng.lognormal(0, 1, size=K)
    if case == "all_aligned":
        f = a * a
    elif case == "all_zero":
        a = np.zeros(K)
        f = np.zeros(K)
    else:
        f = a * a * 0.5
        a[100] *= 2.0 ** 80
        f[100] = a[100] ** 2 * 0.5
    dev = torch.device("cuda:0")
    st = {k: torch.zeros(K if k not in ("x", "y") else n, dtype=torch.float64, device=dev)
          for k in ("x", "y", "a", "s", "mf", "nf", "f")}
    st["a"].copy_(torch.from_numpy(a))
    st["f"].copy_(torch.from_numpy(f))
    off_dev = torch.as_tensor(off, device=dev)
    B = bmm._abi.blocks(off_dev, n, int(nk.max()))
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
    ck = torch.empty(K, dtype=torch.int64, device=dev)
    g = torch.empty(K, dtype=torch.float64, device=dev)
    gw = oracle.g_with_fallback(oracle.g_opt(a, f), a, nk)
    for c in (K, K + 3, n // 2, n - 1, n):
        bmm.bmm_blocksizes(None, None, B, st, bmm._abi.CK_OPT, c, None, None, 0, ck, g, None, ws)
        assert bmm.bmm_read_device_status(ws) == 0
        np.testing.assert_array_equal(host(ck), oracle.apportion(gw, nk, c), err_msg=f"c={c}")


def test_bounded_wait_gives_up_and_reports(bmm):
    """The bounded-wait path of the pipelined kernels, reached on purpose (bmm_wait_selftest): a wait on
    a barrier nothing completes gives up after the bound, a second wait gives up through the abort
    flag, the status word says BMM_ERR_TIMEOUT with both counted, and the context stays usable."""
    import ctypes
    import time
    A = bmm._abi
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda:0")
    t0 = time.perf_counter()
    A.bmm_wait_selftest(ws)
    assert A.bmm_read_device_status(ws) == A.ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert 1.0 < elapsed < 30.0, elapsed
    detail = ctypes.c_int32.from_buffer_copy(bytes(ws[4:8].cpu().numpy())).value
    assert detail == 2
    # the device still answers: a small product runs and its status is clean
    off, M, N, Mt, Nt = _problem(64, 256, 64, 4, seed=13, dtype=np.float64)
    prob = bmm.prepare(Mt, Nt, off, max_draws=16)
    r = bmm.run(prob, "ONC", 16, seed=1, gemm_mode=A.GEMM_F64)
    bmm.check_status(prob)
    assert np.isfinite(host(r["out"])).all()


@pytest.mark.parametrize("unit", ["column", "block"])
def test_sample_batched_equals_single_products(bmm, unit):
    """bmm_sample_batched over 230 products of mixed lengths (one crosses the 200-product launch
    split; some segments longer than one 1024-element scan tile; zero-probability entries; one
    product with no draws) gives each product's bmm_sample draws bit for bit, and the first product
    also equals the oracle's draws."""
    A = bmm._abi
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(91)
    col = unit == "column"
    ps, Bs, cks, cs, seeds, sids, wss, keep = [], [], [], [], [], [], [], []
    for i in range(230):
        n = int(rng.integers(40, 3000)) if i % 7 else int(rng.integers(2100, 5000))
        K = int(rng.integers(1, min(n, 60) + 1))
        off = np.sort(rng.choice(np.arange(1, n), size=K - 1, replace=False)) if K > 1 else np.array([], dtype=np.int64)
        off = np.concatenate([[0], off, [n]]).astype(np.int64)
        p = S.random_probabilities(off if col else np.array([0, K]), seed=1000 + i, zero_frac=0.1)
        c = 0 if i == 17 else (int(rng.integers(K, min(n, 4 * K) + 1)) if col else int(rng.integers(1, 200)))
        ck = oracle.apportion(np.ones(K), np.diff(off), c) if col and c > 0 else np.zeros(K, dtype=np.int64)
        off_dev = to_dev(off)
        keep.append(off_dev)
        B = A.blocks(off_dev, n, int(np.diff(off).max()))
        ps.append(to_dev(p))
        Bs.append(B)
        cks.append(to_dev(ck))
        cs.append(c)
        seeds.append(int(rng.integers(0, 2 ** 62)))
        sids.append(int(rng.integers(0, 2 ** 20)))
        need = 256 + 8 * (n + 64 + K + 1) + 4096
        wss.append(torch.zeros(need, dtype=torch.uint8, device=dev))
    idx_b = [torch.full((max(c, 1),), -1, dtype=torch.int32, device=dev) for c in cs]
    sc_b = [torch.full((max(c, 1),), float("nan"), dtype=torch.float64, device=dev) for c in cs]
    ut = A.UNIT_COLUMN if col else A.UNIT_BLOCK
    A.bmm_sample_batched(ps, ut, Bs, cks if col else None, cs, seeds, sids, idx_b, sc_b, wss)
    for i in range(230):
        assert A.bmm_read_device_status(wss[i]) == A.OK, i
        if cs[i] == 0:
            assert int(idx_b[i][0]) == -1
            continue
        idx1 = torch.empty(cs[i], dtype=torch.int32, device=dev)
        sc1 = torch.empty(cs[i], dtype=torch.float64, device=dev)
        A.bmm_sample(ps[i], ut, Bs[i], cks[i] if col else None, cs[i], seeds[i], sids[i], idx1, sc1, wss[i])
        np.testing.assert_array_equal(host(idx_b[i]), host(idx1), err_msg=str(i))
        np.testing.assert_array_equal(host(sc_b[i]), host(sc1), err_msg=str(i))
    off0 = host(keep[0])
    if col:
        wi, wsc = oracle.sample_alg2(host(ps[0]), off0, host(cks[0]), seeds[0], sids[0])
    else:
        wi, wsc = oracle.sample_blocks(host(ps[0]), cs[0], seeds[0], sids[0])
    np.testing.assert_array_equal(host(idx_b[0]), wi)
    np.testing.assert_array_equal(host(sc_b[0]), wsc)


def test_autograd_step_replays_in_a_cuda_graph(bmm):
    """A forward and backward through sampled_matmul (BF16 mode) captured in a CUDA graph after one
    eager step: each replay recomputes the statistics, draws, product and adjoint, and gives the
    eager step's output and gradients bit for bit (same seed)."""
    off = S.block_offsets_equal(1024, 16)
    M, N = S.scaled_gaussian(192, 1024, 136, off, 1.0, seed=13, dtype=np.float32)
    X = to_dev(M).to(torch.bfloat16).requires_grad_(True)
    W = to_dev(N).to(torch.bfloat16).requires_grad_(True)
    R = to_dev(np.random.default_rng(14).standard_normal((192, 136)).astype(np.float32))

    def step():
        y = bmm.sampled_matmul(X, W, off, method="OPL", c=256, seed=9, mode="bf16")
        (y * R).sum().backward()
        return y

    for t in (X, W):
        t.grad = torch.zeros_like(t)
    y_eager = step().detach().clone()
    gX, gW = X.grad.clone(), W.grad.clone()
    for t in (X, W):
        t.grad.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        y_static = step()
    for t in (X, W):
        t.grad.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y_static, y_eager)
    assert torch.equal(X.grad, gX) and torch.equal(W.grad, gW)
    assert torch.count_nonzero(X.grad) > 0


@pytest.mark.parametrize("mode", ["bf16", "f64"])
@pytest.mark.parametrize("unit", ["column", "block"])
def test_apply_merges_repeated_draws(bmm, mode, unit):
    """bmm_apply reduces the draws to their distinct indices, each weighted by its multiplicity times
    its scale: the product of draws with repeats equals, bit for bit, the product of the distinct
    indices with those weights, stays within the element bound of the oracle's sum over every draw,
    and a repeated index carrying another scale is reported (BMM_ERR_ARG)."""
    A = bmm._abi
    gm = bmm.MODES[mode]
    off, M, N, Mt, Nt = _problem(300, 1500, 264, 15, seed=97, dtype=np.float32 if mode == "bf16" else np.float64,
                                 lo=40, hi=160)
    method, c = ("ONC", 900) if unit == "column" else ("SSM", 20)
    u = A.UNIT_BLOCK if unit == "block" else A.UNIT_COLUMN
    prob = bmm.prepare(Mt, Nt, off, max_draws=c, unit=u, gemm_mode=gm)
    r = bmm.run(prob, method, c, seed=4, gemm_mode=gm, compute_product=False)
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    ui, inv, cnt = np.unique(idx, return_inverse=True, return_counts=True)
    assert cnt.max() > 1  # the sample repeats some index
    usc = np.zeros(len(ui))
    usc[inv] = scale
    dt = torch.float32 if mode == "bf16" else torch.float64
    a = torch.empty(300, 264, dtype=dt, device=Mt.device)
    b = torch.empty(300, 264, dtype=dt, device=Mt.device)
    bmm.bmm_apply(Mt, Nt, prob.B, u, r["idx"], r["scale"], c, gm, a, False, prob.ws)
    bmm.check_status(prob)
    bmm.bmm_apply(Mt, Nt, prob.B, u, to_dev(ui.astype(np.int32)), to_dev(cnt * usc), len(ui), gm, b, False, prob.ws)
    bmm.check_status(prob)
    assert torch.equal(a, b)
    if unit == "column":
        want = oracle.sampled_product_columns(M, N, idx, scale)
        bound = product_bound(M, N, idx, scale)
        L = c
    else:
        want = oracle.sampled_product_blocks(M, N, off, idx, scale)
        bound = product_bound(M, N, idx, scale, offsets=off, unit="block")
        L = int(np.diff(off)[idx].sum())
    assert np.all(np.abs(host(a).astype(np.float64) - want) <= _tol(mode, L) * bound + 1e-300)
    # a repeated index with another scale
    j = int(np.flatnonzero(cnt[inv] > 1)[0])
    bad = scale.copy()
    bad[j] *= 1.5
    A.bmm_clear_device_status(prob.ws)
    bmm.bmm_apply(Mt, Nt, prob.B, u, r["idx"], to_dev(bad), c, gm, a, False, prob.ws)
    assert A.bmm_read_device_status(prob.ws) == A.ERR_ARG
    A.bmm_clear_device_status(prob.ws)

"""The benched product at its full size, in the launch configuration bench.py times, against the
FP64 oracle on sampled outputs.

Workload: M 8192 x 65536 and N 65536 x 8192 FP32 (row-major), N(0,1) * LogNormal(0, 1.5) block
scales, K = 1024 blocks of 16..128, OPL with L = 8192 outer products, fused statistics pass with
tensor-core f_k, BF16 sampled GEMM with the autotuned tile, products two in flight
(pipeline.run_pipelined).  The oracle cannot hold the whole problem in FP64 in seconds, so it
checks what it can compute one piece at a time:
  x_i, y_i, a_k, s_k, ||M^k||_F^2, ||N_k||_F^2, eq. 3.8 p   on 12 sampled blocks, 1e-12 relative
  f_k                       on the same blocks, within the TF32 Gram bound of the off-diagonal trace
  c_k (eq. 3.9)             all K, bit for bit from the GPU's own a_k and f_k
  idx, scale                all L draws, bit for bit from the GPU's p and c_k
  CD                        32 sampled rows x all 8192 columns, within the BF16 element bound
and every product of the pipelined schedule equals pipeline.run with the same seed, bit for bit.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests._gpu_util import host, product_bound, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bmm():
    import paper_2105_04940_gb300 as P
    P.build()
    P._abi.load()
    assert torch.cuda.is_available()
    return P


@pytest.fixture(autouse=True)
def _default_tiles(bmm):
    """These tests tune the GEMM tile table as the bench does; later tests start from the default."""
    yield
    bmm._abi.bmm_autotune_clear()


def _gram_bound(Mb, Nb, round_in):
    """One block: tau_M sum_{i != j} |M|^T|M| |G_N| + tau_N |G_M| |N||N|^T + tau_M tau_N (...), with
    tau = round_in + len 2^-23 (operand rounding, FP32 accumulation over len = m or p)."""
    m, p = Mb.shape[0], Nb.shape[1]
    GM, GN = Mb.T @ Mb, Nb @ Nb.T
    AM, AN = np.abs(Mb).T @ np.abs(Mb), np.abs(Nb) @ np.abs(Nb).T
    tM, tN = round_in + m * 2.0 ** -23, round_in + p * 2.0 ** -23
    E = tM * AM * np.abs(GN) + tN * np.abs(GM) * AN + tM * tN * AM * AN
    np.fill_diagonal(E, 0.0)
    return E.sum()


def test_bench_product_full_size(bmm):
    A = bmm._abi
    m, n, p, K, L = 8192, 65536, 8192, 1024, 8192
    off = S.block_offsets_uneven(n, K, 16, 128, seed=3)
    nk = np.diff(off)
    Mt, Nt, _ = S.scaled_gaussian_torch(m, n, p, off, 1.5, 3, dtype=torch.float32, device="cuda")
    assert bmm.equal_budget(128, n, K) == L
    bmm.autotune([(m, p, L)], A.GEMM_BF16, torch.device("cuda"))
    probs = [bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16) for _ in range(2)]
    outs = [torch.empty(m, p, device="cuda") for _ in range(2)]
    seeds = [71, 72, 73]
    bmm.run_pipelined(probs, L, seeds, outs)
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    piped = {1: outs[1].clone(), 2: outs[0].clone()}
    del outs

    prob = probs[0]
    for i in (1, 2):
        r = bmm.run(prob, "OPL", L, seed=seeds[i], gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
        bmm.check_status(prob)
        assert torch.equal(r["out"], piped[i]), i
    del piped
    st = {k: host(v) for k, v in prob.st.items()}
    p_gpu = host(r["p"])
    seed = seeds[2]

    # statistics, f_k and eq. 3.8 p on sampled blocks (the largest and smallest among them)
    rng = np.random.default_rng(9)
    blocks = np.unique(np.concatenate([rng.choice(K, size=10, replace=False), [int(np.argmax(nk)), int(np.argmin(nk))]]))
    for k in blocks:
        lo, hi = int(off[k]), int(off[k + 1])
        Mb = Mt[:, lo:hi].double().cpu().numpy()
        Nb = Nt[lo:hi, :].double().cpu().numpy()
        loc = np.array([0, hi - lo])
        x, y = oracle.col_row_sq_norms(Mb, Nb)
        ost = oracle.block_stats(x, y, loc)
        assert rel_err(st["x"][lo:hi], x) < 1e-12 and rel_err(st["y"][lo:hi], y) < 1e-12, k
        for key in ("a", "s", "mf", "nf"):
            assert rel_err(st[key][k:k + 1], ost[key]) < 1e-12, (k, key)
        assert rel_err(p_gpu[lo:hi], oracle.p_col_opt(ost["w"], ost["a"], loc)) < 1e-12, k
        f = oracle.block_frob_sq_gram(Mb, Nb, loc)[0]
        assert abs(st["f"][k] - f) <= _gram_bound(Mb, Nb, 2.0 ** -9) + 1e-12 * f, k

    # eq. 3.9 block sizes from the GPU's own a_k and f_k, and the draws from its p and c_k
    ck = host(r["ck"])
    want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
    np.testing.assert_array_equal(ck, want_ck)
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, seed, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)

    # the product on 32 sampled rows, every column, within the BF16 element bound; only the drawn
    # columns of M and rows of N enter, so the oracle gets those (indices remapped)
    rows = np.sort(rng.choice(m, size=32, replace=False))
    cols, loc_idx = np.unique(idx, return_inverse=True)
    cols_t = torch.as_tensor(cols, device="cuda")
    Mr = Mt[torch.as_tensor(rows, device="cuda")][:, cols_t].double().cpu().numpy()
    Nr = Nt[cols_t].double().cpu().numpy()
    want = oracle.sampled_product_columns(Mr, Nr, loc_idx, scale)
    got = r["out"][torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
    tol = 2.0 ** -7 + L * 2.0 ** -22
    assert np.all(np.abs(got - want) <= tol * product_bound(Mr, Nr, loc_idx, scale) + 1e-300)


def test_batched_workload_full_size(bmm):
    """The batched workload at its full size (512 BF16 products, the bench's shapes and seeds), run as
    the bench runs it: an eager batch, the GEMM tile autotuner over the batch, then the whole batch
    captured in one CUDA graph and replayed.  The replay reproduces the eager outputs bit for bit, and
    four products (the largest and smallest m n, two others) are checked against the oracle: the
    statistics and eq. 3.8 p on sampled blocks at 1e-12, f_k within the exact-product Gram bound
    (BF16 products are exact in FP32; FP32 accumulation), every c_k and draw bit for bit from the
    GPU's own statistics, and 16 rows of the product within the BF16 element bound."""
    A = bmm._abi
    shapes = S.batched_products(512, seed=5)
    probs, outs, cs = [], [], []
    for i, sh in enumerate(shapes):
        m, n, p, off = sh["m"], sh["n"], sh["p"], sh["offsets"]
        K = len(off) - 1
        M, N, _ = S.scaled_gaussian_torch(m, n, p, off, 1.0, 5 * 1000003 + 7919 * i, dtype=torch.bfloat16,
                                          device="cuda")
        L = bmm.equal_budget(max(K // 8, 1), n, K)
        probs.append(bmm.prepare(M, N, off, max_draws=L, gemm_mode=A.GEMM_BF16))
        outs.append(torch.empty(m, p, device="cuda", dtype=torch.float32))
        cs.append(L)
    seeds = [11 + i for i in range(len(probs))]
    streams = [torch.cuda.Stream() for _ in range(4)]

    def batch():
        return bmm.run_batched(probs, "OPL", cs, seeds, gemm_mode=A.GEMM_BF16, outs=outs, streams=streams)

    res = batch()
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    mn = np.array([sh["m"] * sh["n"] for sh in shapes])
    rng = np.random.default_rng(13)
    pick = [int(np.argmax(mn)), int(np.argmin(mn))] + [int(i) for i in rng.choice(len(shapes), 2, replace=False)]
    eager = {i: outs[i].clone() for i in pick}
    bmm.autotune_batched(probs, res, cs, A.GEMM_BF16, outs)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        res = batch()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    sid = bmm.stream_id(0, A.PURPOSE_MAIN)
    for i in pick:
        assert torch.equal(outs[i], eager[i]), i
        sh, pr, r = shapes[i], probs[i], res[i]
        m, p, off, L = sh["m"], sh["p"], sh["offsets"], cs[i]
        K, nk = len(off) - 1, np.diff(off)
        st = {k: host(v) for k, v in pr.st.items()}
        p_gpu = host(r["p"])
        for k in np.unique(np.concatenate([rng.choice(K, size=4, replace=False), [int(np.argmax(nk))]])):
            lo, hi = int(off[k]), int(off[k + 1])
            Mb = pr.M[:, lo:hi].double().cpu().numpy()
            Nb = pr.N[lo:hi, :].double().cpu().numpy()
            loc = np.array([0, hi - lo])
            x, y = oracle.col_row_sq_norms(Mb, Nb)
            ost = oracle.block_stats(x, y, loc)
            assert rel_err(st["x"][lo:hi], x) < 1e-12 and rel_err(st["y"][lo:hi], y) < 1e-12, (i, k)
            for key in ("a", "s", "mf", "nf"):
                assert rel_err(st[key][k:k + 1], ost[key]) < 1e-12, (i, k, key)
            assert rel_err(p_gpu[lo:hi], oracle.p_col_opt(ost["w"], ost["a"], loc)) < 1e-12, (i, k)
            f = oracle.block_frob_sq_gram(Mb, Nb, loc)[0]
            assert abs(st["f"][k] - f) <= _gram_bound(Mb, Nb, 0.0) + 1e-12 * f, (i, k)
        ck = host(r["ck"])
        want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
        np.testing.assert_array_equal(ck, want_ck)
        idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
        want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, seeds[i], sid)
        np.testing.assert_array_equal(idx, want_idx)
        np.testing.assert_array_equal(scale, want_scale)
        rows = np.sort(rng.choice(m, size=min(16, m), replace=False))
        cols, loc_idx = np.unique(idx, return_inverse=True)
        cols_t = torch.as_tensor(cols, device="cuda")
        Mr = pr.M[torch.as_tensor(rows, device="cuda")][:, cols_t].double().cpu().numpy()
        Nr = pr.N[cols_t].double().cpu().numpy()
        want = oracle.sampled_product_columns(Mr, Nr, loc_idx, scale)
        got = outs[i][torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        tol = 2.0 ** -7 + L * 2.0 ** -22
        assert np.all(np.abs(got - want) <= tol * product_bound(Mr, Nr, loc_idx, scale) + 1e-300), i


def _e4m3_rows_bound(Aa, Bb, al, be, L):
    """Element-wise error bound of the e4m3 sampled product on a subset of output rows.  Per drawn
    index j: a = M[:, c_j] sqrt(w_j), b = N[c_j, :] sqrt(w_j); the kernel scales a by 2^(e_j + gA) and b
    by 2^(gB - e_j) (e_j balances max|a| and max|b|, gA and gB bring each operand's largest value to
    at most 448) and rounds to e4m3: |q(x) - x| <= 2^-4 |x| in the normal range, or 2^-10 in scaled
    units below it (a factor 4 for an exponent one off from the kernel's).  Aa = |a| on the chosen rows,
    Bb = |b|; al and be are max|a| over all of M's rows and max|b|, recomputed here in FP64."""
    u = 2.0 ** -4
    e = np.zeros(len(al))
    pos = (al > 0) & (be > 0)
    e[pos] = np.clip(np.rint(0.5 * np.log2(be[pos] / al[pos])), -60, 60)
    gA = int(np.floor(np.log2(448.0 / np.max(al * 2.0 ** e))))
    gB = int(np.floor(np.log2(448.0 / np.max(be * 2.0 ** -e))))
    da = 4 * 2.0 ** -10 * 2.0 ** -(e + gA)
    db = 4 * 2.0 ** -10 * 2.0 ** -(gB - e)
    bound = (2 * u + u * u + 1.2 * L * 2.0 ** -23) * (Aa @ Bb)
    bound += (1 + u) * ((da @ Bb)[None, :] + (Aa @ db)[:, None]) + np.sum(da * db)
    return bound


def test_precision_workload_full_size(bmm):
    """The tall-skinny precision configuration at full size, as the bench's precision summary runs it:
    M 4096 x 262144 and N 262144 x 4096 FP32, each rank 32 (Gaussian factors / sqrt 32) plus 1e-3
    N(0,1) noise, K = 4096 blocks of 64, OPL with L = 32768 draws; one sample applied in every GEMM
    mode.  Statistics and eq. 3.8 p on sampled blocks at 1e-12, f_k within the TF32 Gram bound, all
    c_k and draws bit for bit, and each mode's product on 16 rows within its element bound: FP64
    1e-13 + L 2^-52, BF16 2^-7 + L 2^-22, split BF16 2^-14 + L 2^-22 (of sum_t s_t |M||N|), e4m3 the
    bound of its power-of-two scalings and FP8 rounding."""
    A = bmm._abi
    m, n, p = 4096, 262144, 4096
    K = n // 64
    off = np.arange(0, n + 1, 64, dtype=np.int64)
    L = bmm.equal_budget(K // 8, n, K)
    g = torch.Generator(device="cuda")
    g.manual_seed(4)

    def low_rank(r_, c_):
        F = torch.randn(r_, 32, generator=g, device="cuda", dtype=torch.float64)
        G = torch.randn(32, c_, generator=g, device="cuda", dtype=torch.float64)
        return (F @ G / np.sqrt(32.0) + 1e-3 * torch.randn(r_, c_, generator=g, device="cuda",
                                                          dtype=torch.float64)).float()

    Mt, Nt = low_rank(m, n), low_rank(n, p)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L)
    res = bmm.run(prob, "OPL", L, seed=7, gemm_mode=A.GEMM_BF16, compute_product=False)
    bmm.check_status(prob)
    st = {k: host(v) for k, v in prob.st.items()}
    p_gpu = host(res["p"])
    nk = np.diff(off)
    rng = np.random.default_rng(17)
    for k in rng.choice(K, size=8, replace=False):
        lo, hi = int(off[k]), int(off[k + 1])
        Mb = Mt[:, lo:hi].double().cpu().numpy()
        Nb = Nt[lo:hi, :].double().cpu().numpy()
        loc = np.array([0, hi - lo])
        x, y = oracle.col_row_sq_norms(Mb, Nb)
        ost = oracle.block_stats(x, y, loc)
        assert rel_err(st["x"][lo:hi], x) < 1e-12 and rel_err(st["y"][lo:hi], y) < 1e-12, k
        for key in ("a", "s", "mf", "nf"):
            assert rel_err(st[key][k:k + 1], ost[key]) < 1e-12, (k, key)
        assert rel_err(p_gpu[lo:hi], oracle.p_col_opt(ost["w"], ost["a"], loc)) < 1e-12, k
        f = oracle.block_frob_sq_gram(Mb, Nb, loc)[0]
        assert abs(st["f"][k] - f) <= _gram_bound(Mb, Nb, 2.0 ** -9) + 1e-12 * f, k
    ck = host(res["ck"])
    want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
    np.testing.assert_array_equal(ck, want_ck)
    idx, scale = host(res["idx"]).astype(np.int64), host(res["scale"])
    want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, 7, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)

    rows = np.sort(rng.choice(m, size=16, replace=False))
    rows_t = torch.as_tensor(rows, device="cuda")
    cols, loc_idx = np.unique(idx, return_inverse=True)
    cols_t = torch.as_tensor(cols, device="cuda")
    Mr = Mt[rows_t][:, cols_t].double().cpu().numpy()
    Nr = Nt[cols_t].double().cpu().numpy()
    want = oracle.sampled_product_columns(Mr, Nr, loc_idx, scale)
    bound = product_bound(Mr, Nr, loc_idx, scale)
    sw = np.sqrt(scale)
    col_max = Mt[:, cols_t].abs().amax(dim=0).double().cpu().numpy()  # max |M[:, c]| over every row
    al = col_max[loc_idx] * sw
    Bb = np.abs(Nr[loc_idx]) * sw[:, None]
    be = Bb.max(axis=1)
    e4_bound = _e4m3_rows_bound(np.abs(Mr[:, loc_idx]) * sw[None, :], Bb, al, be, L)
    tols = {"f64": 1e-13 + L * 2.0 ** -52, "bf16": 2.0 ** -7 + L * 2.0 ** -22, "split_bf16": 2.0 ** -14 + L * 2.0 ** -22}
    for mode in ("f64", "bf16", "split_bf16", "e4m3"):
        gm = bmm.MODES[mode]
        o = torch.empty(m, p, device="cuda", dtype=torch.float64 if mode == "f64" else torch.float32)
        A.bmm_apply(Mt, Nt, prob.B, res["unit"], res["idx"], res["scale"], L, gm, o, False, prob.ws)
        bmm.check_status(prob)
        got = o[rows_t].double().cpu().numpy()
        lim = e4_bound if mode == "e4m3" else tols[mode] * bound
        assert np.all(np.abs(got - want) <= lim + 1e-300), (mode, float(np.max(np.abs(got - want) / lim)))


def test_mlp_layer_full_size(bmm):
    """One layer of the differentiation workload at full size, through the autograd function as the
    bench's MLP calls it: X 4096 x 16384 BF16 ~ N(0,1), W 16384 x 16384 BF16 ~ N(0, 1/16384), K = 256
    blocks of 64, OPL with c = 64 blocks (L = 4096), BF16 mode, an FP32 upstream gradient.  The draws
    are those of pipeline.run with the same seed; against the oracle: the product on 16 rows, dX on
    16 rows and dW on 16 drawn rows within the BF16 bound of their sums plus the final rounding to
    BF16, and dX, dW exactly zero outside the drawn columns / rows."""
    A = bmm._abi
    m, n, K = 4096, 16384, 256
    off = S.block_offsets_equal(n, K)
    L = bmm.equal_budget(64, n, K)
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    X = torch.randn(m, n, generator=g, device="cuda", dtype=torch.float32).to(torch.bfloat16).requires_grad_(True)
    W = (torch.randn(n, n, generator=g, device="cuda", dtype=torch.float32) / np.sqrt(n)).to(torch.bfloat16) \
        .requires_grad_(True)
    Gup = torch.randn(m, n, generator=g, device="cuda", dtype=torch.float32)
    seed = 1000
    z = bmm.sampled_matmul(X, W, off, method="OPL", c=L, seed=seed, mode="bf16")
    z.backward(Gup)
    torch.cuda.synchronize()
    prob = bmm.prepare(X.detach(), W.detach(), off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "OPL", L, seed=seed, gemm_mode=A.GEMM_BF16, compute_product=False)
    bmm.check_status(prob)
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    cols, loc_idx = np.unique(idx, return_inverse=True)
    cols_t = torch.as_tensor(cols, device="cuda")
    rng = np.random.default_rng(21)
    rows = np.sort(rng.choice(m, size=16, replace=False))
    rows_t = torch.as_tensor(rows, device="cuda")
    Xr = X.detach()[rows_t][:, cols_t].double().cpu().numpy()
    Wc = W.detach()[cols_t].double().cpu().numpy()
    tol = 2.0 ** -7 + n * 2.0 ** -22
    # forward
    want = oracle.sampled_product_columns(Xr, Wc, loc_idx, scale)
    got = z.detach()[rows_t].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= (2.0 ** -7 + L * 2.0 ** -22) * product_bound(Xr, Wc, loc_idx, scale) + 1e-300)
    # dX on 16 rows: only the drawn columns are touched
    Gr = Gup[rows_t].double().cpu().numpy()
    wX, _ = oracle.adjoint_columns(Xr, Wc, loc_idx, scale, Gr)
    bX, _ = oracle.adjoint_columns(np.abs(Xr), np.abs(Wc), loc_idx, scale, np.abs(Gr))
    dXr = X.grad[rows_t].double()
    gotX = dXr[:, cols_t].cpu().numpy()
    assert np.all(np.abs(gotX - wX) <= tol * bX + 2.0 ** -8 * np.abs(wX) + 1e-300)
    dXr[:, cols_t] = 0.0
    assert not torch.any(dXr != 0)
    # dW on 16 drawn rows: every draw of those columns contributes X[:, i]^T G
    pick = np.sort(rng.choice(len(cols), size=16, replace=False))
    sel = np.isin(loc_idx, pick)
    sub_idx = np.searchsorted(pick, loc_idx[sel])
    pick_t = torch.as_tensor(cols[pick], device="cuda")
    Xp = X.detach()[:, pick_t].double().cpu().numpy()
    Wp = W.detach()[pick_t].double().cpu().numpy()
    Gd = Gup.double().cpu().numpy()
    _, wW = oracle.adjoint_columns(Xp, Wp, sub_idx, scale[sel], Gd)
    _, bW = oracle.adjoint_columns(np.abs(Xp), np.abs(Wp), sub_idx, scale[sel], np.abs(Gd))
    gotW = W.grad[pick_t].double().cpu().numpy()
    tolW = 2.0 ** -7 + m * 2.0 ** -22
    assert np.all(np.abs(gotW - wW) <= tolW * bW + 2.0 ** -8 * np.abs(wW) + 1e-300)
    untouched = torch.ones(n, dtype=torch.bool, device="cuda")
    untouched[cols_t] = False
    assert not torch.any(W.grad[untouched] != 0)


@pytest.mark.parametrize("m_layout", ["row", "col"])
def test_element_offsets_beyond_32_bits(bmm, m_layout):
    """A product whose M holds more than 2^32 elements (16500 x 262144 FP32, 17 GB; N 262144 x 256),
    stored row-major or column-major, through the benched OPL path (fused statistics, BF16 apply):
    statistics on blocks at both ends of the range (the last ones at element offsets above 2^32),
    every c_k and draw bit for bit, and the product on rows including the last one."""
    A = bmm._abi
    m, n, p, K = 16500, 262144, 256, 3640
    off = S.block_offsets_uneven(n, K, 16, 128, seed=41)
    nk = np.diff(off)
    Ms, Nt, _ = S.scaled_gaussian_torch(m, n, p, off, 1.0, 43, dtype=torch.float32, device="cuda", m_layout=m_layout)
    Mt = Ms if m_layout == "row" else Ms.t()
    assert Mt.shape == (m, n) and Mt.numel() > 2 ** 32
    L = 8192
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "OPL", L, seed=5, gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
    bmm.check_status(prob)
    st = {k: host(v) for k, v in prob.st.items()}
    p_gpu = host(r["p"])
    for k in (0, 1, K // 2, K - 2, K - 1):
        lo, hi = int(off[k]), int(off[k + 1])
        Mb = Mt[:, lo:hi].double().cpu().numpy()
        Nb = Nt[lo:hi, :].double().cpu().numpy()
        loc = np.array([0, hi - lo])
        x, y = oracle.col_row_sq_norms(Mb, Nb)
        ost = oracle.block_stats(x, y, loc)
        assert rel_err(st["x"][lo:hi], x) < 1e-12 and rel_err(st["y"][lo:hi], y) < 1e-12, k
        for key in ("a", "s", "mf", "nf"):
            assert rel_err(st[key][k:k + 1], ost[key]) < 1e-12, (k, key)
        assert rel_err(p_gpu[lo:hi], oracle.p_col_opt(ost["w"], ost["a"], loc)) < 1e-12, k
        f = oracle.block_frob_sq_gram(Mb, Nb, loc)[0]
        assert abs(st["f"][k] - f) <= _gram_bound(Mb, Nb, 2.0 ** -9) + 1e-12 * f, k
    ck = host(r["ck"])
    want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
    np.testing.assert_array_equal(ck, want_ck)
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, 5, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)
    rng = np.random.default_rng(47)
    rows = np.unique(np.concatenate([rng.choice(m, size=14, replace=False), [0, m - 1]]))
    rows_t = torch.as_tensor(rows, device="cuda")
    cols, loc_idx = np.unique(idx, return_inverse=True)
    cols_t = torch.as_tensor(cols, device="cuda")
    Mr = Mt[rows_t][:, cols_t].double().cpu().numpy()
    Nr = Nt[cols_t].double().cpu().numpy()
    want = oracle.sampled_product_columns(Mr, Nr, loc_idx, scale)
    got = r["out"][rows_t].double().cpu().numpy()
    tol = 2.0 ** -7 + L * 2.0 ** -22
    assert np.all(np.abs(got - want) <= tol * product_bound(Mr, Nr, loc_idx, scale) + 1e-300)

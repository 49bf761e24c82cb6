"""The product path as the benchmark runs it, end to end in one run, against the FP64 oracle.

pipeline.run with OPL composes: the fused statistics pass (x_i, y_i, a_k, s_k, ||M^k||_F^2,
||N_k||_F^2 and f_k = s_k + the off-diagonal trace of tensor-core Grams, F_TC), eq. 3.8
probabilities, eq. 3.9 block sizes from that f, Philox draws, and the BF16 apply (for m p >= 2^24
and >= 4096 draws the row-split, overlapped form).  Each stage is checked against the oracle on
the inputs the stage actually received, so one run pins the whole composition:
  statistics and p            1e-12 relative (FP64-accurate on both sides)
  f_k                         within the TF32 (FP32 inputs) or exact-product (BF16 inputs) Gram
                              bound of the off-diagonal trace
  c_k                         bit for bit: oracle.apportion of eq. 3.9 on the GPU's a_k and f_k
  idx, scale                  bit for bit: oracle.sample_alg2 on the GPU's p and c_k
  CD                          within the BF16 element bound on 64 sampled rows
The block-sampling baseline of eq. 1.2 (WU) under F_TC is checked the same way, with p_k's
tolerance propagated from the f_k bound.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests._gpu_util import host, product_bound, rel_err, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bmm():
    import paper_2105_04940_gb300 as P
    P.build()
    P._abi.load()
    assert torch.cuda.is_available()
    return P


def _gram_bound(M, N, off, round_in):
    """Per block: tau_M sum_{i != j} |M|^T|M| |G_N| + tau_N |G_M| |N||N|^T + tau_M tau_N (...), with
    tau = round_in + len 2^-23 (operand rounding, FP32 accumulation over len = m or p)."""
    m, p = M.shape[0], N.shape[1]
    out = np.empty(len(off) - 1)
    for k, (a_, b_) in enumerate(zip(off[:-1], off[1:])):
        A, B = M[:, a_:b_], N[a_:b_, :]
        GM, GN = A.T @ A, B @ B.T
        AM, AN = np.abs(A).T @ np.abs(A), np.abs(B) @ np.abs(B).T
        tM, tN = round_in + m * 2.0 ** -23, round_in + p * 2.0 ** -23
        E = tM * AM * np.abs(GN) + tN * np.abs(GM) * AN + tM * tN * AM * AN
        np.fill_diagonal(E, 0.0)
        out[k] = E.sum()
    return out


def _inputs(dtype, m, n, p, K, seed):
    off = S.block_offsets_uneven(n, K, 16, 128, seed=seed)
    M, N = S.scaled_gaussian(m, n, p, off, 1.5, seed=seed + 1, dtype=np.float64)
    if dtype == "bf16":
        Mt, Nt = to_dev(M, torch.bfloat16), to_dev(N, torch.bfloat16)
    else:
        Mt, Nt = to_dev(M.astype(np.float32)), to_dev(N.astype(np.float32))
    return off, host(Mt.double()), host(Nt.double()), Mt, Nt


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_benched_opl_path_end_to_end(bmm, dtype):
    A = bmm._abi
    m, n, p, K = 4096, 32768, 4096, 455
    off, M, N, Mt, Nt = _inputs(dtype, m, n, p, K, seed=301 if dtype == "f32" else 311)
    nk = np.diff(off)
    assert len(nk) == K and nk.min() >= 16 and nk.max() <= 128
    L = 4608  # outer products (about c = K/7 blocks' worth)
    assert L >= 4096 and m * p >= 1 << 24  # the overlapped, row-split apply runs
    seed = 7
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "OPL", L, seed=seed, gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
    bmm.check_status(prob)
    st = {k: host(v) for k, v in prob.st.items()}
    # statistics and eq. 3.8 probabilities
    x, y = oracle.col_row_sq_norms(M, N)
    ost = oracle.block_stats(x, y, off)
    assert rel_err(st["x"], x) < 1e-12 and rel_err(st["y"], y) < 1e-12
    for k in ("a", "s", "mf", "nf"):
        assert rel_err(st[k], ost[k]) < 1e-12, k
    p_gpu = host(r["p"])
    assert rel_err(p_gpu, oracle.p_col_opt(ost["w"], ost["a"], off)) < 1e-12
    # f_k from the tensor-core Grams, within the bound of their rounding
    f = oracle.block_frob_sq_gram(M, N, off)
    bound = _gram_bound(M, N, off, 2.0 ** -9 if dtype == "f32" else 0.0)
    err = np.abs(st["f"] - f)
    assert np.all(err <= bound + 1e-12 * f), float(np.max(err / (bound + 1e-12 * f)))
    # eq. 3.9 block sizes from the GPU's own a_k and f_k, bit for bit
    ck = host(r["ck"])
    want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
    np.testing.assert_array_equal(ck, want_ck)
    # the draws from the GPU's p and c_k, bit for bit
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, seed, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)
    # the product on 64 sampled rows, within the BF16 element bound
    rows = np.random.default_rng(5).choice(m, size=64, replace=False)
    want = oracle.sampled_product_columns(M[rows], N, idx, scale)
    got = host(r["out"]).astype(np.float64)[rows]
    tol = 2.0 ** -7 + L * 2.0 ** -22
    assert np.all(np.abs(got - want) <= tol * product_bound(M[rows], N, idx, scale) + 1e-300)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_wu_block_sampling_with_tensor_core_f(bmm, dtype):
    """eq. 1.2 (WU) under F_TC: p_k = sqrt(f_k) / sum_j sqrt(f_j) with f_k from the fused pass.  If
    |f_k - f*_k| <= e_k f*_k, then sqrt(f_k) is within e_k/2 and the normaliser within max_j e_j/2, so
    |p_k - p*_k| <= (e_k + max_j e_j)/2 p*_k to first order (slack 1% plus 1e-12).  The draws are
    then bit-exact given p_k, and the product within the BF16 bound."""
    A = bmm._abi
    m, n, p, K = 1536, 12288, 1280, 170
    off, M, N, Mt, Nt = _inputs(dtype, m, n, p, K, seed=321 if dtype == "f32" else 331)
    c = K // 8
    seed = 11
    prob = bmm.prepare(Mt, Nt, off, max_draws=c, unit=A.UNIT_BLOCK, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "WU", c, seed=seed, gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
    bmm.check_status(prob)
    f = oracle.block_frob_sq_gram(M, N, off)
    bound = _gram_bound(M, N, off, 2.0 ** -9 if dtype == "f32" else 0.0) + 1e-12 * f
    f_gpu = host(prob.st["f"])
    assert np.all(np.abs(f_gpu - f) <= bound)
    e = bound / f
    pk = host(r["p"])
    p_star = oracle.p_blk_prodnorm(f)
    tol = 0.5 * (e + e.max()) * 1.01 + 1e-12
    assert np.all(np.abs(pk - p_star) <= tol * p_star), float(np.max(np.abs(pk - p_star) / (tol * p_star)))
    assert rel_err(pk, oracle.p_blk_prodnorm(f_gpu)) < 1e-12  # eq. 1.2 on the GPU's own f_k
    kidx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    want_idx, want_scale = oracle.sample_blocks(pk, c, seed, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(kidx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)
    rows = np.random.default_rng(6).choice(m, size=64, replace=False)
    want = oracle.sampled_product_blocks(M[rows], N, off, kidx, scale)
    got = host(r["out"]).astype(np.float64)[rows]
    Lcols = int(sum(off[k + 1] - off[k] for k in kidx))
    tolp = 2.0 ** -7 + Lcols * 2.0 ** -22
    bnd = product_bound(M[rows], N, kidx, scale, offsets=off, unit="block")
    assert np.all(np.abs(got - want) <= tolp * bnd + 1e-300)


@pytest.mark.parametrize("dtype,states,nouts", [("f32", 2, 1), ("f32", 3, 5), ("bf16", 2, 2)])
def test_pipelined_products_equal_run(bmm, dtype, states, nouts):
    """run_pipelined (two products in flight over two streams) gives each product exactly what run()
    gives for its seed: same statistics, block sizes, draws and GEMM, only reordered in time."""
    A = bmm._abi
    m, n, p, K = 1000, 16384, 520, 229
    off, _, _, Mt, Nt = _inputs(dtype, m, n, p, K, seed=331)
    L = 2048
    seeds = [41, 42, 43, 44, 45]
    probs = [bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16) for _ in range(states)]
    outs = [torch.full((m, p), float("nan"), device="cuda") for _ in range(nouts)]
    ev = []
    bmm.run_pipelined(probs, L, seeds, outs, events=ev)
    torch.cuda.synchronize()
    names = ("stats_start", "stats_end", "side_start", "design_end", "gathers_end", "gemm_start", "gemm_end")
    assert sorted((n, i) for n, i, _ in ev) == sorted((n, i) for n in names for i in range(len(seeds)))
    at = {(n, i): e for n, i, e in ev}
    for i in range(len(seeds)):  # each product's events in schedule order
        chain = [("stats_start", i), ("stats_end", i), ("side_start", i), ("design_end", i), ("gathers_end", i),
                 ("gemm_start", i), ("gemm_end", i)]
        assert all(at[a].elapsed_time(at[b]) >= 0.0 for a, b in zip(chain[:-1], chain[1:])), i
    for pr in probs:
        bmm.check_status(pr)
    ref = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    # product i lives in outs[i % nouts] until product i + nouts overwrites it
    for i in range(max(0, len(seeds) - nouts), len(seeds)):
        r = bmm.run(ref, "OPL", L, seed=seeds[i], gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
        bmm.check_status(ref)
        assert torch.equal(outs[i % nouts], r["out"]), i


def test_pipelined_rejects_what_it_does_not_run(bmm):
    A = bmm._abi
    off, _, _, Mt, Nt = _inputs("f32", 256, 2048, 128, 32, seed=5)
    pr = bmm.prepare(Mt, Nt, off, max_draws=256, gemm_mode=A.GEMM_BF16)
    out = torch.empty(256, 128, device="cuda")
    with pytest.raises(ValueError):
        bmm.run_pipelined([pr], 256, [1], [out])
    with pytest.raises(ValueError):
        bmm.run_pipelined([pr, pr], 256, [1], [])
    with pytest.raises(ValueError):
        bmm.run_pipelined([pr, pr], 256, [1], [out], gemm_mode=A.GEMM_F64)


def test_pipelined_products_of_different_inputs(bmm):
    """Two states over different matrices (and different block partitions): product i works on
    state i mod 2, so the stream alternates between the two products, each equal to run() on its own
    inputs with the same seed."""
    A = bmm._abi
    L = 1536
    sets = []
    for seed, (m, n, p, K) in ((341, (520, 12288, 776, 170)), (351, (1000, 8192, 264, 120))):
        off, _, _, Mt, Nt = _inputs("f32", m, n, p, K, seed=seed)
        sets.append((off, Mt, Nt))
    probs = [bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16) for off, Mt, Nt in sets]
    outs = [torch.full((int(s[1].shape[0]), int(s[2].shape[1])), float("nan"), device="cuda") for s in sets]
    seeds = [61, 62, 63, 64]
    bmm.run_pipelined(probs, L, seeds, outs)
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    for i in (2, 3):  # the last product of each state
        off, Mt, Nt = sets[i % 2]
        ref = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
        r = bmm.run(ref, "OPL", L, seed=seeds[i], gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
        bmm.check_status(ref)
        assert torch.equal(outs[i % 2], r["out"]), i


@pytest.mark.parametrize("case", ["zero_blocks", "all_zero"])
def test_benched_path_degenerate_inputs(bmm, case):
    """The benched OPL path on the method's degenerate inputs.  zero_blocks: blocks whose M^k or N_k
    is zero (a_k = 0: eq. 3.8 is 0/0 there, read as uniform p; no mass, so nothing drawn there
    matters), and a block with a_k > 0 but M^k N_k = 0 exactly (two outer products that cancel, f_k
    = 0 up to the Gram's rounding).  all_zero: M = 0, so every weight of eq. 3.9 is zero and the
    block sizes fall back to n_k; the product is exactly zero.  Each stage as in the end-to-end test."""
    A = bmm._abi
    m, n, p, K = 300, 4096, 260, 56
    off, M, N, _, _ = _inputs("f32", m, n, p, K, seed=361)
    M, N = M.astype(np.float32).astype(np.float64), N.astype(np.float32).astype(np.float64)
    K = len(off) - 1
    nk = np.diff(off)
    if case == "zero_blocks":
        M[:, off[1]:off[2]] = 0.0
        N[off[2]:off[3], :] = 0.0
        M[:, off[5]:off[6]] = 0.0
        N[off[5]:off[6], :] = 0.0
        lo = int(off[7])
        M[:, lo + 1] = M[:, lo]
        N[lo + 1, :] = -N[lo, :]
        M[:, lo + 2:off[8]] = 0.0
    else:
        M[:] = 0.0
    Mt, Nt = torch.as_tensor(M, dtype=torch.float32, device="cuda"), torch.as_tensor(N, dtype=torch.float32, device="cuda")
    L = 1024
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    r = bmm.run(prob, "OPL", L, seed=3, gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
    bmm.check_status(prob)
    st = {k: host(v) for k, v in prob.st.items()}
    x, y = oracle.col_row_sq_norms(M, N)
    ost = oracle.block_stats(x, y, off)
    for k in ("a", "s", "mf", "nf"):
        np.testing.assert_allclose(st[k], ost[k], rtol=1e-12, atol=0)
    p_gpu = host(r["p"])
    np.testing.assert_allclose(p_gpu, oracle.p_col_opt(ost["w"], ost["a"], off), rtol=1e-12, atol=0)
    f = oracle.block_frob_sq_gram(M, N, off)
    bound = _gram_bound(M, N, off, 2.0 ** -9)
    assert np.all(np.abs(st["f"] - f) <= bound + 1e-12 * f)
    if case == "zero_blocks":
        assert st["a"][1] == 0 and st["a"][2] == 0 and st["a"][5] == 0 and st["a"][7] > 0
        assert st["f"][1] == 0 and st["f"][2] == 0 and st["f"][5] == 0
    ck = host(r["ck"])
    want_ck = oracle.apportion(oracle.g_with_fallback(oracle.g_opt(st["a"], st["f"]), st["a"], nk), nk, L)
    np.testing.assert_array_equal(ck, want_ck)
    idx, scale = host(r["idx"]).astype(np.int64), host(r["scale"])
    want_idx, want_scale = oracle.sample_alg2(p_gpu, off, ck, 3, bmm.stream_id(0, A.PURPOSE_MAIN))
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(scale, want_scale)
    got = host(r["out"]).astype(np.float64)
    if case == "all_zero":
        assert np.all(got == 0.0)
    else:
        want = oracle.sampled_product_columns(M, N, idx, scale)
        tol = 2.0 ** -7 + L * 2.0 ** -22
        assert np.all(np.abs(got - want) <= tol * product_bound(M, N, idx, scale) + 1e-300)


def test_pipelined_products_replay_in_a_cuda_graph(bmm):
    """run_pipelined forks from and joins back into the caller's stream with events only, so a whole
    sequence of pipelined products can be captured in a CUDA graph; each replay recomputes every
    product (statistics, design, draws, gathers, GEMM) and gives run()'s outputs bit for bit."""
    A = bmm._abi
    m, n, p, K = 700, 12288, 392, 170
    off, _, _, Mt, Nt = _inputs("f32", m, n, p, K, seed=371)
    L = 1536
    seeds = [81, 82, 83]
    probs = [bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16) for _ in range(2)]
    outs = [torch.empty(m, p, device="cuda") for _ in range(3)]
    bmm.run_pipelined(probs, L, seeds, outs)  # eager once: the side stream exists before the capture
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bmm.run_pipelined(probs, L, seeds, outs)
    for o in outs:
        o.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for pr in probs:
        bmm.check_status(pr)
    ref = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
    for i, sd in enumerate(seeds):
        r = bmm.run(ref, "OPL", L, seed=sd, gemm_mode=A.GEMM_BF16, fmode=A.F_TC, fused_stats=True)
        bmm.check_status(ref)
        assert torch.equal(outs[i], r["out"]), i


def test_concurrent_host_threads(bmm):
    """Two host threads issue products through the C ABI at the same time, each on its own stream
    and problem (the ctypes calls release the interpreter lock, so the launches' host staging runs
    concurrently): each thread's products equal run() of the same problem and seed issued alone.
    One thread takes the fused tensor-core statistics pass, the other the separate norm pass and
    exact f, so every kernel-parameter staging table is filled from both threads."""
    import threading
    A = bmm._abi
    L = 1536
    cfgs = (("f32", (520, 8192, 264, 120), 391, dict(fmode=A.F_TC, fused_stats=True)),
            ("bf16", (776, 12288, 200, 170), 401, dict(fmode=A.F_EXACT, fused_stats=False)))
    jobs = []
    for dtype, (m, n, p, K), seed, kw in cfgs:
        off, _, _, Mt, Nt = _inputs(dtype, m, n, p, K, seed=seed)
        jobs.append((off, Mt, Nt, kw, [seed + 7 * i for i in range(6)]))
    got = [[] for _ in jobs]
    errors = []
    start = threading.Barrier(len(jobs))

    def work(j):
        try:
            off, Mt, Nt, kw, seeds = jobs[j]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                pr = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
                start.wait()
                for sd in seeds:
                    r = bmm.run(pr, "OPL", L, seed=sd, gemm_mode=A.GEMM_BF16, **kw)
                    got[j].append((r["ck"].clone(), r["idx"].clone(), r["out"].clone()))
            s.synchronize()
            bmm.check_status(pr)
        except Exception as e:  # reported below, on the test's thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(j,)) for j in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for j, (off, Mt, Nt, kw, seeds) in enumerate(jobs):
        ref = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=A.GEMM_BF16)
        assert len(got[j]) == len(seeds)
        for (ck, idx, out), sd in zip(got[j], seeds):
            r = bmm.run(ref, "OPL", L, seed=sd, gemm_mode=A.GEMM_BF16, **kw)
            bmm.check_status(ref)
            assert torch.equal(ck, r["ck"]) and torch.equal(idx, r["idx"]), (j, sd)
            assert torch.equal(out, r["out"]), (j, sd)

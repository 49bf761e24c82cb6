"""GEMM tile autotuner on the GPU: every (tile width, raster group) choice gives the same sampled
product bit for bit (single and grouped launches), and the tuner records one of the candidates."""
import numpy as np
import pytest

import synthetic as S
from tests._gpu_util import host, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHOICES = [(bn, r) for bn in (128, 256, 512, 1024) for r in (4, 8, 16)]  # 512, 1024: CTA-pair tiles


@pytest.fixture(scope="module")
def bmm():
    import paper_2105_04940_gb300 as P
    P.build()
    P._abi.load()
    return P


@pytest.mark.parametrize("mode", ["bf16", "split_bf16", "e4m3"])
def test_tile_choices_do_not_change_results(bmm, mode):
    A = bmm._abi
    gm = bmm.MODES[mode]
    off = S.block_offsets_uneven(6000, 60, 40, 160, seed=61)
    M, N = S.scaled_gaussian(700, 6000, 520, off, 1.0, seed=62, dtype=np.float32)
    Mt, Nt = to_dev(M), to_dev(N)
    L = 1100
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=gm)
    r = bmm.run(prob, "ONC", L, seed=3, compute_product=False)
    A.bmm_autotune_clear()
    outs = []
    for bn, ra in CHOICES:
        A.bmm_autotune_set(700, 520, L, gm, bn, ra)
        out = torch.full((700, 520), float("nan"), dtype=torch.float32, device=Mt.device)
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, False, prob.ws)
        bmm.check_status(prob)
        outs.append(host(out))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    assert np.all(np.isfinite(outs[0]))
    # the tuner picks one candidate and records it for the shape
    ws = torch.empty(A.bmm_autotune_workspace_size(700, 520, L, gm), dtype=torch.uint8, device=Mt.device)
    res = A.bmm_autotune_gemm(700, 520, L, gm, ws)
    assert (res["bn"], res["raster"]) in CHOICES and res["ms"] > 0
    assert A.bmm_autotune_get(700, 520, L, gm) == {"bn": res["bn"], "raster": res["raster"]}
    out = torch.empty(700, 520, dtype=torch.float32, device=Mt.device)
    A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, False, prob.ws)
    np.testing.assert_array_equal(host(out), outs[0])
    A.bmm_autotune_clear()


@pytest.mark.parametrize("mode", ["bf16", "e4m3"])
@pytest.mark.parametrize("m,p", [(64, 40), (130, 260), (256, 256), (390, 129)])
def test_pair_tile_edges_accumulate(bmm, mode, m, p):
    """The CTA-pair tiles (256 x 256 and 256 x 512) against the single-CTA 128 x 128 tile, bit for bit,
    on shapes where the odd CTA's rows of A or of B lie wholly or partly past the matrix (m < 128,
    ragged m and p), adding into a prefilled output."""
    A = bmm._abi
    gm = bmm.MODES[mode]
    off = S.block_offsets_uneven(2000, 25, 40, 120, seed=m + p)
    M, N = S.scaled_gaussian(m, 2000, p, off, 1.0, seed=m * p, dtype=np.float32)
    Mt, Nt = to_dev(M), to_dev(N)
    L = 300
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=gm)
    r = bmm.run(prob, "ONC", L, seed=5, compute_product=False)
    base = torch.from_numpy(np.random.default_rng(m).standard_normal((m, p)).astype(np.float32)).to(Mt.device)
    outs = []
    for bn in (128, A.TILE_PAIR, A.TILE_PAIR_WIDE):
        A.bmm_autotune_clear()
        A.bmm_autotune_set(m, p, L, gm, bn, 8)
        out = base.clone()
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, True, prob.ws)
        bmm.check_status(prob)
        outs.append(host(out))
    A.bmm_autotune_clear()
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])
    assert not np.array_equal(outs[0], host(base))


@pytest.mark.parametrize("mode", ["bf16", "e4m3"])
@pytest.mark.parametrize("bn", [128, 256, 512, 1024])
@pytest.mark.parametrize("accumulate", [False, True])
def test_tma_store_epilogue_matches_plain_stores(bmm, mode, bn, accumulate):
    """An output whose base and row stride are 16-byte aligned is written by the epilogue's TMA tile
    stores (TMA reduce-adds when accumulating); one that is not takes plain stores.  Both give the
    same bits, for every tile width and element kind (e4m3 scales its product in the epilogue), on
    ragged m and p."""
    A = bmm._abi
    gm = bmm.MODES[mode]
    m, p, L = 333, 272, 500
    off = S.block_offsets_uneven(3000, 30, 40, 160, seed=17)
    M, N = S.scaled_gaussian(m, 3000, p, off, 1.0, seed=18, dtype=np.float32)
    Mt, Nt = to_dev(M), to_dev(N)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=gm)
    r = bmm.run(prob, "ONC", L, seed=9, compute_product=False)
    A.bmm_autotune_clear()
    A.bmm_autotune_set(m, p, L, gm, bn, 8)
    base = torch.from_numpy(np.random.default_rng(4).standard_normal((m, p)).astype(np.float32)).to(Mt.device)
    aligned = base.clone()
    assert aligned.data_ptr() % 16 == 0 and aligned.stride(0) % 4 == 0
    offset = torch.empty(m * p + 1, dtype=torch.float32, device=Mt.device)[1:].view(m, p)  # base 4 bytes off
    padded = torch.empty(m, p + 1, dtype=torch.float32, device=Mt.device)[:, :p]  # row stride p + 1
    outs = []
    for out in (aligned, offset, padded):
        out.copy_(base)
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, accumulate, prob.ws)
        bmm.check_status(prob)
        outs.append(host(out))
    A.bmm_autotune_clear()
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])


@pytest.mark.parametrize("bn", [128, 256, 512, 1024])
@pytest.mark.parametrize("p", [272, 300])
def test_tma_epilogue_repeatable_at_ragged_edges(bmm, bn, p):
    """Where the last column tile holds chunks wholly past the matrix (p = 272, 300), the epilogue
    stages and stores only the others, so a staging buffer is never refilled while a store that
    reads it is in flight: twelve repetitions of the TMA-store product (plain and accumulating)
    equal the plain-store product bit for bit every time."""
    A = bmm._abi
    gm = A.GEMM_BF16
    m, L = 700, 900
    off = S.block_offsets_uneven(3000, 40, 40, 110, seed=81)
    M, N = S.scaled_gaussian(m, 3000, p, off, 1.0, seed=82, dtype=np.float32)
    Mt, Nt = to_dev(M), to_dev(N)
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=gm)
    r = bmm.run(prob, "ONC", L, seed=4, compute_product=False)
    A.bmm_autotune_clear()
    A.bmm_autotune_set(m, p, L, gm, bn, 8)
    plain = torch.empty(m * p + 1, dtype=torch.float32, device=Mt.device)[1:].view(m, p)  # no TMA: base 4 bytes off
    A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, plain, False, prob.ws)
    want = host(plain).copy()
    out = torch.empty(m, p, dtype=torch.float32, device=Mt.device)
    for rep in range(12):
        out.fill_(float("nan"))
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, False, prob.ws)
        A.bmm_apply(Mt, Nt, prob.B, A.UNIT_COLUMN, r["idx"], r["scale"], L, gm, out, True, prob.ws)
        bmm.check_status(prob)
        np.testing.assert_array_equal(host(out), 2 * want, err_msg=f"repetition {rep}")
    A.bmm_autotune_clear()


def test_grouped_launch_mixed_choices(bmm):
    """bmm_apply_batched with products whose recorded tile widths differ: each product lands in the
    launch of its own width and equals its single-product result."""
    A = bmm._abi
    gm = A.GEMM_BF16
    A.bmm_autotune_clear()
    probs, samples, cs, shapes = [], [], [], [(300, 200), (520, 136), (128, 520), (700, 300)]
    for i, (m, p) in enumerate(shapes):
        off = S.block_offsets_uneven(3000, 30, 40, 160, seed=70 + i)
        M, N = S.scaled_gaussian(m, 3000, p, off, 1.0, seed=80 + i, dtype=np.float32)
        pr = bmm.prepare(to_dev(M), to_dev(N), off, max_draws=600, gemm_mode=gm)
        r = bmm.run(pr, "ONC", 600, seed=i, compute_product=False)
        probs.append(pr)
        samples.append(r)
        cs.append(600)
        A.bmm_autotune_set(m, p, 600, gm, (128, 256, A.TILE_PAIR, A.TILE_PAIR_WIDE)[i % 4], (4, 8, 16)[(i + 1) % 3])
    single = []
    for pr, r in zip(probs, samples):
        out = torch.empty(pr.M.shape[0], pr.N.shape[1], dtype=torch.float32, device=pr.M.device)
        A.bmm_apply(pr.M, pr.N, pr.B, A.UNIT_COLUMN, r["idx"], r["scale"], 600, gm, out, False, pr.ws)
        single.append(host(out))
    outs = [torch.empty(pr.M.shape[0], pr.N.shape[1], dtype=torch.float32, device=pr.M.device) for pr in probs]
    A.bmm_apply_batched([pr.M for pr in probs], [pr.N for pr in probs], [pr.B for pr in probs], A.UNIT_COLUMN,
                        [r["idx"] for r in samples], [r["scale"] for r in samples], cs, gm, outs, False,
                        [pr.ws for pr in probs])
    for pr in probs:
        bmm.check_status(pr)
    for a_, b_ in zip(single, outs):
        np.testing.assert_array_equal(host(b_), a_)
    A.bmm_autotune_clear()


def test_batch_level_tuning_keeps_results(bmm):
    """autotune_batched times the batch's own grouped launch under each tile policy and keeps the
    fastest; the products are unchanged bit for bit."""
    A = bmm._abi
    A.bmm_autotune_clear()
    probs, cs = [], []
    for i, (m, p) in enumerate([(256, 384), (640, 128), (384, 512)]):
        off = S.block_offsets_uneven(4096, 64, 32, 100, seed=90 + i)
        M, N = S.scaled_gaussian(m, 4096, p, off, 1.0, seed=95 + i, dtype=np.float32)
        probs.append(bmm.prepare(to_dev(M), to_dev(N), off, max_draws=512, gemm_mode=A.GEMM_BF16))
        cs.append(512)
    res = bmm.run_batched(probs, "ONC", cs, [1, 2, 3], gemm_mode=A.GEMM_BF16)
    before = [host(r["out"]).copy() for r in res]
    tune = bmm.autotune_batched(probs, res, cs, A.GEMM_BF16)
    assert tune["choice"] in tune["ms"] and len(tune["ms"]) == 14
    res2 = bmm.run_batched(probs, "ONC", cs, [1, 2, 3], gemm_mode=A.GEMM_BF16)
    for a_, r in zip(before, res2):
        np.testing.assert_array_equal(host(r["out"]), a_)
    A.bmm_autotune_clear()


@pytest.mark.parametrize("m,p", [(300, 264), (100, 70), (520, 1000)])
def test_adjoint_tile_choices_do_not_change_gradients(bmm, m, p):
    """The adjoint's GEMMs -- dM with G as a K-major A, dN with G as an MN-major B (rows of K, boxes
    of 64 columns) -- give the same gradients bit for bit under every tile choice, on ragged shapes
    (p not a multiple of 64, m below one 128-row tile)."""
    A = bmm._abi
    gm = A.GEMM_BF16
    n = 3000
    off = S.block_offsets_uneven(n, 30, 40, 160, seed=71)
    M, N = S.scaled_gaussian(m, n, p, off, 1.0, seed=72, dtype=np.float32)
    Mt, Nt = to_dev(M), to_dev(N)
    L = 700
    prob = bmm.prepare(Mt, Nt, off, max_draws=L, gemm_mode=gm)
    r = bmm.run(prob, "ONC", L, seed=5, gemm_mode=gm, compute_product=False)
    Gt = to_dev(np.random.default_rng(73).standard_normal((m, p)).astype(np.float32))
    lmax = min(L, n)  # rows of the gathered operands: at most one per distinct draw
    A.bmm_autotune_clear()
    grads = []
    for bn, ra in CHOICES:
        A.bmm_autotune_set(m, lmax, p, gm, bn, ra)    # dM = G (m x p) times the drawn rows of N
        A.bmm_autotune_set(lmax, p, m, gm, bn, ra)    # dN = drawn columns of M (transposed) times G
        dM = torch.full((m, n), float("nan"), dtype=torch.float32, device=Mt.device)
        dN = torch.full((n, p), float("nan"), dtype=torch.float32, device=Mt.device)
        bmm.bmm_backward(Gt, Mt, Nt, prob.B, r["unit"], r["p"], r["ck"], L, 5, r["sid"], gm, dM, dN, False, prob.ws)
        bmm.check_status(prob)
        grads.append((host(dM), host(dN)))
    A.bmm_autotune_clear()
    for gM, gN in grads[1:]:
        np.testing.assert_array_equal(gM, grads[0][0])
        np.testing.assert_array_equal(gN, grads[0][1])
    assert np.all(np.isfinite(grads[0][0])) and np.all(np.isfinite(grads[0][1]))

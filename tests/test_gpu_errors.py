"""Error bars through the C ABI (bmm_entry_variance, bmm_entry_estimate, bmm_error_report) against the
FP64 oracle, on the same seeded inputs and the same draws.

Tolerances: FP64 sums on both sides in different orders; eq. 3.7 subtracts the squared block dot
product from the sum of squares and the estimate subtracts a mean, so entries are compared to
1e-10 of the entry's scale (the sum of its non-negative terms), the report to 1e-12 relative."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from tests._gpu_util import as_layout, host, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bmm():
    import paper_2105_04940_gb300 as P
    P.build()
    P._abi.load()
    assert torch.cuda.is_available()
    return P


def _problem(m, n, p, K, seed, dtype):
    off = S.block_offsets_uneven(n, K, 1, 2 * n // K, seed=seed)
    M, N = S.scaled_gaussian(m, n, p, off, 1.0, seed=seed + 1, dtype=np.float64)
    if dtype == "bf16":
        Mt, Nt = to_dev(M, torch.bfloat16), to_dev(N, torch.bfloat16)
    else:
        Mt, Nt = to_dev(M.astype(dtype)), to_dev(N.astype(dtype))
    return off, host(Mt.double()), host(Nt.double()), Mt, Nt


def _entries(m, p, count, seed):
    rng = np.random.default_rng(seed)
    e = np.stack([rng.integers(0, m, count), rng.integers(0, p, count)], axis=1).astype(np.int64)
    e[:3] = [(0, 0), (m - 1, p - 1), (m - 1, 0)]
    return e


def _scale_col(M, N, off, p, ck, ent):
    # the positive part of eq. 3.7 per entry: what cancellation is measured against
    ckd = np.repeat(ck, np.diff(off)).astype(np.float64)
    q = np.where(p > 0, 1.0 / np.where(p > 0, p, 1.0), 0.0) / ckd
    return np.array([np.sum((M[h] * N[:, f]) ** 2 * q) for h, f in ent])


@pytest.mark.parametrize("dtype", [np.float64, np.float32, "bf16"])
@pytest.mark.parametrize("layouts", [("row", "row"), ("col", "row"), ("row", "col")])
def test_entry_variance_columns(bmm, dtype, layouts):
    off, M, N, Mt, Nt = _problem(41, 733, 29, 23, seed=71, dtype=dtype)
    Mt, Nt = as_layout(Mt, layouts[0]), as_layout(Nt, layouts[1])
    p = S.random_probabilities(off, seed=72, zero_frac=0.1)
    ck = np.random.default_rng(73).integers(1, 6, len(off) - 1).astype(np.int64)
    ent = _entries(41, 29, 150, seed=74)
    prob = bmm.prepare(Mt, Nt, off, max_draws=16)
    out = torch.empty(len(ent), dtype=torch.float64, device=Mt.device)
    bmm.bmm_entry_variance(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, to_dev(p), to_dev(ck), int(ck.sum()),
                           to_dev(ent), out)
    want = oracle.entry_variance_columns(M, N, off, p, ck, ent)
    scale = _scale_col(M, N, off, p, ck, ent)
    assert np.all(np.abs(host(out) - want) <= 1e-10 * scale + 1e-300)


@pytest.mark.parametrize("dtype", [np.float64, "bf16"])
def test_entry_variance_blocks(bmm, dtype):
    off, M, N, Mt, Nt = _problem(23, 500, 17, 31, seed=81, dtype=dtype)
    pblk = S.random_probabilities(np.array([0, len(off) - 1]), seed=82, zero_frac=0.1)
    ent = _entries(23, 17, 90, seed=83)
    c = 37
    prob = bmm.prepare(Mt, Nt, off, max_draws=c, unit=bmm._abi.UNIT_BLOCK)
    out = torch.empty(len(ent), dtype=torch.float64, device=Mt.device)
    bmm.bmm_entry_variance(Mt, Nt, prob.B, bmm._abi.UNIT_BLOCK, to_dev(pblk), None, c, to_dev(ent), out)
    want = oracle.entry_variance_blocks(M, N, off, pblk, c, ent)
    d = [np.array([M[h, off[k]:off[k + 1]] @ N[off[k]:off[k + 1], f] for k in range(len(off) - 1)]) for h, f in ent]
    scale = np.array([np.sum(np.where(pblk > 0, di * di / np.where(pblk > 0, pblk, 1), 0)) / c for di in d])
    assert np.all(np.abs(host(out) - want) <= 1e-10 * scale + 1e-300)


@pytest.mark.parametrize("dtype", [np.float64, np.float32, "bf16"])
def test_entry_estimate_columns(bmm, dtype):
    off, M, N, Mt, Nt = _problem(37, 900, 21, 30, seed=91, dtype=dtype)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = np.random.default_rng(92).integers(1, 7, len(off) - 1).astype(np.int64)
    ck[:3] = 1  # single-draw blocks add value but no variance
    idx, scale = oracle.sample_alg2(p, off, ck, 93, 0)
    ent = _entries(37, 21, 120, seed=94)
    prob = bmm.prepare(Mt, Nt, off, max_draws=int(ck.sum()))
    cd = torch.empty(len(ent), dtype=torch.float64, device=Mt.device)
    s2 = torch.empty_like(cd)
    bmm.bmm_entry_estimate(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, to_dev(ck), to_dev(idx.astype(np.int32)),
                           to_dev(scale), len(idx), to_dev(ent), cd, s2, prob.ws)
    bmm.check_status(prob)
    w_cd, w_s2, _ = oracle.entry_estimate_columns(M, N, off, ck, idx, scale, ent)
    mag = np.array([np.sum(np.abs(scale * M[h, idx] * N[idx, f])) for h, f in ent])
    assert np.all(np.abs(host(cd) - w_cd) <= 1e-12 * mag + 1e-300)
    assert np.all(np.abs(host(s2) - w_s2) <= 1e-10 * (mag * mag) + 1e-300)


def test_entry_estimate_blocks_and_edges(bmm):
    off, M, N, Mt, Nt = _problem(19, 400, 13, 25, seed=101, dtype=np.float64)
    pblk = S.random_probabilities(np.array([0, len(off) - 1]), seed=102)
    kidx, scale = oracle.sample_blocks(pblk, 40, 103, 0)
    ent = _entries(19, 13, 60, seed=104)
    prob = bmm.prepare(Mt, Nt, off, max_draws=40, unit=bmm._abi.UNIT_BLOCK)
    cd = torch.empty(len(ent), dtype=torch.float64, device=Mt.device)
    s2 = torch.empty_like(cd)
    bmm.bmm_entry_estimate(Mt, Nt, prob.B, bmm._abi.UNIT_BLOCK, None, to_dev(kidx.astype(np.int32)), to_dev(scale),
                           len(kidx), to_dev(ent), cd, s2, prob.ws)
    w_cd, w_s2 = oracle.entry_estimate_blocks(M, N, off, kidx, scale, ent)
    mag = np.array([sum(abs(s * (M[h, off[k]:off[k + 1]] @ N[off[k]:off[k + 1], f])) for s, k in zip(scale, kidx))
                    for h, f in ent])
    assert np.all(np.abs(host(cd) - w_cd) <= 1e-12 * mag + 1e-300)
    assert np.all(np.abs(host(s2) - w_s2) <= 1e-10 * mag * mag + 1e-300)
    # entries outside the product come back NaN; an empty list is a no-op
    bad = to_dev(np.array([[19, 0], [0, 13], [-1, 2]], dtype=np.int64))
    out = torch.zeros(3, dtype=torch.float64, device=Mt.device)
    bmm.bmm_entry_variance(Mt, Nt, prob.B, bmm._abi.UNIT_BLOCK, to_dev(pblk), None, 40, bad, out)
    assert torch.isnan(out).all()
    bmm.bmm_entry_estimate(Mt, Nt, prob.B, bmm._abi.UNIT_BLOCK, None, to_dev(kidx.astype(np.int32)), to_dev(scale),
                           len(kidx), bad, out, torch.empty_like(out), prob.ws)
    assert torch.isnan(out).all()
    empty = torch.empty((0, 2), dtype=torch.int64, device=Mt.device)
    bmm.bmm_entry_variance(Mt, Nt, prob.B, bmm._abi.UNIT_BLOCK, to_dev(pblk), None, 40, empty, out[:0])
    torch.cuda.synchronize()


def test_entry_estimate_draw_count_mismatch_is_reported(bmm):
    off, M, N, Mt, Nt = _problem(8, 200, 6, 10, seed=111, dtype=np.float64)
    ck = np.full(len(off) - 1, 2, dtype=np.int64)
    prob = bmm.prepare(Mt, Nt, off, max_draws=64)
    idx = to_dev(np.zeros(5, dtype=np.int32))
    ent = to_dev(np.array([[0, 0]], dtype=np.int64))
    cd = torch.empty(1, dtype=torch.float64, device=Mt.device)
    bmm.bmm_entry_estimate(Mt, Nt, prob.B, bmm._abi.UNIT_COLUMN, to_dev(ck), idx, to_dev(np.ones(5)), 5, ent, cd,
                           torch.empty_like(cd), prob.ws)
    assert bmm._abi.bmm_read_device_status(prob.ws) == bmm._abi.ERR_SHAPE
    bmm._abi.bmm_clear_device_status(prob.ws)


@pytest.mark.parametrize("with_fhat", [False, True])
def test_error_report(bmm, with_fhat):
    off, M, N, Mt, Nt = _problem(30, 1200, 26, 40, seed=121, dtype=np.float64)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    f = oracle.block_frob_sq(M, N, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    p[5] *= 0.5  # beta < 1 (still a valid estimator: p_5 > 0)
    ck = oracle.apportion(oracle.g_opt(st["a"], f), np.diff(off), 160)
    fhat = f * np.random.default_rng(122).uniform(0.5, 1.5, len(f)) if with_fhat else None
    want = oracle.error_report(x, y, p, off, ck, st["a"], f, st["mf"], st["nf"], int(ck.sum()), 0.05, fhat=fhat)
    dst = {k: to_dev(np.asarray(v, dtype=np.float64)) for k, v in (("x", x), ("y", y), ("a", st["a"]), ("s", st["s"]),
                                                                    ("mf", st["mf"]), ("nf", st["nf"]), ("f", f))}
    prob = bmm.prepare(Mt, Nt, off, max_draws=16)
    out = torch.empty(bmm._abi.REPORT_LEN, dtype=torch.float64, device=Mt.device)
    bmm._abi.bmm_error_report(prob.B, dst, to_dev(p), to_dev(ck), int(ck.sum()),
                              to_dev(fhat) if fhat is not None else None, 0.05, out)
    got = dict(zip(bmm._abi.REPORT_FIELDS, host(out).tolist()))
    assert tuple(oracle.REPORT_FIELDS) == tuple(bmm._abi.REPORT_FIELDS)
    for k in oracle.REPORT_FIELDS:
        if math.isnan(want[k]):
            assert math.isnan(got[k]), k
        else:
            assert got[k] == pytest.approx(want[k], rel=1e-12), k
    # without f only beta and the Frobenius norms are defined
    dst["f"] = None
    bmm._abi.bmm_error_report(prob.B, dst, to_dev(p), to_dev(ck), int(ck.sum()), None, 0.05, out)
    got = host(out)
    assert got[4] == pytest.approx(want["beta"], rel=1e-12) and not math.isnan(got[5])
    assert np.isnan(got[[0, 1, 2, 3, 7, 8]]).all()


def test_error_bars_on_a_run(bmm):
    """End to end on one OPL product: the one-sample intervals cover about 95% of the entries of MN
    (Thm 3.1), and eq. 3.7 summed over every entry equals the report's E||MN - CD||_F^2 (Remark 2.2),
    both computed on the GPU from the run's own design."""
    off = S.block_offsets_equal(4096, 32)
    M, N = S.scaled_gaussian(48, 4096, 40, off, 1.0, seed=131, dtype=np.float64)
    Mt, Nt = to_dev(M), to_dev(N)
    prob = bmm.prepare(Mt, Nt, off, max_draws=2048, gemm_mode=bmm._abi.GEMM_F64)
    res = bmm.run(prob, "OPL", 2048, seed=5, gemm_mode=bmm._abi.GEMM_F64, fmode=bmm._abi.F_EXACT)
    bmm.check_status(prob)
    rep = bmm.error_report(prob, res, delta=0.1)
    ent = np.array([(h, f) for h in range(48) for f in range(40)], dtype=np.int64)
    eb = bmm.error_bars(prob, res, ent, exact=True)
    var = host(eb["var"])
    assert var.sum() == pytest.approx(rep["expected_sq_error"], rel=1e-9)
    assert rep["expected_sq_error"] <= rep["eq312"]
    MN = M @ N
    lo, hi = host(eb["lo"]), host(eb["hi"])
    cover = np.mean((MN.ravel() >= lo) & (MN.ravel() <= hi))
    assert 0.90 <= cover <= 0.985, cover
    np.testing.assert_allclose(host(eb["value"]), host(res["out"]).ravel(), rtol=1e-9, atol=1e-9 * np.abs(MN).max())


def test_error_report_hand_worked_example(bmm):
    """bmm_error_report on the hand-worked example of tests/golden/error_report_thm33_thm44.json
    (theta_1 != theta_2, beta < 1, theta-hat_1 != theta-hat_2): every field against the values
    simplified by hand from Remark 2.2, eq. 3.10 and Thms 3.3, 4.2 and 4.4."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "error_report_thm33_thm44.json")
    with open(path) as fh:
        fx = json.load(fh)
    i = fx["inputs"]
    off = np.asarray(i["offsets"], dtype=np.int64)
    off_dev = to_dev(off)
    B = bmm._abi.blocks(off_dev, int(off[-1]), int(np.diff(off).max()))
    dst = {k: to_dev(np.asarray(i[k], dtype=np.float64)) for k in ("x", "y", "a", "mf", "nf", "f")}
    out = torch.empty(bmm._abi.REPORT_LEN, dtype=torch.float64, device=off_dev.device)
    bmm._abi.bmm_error_report(B, dst, to_dev(np.asarray(i["p"], dtype=np.float64)),
                              to_dev(np.asarray(i["ck"], dtype=np.int64)), int(i["c"]),
                              to_dev(np.asarray(i["fhat"], dtype=np.float64)), math.exp(-1.0), out)
    got = dict(zip(bmm._abi.REPORT_FIELDS, host(out).tolist()))
    for name, e in fx["expected"].items():
        assert got[name] == pytest.approx(e["value"], rel=1e-13, abs=0.0), name

"""bmm_probs_static, the workspace-free statistics entry point, against bmm_probs.

Callers that cannot allocate device memory at call time use bmm_probs_static; its results must
be those of bmm_probs, which takes a caller workspace.  Two calls in a row check that the shared
fixed scratch array, which keeps the previous call's contents, does not leak into the next result.
This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def test_static_scratch_matches_workspace_entry_point():
    import paper_2105_04940_gb300 as P
    P.build()
    A = P._abi
    A.load()
    dev = torch.device("cuda:0")
    # row-major M wide enough that the column pass splits rows into slices (uses the scratch)
    off = S.block_offsets_uneven(40000, 300, 40, 250, seed=7)
    Mh, Nh = S.scaled_gaussian(3000, 40000, 500, off, 1.0, seed=8, dtype=np.float32)
    M, N = torch.from_numpy(Mh).to(dev), torch.from_numpy(Nh).to(dev)
    off_dev = torch.as_tensor(off, device=dev)
    B = A.blocks(off_dev, 40000, int(np.diff(off).max()))
    f64 = dict(dtype=torch.float64, device=dev)

    def fresh_stats():
        return {k: torch.full((40000 if k in ("x", "y") else 300,), float("nan"), **f64)
                for k in ("x", "y", "a", "s", "mf", "nf")}

    ws = torch.zeros(A.bmm_workspace_size(M, N, B, A.UNIT_COLUMN, 1, A.GEMM_BF16), dtype=torch.uint8, device=dev)
    st_ref, p_ref = fresh_stats(), torch.empty(40000, **f64)
    A.bmm_probs(M, N, B, A.P_COL_OPT, A.F_NONE, p_ref, st_ref, ws)
    assert A.bmm_read_device_status(ws) == A.OK

    for call in range(2):
        st, p = fresh_stats(), torch.empty(40000, **f64)
        status = torch.zeros(2, dtype=torch.int32, device=dev)
        A.bmm_probs_static(M, N, B, A.P_COL_OPT, p, st, status)
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0], call
        for k in st:
            assert _rel(st[k].cpu().numpy(), st_ref[k].cpu().numpy()) <= 1e-12, (call, k)
        assert _rel(p.cpu().numpy(), p_ref.cpu().numpy()) <= 1e-12, call

    # A problem whose partial sums exceed the fixed scratch is refused before any launch:
    # BF16 M of 128 x 1,049,600 splits its rows into 2 slices -> 2 * 1,049,600 doubles = 16.79 MB.
    # Every buffer is real and large enough, so nothing could be read out of bounds either way.
    nbig, mbig, kbig = 1_049_600, 128, 1025
    big_off = S.block_offsets_equal(nbig, kbig)
    Mb = torch.zeros((mbig, nbig), dtype=torch.bfloat16, device=dev)
    Nb = torch.zeros((nbig, 8), dtype=torch.bfloat16, device=dev)
    big_off_dev = torch.as_tensor(big_off, device=dev)  # kept alive: the struct holds only its address
    Bb = A.blocks(big_off_dev, nbig, int(np.diff(big_off).max()))
    st_big = {k: torch.zeros(nbig if k in ("x", "y") else kbig, **f64) for k in ("x", "y", "a", "s", "mf", "nf")}
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    with pytest.raises(A.BmmError) as err:
        A.bmm_probs_static(Mb, Nb, Bb, A.P_COL_OPT, None, st_big, status)
    assert err.value.code == A.ERR_WORKSPACE


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m_layout,n_layout", [("row", "row"), ("col", "col"), ("col", "row"), ("row", "col")])
@pytest.mark.parametrize("pkind", ["col_opt", "col_uniform", "blk_normprod"])
def test_static_scratch_every_type_layout_and_kind(dtype, m_layout, n_layout, pkind):
    """The same comparison over every element type, both storage orders of M and N (which decide
    whether the column pass needs the partial sums at all) and the three probability kinds the
    static form offers; the FP64 row-major case of each kind runs without p_out (which must then stay
    untouched)."""
    import paper_2105_04940_gb300 as P
    P.build()
    A = P._abi
    A.load()
    dev = torch.device("cuda:0")
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    pk = {"col_opt": A.P_COL_OPT, "col_uniform": A.P_COL_UNIFORM, "blk_normprod": A.P_BLK_NORMPROD}[pkind]
    m, n, p = 1100, 6000, 300
    off = S.block_offsets_uneven(n, 70, 40, 130, seed=21)
    K = len(off) - 1
    Mh, Nh = S.scaled_gaussian(m, n, p, off, 1.0, seed=22)
    M = torch.from_numpy(Mh).to(dev).to(tdt)
    N = torch.from_numpy(Nh).to(dev).to(tdt)
    if m_layout == "col":
        M = M.t().contiguous().t()
    if n_layout == "col":
        N = N.t().contiguous().t()
    off_dev = torch.as_tensor(off, device=dev)
    B = A.blocks(off_dev, n, int(np.diff(off).max()))
    f64 = dict(dtype=torch.float64, device=dev)
    plen = n if pk != A.P_BLK_NORMPROD else K

    def fresh_stats():
        return {k: torch.full((n if k in ("x", "y") else K,), float("nan"), **f64)
                for k in ("x", "y", "a", "s", "mf", "nf")}

    ws = torch.zeros(A.bmm_workspace_size(M, N, B, A.UNIT_COLUMN, 1, A.GEMM_BF16), dtype=torch.uint8, device=dev)
    st_ref, p_ref = fresh_stats(), torch.empty(plen, **f64)
    A.bmm_probs(M, N, B, pk, A.F_NONE, p_ref, st_ref, ws)
    assert A.bmm_read_device_status(ws) == A.OK
    with_p = not (m_layout == "row" and n_layout == "row" and dtype == "f64")
    for call in range(2):
        st, pv = fresh_stats(), torch.full((plen,), float("nan"), **f64)
        status = torch.zeros(2, dtype=torch.int32, device=dev)
        A.bmm_probs_static(M, N, B, pk, pv if with_p else None, st, status)
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0], call
        for k in st:
            assert _rel(st[k].cpu().numpy(), st_ref[k].cpu().numpy()) <= 1e-12, (call, k)
        if with_p:
            assert _rel(pv.cpu().numpy(), p_ref.cpu().numpy()) <= 1e-12, call
        else:
            assert torch.isnan(pv).all()

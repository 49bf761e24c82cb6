"""The C ABI library builds, loads without a GPU and exports every entry point of include/bmm.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_04940_gb300 import build, _abi
    build()
    return _abi.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "bmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bmm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2105_04940_gb300 import _abi
    declared = _declared()
    assert declared == sorted(_abi.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_only_the_abi_is_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2105_04940_gb300", "libbmm.so")],
                         capture_output=True, text=True).stdout
    funcs = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert funcs == _declared()


def test_status_strings_and_workspace_size_on_host(lib):
    from paper_2105_04940_gb300 import _abi
    assert _abi.status_string(0) == "ok"
    assert "workspace" in _abi.status_string(_abi.ERR_WORKSPACE)
    fake = 1 << 20  # never dereferenced: the size query only reads the descriptors
    M = _abi.Mat(fake, 256, 4096, 4096, _abi.F32, _abi.ROW_MAJOR)
    N = _abi.Mat(fake, 4096, 256, 256, _abi.F32, _abi.ROW_MAJOR)
    B = _abi.Blocks(64, 4096, 64, fake)
    sz = lib.bmm_workspace_size(ctypes.byref(M), ctypes.byref(N), ctypes.byref(B), _abi.UNIT_COLUMN, 1024,
                                _abi.GEMM_SPLIT_BF16)
    # at least the two split-BF16 operands (256 x 3*1024 bf16 each) plus the status block
    assert sz >= 2 * 256 * 3 * 1024 * 2 + 256
    bad = _abi.Mat(fake, 256, 4000, 4096, _abi.F32, _abi.ROW_MAJOR)
    assert lib.bmm_workspace_size(ctypes.byref(bad), ctypes.byref(N), ctypes.byref(B), 0, 1024, 1) == 0
    blk = lib.bmm_workspace_size(ctypes.byref(M), ctypes.byref(N), ctypes.byref(B), _abi.UNIT_BLOCK, 16,
                                 _abi.GEMM_BF16)
    assert blk >= 2 * 256 * 16 * 64 * 2


def test_product_path_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_2105_04940_gb300 as P
    with pytest.raises(RuntimeError):
        P.prepare(torch.zeros(4, 4), torch.zeros(4, 4), np.array([0, 2, 4]), max_draws=2)


def test_autotune_table_host_side():
    """The GEMM tile table (no device access): untuned shapes take the default rule, a recorded
    choice covers its whole bucket (rounded-up log2 of m, p and the GEMM depth), invalid choices and
    modes are refused, and clear forgets everything."""
    import paper_2105_04940_gb300 as P
    A = P._abi
    A.load()
    A.bmm_autotune_clear()
    assert A.bmm_autotune_get(300, 100, 517, A.GEMM_BF16) == {"bn": 128, "raster": 8}
    assert A.bmm_autotune_get(100, 520, 517, A.GEMM_BF16) == {"bn": 256, "raster": 8}  # m <= 128: one CTA
    assert A.bmm_autotune_get(300, 520, 517, A.GEMM_BF16) == {"bn": A.TILE_PAIR, "raster": 8}
    A.bmm_autotune_set(300, 520, 517, A.GEMM_BF16, 128, 16)
    assert A.bmm_autotune_get(300, 520, 600, A.GEMM_BF16) == {"bn": 128, "raster": 16}  # same bucket
    assert A.bmm_autotune_get(300, 520, 2000, A.GEMM_BF16) == {"bn": A.TILE_PAIR, "raster": 8}  # depth bucket differs
    assert A.bmm_autotune_get(300, 520, 517, A.GEMM_E4M3) == {"bn": A.TILE_PAIR, "raster": 8}  # element kind differs
    A.bmm_autotune_set(300, 520, 517, A.GEMM_BF16, A.TILE_PAIR, 4)
    assert A.bmm_autotune_get(300, 520, 517, A.GEMM_BF16) == {"bn": A.TILE_PAIR, "raster": 4}
    for bad in ((300, 520, 517, A.GEMM_BF16, 192, 8), (300, 520, 517, A.GEMM_BF16, 128, 5), (300, 520, 517, A.GEMM_BF16, 2048, 8),
                (300, 520, 517, A.GEMM_F64, 128, 8), (0, 520, 517, A.GEMM_BF16, 128, 8)):
        with pytest.raises(A.BmmError):
            A.bmm_autotune_set(*bad)
    assert A.bmm_autotune_workspace_size(300, 520, 517, A.GEMM_F64) == 0
    assert A.bmm_autotune_workspace_size(300, 520, 517, A.GEMM_BF16) > 256 + 2 * (300 + 520) * 576
    A.bmm_autotune_clear()
    assert A.bmm_autotune_get(300, 520, 517, A.GEMM_BF16) == {"bn": A.TILE_PAIR, "raster": 8}


def test_error_bar_calls_validate_arguments_on_host(lib):
    """The error-bar entry points reject bad arguments before any device work (no GPU needed), and
    the report's field names match the BMM_REPORT_* indices of include/bmm.h."""
    from paper_2105_04940_gb300 import _abi
    fake = 1 << 20  # never dereferenced
    M = _abi.Mat(fake, 8, 64, 64, _abi.F64, _abi.ROW_MAJOR)
    N = _abi.Mat(fake, 64, 8, 8, _abi.F64, _abi.ROW_MAJOR)
    B = _abi.Blocks(4, 64, 16, fake)
    st = _abi.Stats(fake, fake, fake, fake, fake, fake, None)
    ok = dict(p=fake, ck=fake, out=fake)
    assert lib.bmm_error_report(ctypes.byref(B), ctypes.byref(st), fake, fake, 16, None, 1.5, fake, None) == _abi.ERR_ARG
    assert lib.bmm_error_report(ctypes.byref(B), ctypes.byref(st), fake, fake, 0, None, 0.1, fake, None) == _abi.ERR_ARG
    assert lib.bmm_error_report(ctypes.byref(B), None, fake, fake, 16, None, 0.1, fake, None) == _abi.ERR_ARG
    assert lib.bmm_entry_variance(ctypes.byref(M), ctypes.byref(N), ctypes.byref(B), 7, ok["p"], ok["ck"], 16, fake,
                                  3, fake, None) == _abi.ERR_ARG
    assert lib.bmm_entry_variance(ctypes.byref(M), ctypes.byref(N), ctypes.byref(B), _abi.UNIT_COLUMN, ok["p"], None,
                                  16, fake, 3, fake, None) == _abi.ERR_ARG
    badN = _abi.Mat(fake, 63, 8, 8, _abi.F64, _abi.ROW_MAJOR)
    assert lib.bmm_entry_variance(ctypes.byref(M), ctypes.byref(badN), ctypes.byref(B), _abi.UNIT_COLUMN, ok["p"],
                                  ok["ck"], 16, fake, 3, fake, None) == _abi.ERR_SHAPE
    assert lib.bmm_entry_estimate(ctypes.byref(M), ctypes.byref(N), ctypes.byref(B), _abi.UNIT_COLUMN, fake, fake,
                                  fake, 16, fake, 3, fake, fake, None, 0, None) == _abi.ERR_WORKSPACE
    text = open(os.path.join(ROOT, "include", "bmm.h")).read()
    idx = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"BMM_REPORT_([A-Z0-9_]+) = (\d+)", text)}
    assert idx.pop("len") == _abi.REPORT_LEN
    assert [k for k, _ in sorted(idx.items(), key=lambda kv: kv[1])] == list(_abi.REPORT_FIELDS)


def test_blocksizes_batched_validates_on_host(lib):
    """bmm_blocksizes_batched refuses bad arguments before any device work: a negative count, the
    pilot kind (which needs bmm_blocksizes), missing statistics, an infeasible c, a short workspace."""
    from paper_2105_04940_gb300 import _abi
    fake = 1 << 20  # never dereferenced
    B = (_abi.Blocks * 1)(_abi.Blocks(4, 64, 16, fake))
    st = (_abi.Stats * 1)(_abi.Stats(None, None, fake, None, None, None, fake))
    cs = (ctypes.c_int64 * 1)(16)
    ck = (ctypes.c_void_p * 1)(fake)
    ws = (ctypes.c_void_p * 1)(1 << 21)  # 256-byte aligned
    big = (ctypes.c_size_t * 1)(1 << 20)
    small = (ctypes.c_size_t * 1)(64)
    call = lib.bmm_blocksizes_batched
    assert call(-1, B, st, _abi.CK_OPT, cs, ck, None, ws, big, None) == _abi.ERR_ARG
    assert call(0, None, None, _abi.CK_OPT, None, None, None, None, None, None) == _abi.OK
    assert call(1, B, st, _abi.CK_TILDE, cs, ck, None, ws, big, None) == _abi.ERR_ARG
    assert call(1, B, None, _abi.CK_OPT, cs, ck, None, ws, big, None) == _abi.ERR_ARG
    no_f = (_abi.Stats * 1)(_abi.Stats(None, None, fake, None, None, None, None))
    assert call(1, B, no_f, _abi.CK_OPT, cs, ck, None, ws, big, None) == _abi.ERR_ARG
    bad_c = (ctypes.c_int64 * 1)(3)  # below K
    assert call(1, B, st, _abi.CK_OPT, bad_c, ck, None, ws, big, None) == _abi.ERR_INFEASIBLE
    assert call(1, B, st, _abi.CK_OPT, cs, ck, None, ws, small, None) == _abi.ERR_WORKSPACE


def test_static_entry_point_checks_arguments_like_bmm_probs(lib):
    """bmm_probs_static and bmm_probs refuse the same bad descriptors with the same status codes,
    before anything is launched (host only: no pointer below is ever dereferenced).  bmm_probs is
    called first with no workspace, so a case that slipped past the descriptor checks would fail
    there (BMM_ERR_WORKSPACE) before bmm_probs_static could launch anything on the fake pointers."""
    from paper_2105_04940_gb300 import _abi
    fake = 1 << 20
    n, K = 4096, 64

    def M_(**kw):
        d = dict(data=fake, rows=256, cols=n, ld=n, dtype=_abi.F32, layout=_abi.ROW_MAJOR)
        d.update(kw)
        return _abi.Mat(d["data"], d["rows"], d["cols"], d["ld"], d["dtype"], d["layout"])

    def N_(**kw):
        d = dict(data=fake, rows=n, cols=256, ld=256, dtype=_abi.F32, layout=_abi.ROW_MAJOR)
        d.update(kw)
        return _abi.Mat(d["data"], d["rows"], d["cols"], d["ld"], d["dtype"], d["layout"])

    def B_(**kw):
        d = dict(K=K, n=n, max_nk=64, offsets=fake)
        d.update(kw)
        return _abi.Blocks(d["K"], d["n"], d["max_nk"], d["offsets"])

    good_st = _abi.Stats(*([fake] * 6 + [None]))
    big = 1 << 31
    cases = {
        "M null": (M_(data=None), N_(), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_ARG),
        "M dtype": (M_(dtype=7), N_(), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_DTYPE),
        "M misaligned for F32": (M_(data=fake + 2), N_(), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_ARG),
        "F64 N misaligned": (M_(dtype=_abi.F64), N_(dtype=_abi.F64, data=fake + 4), B_(), _abi.P_COL_OPT, good_st,
                             _abi.ERR_ARG),
        "N layout": (M_(), N_(layout=5), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_ARG),
        "M negative rows": (M_(rows=-1), N_(), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_SHAPE),
        "M short ld": (M_(ld=n - 1), N_(), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_SHAPE),
        "K = 0": (M_(), N_(), B_(K=0), _abi.P_COL_OPT, good_st, _abi.ERR_SHAPE),
        "offsets null": (M_(), N_(), B_(offsets=None), _abi.P_COL_OPT, good_st, _abi.ERR_ARG),
        "n above INT32_MAX": (M_(cols=big, ld=big), N_(rows=big), B_(n=big), _abi.P_COL_OPT, good_st,
                              _abi.ERR_UNSUPPORTED),
        "cols(M) != rows(N)": (M_(), N_(rows=n - 1), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_SHAPE),
        "dtype mismatch": (M_(), N_(dtype=_abi.BF16, ld=256), B_(), _abi.P_COL_OPT, good_st, _abi.ERR_DTYPE),
        "unknown pkind": (M_(), N_(), B_(), 9, good_st, _abi.ERR_ARG),
        "stats without x": (M_(), N_(), B_(), _abi.P_COL_OPT, _abi.Stats(*([None] + [fake] * 5 + [None])),
                            _abi.ERR_ARG),
    }
    by = ctypes.byref
    for name, (M, N, B, pk, st, want) in cases.items():
        got = lib.bmm_probs(by(M), by(N), by(B), pk, _abi.F_NONE, None, by(st), None, 0, None)
        assert got == want, (name, got)
        status = ctypes.c_void_p(fake)
        got_static = lib.bmm_probs_static(by(M), by(N), by(B), pk, None, by(st), status, None)
        assert got_static == want, (name, got_static)
    # the status word of the static form is updated with 32-bit atomics: null or misaligned is refused
    Mg, Ng, Bg = M_(), N_(), B_()
    assert lib.bmm_probs(by(Mg), by(Ng), by(Bg), _abi.P_COL_OPT, _abi.F_NONE, None, by(good_st), None, 0,
                         None) == _abi.ERR_WORKSPACE
    for bad in (None, ctypes.c_void_p(fake + 2)):
        assert lib.bmm_probs_static(by(Mg), by(Ng), by(Bg), _abi.P_COL_OPT, None, by(good_st), bad,
                                    None) == _abi.ERR_ARG


def test_apply_part_refuses_bad_parts_and_row_ranges(lib):
    """bmm_apply_part checks its part and row range on the host, before anything is launched (the
    fake pointers below are never dereferenced)."""
    from paper_2105_04940_gb300 import _abi
    fake = 1 << 20
    M = _abi.Mat(fake, 512, 4096, 4096, _abi.F32, _abi.ROW_MAJOR)
    N = _abi.Mat(fake, 4096, 256, 256, _abi.F32, _abi.ROW_MAJOR)
    out = _abi.Mat(fake, 512, 256, 256, _abi.F32, _abi.ROW_MAJOR)
    B = _abi.Blocks(64, 4096, 64, fake)
    by = ctypes.byref
    call = lambda part, r0, r1, count=100: lib.bmm_apply_part(by(M), by(N), by(B), fake, fake, count, by(out), 0, part,
                                                             r0, r1, None, 0, None)
    assert call(4, 0, 128) == _abi.ERR_ARG
    assert call(-1, 0, 128) == _abi.ERR_ARG
    assert call(_abi.APPLY_GEMM, 0, 128, count=0) == _abi.ERR_ARG
    assert call(_abi.APPLY_GATHER_A, 64, 128) == _abi.ERR_SHAPE   # row0 not a multiple of 128
    assert call(_abi.APPLY_GEMM, 0, 100) == _abi.ERR_SHAPE        # row1 neither a multiple of 128 nor m
    assert call(_abi.APPLY_GEMM, 256, 128) == _abi.ERR_SHAPE      # row1 < row0
    assert call(_abi.APPLY_GEMM, 0, 640) == _abi.ERR_SHAPE        # row1 > m
    # a well-formed request passes these checks and stops at the device (none here) or workspace check;
    # REDUCE and GATHER_B ignore the rows
    assert call(_abi.APPLY_GEMM, 0, 512) in (_abi.ERR_UNSUPPORTED, _abi.ERR_WORKSPACE)
    assert call(_abi.APPLY_REDUCE, 64, 100) in (_abi.ERR_UNSUPPORTED, _abi.ERR_WORKSPACE)
    assert call(_abi.APPLY_GATHER_B, 64, 100) in (_abi.ERR_UNSUPPORTED, _abi.ERR_WORKSPACE)


def test_f_tc_query_on_the_host(lib):
    """bmm_f_tc_supported answers from the descriptors alone (no launch): without an sm_103 device it
    reports the exact fallback; bad descriptors get bmm_probs's codes; a null answer pointer is refused."""
    from paper_2105_04940_gb300 import _abi
    import torch
    fake = 1 << 20
    M = _abi.Mat(fake, 256, 4096, 4096, _abi.F32, _abi.ROW_MAJOR)
    N = _abi.Mat(fake, 4096, 256, 256, _abi.F32, _abi.ROW_MAJOR)
    B = _abi.Blocks(64, 4096, 64, fake)
    r = ctypes.c_int32(-1)
    by = ctypes.byref
    assert lib.bmm_f_tc_supported(by(M), by(N), by(B), by(r)) == _abi.OK
    if not torch.cuda.is_available():
        assert r.value == 0
    bad = _abi.Mat(fake, 256, 4000, 4096, _abi.F32, _abi.ROW_MAJOR)
    assert lib.bmm_f_tc_supported(by(bad), by(N), by(B), by(r)) == _abi.ERR_SHAPE
    assert lib.bmm_f_tc_supported(by(M), by(N), by(B), None) == _abi.ERR_ARG


def test_core_entry_points_validate_on_host(lib):
    """bmm_blocksizes, bmm_sample and bmm_backward refuse bad arguments with the documented codes
    before anything is launched (host only: the fake pointers are never dereferenced; a case that
    slipped past the checks would stop at the missing workspace, BMM_ERR_WORKSPACE, instead)."""
    from paper_2105_04940_gb300 import _abi
    fake = 1 << 20
    n, K, m, p = 4096, 64, 256, 128
    M = _abi.Mat(fake, m, n, n, _abi.F32, _abi.ROW_MAJOR)
    N = _abi.Mat(fake, n, p, p, _abi.F32, _abi.ROW_MAJOR)
    B = _abi.Blocks(K, n, 64, fake)
    st = _abi.Stats(*([fake] * 7))
    st_nof = _abi.Stats(*([fake] * 6 + [None]))
    by = ctypes.byref
    vp = ctypes.c_void_p

    def bs(ckind, c, stats=st, ck=fake, Bk=B):
        return lib.bmm_blocksizes(by(M), by(N), by(Bk), by(stats), ckind, c, None, None, 0, vp(ck) if ck else None,
                                  vp(fake), None, None, 0, None)

    assert bs(9, 1024) == _abi.ERR_ARG                                  # unknown kind
    assert bs(_abi.CK_OPT, 1024, ck=None) == _abi.ERR_ARG               # no output
    assert bs(_abi.CK_OPT, 1024, stats=st_nof) == _abi.ERR_ARG          # eq. 3.9 needs f
    assert bs(_abi.CK_TILDE, 1024) == _abi.ERR_ARG                      # Alg. 3 needs its pilot
    assert bs(_abi.CK_OPT, K - 1) == _abi.ERR_INFEASIBLE                # fewer draws than blocks
    assert bs(_abi.CK_OPT, n + 1) == _abi.ERR_INFEASIBLE                # more draws than vectors
    assert bs(_abi.CK_OPT, 1024, Bk=_abi.Blocks(0, n, 64, fake)) == _abi.ERR_SHAPE
    assert bs(_abi.CK_OPT, 1024) == _abi.ERR_WORKSPACE                  # well formed: stops at the workspace

    def smp(unit, c, p_=fake, ck=fake, idx=fake):
        return lib.bmm_sample(vp(p_) if p_ else None, unit, by(B), vp(ck) if ck else None, c, 1, 0,
                              vp(idx) if idx else None, vp(fake), None, 0, None)

    assert smp(_abi.UNIT_COLUMN, 100, p_=None) == _abi.ERR_ARG
    assert smp(_abi.UNIT_COLUMN, 100, idx=None) == _abi.ERR_ARG
    assert smp(_abi.UNIT_COLUMN, -1) == _abi.ERR_ARG
    assert smp(7, 100) == _abi.ERR_ARG                                  # unknown unit
    assert smp(_abi.UNIT_COLUMN, 100, ck=None) == _abi.ERR_ARG          # column draws need c_k
    assert smp(_abi.UNIT_COLUMN, 1 << 31) == _abi.ERR_UNSUPPORTED       # beyond int32 indices
    assert smp(_abi.UNIT_BLOCK, 100, ck=None) == _abi.ERR_WORKSPACE     # block draws take no c_k

    def bwd(G, gemm=_abi.GEMM_BF16, unit=_abi.UNIT_COLUMN, dM=None, dN=None, c=100):
        return lib.bmm_backward(by(G), by(M), by(N), by(B), unit, vp(fake), vp(fake), c, 1, 0, gemm,
                                by(dM) if dM else None, by(dN) if dN else None, 0, None, 0, None)

    G = _abi.Mat(fake, m, p, p, _abi.F32, _abi.ROW_MAJOR)
    assert bwd(G, unit=5) == _abi.ERR_ARG
    assert bwd(G, gemm=17) == _abi.ERR_ARG
    assert bwd(G, c=-1) == _abi.ERR_ARG
    assert bwd(G, gemm=_abi.GEMM_SPLIT_BF16) == _abi.ERR_UNSUPPORTED    # the adjoint runs BF16 or FP64
    assert bwd(_abi.Mat(fake, m, p - 1, p, _abi.F32, _abi.ROW_MAJOR)) == _abi.ERR_SHAPE
    assert bwd(_abi.Mat(fake, m, p, p, _abi.F64, _abi.ROW_MAJOR)) == _abi.ERR_DTYPE  # BF16 mode takes FP32 G
    assert bwd(G, dM=_abi.Mat(fake, m, n - 1, n, _abi.F32, _abi.ROW_MAJOR)) == _abi.ERR_SHAPE
    assert bwd(G, dN=_abi.Mat(fake, n, p, p, 9, _abi.ROW_MAJOR)) == _abi.ERR_DTYPE


def test_run_pipelined_refuses_on_the_host():
    """run_pipelined checks its arguments before it touches a device."""
    import paper_2105_04940_gb300 as P
    with pytest.raises(ValueError):
        P.run_pipelined([], 100, [1], [object()])
    with pytest.raises(ValueError):
        P.run_pipelined([object()], 100, [1], [object()])
    with pytest.raises(ValueError):
        P.run_pipelined([object(), object()], 100, [1], [])
    with pytest.raises(ValueError):
        P.run_pipelined([object(), object()], 100, [1], [object()], gemm_mode=P._abi.GEMM_F64)


def test_upload_cache_is_safe_across_host_threads(monkeypatch):
    """pipeline._upload (the per-content cache of block offsets, at most 64 entries) is shared by
    host threads that prepare problems at the same time: many threads uploading more distinct
    arrays than the cache holds get each array back intact and no thread fails on an entry that
    another thread evicted.  The cache's host logic runs here with CPU tensors (the package's
    refusal to run without a GPU is lifted for this function only)."""
    import threading

    import numpy as np
    import torch

    from paper_2105_04940_gb300 import pipeline
    monkeypatch.setattr(pipeline, "_torch", lambda: torch)
    monkeypatch.setattr(pipeline, "_UPLOADS", {})
    dev = torch.device("cpu")
    errors, bad = [], []
    start = threading.Barrier(8)

    def work(t):
        try:
            start.wait()
            for k in range(150):
                arr = np.arange(k, k + 5 + t, dtype=np.int64) * (t + 1)
                if not np.array_equal(pipeline._upload(arr, dev).numpy(), arr):
                    bad.append((t, k))
        except Exception as e:  # reported on the test's thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(8)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors and not bad, (errors[:3], bad[:3])
    assert len(pipeline._UPLOADS) <= 64


def test_binding_constants_match_the_header():
    """Every enumerator and #define of include/bmm.h has the same value in the ctypes binding (name
    without the BMM_ prefix; the report fields by position in REPORT_FIELDS), so the two cannot
    drift apart."""
    from paper_2105_04940_gb300 import _abi
    text = open(os.path.join(ROOT, "include", "bmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = dict(re.findall(r"\b(BMM_[A-Z0-9_]+)\s*=\s*(0x[0-9a-fA-F]+|\d+)", text))
    found.update(re.findall(r"#define\s+(BMM_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)\b", text))
    assert len(found) > 50
    fields = [f.upper() for f in _abi.REPORT_FIELDS]
    for name, val in sorted(found.items()):
        v = int(val, 0)
        short = name[len("BMM_"):]
        if short.startswith("REPORT_") and short != "REPORT_LEN":
            assert fields[v] == short[len("REPORT_"):], name
        else:
            assert getattr(_abi, short) == v, name


def _c_params(text):
    """(return type, name, [parameter types]) of every function prototype in a comment-free header."""
    out = []
    for ret, name, params in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(bmm_\w+)\s*\(([^;{}]*?)\)\s*;", text):
        ps = [] if params.strip() in ("", "void") else [p.strip() for p in params.split(",")]
        # drop the parameter name: the last identifier unless the declarator is only a type
        types = [re.sub(r"\s*\b\w+$", "", p) if re.search(r"[\w\*]\s+\w+$", p) else p for p in ps]
        norm = lambda t: " ".join(t.replace("*", " * ").split())
        out.append((norm(ret), name, [norm(t) for t in types]))
    return out


def test_binding_signatures_match_the_header(lib):
    """Each prototype of include/bmm.h against the argtypes and restype the ctypes binding declares:
    same arity; integers and floats of the same width and signedness; descriptor structs by pointer;
    arrays of pointers as pointers to c_void_p; other pointers as c_void_p or a pointer to the same
    scalar type.  A binding that passed an int64 where the header takes int32 would fail here."""
    import ctypes

    from paper_2105_04940_gb300 import _abi
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bmm.h")).read(), flags=re.S)
    protos = _c_params(text)
    assert sorted(name for _, name, _ in protos) == sorted(_abi.EXPORTED)
    scalars = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
               "size_t": ctypes.c_size_t, "double": ctypes.c_double, "float": ctypes.c_float,
               "bmm_status": ctypes.c_int32}
    structs = {"bmm_mat": _abi.Mat, "bmm_blocks": _abi.Blocks, "bmm_stats": _abi.Stats}

    def ok(ctype, t):
        base = t.replace("const", "").replace("*", "").split()
        stars = t.count("*")
        if t == "bmm_stream_t" or (stars == 1 and base == ["void"]):
            return ctype is ctypes.c_void_p
        if stars == 0:
            return ctype is scalars[base[0]]
        if stars >= 2:
            return ctype is ctypes.POINTER(ctypes.c_void_p)
        if base[0] in structs:
            return ctype is ctypes.POINTER(structs[base[0]])
        return ctype is ctypes.c_void_p or ctype is ctypes.POINTER(scalars[base[0]])

    for ret, name, types in protos:
        fn = getattr(lib, name)
        assert len(fn.argtypes) == len(types), name
        for i, (ct, t) in enumerate(zip(fn.argtypes, types)):
            assert ok(ct, t), (name, i, t, ct)
        want = {"bmm_status": ctypes.c_int32, "size_t": ctypes.c_size_t, "const char *": ctypes.c_char_p,
                "uint64_t": ctypes.c_uint64, "void": None}[ret]
        assert fn.restype is want, (name, ret, fn.restype)


def test_descriptor_structs_match_the_header(tmp_path):
    """bmm_mat, bmm_blocks and bmm_stats as a C compiler lays them out from include/bmm.h (sizes and
    every field's offset, from a small program built with the host compiler) against the binding's
    ctypes structures."""
    import ctypes
    import shutil
    import subprocess

    from paper_2105_04940_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    layouts = {"bmm_mat": _abi.Mat, "bmm_blocks": _abi.Blocks, "bmm_stats": _abi.Stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "bmm.h"', "int main(void) {"]
    for cname, cls in layouts.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, cls in layouts.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_header_stands_alone_in_c_and_cpp(tmp_path):
    """include/bmm.h compiles on its own, as C and as C++ (C linkage: the exported names are the
    plain function names), with warnings treated as errors."""
    import shutil
    import subprocess
    for lang, comp in (("c", shutil.which("gcc")), ("c++", shutil.which("g++"))):
        if comp is None:
            pytest.skip("no host compiler")
        src = tmp_path / ("h." + ("c" if lang == "c" else "cpp"))
        src.write_text('#include "bmm.h"\nint main(void) { return (int)sizeof(bmm_mat) == 0; }\n')
        subprocess.run([comp, "-x", lang, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-fsyntax-only", str(src)], check=True)

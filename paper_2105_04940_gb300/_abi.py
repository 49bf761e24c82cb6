"""ctypes binding of include/bmm.h -- argument marshalling only.

Every function below calls the C entry point of the same name in libbmm.so and raises
BmmError on a non-OK status.  Tensors are torch CUDA tensors; their device pointers,
shapes and strides are passed through, nothing is computed here.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbmm.so")

# enums of include/bmm.h
OK, ERR_ARG, ERR_SHAPE, ERR_DTYPE, ERR_INFEASIBLE, ERR_NONFINITE, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(10)
F64, F32, BF16 = 0, 1, 2
ROW_MAJOR, COL_MAJOR = 0, 1
P_COL_OPT, P_COL_UNIFORM, P_BLK_PRODNORM, P_BLK_NORMPROD = 0, 1, 2, 3
CK_OPT, CK_HAT, CK_TILDE, CK_EQUAL = 0, 1, 2, 3
F_NONE, F_EXACT, F_TC = 0, 1, 2
REUSE_STATS = 0x100
UNIT_COLUMN, UNIT_BLOCK = 0, 1
GEMM_F64, GEMM_BF16, GEMM_SPLIT_BF16, GEMM_E4M3 = 0, 1, 2, 3
PURPOSE_MAIN, PURPOSE_PILOT = 0, 1
APPLY_GATHER_B, APPLY_GATHER_A, APPLY_GEMM, APPLY_REDUCE = 0, 1, 2, 3
TILE_PAIR = 512  # GEMM tile choice: a CTA pair per 256 x 256 tile
TILE_PAIR_WIDE = 1024  # a CTA pair per 256 x 512 tile

EXPORTED = (
    "bmm_workspace_size", "bmm_probs", "bmm_blocksizes", "bmm_sample", "bmm_apply", "bmm_backward",
    "bmm_read_device_status", "bmm_clear_device_status", "bmm_status_string", "bmm_launch_count",
    "bmm_probs_static", "bmm_apply_batched", "bmm_probs_batched",
    "bmm_autotune_workspace_size", "bmm_autotune_gemm", "bmm_autotune_get", "bmm_autotune_set", "bmm_autotune_clear",
    "bmm_error_report", "bmm_entry_variance", "bmm_entry_estimate", "bmm_blocksizes_batched", "bmm_apply_part",
    "bmm_f_tc_supported", "bmm_wait_selftest", "bmm_sample_batched",
)

# fields of the bmm_error_report output, in order (BMM_REPORT_* of include/bmm.h)
REPORT_FIELDS = (
    "expected_sq_error", "eq310", "theta1", "theta2", "beta", "m_fro2", "n_fro2", "phi", "eq311", "eta312", "eq312",
    "phihat", "eq43", "eta44", "eq44", "theta1hat", "theta2hat", "phitilde", "eq48", "eta49", "eq49",
)
REPORT_LEN = len(REPORT_FIELDS)


class BmmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


class Mat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32)]


class Blocks(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("n", ctypes.c_int64), ("max_nk", ctypes.c_int64),
                ("offsets", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("x", "y", "a", "s", "mf", "nf", "f")]


_lib = None


def load(path: str = LIB_PATH):
    """Load libbmm.so and declare the signatures; fails loudly if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2105_04940_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    lib.bmm_workspace_size.argtypes = [P(Mat), P(Mat), P(Blocks), i32, i64, i32]
    lib.bmm_workspace_size.restype = sz
    lib.bmm_probs.argtypes = [P(Mat), P(Mat), P(Blocks), i32, i32, vp, P(Stats), vp, sz, vp]
    lib.bmm_blocksizes.argtypes = [P(Mat), P(Mat), P(Blocks), P(Stats), i32, i64, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    lib.bmm_sample.argtypes = [vp, i32, P(Blocks), vp, i64, u64, u64, vp, vp, vp, sz, vp]
    lib.bmm_apply.argtypes = [P(Mat), P(Mat), P(Blocks), i32, vp, vp, i64, i32, P(Mat), i32, vp, sz, vp]
    lib.bmm_apply_part.argtypes = [P(Mat), P(Mat), P(Blocks), vp, vp, i64, P(Mat), i32, i32, i64, i64, vp, sz, vp]
    lib.bmm_apply_part.restype = i32
    lib.bmm_f_tc_supported.argtypes = [P(Mat), P(Mat), P(Blocks), P(i32)]
    lib.bmm_f_tc_supported.restype = i32
    lib.bmm_wait_selftest.argtypes = [vp, sz, vp]
    lib.bmm_wait_selftest.restype = i32
    lib.bmm_sample_batched.argtypes = [i64, P(vp), i32, P(Blocks), P(vp), P(i64), P(u64), P(u64), P(vp), P(vp), P(vp),
                                       P(sz), vp]
    lib.bmm_sample_batched.restype = i32
    lib.bmm_backward.argtypes = [P(Mat), P(Mat), P(Mat), P(Blocks), i32, vp, vp, i64, u64, u64, i32,
                                 P(Mat), P(Mat), i32, vp, sz, vp]
    lib.bmm_read_device_status.argtypes = [vp, vp]
    lib.bmm_clear_device_status.argtypes = [vp, vp]
    lib.bmm_status_string.argtypes = [i32]
    lib.bmm_status_string.restype = ctypes.c_char_p
    lib.bmm_probs_static.argtypes = [P(Mat), P(Mat), P(Blocks), i32, vp, P(Stats), vp, vp]
    lib.bmm_probs_static.restype = i32
    lib.bmm_apply_batched.argtypes = [i64, P(Mat), P(Mat), P(Blocks), i32, P(vp), P(vp), P(i64), i32, P(Mat), i32,
                                      P(vp), P(sz), vp]
    lib.bmm_apply_batched.restype = i32
    lib.bmm_probs_batched.argtypes = [i64, P(Mat), P(Mat), P(Blocks), i32, i32, P(vp), P(Stats), P(vp), P(sz), vp]
    lib.bmm_probs_batched.restype = i32
    lib.bmm_launch_count.argtypes = []
    lib.bmm_launch_count.restype = ctypes.c_uint64
    lib.bmm_autotune_workspace_size.argtypes = [i64, i64, i64, i32]
    lib.bmm_autotune_workspace_size.restype = sz
    lib.bmm_autotune_gemm.argtypes = [i64, i64, i64, i32, vp, sz, vp, P(i32), P(i32), P(ctypes.c_float)]
    lib.bmm_autotune_gemm.restype = i32
    lib.bmm_autotune_get.argtypes = [i64, i64, i64, i32, P(i32), P(i32)]
    lib.bmm_autotune_get.restype = i32
    lib.bmm_autotune_set.argtypes = [i64, i64, i64, i32, i32, i32]
    lib.bmm_autotune_set.restype = i32
    lib.bmm_autotune_clear.argtypes = []
    lib.bmm_autotune_clear.restype = None
    lib.bmm_blocksizes_batched.argtypes = [i64, P(Blocks), P(Stats), i32, P(i64), P(vp), P(vp), P(vp), P(sz), vp]
    lib.bmm_blocksizes_batched.restype = i32
    lib.bmm_error_report.argtypes = [P(Blocks), P(Stats), vp, vp, i64, vp, ctypes.c_double, vp, vp]
    lib.bmm_error_report.restype = i32
    lib.bmm_entry_variance.argtypes = [P(Mat), P(Mat), P(Blocks), i32, vp, vp, i64, vp, i64, vp, vp]
    lib.bmm_entry_variance.restype = i32
    lib.bmm_entry_estimate.argtypes = [P(Mat), P(Mat), P(Blocks), i32, vp, vp, vp, i64, vp, i64, vp, vp, vp, sz, vp]
    lib.bmm_entry_estimate.restype = i32
    for name in ("bmm_probs", "bmm_blocksizes", "bmm_sample", "bmm_apply", "bmm_backward",
                 "bmm_read_device_status", "bmm_clear_device_status"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().bmm_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != OK:
        raise BmmError(code, where)


# ---------------------------------------------------------------- marshalling helpers
_DT = None


def _dtypes():
    global _DT
    if _DT is None:
        import torch
        _DT = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}
    return _DT


def mat(t) -> Mat:
    """bmm_mat of a 2-D tensor: row-major if its last stride is 1, column-major if its first is."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    dt = _dtypes().get(t.dtype)
    if dt is None:
        raise TypeError(f"unsupported dtype {t.dtype}")
    r, c = t.shape
    s0, s1 = t.stride()
    if s1 == 1 or c <= 1:
        return Mat(t.data_ptr(), r, c, max(s0, c, 1), dt, ROW_MAJOR)
    if s0 == 1 or r <= 1:
        return Mat(t.data_ptr(), r, c, max(s1, r, 1), dt, COL_MAJOR)
    raise ValueError("tensor must have a unit stride in one dimension")


def blocks(offsets_dev, n: int, max_nk: int) -> Blocks:
    """bmm_blocks of a device int64 offsets tensor.  The struct keeps a reference to the tensor:
    it holds only the raw device address, and a temporary tensor freed after this call would
    hand that memory to the next allocation."""
    b = Blocks(len(offsets_dev) - 1, n, max_nk, offsets_dev.data_ptr())
    b._offsets_ref = offsets_dev
    return b


def stats(d: dict) -> Stats:
    return Stats(*[(d[k].data_ptr() if d.get(k) is not None else None) for k in ("x", "y", "a", "s", "mf", "nf", "f")])


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- the entry points
def bmm_workspace_size(M, N, B: Blocks, unit: int, max_draws: int, gemm_mode: int) -> int:
    return int(load().bmm_workspace_size(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B),
                                         unit, max_draws, gemm_mode))


def bmm_probs(M, N, B: Blocks, pkind: int, fmode: int, p_out, st: dict, ws, stream=None):
    Mm = ctypes.byref(mat(M)) if M is not None else None
    Nm = ctypes.byref(mat(N)) if N is not None else None
    sp = ctypes.byref(stats(st)) if st is not None else None
    _check(load().bmm_probs(Mm, Nm, ctypes.byref(B), pkind, fmode, _ptr(p_out), sp, ws.data_ptr(), ws.numel(),
                            _stream(stream)), "bmm_probs")


def bmm_probs_batched(Ms, Ns, Bs, pkind: int, fmode: int, p_outs, sts, wss, stream=None):
    """bmm_probs over many independent products (lists of equal length; p_outs entries may be None)."""
    n = len(Ms)
    MatA, BlkA, VpA = Mat * n, Blocks * n, ctypes.c_void_p * n
    pp = VpA(*[_ptr(p) for p in p_outs]) if p_outs is not None else None
    _check(load().bmm_probs_batched(
        n, MatA(*[mat(m) for m in Ms]), MatA(*[mat(x) for x in Ns]), BlkA(*Bs), pkind, fmode, pp,
        (Stats * n)(*[stats(st) for st in sts]), VpA(*[w.data_ptr() for w in wss]),
        (ctypes.c_size_t * n)(*[w.numel() for w in wss]), _stream(stream)), "bmm_probs_batched")


def bmm_blocksizes(M, N, B: Blocks, st: dict, ckind: int, c: int, pilot_idx, pilot_scale, pilot_per_block: int,
                   ck_out, g_out, fhat_out, ws, stream=None):
    Mm = ctypes.byref(mat(M)) if M is not None else None
    Nm = ctypes.byref(mat(N)) if N is not None else None
    sp = ctypes.byref(stats(st)) if st is not None else None
    _check(load().bmm_blocksizes(Mm, Nm, ctypes.byref(B), sp, ckind, c, _ptr(pilot_idx), _ptr(pilot_scale),
                                 pilot_per_block, _ptr(ck_out), _ptr(g_out), _ptr(fhat_out), ws.data_ptr(),
                                 ws.numel(), _stream(stream)), "bmm_blocksizes")


def bmm_sample(p, unit: int, B: Blocks, ck, c: int, seed: int, stream_id: int, idx_out, scale_out, ws, stream=None):
    _check(load().bmm_sample(_ptr(p), unit, ctypes.byref(B), _ptr(ck), c, seed & 0xFFFFFFFFFFFFFFFF,
                             stream_id & 0xFFFFFFFFFFFFFFFF, _ptr(idx_out), _ptr(scale_out), ws.data_ptr(),
                             ws.numel(), _stream(stream)), "bmm_sample")


def bmm_sample_batched(ps, unit: int, Bs, cks, cs, seeds, stream_ids, idx_outs, scale_outs, wss, stream=None):
    """bmm_sample over many independent products (lists of equal length; cks None for the block unit)."""
    n = len(ps)
    VpA, I64A, U64A = ctypes.c_void_p * n, ctypes.c_int64 * n, ctypes.c_uint64 * n
    ckp = VpA(*[_ptr(c) for c in cks]) if cks is not None else None
    _check(load().bmm_sample_batched(
        n, VpA(*[_ptr(x) for x in ps]), unit, (Blocks * n)(*Bs), ckp, I64A(*[int(c) for c in cs]),
        U64A(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds]), U64A(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in stream_ids]),
        VpA(*[_ptr(x) for x in idx_outs]), VpA(*[_ptr(x) for x in scale_outs]), VpA(*[w.data_ptr() for w in wss]),
        (ctypes.c_size_t * n)(*[w.numel() for w in wss]), _stream(stream)), "bmm_sample_batched")


def bmm_apply(M, N, B: Blocks, unit: int, idx, scale, count: int, gemm_mode: int, out, accumulate: bool, ws,
              stream=None):
    _check(load().bmm_apply(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), unit, _ptr(idx),
                            _ptr(scale), count, gemm_mode, ctypes.byref(mat(out)), int(bool(accumulate)),
                            ws.data_ptr(), ws.numel(), _stream(stream)), "bmm_apply")


def bmm_apply_part(M, N, B: Blocks, idx, scale, count: int, out, accumulate: bool, part: int, row0: int, row1: int,
                   ws, stream=None):
    """One part (APPLY_REDUCE first, then APPLY_GATHER_B / APPLY_GATHER_A, then APPLY_GEMM) of a
    column-sampled BF16 bmm_apply."""
    _check(load().bmm_apply_part(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), _ptr(idx), _ptr(scale),
                                 count, ctypes.byref(mat(out)), int(bool(accumulate)), part, row0, row1, ws.data_ptr(),
                                 ws.numel(), _stream(stream)), "bmm_apply_part")


def bmm_backward(G, M, N, B: Blocks, unit: int, p, ck, c: int, seed: int, stream_id: int, gemm_mode: int, dM, dN,
                 accumulate: bool, ws, stream=None):
    dMm = ctypes.byref(mat(dM)) if dM is not None else None
    dNm = ctypes.byref(mat(dN)) if dN is not None else None
    _check(load().bmm_backward(ctypes.byref(mat(G)), ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B),
                               unit, _ptr(p), _ptr(ck), c, seed & 0xFFFFFFFFFFFFFFFF, stream_id & 0xFFFFFFFFFFFFFFFF,
                               gemm_mode, dMm, dNm, int(bool(accumulate)), ws.data_ptr(), ws.numel(),
                               _stream(stream)), "bmm_backward")


def bmm_blocksizes_batched(Bs, sts, ckind: int, cs, ck_outs, g_outs, wss, stream=None):
    """bmm_blocksizes for many products in one launch (lists of equal length; sts may be None for
    CK_EQUAL, g_outs None or a list with None entries)."""
    n = len(Bs)
    BlkA, VpA = Blocks * n, ctypes.c_void_p * n
    st = (Stats * n)(*[stats(d) for d in sts]) if sts is not None else None
    gp = VpA(*[_ptr(g) for g in g_outs]) if g_outs is not None else None
    _check(load().bmm_blocksizes_batched(n, BlkA(*Bs), st, ckind, (ctypes.c_int64 * n)(*[int(c) for c in cs]),
                                         VpA(*[_ptr(c) for c in ck_outs]), gp, VpA(*[w.data_ptr() for w in wss]),
                                         (ctypes.c_size_t * n)(*[w.numel() for w in wss]), _stream(stream)),
           "bmm_blocksizes_batched")


def bmm_error_report(B: Blocks, st: dict, p, ck, c: int, fhat, delta: float, report_out, stream=None):
    """report_out: device FP64 [REPORT_LEN] (fields REPORT_FIELDS)."""
    _check(load().bmm_error_report(ctypes.byref(B), ctypes.byref(stats(st)), _ptr(p), _ptr(ck), c, _ptr(fhat),
                                   float(delta), _ptr(report_out), _stream(stream)), "bmm_error_report")


def bmm_entry_variance(M, N, B: Blocks, unit: int, p, ck, c: int, entries, sigma2_out, stream=None):
    """entries: device int64 [count, 2] of (h, f); sigma2_out: device FP64 [count]."""
    count = 0 if entries is None else int(entries.shape[0])
    _check(load().bmm_entry_variance(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), unit, _ptr(p),
                                     _ptr(ck), c, _ptr(entries), count, _ptr(sigma2_out), _stream(stream)),
           "bmm_entry_variance")


def bmm_entry_estimate(M, N, B: Blocks, unit: int, ck, idx, scale, draws: int, entries, cd_out, s2_out, ws,
                       stream=None):
    """entries: device int64 [count, 2]; cd_out, s2_out: device FP64 [count]."""
    count = 0 if entries is None else int(entries.shape[0])
    _check(load().bmm_entry_estimate(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), unit, _ptr(ck),
                                     _ptr(idx), _ptr(scale), draws, _ptr(entries), count, _ptr(cd_out), _ptr(s2_out),
                                     ws.data_ptr(), ws.numel(), _stream(stream)), "bmm_entry_estimate")


def bmm_f_tc_supported(M, N, B: Blocks) -> bool:
    """Whether bmm_probs with F_TC computes f_k of this problem on the tensor cores (else exactly)."""
    r = ctypes.c_int32(-1)
    _check(load().bmm_f_tc_supported(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), ctypes.byref(r)),
           "bmm_f_tc_supported")
    return r.value == 1


def bmm_wait_selftest(ws, stream=None):
    """Launch the bounded-wait self-test (gives up after the library's wait bound, about 2 s)."""
    _check(load().bmm_wait_selftest(ws.data_ptr(), ws.numel(), _stream(stream)), "bmm_wait_selftest")


def bmm_read_device_status(ws, stream=None) -> int:
    return int(load().bmm_read_device_status(ws.data_ptr(), _stream(stream)))


def bmm_clear_device_status(ws, stream=None):
    _check(load().bmm_clear_device_status(ws.data_ptr(), _stream(stream)), "bmm_clear_device_status")


def bmm_launch_count() -> int:
    """Kernels launched by libbmm.so since it was loaded (diagnostic)."""
    return int(load().bmm_launch_count())


def bmm_autotune_workspace_size(m: int, p: int, L: int, gemm_mode: int) -> int:
    """Workspace bytes bmm_autotune_gemm needs for an m x p product of L outer products."""
    return int(load().bmm_autotune_workspace_size(m, p, L, gemm_mode))


def bmm_autotune_gemm(m: int, p: int, L: int, gemm_mode: int, ws, stream=None) -> dict:
    """Time the GEMM tile candidates for this shape and record the fastest (see include/bmm.h)."""
    bn, ra, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().bmm_autotune_gemm(m, p, L, gemm_mode, ws.data_ptr(), ws.numel(), _stream(stream), ctypes.byref(bn),
                                    ctypes.byref(ra), ctypes.byref(ms)), "bmm_autotune_gemm")
    return {"bn": bn.value, "raster": ra.value, "ms": ms.value}


def bmm_autotune_get(m: int, p: int, L: int, gemm_mode: int) -> dict:
    """The tile choice the next GEMM of this shape will use."""
    bn, ra = ctypes.c_int32(), ctypes.c_int32()
    _check(load().bmm_autotune_get(m, p, L, gemm_mode, ctypes.byref(bn), ctypes.byref(ra)), "bmm_autotune_get")
    return {"bn": bn.value, "raster": ra.value}


def bmm_autotune_set(m: int, p: int, L: int, gemm_mode: int, bn: int, raster: int):
    _check(load().bmm_autotune_set(m, p, L, gemm_mode, bn, raster), "bmm_autotune_set")


def bmm_autotune_clear():
    load().bmm_autotune_clear()


def bmm_probs_static(M, N, B: Blocks, pkind: int, p_out, st: dict, status_out, stream=None):
    """bmm_probs with the library's fixed device scratch instead of a workspace (see include/bmm.h)."""
    _check(load().bmm_probs_static(ctypes.byref(mat(M)), ctypes.byref(mat(N)), ctypes.byref(B), pkind, _ptr(p_out),
                                   ctypes.byref(stats(st)), _ptr(status_out), _stream(stream)), "bmm_probs_static")


def bmm_apply_batched(Ms, Ns, Bs, unit: int, idxs, scales, draws, gemm_mode: int, outs, accumulate: bool, wss,
                      stream=None):
    """bmm_apply over many independent products (lists of equal length; see include/bmm.h)."""
    n = len(Ms)
    MatA, BlkA, VpA = Mat * n, Blocks * n, ctypes.c_void_p * n
    _check(load().bmm_apply_batched(
        n, MatA(*[mat(m) for m in Ms]), MatA(*[mat(x) for x in Ns]), BlkA(*Bs), unit,
        VpA(*[i.data_ptr() for i in idxs]), VpA(*[s.data_ptr() for s in scales]),
        (ctypes.c_int64 * n)(*[int(d) for d in draws]), gemm_mode, MatA(*[mat(o) for o in outs]),
        int(bool(accumulate)), VpA(*[w.data_ptr() for w in wss]), (ctypes.c_size_t * n)(*[w.numel() for w in wss]),
        _stream(stream)), "bmm_apply_batched")

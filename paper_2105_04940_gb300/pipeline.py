"""The sampled product as a sequence of C-ABI calls, and its torch.autograd.Function.

Method presets (Table 2 of the paper, plus the block-sampling baselines of Sec. 1):

  OPL     p eq. 3.8, c_k eq. 3.9 (needs ||M^k N_k||_F)        Alg. 2
  ONC     p eq. 3.8, c_k eq. 4.2                               Alg. 2
  ONU     p eq. 3.8, c_k eq. 4.7, pilot p0 = 1/n_k             Alg. 3
  ONMCNR  p eq. 3.8, c_k eq. 4.7, pilot p0 = eq. 3.8           Alg. 3
  UU      p = 1/n_k, c_k = c/K                                 Alg. 2
  SSM     c whole blocks, p_k eq. 1.4                          block sampling
  WU      c whole blocks, p_k eq. 1.2                          block sampling

Only memory allocation and argument passing happen here; every arithmetic step runs in
the CUDA kernels behind include/bmm.h.  For the Alg. 2/3 methods ``c`` counts outer
products (the paper's c); for SSM/WU it counts blocks.
"""
from __future__ import annotations

import threading
from dataclasses import dataclass, field

import numpy as np

from . import _abi as A

COLUMN_METHODS = ("OPL", "ONC", "ONU", "ONMCNR", "UU")
BLOCK_METHODS = ("SSM", "WU")
METHODS = COLUMN_METHODS + BLOCK_METHODS
MODES = {"f64": A.GEMM_F64, "bf16": A.GEMM_BF16, "split_bf16": A.GEMM_SPLIT_BF16, "e4m3": A.GEMM_E4M3}


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the sampled product runs on the GPU only: no CUDA device is available")
    return torch


def stream_id(replicate: int, purpose: int) -> int:
    return (int(replicate) << 8) | int(purpose)


def equal_budget(c_blocks: int, n: int, K: int) -> int:
    """Outer products matching c whole blocks: L = round(c n / K)."""
    return int(np.floor(c_blocks * n / K + 0.5))


@dataclass
class Problem:
    """Device-resident M, N, block offsets, statistics buffers and one workspace."""
    M: object
    N: object
    offsets: np.ndarray
    offsets_dev: object
    B: A.Blocks
    ws: object
    st: dict = field(default_factory=dict)
    pilot_counts: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return len(self.offsets) - 1

    @property
    def n(self) -> int:
        return int(self.offsets[-1])


_UPLOADS: dict = {}
_UPLOADS_LOCK = threading.Lock()


def _upload(arr: np.ndarray, dev):
    """Device copy of a small host int64 array, without making the host wait for the stream (a
    pageable copy would): pinned staging and a non-blocking copy, cached per content and device so
    that repeated products with the same blocks (every layer, every step) upload once.  Once the copy
    has landed no stream waits for it again, so calls captured in a CUDA graph after one eager call
    depend on no work outside the capture."""
    torch = _torch()
    key = (str(dev), arr.dtype.str, arr.tobytes())
    with _UPLOADS_LOCK:  # host threads may prepare problems at the same time
        hit = _UPLOADS.get(key)
        if hit is None:
            if len(_UPLOADS) >= 64:
                _UPLOADS.pop(next(iter(_UPLOADS)))
            host_t = torch.from_numpy(np.ascontiguousarray(arr))
            ev = None
            if dev.type == "cuda":
                t = host_t.pin_memory().to(dev, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record()
            else:
                t = host_t.to(dev)
            hit = _UPLOADS[key] = (t, ev)
        t, ev = hit
        if ev is not None:
            if ev.query():  # the copy has landed: no stream needs to wait for it again
                _UPLOADS[key] = (t, None)
            else:  # issued on some stream and still in flight
                torch.cuda.current_stream(dev).wait_event(ev)
    return t


def prepare(M, N, offsets, max_draws: int, unit: int = A.UNIT_COLUMN, gemm_mode: int | None = None,
            ws=None) -> Problem:
    """Upload the offsets, allocate statistics and a workspace large enough for ``gemm_mode``
    (all modes when None) and for draws of ``unit`` up to ``max_draws``."""
    torch = _torch()
    modes = (A.GEMM_F64, A.GEMM_SPLIT_BF16, A.GEMM_E4M3) if gemm_mode is None else (gemm_mode,)
    off = np.asarray(offsets, dtype=np.int64)
    n = int(off[-1])
    max_nk = int(np.diff(off).max())
    dev = M.device
    off_dev = _upload(off, dev)
    B = A.blocks(off_dev, n, max_nk)
    if ws is None:
        need = max(A.bmm_workspace_size(M, N, B, unit, max_draws, md) for md in modes)
        if need == 0:
            raise ValueError("invalid problem description")
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    if ws.data_ptr() % 256:
        raise ValueError("workspace must be 256-byte aligned")
    K = len(off) - 1
    f64 = dict(dtype=torch.float64, device=dev)
    st = {"x": torch.empty(n, **f64), "y": torch.empty(n, **f64), "a": torch.empty(K, **f64),
          "s": torch.empty(K, **f64), "mf": torch.empty(K, **f64), "nf": torch.empty(K, **f64),
          "f": torch.empty(K, **f64)}
    A.bmm_clear_device_status(ws)
    return Problem(M, N, off, off_dev, B, ws, st)


_SIDE = threading.local()


def _side_stream(dev):
    """A high-priority stream per device and host thread for the GEMM halves of the overlapped apply
    and for the design and gathers of run_pipelined (created once, outside any graph capture that
    uses it).  Per thread, so that callers on different threads neither wait on each other's work
    nor enqueue onto a stream that another thread is capturing."""
    torch = _torch()
    streams = _SIDE.__dict__.setdefault("streams", {})
    s = streams.get(str(dev))
    if s is None:
        s = streams[str(dev)] = torch.cuda.Stream(device=dev, priority=-1)
    return s


def overlapped_apply_wanted(M, N, count: int, gemm_mode: int, unit: int) -> bool:
    """Large column-sampled BF16 products (>= 4096 draws, m >= 256, m p >= 2^24) gain from overlapping
    the gather of M's columns (memory-bound) with the GEMM (tensor-bound)."""
    m, p = int(M.shape[0]), int(N.shape[1])
    return gemm_mode == A.GEMM_BF16 and unit == A.UNIT_COLUMN and count >= 4096 and m >= 256 and m * p >= 1 << 24


def apply_columns(prob: Problem, idx, scale, count: int, gemm_mode: int, out, accumulate: bool = False):
    """CD of Alg. 2's draws (bmm_apply).  For large BF16 products the output rows are split in two:
    the draws are reduced to distinct indices, N's rows and the first half's columns of M are
    gathered on the current stream, the first half's GEMM runs on a high-priority side stream while
    the second half's columns are gathered, then the second half's GEMM -- all through
    bmm_apply_part, ordered by events (a fork and a join of the current stream, so the sequence can be
    captured in a graph).  The result is bit-identical to one bmm_apply: every output element is the
    same full-depth dot product."""
    torch = _torch()
    M, N, B, ws = prob.M, prob.N, prob.B, prob.ws
    if not overlapped_apply_wanted(M, N, count, gemm_mode, A.UNIT_COLUMN):
        A.bmm_apply(M, N, B, A.UNIT_COLUMN, idx, scale, count, gemm_mode, out, accumulate, ws)
        return out
    main = torch.cuda.current_stream(M.device)
    side = _side_stream(M.device)
    m = int(M.shape[0])
    half = min(m, ((m + 1) // 2 + 127) // 128 * 128)
    side.wait_stream(main)
    A.bmm_apply_part(M, N, B, idx, scale, count, out, accumulate, A.APPLY_REDUCE, 0, 0, ws, main)
    A.bmm_apply_part(M, N, B, idx, scale, count, out, accumulate, A.APPLY_GATHER_B, 0, 0, ws, main)
    done = []
    for lo, hi in ((0, half), (half, m)):
        A.bmm_apply_part(M, N, B, idx, scale, count, out, accumulate, A.APPLY_GATHER_A, lo, hi, ws, main)
        ev = torch.cuda.Event()
        ev.record(main)
        done.append((lo, hi, ev))
    for lo, hi, ev in done:
        side.wait_event(ev)
        A.bmm_apply_part(M, N, B, idx, scale, count, out, accumulate, A.APPLY_GEMM, lo, hi, ws, side)
    main.wait_stream(side)
    return out


def run(prob: Problem, method: str, c: int, seed: int, replicate: int = 0, c0: int | None = None,
        gemm_mode: int = A.GEMM_BF16, out=None, compute_product: bool = True, events: list | None = None,
        fmode: int = A.F_TC, fused_stats: bool = True, p_ready=None, sizes_ready=None) -> dict:
    """One approximate product CD of prob.M @ prob.N by ``method`` (see module docstring).

    fmode: how OPL and WU compute ||M^k N_k||_F^2 -- A.F_TC (tensor-core Grams when the inputs
    allow it, else exact) or A.F_EXACT.  fused_stats (default): with F_TC, one pass computes the
    statistics and f together; otherwise the norm pass runs first and the Gram pass reuses its
    statistics (two reads of M and N, slower on one large product).

    events: if a list, (stage name, torch.cuda.Event) pairs are appended at the stage
    boundaries (recorded on the current stream; used for timing only).
    sizes_ready (OPL only): a (c_k, g_k) pair already computed for this product and this c.
    p_ready (OPL only): probabilities already computed, with prob.st holding the statistics and f
    (run_batched computes them for many products at once); the statistics calls are skipped.
    """
    torch = _torch()
    M, N, B, ws, st = prob.M, prob.N, prob.B, prob.ws, prob.st
    dev = M.device
    K, n = prob.K, prob.n
    sid = stream_id(replicate, A.PURPOSE_MAIN)
    res = {"method": method, "c": c, "seed": seed, "sid": sid}

    def mark(name):
        if events is not None:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            events.append((name, ev))

    mark("start")
    if out is None and compute_product:
        out = torch.empty(M.shape[0], N.shape[1], device=dev,
                          dtype=torch.float64 if gemm_mode == A.GEMM_F64 else torch.float32)
    if method in BLOCK_METHODS:
        pblk = torch.empty(K, dtype=torch.float64, device=dev)
        if method == "SSM":
            A.bmm_probs(M, N, B, A.P_BLK_NORMPROD, A.F_NONE, pblk, st, ws)
            mark("stats")
        elif fmode == A.F_TC and fused_stats:
            A.bmm_probs(M, N, B, A.P_BLK_PRODNORM, A.F_TC, pblk, st, ws)
            mark("stats_f")
        else:
            A.bmm_probs(M, N, B, A.P_BLK_NORMPROD, A.F_NONE, None, st, ws)
            mark("stats")
            A.bmm_probs(M, N, B, A.P_BLK_PRODNORM, fmode | A.REUSE_STATS, pblk, st, ws)
            mark("exact_f" if fmode == A.F_EXACT else "gram_f")
        idx = torch.empty(c, dtype=torch.int32, device=dev)
        scale = torch.empty(c, dtype=torch.float64, device=dev)
        A.bmm_sample(pblk, A.UNIT_BLOCK, B, None, c, seed, sid, idx, scale, ws)
        mark("sample")
        if compute_product:
            A.bmm_apply(M, N, B, A.UNIT_BLOCK, idx, scale, c, gemm_mode, out, False, ws)
            mark("apply")
        res.update(p=pblk, idx=idx, scale=scale, unit=A.UNIT_BLOCK, out=out, ck=None)
        return res
    if method not in COLUMN_METHODS:
        raise ValueError(f"unknown method {method}")
    p = torch.empty(n, dtype=torch.float64, device=dev)
    ck = torch.empty(K, dtype=torch.int64, device=dev)
    g = torch.empty(K, dtype=torch.float64, device=dev)
    if method == "UU":
        A.bmm_probs(None, None, B, A.P_COL_UNIFORM, A.F_NONE, p, None, ws)
        mark("stats")
        A.bmm_blocksizes(None, None, B, None, A.CK_EQUAL, c, None, None, 0, ck, g, None, ws)
        mark("blocksizes")
    elif method == "OPL":
        if p_ready is not None:
            p = p_ready
        elif fmode == A.F_TC and fused_stats:
            A.bmm_probs(M, N, B, A.P_COL_OPT, A.F_TC, p, st, ws)
            mark("stats_f")
        else:
            A.bmm_probs(M, N, B, A.P_COL_OPT, A.F_NONE, p, st, ws)
            mark("stats")
            A.bmm_probs(M, N, B, A.P_COL_OPT, fmode | A.REUSE_STATS, None, st, ws)
            mark("exact_f" if fmode == A.F_EXACT else "gram_f")
        if sizes_ready is not None:  # (c_k, g_k) already computed for this product (run_batched)
            ck, g = sizes_ready
        else:
            A.bmm_blocksizes(M, N, B, st, A.CK_OPT, c, None, None, 0, ck, g, None, ws)
        mark("blocksizes")
    elif method == "ONC":
        A.bmm_probs(M, N, B, A.P_COL_OPT, A.F_NONE, p, st, ws)
        mark("stats")
        A.bmm_blocksizes(M, N, B, st, A.CK_HAT, c, None, None, 0, ck, g, None, ws)
        mark("blocksizes")
    else:  # Alg. 3: pilot sample, then c~_k
        if c0 is None:
            raise ValueError("two-step methods need c0")
        A.bmm_probs(M, N, B, A.P_COL_OPT, A.F_NONE, p, st, ws)
        mark("stats")
        if method == "ONU":
            p0 = torch.empty(n, dtype=torch.float64, device=dev)
            A.bmm_probs(None, None, B, A.P_COL_UNIFORM, A.F_NONE, p0, None, ws)
        else:
            p0 = p
        per = max(1, c0 // K)
        ck0 = prob.pilot_counts.get(per)
        if ck0 is None:  # uploaded once per problem, outside any timed loop
            ck0 = _upload(np.full(K, per, dtype=np.int64), dev)
            prob.pilot_counts[per] = ck0
        pidx = torch.empty(K * per, dtype=torch.int32, device=dev)
        pscale = torch.empty(K * per, dtype=torch.float64, device=dev)
        A.bmm_sample(p0, A.UNIT_COLUMN, B, ck0, K * per, seed, stream_id(replicate, A.PURPOSE_PILOT), pidx, pscale, ws)
        fhat = torch.empty(K, dtype=torch.float64, device=dev)
        A.bmm_blocksizes(M, N, B, st, A.CK_TILDE, c, pidx, pscale, per, ck, g, fhat, ws)
        mark("pilot_blocksizes")
        res.update(p0=p0, pilot_idx=pidx, pilot_scale=pscale, fhat=fhat)
    idx = torch.empty(c, dtype=torch.int32, device=dev)
    scale = torch.empty(c, dtype=torch.float64, device=dev)
    A.bmm_sample(p, A.UNIT_COLUMN, B, ck, c, seed, sid, idx, scale, ws)
    mark("sample")
    if compute_product:
        apply_columns(prob, idx, scale, c, gemm_mode, out)
        mark("apply")
    res.update(p=p, ck=ck, g=g, idx=idx, scale=scale, unit=A.UNIT_COLUMN, out=out)
    return res


def run_pipelined(probs: list, c: int, seeds, outs: list, gemm_mode: int = A.GEMM_BF16, replicate: int = 0,
                  events: list | None = None) -> None:
    """Alg. 2 with eq. 3.8 / 3.9 (OPL, tensor-core f_k, fused statistics pass, column sampling) on a
    sequence of independent products, two in flight: product i + 1's statistics pass (bound by
    shared-memory traffic, leaving HBM bandwidth free) runs beside product i's block sizes, draws and
    gathers (on a high-priority side stream), and product i's GEMM follows, so a long sequence takes
    about a statistics pass plus a GEMM per product instead of the whole chain.  Every product is the
    same computation as run() with its seed, bit for bit.

    probs: two or more Problem states (prepared with max_draws >= c) over the inputs, used round-robin
    (product i works in probs[i % len(probs)]); seeds: one per product; outs: output matrices used
    round-robin (product i writes outs[i % len(outs)], which keeps it until product i + len(outs)
    overwrites it); replicate: as in run().  Enqueues everything on the current stream and the side
    stream and returns; the current stream has joined the side stream when it returns, so a whole
    sequence can be captured in a CUDA graph (after one eager call has created the side stream) and
    replayed.  Device status is read with check_status() on each state, as after run().

    events: if a list, (name, product, torch.cuda.Event) triples are appended for a timeline (timing
    only): stats_start / stats_end and gemm_start / gemm_end on the current stream, side_start /
    design_end / gathers_end on the side stream."""
    if len(probs) < 2 or not outs:
        raise ValueError("run_pipelined needs two or more problem states and an output")
    if gemm_mode != A.GEMM_BF16:
        raise ValueError("run_pipelined runs the BF16 sampled GEMM")
    torch = _torch()
    seeds = list(seeds)
    dev = probs[0].M.device
    main = torch.cuda.current_stream(dev)
    side = _side_stream(dev)
    sid = stream_id(replicate, A.PURPOSE_MAIN)
    bufs = []
    for pr in probs:
        K, n = pr.B.K, pr.B.n
        bufs.append(dict(p=torch.empty(n, dtype=torch.float64, device=dev), ck=torch.empty(K, dtype=torch.int64, device=dev),
                         g=torch.empty(K, dtype=torch.float64, device=dev), idx=torch.empty(c, dtype=torch.int32, device=dev),
                         scale=torch.empty(c, dtype=torch.float64, device=dev)))

    def mark(name, i, stream):
        ev = torch.cuda.Event(enable_timing=events is not None)
        ev.record(stream)
        if events is not None:
            events.append((name, i, ev))
        return ev

    def stats(i):
        pr, b = probs[i % len(probs)], bufs[i % len(probs)]
        if events is not None:
            mark("stats_start", i, main)
        A.bmm_probs(pr.M, pr.N, pr.B, A.P_COL_OPT, A.F_TC, b["p"], pr.st, pr.ws, main)
        return mark("stats_end", i, main)

    if not seeds:
        return
    side.wait_stream(main)
    ev_stats = stats(0)
    for i, seed in enumerate(seeds):
        pr, b, out = probs[i % len(probs)], bufs[i % len(probs)], outs[i % len(outs)]
        m = int(pr.M.shape[0])
        side.wait_event(ev_stats)
        if events is not None:
            mark("side_start", i, side)
        A.bmm_blocksizes(pr.M, pr.N, pr.B, pr.st, A.CK_OPT, c, None, None, 0, b["ck"], b["g"], None, pr.ws, side)
        A.bmm_sample(b["p"], A.UNIT_COLUMN, pr.B, b["ck"], c, seed, sid, b["idx"], b["scale"], pr.ws, side)
        if events is not None:
            mark("design_end", i, side)
        A.bmm_apply_part(pr.M, pr.N, pr.B, b["idx"], b["scale"], c, out, False, A.APPLY_REDUCE, 0, 0, pr.ws, side)
        A.bmm_apply_part(pr.M, pr.N, pr.B, b["idx"], b["scale"], c, out, False, A.APPLY_GATHER_B, 0, 0, pr.ws, side)
        A.bmm_apply_part(pr.M, pr.N, pr.B, b["idx"], b["scale"], c, out, False, A.APPLY_GATHER_A, 0, m, pr.ws, side)
        ev_g = mark("gathers_end", i, side)
        if i + 1 < len(seeds):
            # the next product's state is free: its previous user (product i + 1 - len(probs)) finished
            # its GEMM on this stream, and its side work before that GEMM started
            ev_stats = stats(i + 1)
        main.wait_event(ev_g)
        if events is not None:
            mark("gemm_start", i, main)
        A.bmm_apply_part(pr.M, pr.N, pr.B, b["idx"], b["scale"], c, out, False, A.APPLY_GEMM, 0, m, pr.ws, main)
        if events is not None:
            mark("gemm_end", i, main)
    main.wait_stream(side)


def error_report(prob: Problem, res: dict, delta: float = 0.05, stream=None) -> dict:
    """Whole-matrix error quantities of one Alg. 2 run (a run() result with res["unit"] column):
    E||MN - CD||_F^2 (Remark 2.2), eq. 3.10, theta_1, theta_2, beta and the bounds of eq. 3.11 / 3.12,
    eq. 4.3 / 4.4 and, for the two-step methods, eq. 4.8 / 4.9, as a dict keyed by _abi.REPORT_FIELDS
    (NaN where ||M^k N_k||_F^2 was not computed by the method).  Synchronises to read the values."""
    torch = _torch()
    if res["unit"] != A.UNIT_COLUMN:
        raise ValueError("the error report covers Alg. 2 (column sampling)")
    out = torch.empty(A.REPORT_LEN, dtype=torch.float64, device=prob.M.device)
    st = dict(prob.st)
    if res["method"] != "OPL":  # f_k of this run exists only where the method computed it
        st["f"] = None
    A.bmm_error_report(prob.B, st, res["p"], res["ck"], int(res["c"]), res.get("fhat") if st["f"] is not None else None,
                       delta, out, stream)
    return dict(zip(A.REPORT_FIELDS, out.cpu().tolist()))


def error_bars(prob: Problem, res: dict, entries, z: float = 1.96, exact: bool = False, stream=None) -> dict:
    """Normal intervals (Thm 3.1) for chosen entries of one sampled product: for entries (int64
    [count, 2] of (h, f), any device) the value (CD)_hf and the one-sample variance estimate from
    the run's own draws (bmm_entry_estimate), the interval value +- z sqrt(estimate), and with
    exact=True also the variance of eq. 3.7 (bmm_entry_variance; reads O(n) elements per entry).
    Tensors stay on the device."""
    torch = _torch()
    dev = prob.M.device
    ent = torch.as_tensor(entries, dtype=torch.int64).to(dev).reshape(-1, 2).contiguous()
    cnt = ent.shape[0]
    cd = torch.empty(cnt, dtype=torch.float64, device=dev)
    s2 = torch.empty(cnt, dtype=torch.float64, device=dev)
    unit = res["unit"]
    A.bmm_entry_estimate(prob.M, prob.N, prob.B, unit, res.get("ck"), res["idx"], res["scale"], int(res["idx"].numel()),
                         ent, cd, s2, prob.ws, stream)
    half = z * torch.sqrt(torch.clamp(s2, min=0.0))
    out = {"entries": ent, "value": cd, "var_est": s2, "lo": cd - half, "hi": cd + half}
    if exact:
        var = torch.empty(cnt, dtype=torch.float64, device=dev)
        A.bmm_entry_variance(prob.M, prob.N, prob.B, unit, res["p"], res.get("ck"), int(res["idx"].numel()), ent, var,
                             stream)
        out["var"] = var
    return out


def check_status(prob: Problem):
    code = A.bmm_read_device_status(prob.ws)
    if code != A.OK:
        raise A.BmmError(code, "device status")


def sampled_matmul(M, N, offsets, method: str = "ONC", c: int = None, seed: int = 0, replicate: int = 0,
                   c0: int | None = None, mode: str = "bf16"):
    """CD approximating M @ N, differentiable in M and N (the sample and p are held fixed)."""
    return SampledMatmul.apply(M, N, dict(offsets=offsets, method=method, c=c, seed=seed, replicate=replicate,
                                          c0=c0, mode=mode))


def _autograd_function():
    torch = _torch()

    class _SampledMatmul(torch.autograd.Function):
        @staticmethod
        def forward(ctx, M, N, cfg):
            gm = MODES[cfg["mode"]]
            prob = prepare(M.detach(), N.detach(), cfg["offsets"], cfg["c"], gemm_mode=gm)
            res = run(prob, cfg["method"], cfg["c"], cfg["seed"], cfg["replicate"], cfg["c0"], gemm_mode=gm)
            ctx.prob = prob
            ctx.cfg = cfg
            ctx.res = {k: res[k] for k in ("p", "ck", "unit", "sid")}
            return res["out"]

        @staticmethod
        def backward(ctx, G):
            prob, cfg, res = ctx.prob, ctx.cfg, ctx.res
            gm = MODES[cfg["mode"]]
            gdt = torch.float64 if gm == A.GEMM_F64 else torch.float32
            G = G.to(gdt).contiguous()

            def grad_dtype(t):  # BF16 inputs get BF16 gradients written by the library (one rounding)
                return torch.bfloat16 if gm == A.GEMM_BF16 and t.dtype == torch.bfloat16 else gdt

            dM = torch.empty(prob.M.shape, dtype=grad_dtype(prob.M), device=G.device) if ctx.needs_input_grad[0] else None
            dN = torch.empty(prob.N.shape, dtype=grad_dtype(prob.N), device=G.device) if ctx.needs_input_grad[1] else None
            A.bmm_backward(G, prob.M, prob.N, prob.B, res["unit"], res["p"], res["ck"], cfg["c"], cfg["seed"],
                           res["sid"], gm, dM, dN, False, prob.ws)
            if dM is not None and dM.dtype != prob.M.dtype:
                dM = dM.to(prob.M.dtype)
            if dN is not None and dN.dtype != prob.N.dtype:
                dN = dN.to(prob.N.dtype)
            return dM, dN, None

    return _SampledMatmul


class _Lazy:
    _fn = None

    def apply(self, *args):
        if _Lazy._fn is None:
            _Lazy._fn = _autograd_function()
        return _Lazy._fn.apply(*args)


SampledMatmul = _Lazy()


def autotune(shapes, gemm_mode: int = A.GEMM_BF16, device=None) -> dict:
    """Tune the tensor-core GEMM tiles for the sampled products of ``shapes`` ((m, p, L) triples):
    one bmm_autotune_gemm call per distinct (log2 m, log2 p, log2 K) bucket, on a scratch tensor
    allocated here.  Synchronises; call it before timing or capturing a graph.  Returns
    {(m, p, L): {"bn", "raster", "ms"}} for the shapes that were timed (one per bucket)."""
    torch = _torch()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    done, out, ws = set(), {}, None

    def lg(v):
        return int(np.ceil(np.log2(max(int(v), 1))))

    unit = 128 if gemm_mode == A.GEMM_E4M3 else 64
    mult = 3 if gemm_mode == A.GEMM_SPLIT_BF16 else 1
    for m, p, L in shapes:
        key = (lg(m), lg(p), lg(mult * ((int(L) + unit - 1) // unit) * unit))
        if key in done:
            continue
        done.add(key)
        need = A.bmm_autotune_workspace_size(int(m), int(p), int(L), gemm_mode)
        if need == 0:
            raise ValueError(f"cannot tune shape {(m, p, L)} in mode {gemm_mode}")
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        out[(int(m), int(p), int(L))] = A.bmm_autotune_gemm(int(m), int(p), int(L), gemm_mode, ws)
    return out


def autotune_batched(probs: list, results: list, cs, gemm_mode: int = A.GEMM_BF16, outs=None, reps: int = 3) -> dict:
    """Tune the GEMM tiles of a batch for its grouped launch, whose best tiles differ from those of
    each product alone (many products share the GPU).  Times the batch's own bmm_apply_batched
    (the draws of ``results``, eager, CUDA events, best of ``reps``) under each policy: the default
    rule, every uniform (tile width, raster group), and the per-shape choices of autotune(); keeps
    the fastest in the library's table.  Synchronises; call it before capturing a graph.  The
    outputs are overwritten.  Returns {"choice": name, "ms": {policy: ms}}."""
    torch = _torch()
    shapes = [(int(p.M.shape[0]), int(p.N.shape[1]), int(c)) for p, c in zip(probs, cs)]
    if outs is None:
        outs = [r["out"] for r in results]
    unit = results[0]["unit"] if results else A.UNIT_COLUMN

    def apply():
        A.bmm_apply_batched([p.M for p in probs], [p.N for p in probs], [p.B for p in probs], unit,
                            [r["idx"] for r in results], [r["scale"] for r in results], [c for *_, c in shapes],
                            gemm_mode, outs, False, [p.ws for p in probs])

    def timed():
        apply()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(max(1, reps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            apply()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def uniform(bn, ra):
        A.bmm_autotune_clear()
        for m, p, L in shapes:
            A.bmm_autotune_set(m, p, L, gemm_mode, bn, ra)

    policies = {"default": A.bmm_autotune_clear}
    for bn in (128, 256, A.TILE_PAIR, A.TILE_PAIR_WIDE):
        for ra in (4, 8, 16):
            policies[f"bn{bn}/r{ra}"] = (lambda bn=bn, ra=ra: uniform(bn, ra))
    policies["per_shape"] = lambda: (A.bmm_autotune_clear(), autotune(shapes, gemm_mode, probs[0].M.device))
    ms = {}
    for name, setp in policies.items():
        setp()
        ms[name] = timed()
    best = min(ms, key=ms.get)
    policies[best]()
    return {"choice": best, "ms": ms}


def run_batched(probs: list, method: str, cs, seeds, gemm_mode: int = A.GEMM_BF16, outs=None, streams=None,
                c0: int | None = None, fmode: int = A.F_TC, fused_stats: bool = False,
                grouped_stats: bool = True) -> list:
    """Many independent products (the batched configuration).

    With OPL and tensor-core f_k (``grouped_stats``) every stage runs as grouped launches over all the
    products: statistics (bmm_probs_batched), block sizes (bmm_blocksizes_batched), draws
    (bmm_sample_batched) and the products (bmm_apply_batched, whose BF16 GEMMs share persistent
    tensor-core launches), so the number of launches does not grow with the number of products.
    Other methods run each product's design and draws on its own, spread round-robin over
    ``streams`` so that small products overlap, and then the grouped products.
    Every step is an asynchronous C-ABI call, so the whole sequence can be captured with
    torch.cuda.graph and replayed as one graph launch.  Each Problem needs its own workspace.
    ``grouped_stats`` (OPL with tensor-core f_k): the statistics passes of all products share
    launches of many products (bmm_probs_batched): the norm pass of every product, then the Gram
    pass, whose CTAs pull blocks from one work list instead of one small launch per product.
    ``fused_stats`` computes each product's norms and f_k in one tensor-core pass instead; with
    many products in flight the two separate grouped passes are faster (each runs closer to its
    own limit), so the split form is the default here, unlike run() for one product.
    """
    torch = _torch()
    main = torch.cuda.current_stream()
    if streams is None:
        streams = [main]
    for s in streams:
        if s is not main:
            s.wait_stream(main)
    results = []
    ready = [None] * len(probs)
    sizes = [None] * len(probs)
    if grouped_stats and method == "OPL" and fmode == A.F_TC and probs:
        ready = [torch.empty(pr.n, dtype=torch.float64, device=pr.M.device) for pr in probs]
        Ms, Ns, Bs = [pr.M for pr in probs], [pr.N for pr in probs], [pr.B for pr in probs]
        sts, wss = [pr.st for pr in probs], [pr.ws for pr in probs]
        if fused_stats:
            A.bmm_probs_batched(Ms, Ns, Bs, A.P_COL_OPT, A.F_TC, ready, sts, wss)
        else:
            # the norm passes of all products grouped, then the Gram passes grouped
            A.bmm_probs_batched(Ms, Ns, Bs, A.P_COL_OPT, A.F_NONE, ready, sts, wss)
            A.bmm_probs_batched(Ms, Ns, Bs, A.P_COL_OPT, A.F_TC | A.REUSE_STATS, None, sts, wss)
        # every product's eq. 3.9 block sizes in one launch
        cks = [torch.empty(pr.K, dtype=torch.int64, device=pr.M.device) for pr in probs]
        gs = [torch.empty(pr.K, dtype=torch.float64, device=pr.M.device) for pr in probs]
        A.bmm_blocksizes_batched(Bs, sts, A.CK_OPT, [int(x) for x in cs], cks, gs, wss)
        sizes = list(zip(cks, gs))
        for s in streams:
            if s is not main:
                s.wait_stream(main)
    if probs and sizes[0] is not None:
        # every product's draws in grouped launches (bmm_sample_batched) on the current stream
        sid = stream_id(0, A.PURPOSE_MAIN)
        idxs = [torch.empty(int(c), dtype=torch.int32, device=pr.M.device) for pr, c in zip(probs, cs)]
        scales = [torch.empty(int(c), dtype=torch.float64, device=pr.M.device) for pr, c in zip(probs, cs)]
        A.bmm_sample_batched(ready, A.UNIT_COLUMN, [pr.B for pr in probs], [ck for ck, _ in sizes],
                             [int(c) for c in cs], [int(sd) for sd in seeds], [sid] * len(probs), idxs, scales,
                             [pr.ws for pr in probs])
        for i, pr in enumerate(probs):
            results.append({"method": method, "c": int(cs[i]), "seed": int(seeds[i]), "sid": sid, "p": ready[i],
                            "ck": sizes[i][0], "g": sizes[i][1], "idx": idxs[i], "scale": scales[i],
                            "unit": A.UNIT_COLUMN, "out": None})
    else:
        for i, prob in enumerate(probs):
            with torch.cuda.stream(streams[i % len(streams)]):
                results.append(run(prob, method, int(cs[i]), int(seeds[i]), c0=c0, gemm_mode=gemm_mode,
                                   compute_product=False, fmode=fmode, fused_stats=fused_stats, p_ready=ready[i],
                                   sizes_ready=sizes[i]))
    for s in streams:
        if s is not main:
            main.wait_stream(s)
    if outs is None:
        dt = torch.float64 if gemm_mode == A.GEMM_F64 else torch.float32
        outs = [torch.empty(p.M.shape[0], p.N.shape[1], dtype=dt, device=p.M.device) for p in probs]
    unit = results[0]["unit"] if results else A.UNIT_COLUMN
    A.bmm_apply_batched([p.M for p in probs], [p.N for p in probs], [p.B for p in probs], unit,
                        [r["idx"] for r in results], [r["scale"] for r in results], [int(c) for c in cs],
                        gemm_mode, outs, False, [p.ws for p in probs])
    for r, o in zip(results, outs):
        r["out"] = o
    return results

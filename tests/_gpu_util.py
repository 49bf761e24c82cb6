"""Shared helpers for the GPU parity tests (test infrastructure)."""
import numpy as np


def device():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device())


def host(t):
    return t.detach().cpu().numpy()


def as_layout(t, layout):
    """Same logical matrix stored row-major ('row') or column-major ('col', a transposed view)."""
    if layout == "row":
        return t.contiguous()
    return t.t().contiguous().t()


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    s = np.maximum(np.abs(b), 1e-300)
    return float(np.max(d / s))


def product_bound(M, N, idx, scale, offsets=None, unit="column"):
    """sum_t scale_t |M^{(i_t)}| |N_{(i_t)}|: the scale of each output entry's rounding error."""
    M = np.abs(np.asarray(M, dtype=np.float64))
    N = np.abs(np.asarray(N, dtype=np.float64))
    if unit == "column":
        cols, w = np.asarray(idx), np.asarray(scale)
    else:
        off = np.asarray(offsets)
        cols = np.concatenate([np.arange(off[k], off[k + 1]) for k in idx])
        w = np.concatenate([np.full(off[k + 1] - off[k], s) for k, s in zip(idx, scale)])
    return (M[:, cols] * w[None, :]) @ N[cols, :]

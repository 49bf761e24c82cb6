"""GB300 (sm_103a) randomized block matrix multiplication (Niu & Li, "Optimal Sampling
Algorithms for Block Matrix Multiplication").

The compute lives in libbmm.so (C ABI: include/bmm.h); this package is its thin Python
binding (``_abi``, the same entry-point names) plus the call sequence of a product and a
torch.autograd.Function (``pipeline``).  There is no CPU path: without a CUDA device or
without the built library every call raises.
"""
from . import _abi
from ._abi import (BmmError, bmm_apply, bmm_apply_batched, bmm_backward, bmm_blocksizes, bmm_blocksizes_batched,
                   bmm_clear_device_status,
                   bmm_entry_estimate, bmm_entry_variance, bmm_error_report, bmm_probs, bmm_probs_batched,
                   bmm_read_device_status, bmm_sample, bmm_workspace_size)
from .pipeline import (METHODS, MODES, Problem, SampledMatmul, autotune, autotune_batched, check_status, equal_budget,
                       error_bars, error_report, prepare, run, run_batched, run_pipelined, sampled_matmul,
                       stream_id)

__all__ = [
    "BmmError", "bmm_apply", "bmm_apply_batched", "bmm_backward", "bmm_blocksizes", "bmm_blocksizes_batched",
    "bmm_clear_device_status",
    "bmm_entry_estimate", "bmm_entry_variance", "bmm_error_report", "bmm_probs", "bmm_probs_batched",
    "bmm_read_device_status", "bmm_sample", "bmm_workspace_size", "METHODS", "MODES", "Problem",
    "SampledMatmul", "autotune", "autotune_batched", "check_status", "equal_budget", "error_bars", "error_report",
    "prepare", "run", "run_batched", "sampled_matmul", "stream_id",
]


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile the CUDA library in-tree (see buildlib.py)."""
    from .buildlib import build as _build
    return _build(verbose=verbose, force=force)

"""Boxcar search of a transform output (``fdmt_search``): argument marshalling only.

Section 4.2 ("Pulse profile"): a uniform pulse profile convolved with the
time axis commutes with the transform, so widths w = 2^k are tested on its
output A [nd, nt]; per row and width the maximum window sum and the first
time that reaches it.
"""
from __future__ import annotations

import ctypes

from . import _native as N
from .plan import _ptr, _stream_handle

MAX_WIDTHS = 13


def search_workspace_bytes(nd: int, nt: int, n_widths: int) -> int:
    v = ctypes.c_size_t()
    N.check(N.load().fdmt_search_workspace_bytes(nd, nt, n_widths, ctypes.byref(v)),
            "fdmt_search_workspace_bytes")
    return v.value


def search(A, n_widths: int, value_bound: int = 0, peak=None, time=None, workspace=None, stream=None):
    """(peak [nd, K], time [nd, K]) of the boxcar search on the device.

    A: int32 (a uint8 plan's output; peaks are int64) or float32 (peaks
    float32), [nd, nt], contiguous, on a CUDA device.  value_bound (int32 A
    only): 0, or a guaranteed bound on |A| that lets the sums run in int32
    (``Plan.search`` passes the one of its plan).
    """
    import torch
    if A.dim() != 2 or not A.is_contiguous() or A.dtype not in (torch.int32, torch.float32):
        raise ValueError("A must be a contiguous int32 or float32 tensor of shape (nd, nt)")
    nd, nt = A.shape
    integer = A.dtype == torch.int32
    if peak is None:
        peak = torch.empty((nd, n_widths), dtype=torch.int64 if integer else torch.float32, device=A.device)
    if time is None:
        time = torch.empty((nd, n_widths), dtype=torch.int32, device=A.device)
    if workspace is None:
        workspace = torch.empty(max(search_workspace_bytes(nd, nt, n_widths), 16), dtype=torch.uint8,
                                device=A.device)
    N.check(N.load().fdmt_search(_ptr(A), N.U8_I32 if integer else N.F32_F32, nd, nt, n_widths, value_bound, _ptr(peak),
                                 _ptr(time), _ptr(workspace), workspace.numel(), _stream_handle(stream)),
            "fdmt_search")
    return peak, time

"""Overlap-save streaming (``fdmt_stream_*``): argument marshalling only.

Each push transforms the next chunk of a continuous stream; its output equals
the matching columns of one transform of the whole stream.
"""
from __future__ import annotations

import ctypes

from . import _native as N
from .plan import _DTYPES, _SCHEDULES, _ptr, _stream_handle


class Stream:
    """A chunked transform (``fdmt_stream_create``): nf channels, nd delay
    rows, `chunk` samples per push (a multiple of 16)."""

    def __init__(self, f_min, f_max, nf, chunk, nd, dtype="f32", schedule="plain"):
        self._lib = N.load()
        self.nf, self.chunk, self.nd, self.dtype = int(nf), int(chunk), int(nd), dtype
        h = ctypes.c_void_p()
        N.check(self._lib.fdmt_stream_create(float(f_min), float(f_max), self.nf, self.chunk, self.nd,
                                             _DTYPES[dtype], _SCHEDULES[schedule], ctypes.byref(h)),
                "fdmt_stream_create")
        self._h = h
        carry, window = ctypes.c_int64(), ctypes.c_int64()
        N.check(self._lib.fdmt_stream_info(self._h, ctypes.byref(carry), ctypes.byref(window)), "fdmt_stream_info")
        self.carry, self.window = carry.value, window.value

    def push(self, x, out=None, stream=None):
        """Transform the next chunk x [nf, chunk] (device); returns [nd, chunk]."""
        import torch
        want = torch.uint8 if self.dtype == "u8" else torch.float32
        if tuple(x.shape) != (self.nf, self.chunk) or x.dtype != want or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {want} tensor of shape ({self.nf}, {self.chunk})")
        if out is None:
            out = torch.empty((self.nd, self.chunk), dtype=torch.int32 if self.dtype == "u8" else torch.float32,
                              device=x.device)
        N.check(self._lib.fdmt_stream_push(self._h, _ptr(x), _ptr(out), _stream_handle(stream)), "fdmt_stream_push")
        return out

    def reset(self, stream=None):
        N.check(self._lib.fdmt_stream_reset(self._h, _stream_handle(stream)), "fdmt_stream_reset")

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.fdmt_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

"""FFT-FDMT (``fdmt_fft_*``, section 5, Algorithm 2): argument marshalling only.

The transform computed bin by bin in the Fourier domain of the time axis;
the result equals the direct transform's (``Plan``) up to float32 FFT
rounding.  Overlapping FFT blocks of N samples (hop N - (Nd - 1)), two blocks
per complex FFT.
"""
from __future__ import annotations

import ctypes

from . import _native as N
from .plan import _ptr, _stream_handle

_IN_DTYPES = {"f32": N.F32_F32, "u8": N.U8_I32}


class FFTPlan:
    """FFT-FDMT of nf channels x nt samples into nd delay rows.

    dtype: input type, "f32" or "u8" (the output is float32 either way).
    block: FFT length N (0: picked from nd); bins: Fourier bins per merge
    block (0: picked).  host_only: shape and workspace only."""

    def __init__(self, f_min, f_max, nf, nt, nd, dtype="f32", block=0, bins=0, host_only=False):
        self._lib = N.load()
        if dtype not in _IN_DTYPES:
            raise ValueError(f"dtype must be one of {sorted(_IN_DTYPES)}")
        self.nf, self.nt, self.nd, self.dtype = int(nf), int(nt), int(nd), dtype
        h = ctypes.c_void_p()
        N.check(self._lib.fdmt_fft_plan(float(f_min), float(f_max), self.nf, self.nt, self.nd, _IN_DTYPES[dtype],
                                        int(block), int(bins), N.PLAN_HOST_ONLY if host_only else 0,
                                        ctypes.byref(h)), "fdmt_fft_plan")
        self._h = h
        blk, hop, pairs, b = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        N.check(self._lib.fdmt_fft_info(self._h, ctypes.byref(blk), ctypes.byref(hop), ctypes.byref(pairs),
                                        ctypes.byref(b)), "fdmt_fft_info")
        self.block, self.hop, self.pairs, self.bins = blk.value, hop.value, pairs.value, b.value
        ws = ctypes.c_size_t()
        N.check(self._lib.fdmt_fft_workspace_bytes(self._h, ctypes.byref(ws)), "fdmt_fft_workspace_bytes")
        self.workspace_bytes = ws.value

    def __call__(self, x, out=None, workspace=None, stream=None):
        """x [nf, nt] (device, float32 or uint8 as the plan says) -> float32 [nd, nt]."""
        import torch
        want = torch.uint8 if self.dtype == "u8" else torch.float32
        if tuple(x.shape) != (self.nf, self.nt) or x.dtype != want or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {want} tensor of shape ({self.nf}, {self.nt})")
        if out is None:
            out = torch.empty((self.nd, self.nt), dtype=torch.float32, device=x.device)
        if workspace is None:
            workspace = torch.empty(max(self.workspace_bytes, 16), dtype=torch.uint8, device=x.device)
        N.check(self._lib.fdmt_fft_execute(self._h, _ptr(x), _ptr(out), _ptr(workspace), workspace.numel(),
                                           _stream_handle(stream)), "fdmt_fft_execute")
        return out

    def profile_enable(self, capacity: int):
        """Record the device time of each launch in a ring of `capacity` (0: off)."""
        N.check(self._lib.fdmt_fft_profile_enable(self._h, int(capacity)), "fdmt_fft_profile_enable")
        self._prof_cap = int(capacity)

    def profile_read(self):
        """(launches recorded, [(kernel name, ms), ...]) since enable or the last read."""
        cap = max(getattr(self, "_prof_cap", 0), 1)
        ids = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int64()
        N.check(self._lib.fdmt_fft_profile_read(self._h, ids, ms, cap, ctypes.byref(n)), "fdmt_fft_profile_read")
        have = min(n.value, getattr(self, "_prof_cap", 0))
        return n.value, [(self._lib.fdmt_kernel_name(ids[i]).decode(), float(ms[i])) for i in range(have)]

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.fdmt_fft_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

"""Pipelined host execution (``fdmt_pipeline_*``): argument marshalling only.

Transforms of host-resident data with the copies of consecutive steps
overlapped with compute (two device slots, three CUDA streams)."""
from __future__ import annotations

import ctypes

from . import _native as N
from .plan import _ptr


class Pipeline:
    """Queue transforms of `plan` on page-locked host tensors; ``wait()``
    before reading the outputs."""

    def __init__(self, plan):
        self._lib = N.load()
        self.plan = plan  # kept alive: the pipeline borrows its handle
        h = ctypes.c_void_p()
        N.check(self._lib.fdmt_pipeline_create(plan._h, ctypes.byref(h)), "fdmt_pipeline_create")
        self._h = h

    def push(self, host_in, host_out):
        N.check(self._lib.fdmt_pipeline_push(self._h, _ptr(host_in), _ptr(host_out)), "fdmt_pipeline_push")

    def wait(self):
        N.check(self._lib.fdmt_pipeline_wait(self._h), "fdmt_pipeline_wait")

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.fdmt_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

"""Python binding of the batched FDMT (fdmt_plan_batch / fdmt_execute_batch):
argument marshalling only.  Many independent beams with their own band,
channel count, length and delay range are transformed by one persistent
kernel launch, recorded once as a CUDA graph and replayed afterwards."""
from __future__ import annotations

import ctypes

from . import _native as N
from .plan import _DTYPES, _stream_handle


class BatchPlan:
    """Plan of a batch of beams; beams = [(f_min, f_max, nf, nt, nd), ...].

    schedule "levels": one merge level per work item (rows_per_item, tile);
    "fused": every beam's fused cone programme (fused_tile, smem_budget),
    uint8 and float32 only.  Both run as one persistent launch.  "launches":
    one plan per beam, their launches spread over four streams forked from
    the caller's stream (fused_tile, smem_budget apply to the fused plans)."""

    def __init__(self, beams, dtype: str = "u8", rows_per_item: int = 0, tile: int = 0,
                 blocks_per_sm: int = 0, wait_ms: int = 0, schedule: str = "levels",
                 fused_tile: int = 0, smem_budget: int = 0):
        self._lib = N.load()
        self.beams = [tuple(b) for b in beams]
        self.dtype = dtype
        arr = (N.BeamDesc * len(self.beams))()
        for i, (f_min, f_max, nf, nt, nd) in enumerate(self.beams):
            arr[i] = N.BeamDesc(float(f_min), float(f_max), int(nf), int(nd), int(nt))
        codes = {"levels": 0, "fused": 1, "launches": 2}
        if schedule not in codes:
            raise ValueError("schedule must be 'levels', 'fused' or 'launches'")
        self.schedule = schedule
        prm = N.BatchParams(int(rows_per_item), int(tile), int(blocks_per_sm), int(wait_ms),
                            codes[schedule], int(fused_tile), int(smem_budget))
        h = ctypes.c_void_p()
        N.check(self._lib.fdmt_plan_batch(len(self.beams), arr, _DTYPES[dtype], 0, ctypes.byref(prm),
                                          ctypes.byref(h)), "fdmt_plan_batch")
        self._h = h
        self._ws = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fdmt_destroy_batch(self._h)
        self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        N.check(self._lib.fdmt_batch_workspace_bytes(self._h, ctypes.byref(v)), "fdmt_batch_workspace_bytes")
        return v.value

    def workspace(self, device=None):
        import torch
        need = self.workspace_bytes
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device or "cuda")
        return self._ws

    def outputs(self, device=None):
        """Freshly allocated output tensors, one [nd, nt] per beam."""
        import torch
        dt = torch.int32 if self.dtype == "u8" else torch.float32
        return [torch.empty((nd, nt), dtype=dt, device=device or "cuda") for (_, _, _, nt, nd) in self.beams]

    def execute(self, inputs, outputs, workspace=None, stream=None):
        """Transform every beam (``fdmt_execute_batch``); waits for the stream."""
        n = len(self.beams)
        if len(inputs) != n or len(outputs) != n:
            raise ValueError("one input and one output per beam")
        ins = (ctypes.c_void_p * n)(*[x.data_ptr() for x in inputs])
        outs = (ctypes.c_void_p * n)(*[y.data_ptr() for y in outputs])
        ws = self.workspace(inputs[0].device) if workspace is None else workspace
        N.check(self._lib.fdmt_execute_batch(self._h, ins, outs, ctypes.c_void_p(ws.data_ptr()),
                                             ws.numel() * ws.element_size(), _stream_handle(stream)),
                "fdmt_execute_batch")
        return outputs

    def levels(self, beam: int, sizes: bool = False):
        """Level boundaries beam `beam` is computed in (``fdmt_batch_levels``);
        with sizes=True also the bytes per sample stored at each."""
        g = ctypes.c_int32()
        N.check(self._lib.fdmt_batch_levels(self._h, int(beam), ctypes.byref(g), None, None, 0),
                "fdmt_batch_levels")
        buf = (ctypes.c_int32 * (g.value + 1))()
        sz = (ctypes.c_int32 * (g.value + 1))()
        N.check(self._lib.fdmt_batch_levels(self._h, int(beam), ctypes.byref(g), buf, sz, g.value + 1),
                "fdmt_batch_levels")
        return (list(buf), list(sz)) if sizes else list(buf)

    def drop_level(self, beam: int, level: int) -> None:
        """Test hook: remove the work items of (beam, level) (-1 restores)."""
        N.check(self._lib.fdmt_batch_drop_level(self._h, int(beam), int(level)), "fdmt_batch_drop_level")

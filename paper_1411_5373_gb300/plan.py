"""Python binding of the FDMT C ABI: argument marshalling only.

Every step of the transform runs in the CUDA library; torch supplies device
memory (outputs, workspace) and the current stream.  Names follow the C ABI:
``Plan`` wraps ``fdmt_plan``/``fdmt_destroy``, ``Plan.execute`` wraps
``fdmt_execute``, ``Plan.adjoint`` wraps ``fdmt_adjoint``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N

_DTYPES = {"u8": N.U8_I32, "f32": N.F32_F32, "f16state": N.F32_F16STATE}
_SCHEDULES = {"plain": N.SCHED_PLAIN, "fused": N.SCHED_FUSED}
_STAGING = {"auto": 0, "boxes": 1, "blocks": 2}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Delay tables and schedule for one transform shape (``fdmt_plan``).

    dtype: "u8" (uint8 -> int32, exact), "f32" (float32 throughout) or
    "f16state" (float32 in/out, intermediate state stored as fp16).
    schedule: "plain" (one launch per level) or "fused".
    host_only: build the tables without touching the GPU (inspection only).
    tile, smem_budget, bounds, group_tiles, group_budgets, staging, state16:
    fused schedule parameters (fdmt_schedule_params); staging "auto", "boxes"
    or "blocks" selects how staged rows are copied; state16 (uint8 only)
    stores the levels between launches as uint16 where their sums fit.
    gamma: the curves' power law Dt ~ f^gamma (-2, the default, is
    cold-plasma dispersion; ``fdmt_plan_curve``).
    d_min: delay of output row 0 in samples (the input is pre-shifted by the
    delay of d_min, section 4.2).  descending: input row j holds channel
    nf - 1 - j (f_max first).  Weights stay indexed by ascending channel.
    adjoint: "fused" (the default; fused float plans: several transposed
    levels per launch) or "plain" (one or two transposed levels per launch);
    adjoint_tile, adjoint_smem_budget, adjoint_bounds (with
    adjoint_group_tiles / adjoint_group_budgets per launch, indexed as the
    bounds) set the fused adjoint's launches (fdmt_schedule_params).
    """

    def __init__(self, f_min: float, f_max: float, nf: int, nt: int, nd: int,
                 dtype: str = "f32", schedule: str = "plain", host_only: bool = False,
                 tile: int = 0, smem_budget: int = 0, bounds=None, group_tiles=None,
                 group_budgets=None, staging: str = "auto", state16: bool = True, gamma: float = -2.0,
                 d_min: int = 0, descending: bool = False, search_widths: int = 0, adjoint: str = "fused",
                 adjoint_tile: int = 0, adjoint_smem_budget: int = 0, adjoint_bounds=None,
                 adjoint_group_tiles=None, adjoint_group_budgets=None):
        self._lib = N.load()
        if dtype not in _DTYPES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPES)}")
        if schedule not in _SCHEDULES:
            raise ValueError(f"schedule must be one of {sorted(_SCHEDULES)}")
        self.f_min, self.f_max = float(f_min), float(f_max)
        self.nf, self.nt, self.nd = int(nf), int(nt), int(nd)
        self.dtype, self.schedule, self.host_only = dtype, schedule, host_only
        flags = _SCHEDULES[schedule] | (N.PLAN_HOST_ONLY if host_only else 0)
        h = ctypes.c_void_p()
        params = None
        if staging not in _STAGING:
            raise ValueError(f"staging must be one of {sorted(_STAGING)}")
        self.search_widths = int(search_widths)
        if adjoint not in ("fused", "plain"):
            raise ValueError("adjoint must be 'fused' or 'plain'")
        if (tile or smem_budget or bounds or staging != "auto" or not state16 or search_widths or adjoint != "fused"
                or adjoint_tile or adjoint_smem_budget or adjoint_bounds):
            params = N.ScheduleParams()
            params.adjoint_schedule = 2 if adjoint == "fused" else 1
            params.adjoint_tile = int(adjoint_tile)
            params.adjoint_smem_budget = int(adjoint_smem_budget)
            ab = list(adjoint_bounds or [])
            params.adjoint_n_bounds = len(ab)
            for i, v in enumerate(ab):
                params.adjoint_bounds[i] = int(v)
            for i, v in enumerate(adjoint_group_tiles or []):
                params.adjoint_group_tile[i] = int(v)
            for i, v in enumerate(adjoint_group_budgets or []):
                params.adjoint_group_budget[i] = int(v)
            params.staging = _STAGING[staging]
            params.state16 = 0 if state16 else 1
            params.search_widths = int(search_widths)
            params.tile = int(tile)
            params.smem_budget = int(smem_budget)
            b = list(bounds or [])
            params.n_bounds = len(b)
            for i, v in enumerate(b):
                params.bounds[i] = int(v)
            for i, v in enumerate(group_tiles or []):
                params.group_tile[i] = int(v)
            for i, v in enumerate(group_budgets or []):
                params.group_budget[i] = int(v)
            params = ctypes.byref(params)
        self.gamma, self.d_min, self.descending = float(gamma), int(d_min), bool(descending)
        curve = None
        if self.gamma != -2.0 or self.d_min or self.descending:
            curve = ctypes.byref(N.CurveParams(self.gamma, self.d_min, int(self.descending)))
        N.check(self._lib.fdmt_plan_curve(self.f_min, self.f_max, self.nf, self.nt, self.nd,
                                          _DTYPES[dtype], flags, curve, params, ctypes.byref(h)), "fdmt_plan")
        self._h = h
        self._ws = None
        self._adj_ws = None

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fdmt_destroy(self._h)
        self._h = None
        self._ws = None
        self._adj_ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- sizes and tables ---------------------------------------------------
    @property
    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        N.check(self._lib.fdmt_workspace_bytes(self._h, ctypes.byref(v)), "fdmt_workspace_bytes")
        return v.value

    @property
    def adjoint_workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        N.check(self._lib.fdmt_adjoint_workspace_bytes(self._h, ctypes.byref(v)),
                "fdmt_adjoint_workspace_bytes")
        return v.value

    @property
    def levels(self) -> int:
        v = ctypes.c_int32()
        N.check(self._lib.fdmt_num_levels(self._h, ctypes.byref(v)), "fdmt_num_levels")
        return v.value

    def band_rows(self, level: int) -> np.ndarray:
        n = -(-self.nf // (1 << level))  # ceil(nf / 2^level) bands
        buf = (ctypes.c_int32 * n)()
        N.check(self._lib.fdmt_band_rows(self._h, level, buf, n), "fdmt_band_rows")
        return np.frombuffer(buf, dtype=np.int32).copy()

    def input_map(self):
        """(per-channel input delay s_k, descending) of the plan (``fdmt_input_map``)."""
        buf = (ctypes.c_int32 * self.nf)()
        desc = ctypes.c_int32()
        N.check(self._lib.fdmt_input_map(self._h, buf, self.nf, ctypes.byref(desc)), "fdmt_input_map")
        return np.frombuffer(buf, dtype=np.int32).copy(), bool(desc.value)

    def band_dl(self, level: int, band: int) -> np.ndarray:
        n = int(self.band_rows(level)[band])
        buf = (ctypes.c_int32 * n)()
        N.check(self._lib.fdmt_band_dl(self._h, level, band, buf, n), "fdmt_band_dl")
        return np.frombuffer(buf, dtype=np.int32).copy()

    def schedule_info(self):
        """(tile, [level boundaries]) of the fused schedule; (0, []) if plain."""
        g = ctypes.c_int32()
        w = ctypes.c_int32()
        N.check(self._lib.fdmt_schedule_info(self._h, ctypes.byref(g), None, 0, ctypes.byref(w)),
                "fdmt_schedule_info")
        if g.value == 0:
            return 0, []
        buf = (ctypes.c_int32 * (g.value + 1))()
        N.check(self._lib.fdmt_schedule_info(self._h, ctypes.byref(g), buf, g.value + 1, ctypes.byref(w)),
                "fdmt_schedule_info")
        return w.value, list(buf)

    def fused_table(self, kind: int) -> np.ndarray:
        """One table of the fused schedule as int32 (see fdmt_fused_tables)."""
        cnt = ctypes.c_int64()
        N.check(self._lib.fdmt_fused_tables(self._h, kind, None, 0, ctypes.byref(cnt)), "fdmt_fused_tables")
        buf = (ctypes.c_int32 * max(1, cnt.value))()
        N.check(self._lib.fdmt_fused_tables(self._h, kind, buf, cnt.value, ctypes.byref(cnt)),
                "fdmt_fused_tables")
        return np.frombuffer(buf, dtype=np.int32)[: cnt.value].copy()

    def device_status(self, stream=None) -> None:
        """Raise FdmtError(FDMT_ERR_TIMEOUT) if a bounded device wait gave up."""
        N.check(self._lib.fdmt_device_status(self._h, _stream_handle(stream)), "fdmt_device_status")

    # -- device memory helpers (torch) ----------------------------------------
    @property
    def in_dtype(self):
        import torch
        return torch.uint8 if self.dtype == "u8" else torch.float32

    @property
    def out_dtype(self):
        import torch
        return torch.int32 if self.dtype == "u8" else torch.float32

    def workspace(self, device=None):
        """A cached device workspace of workspace_bytes (allocated by torch)."""
        import torch
        need = self.workspace_bytes
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device or "cuda")
        return self._ws

    def adjoint_workspace(self, device=None):
        import torch
        need = self.adjoint_workspace_bytes
        if self._adj_ws is None or self._adj_ws.numel() < need:
            self._adj_ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device or "cuda")
        return self._adj_ws

    # -- transforms -----------------------------------------------------------
    def execute(self, x, out=None, weights=None, workspace=None, stream=None):
        """A = FDMT(w .* x) on the device (``fdmt_execute``).  x: [nf, nt]."""
        import torch
        if tuple(x.shape) != (self.nf, self.nt) or x.dtype != self.in_dtype or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {self.in_dtype} tensor of shape ({self.nf}, {self.nt})")
        if out is None:
            out = torch.empty((self.nd, self.nt), dtype=self.out_dtype, device=x.device)
        ws = self.workspace(x.device) if workspace is None else workspace
        N.check(self._lib.fdmt_execute(self._h, _ptr(x), _ptr(weights), _ptr(out), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream_handle(stream)),
                "fdmt_execute")
        return out

    def execute_host(self, x_host, out_host, dev_in, dev_out, weights_host=None,
                     dev_weights=None, workspace=None, stream=None):
        """Host-buffer transform (``fdmt_execute_host``): H2D copy, transform,
        D2H copy, stream synchronise.  All tensors preallocated by the caller."""
        ws = self.workspace(dev_in.device) if workspace is None else workspace
        N.check(self._lib.fdmt_execute_host(self._h, _ptr(x_host), _ptr(weights_host), _ptr(out_host),
                                            _ptr(dev_in), _ptr(dev_weights), _ptr(dev_out), _ptr(ws),
                                            ws.numel() * ws.element_size(), _stream_handle(stream)),
                "fdmt_execute_host")
        return out_host

    def search(self, out, n_widths: int, **kw):
        """Boxcar search of this plan's output (``fdmt_search``).  A uint8
        plan passes the bound 255 * (nf + nd - 1) on |out| (no output cell
        sums more input samples), so the sums run in int32 where that is
        exact."""
        from .search import search
        bound = 255 * (self.nf + self.nd - 1) if self.dtype == "u8" else 0
        return search(out, n_widths, value_bound=bound, **kw)

    def execute_search(self, x, n_widths: int, out=None, weights=None, peak=None, time=None, workspace=None,
                       stream=None):
        """(A, peak [nd, K], time [nd, K]): the transform and the boxcar search
        of its output (``fdmt_execute_search``); in the last fused launch
        when the plan was made with search_widths == n_widths."""
        import torch
        if tuple(x.shape) != (self.nf, self.nt) or x.dtype != self.in_dtype or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {self.in_dtype} tensor of shape ({self.nf}, {self.nt})")
        if out is None:
            out = torch.empty((self.nd, self.nt), dtype=self.out_dtype, device=x.device)
        if peak is None:
            peak = torch.empty((self.nd, n_widths), dtype=torch.int64 if self.dtype == "u8" else torch.float32,
                               device=x.device)
        if time is None:
            time = torch.empty((self.nd, n_widths), dtype=torch.int32, device=x.device)
        if workspace is None:
            workspace = torch.empty(max(self.search_workspace_bytes(n_widths), 256), dtype=torch.uint8,
                                    device=x.device)
        N.check(self._lib.fdmt_execute_search(self._h, _ptr(x), _ptr(weights), _ptr(out), int(n_widths), _ptr(peak),
                                              _ptr(time), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                              _stream_handle(stream)),
                "fdmt_execute_search")
        return out, peak, time

    def search_workspace_bytes(self, n_widths: int) -> int:
        """Workspace of execute_search (``fdmt_execute_search_workspace_bytes``)."""
        v = ctypes.c_size_t()
        N.check(self._lib.fdmt_execute_search_workspace_bytes(self._h, int(n_widths), ctypes.byref(v)),
                "fdmt_execute_search_workspace_bytes")
        return v.value

    def adjoint(self, grad_out, x=None, weights=None, grad_in=None, grad_weights=None,
                workspace=None, stream=None):
        """grad_in = w .* FDMT^T(grad_out); grad_weights[k] = <x[k], FDMT^T(grad_out)[k]>
        when a grad_weights tensor is passed (``fdmt_adjoint``)."""
        import torch
        if tuple(grad_out.shape) != (self.nd, self.nt) or grad_out.dtype != torch.float32:
            raise ValueError("grad_out must be float32 of shape (nd, nt)")
        grad_out = grad_out.contiguous()
        if grad_in is None:
            grad_in = torch.empty((self.nf, self.nt), dtype=torch.float32, device=grad_out.device)
        ws = self.adjoint_workspace(grad_out.device) if workspace is None else workspace
        N.check(self._lib.fdmt_adjoint(self._h, _ptr(grad_out), _ptr(x), _ptr(weights), _ptr(grad_in),
                                       _ptr(grad_weights), _ptr(ws), ws.numel() * ws.element_size(),
                                       _stream_handle(stream)),
                "fdmt_adjoint")
        return grad_in

    # -- launch profiler --------------------------------------------------------
    def profile_enable(self, capacity: int) -> None:
        """Record device time of every kernel launch (``fdmt_profile_enable``)."""
        N.check(self._lib.fdmt_profile_enable(self._h, int(capacity)), "fdmt_profile_enable")
        self._prof_cap = int(capacity)

    def profile_read(self):
        """Return (launches, [(kernel_name, level, ms), ...]) for the recorded
        launches, oldest first (``fdmt_profile_read``); resets the record."""
        n = max(1, getattr(self, "_prof_cap", 0))
        ids = (ctypes.c_int32 * n)()
        lv = (ctypes.c_int32 * n)()
        ms = (ctypes.c_float * n)()
        cnt = ctypes.c_int64()
        N.check(self._lib.fdmt_profile_read(self._h, ids, lv, ms, n, ctypes.byref(cnt)), "fdmt_profile_read")
        have = min(cnt.value, getattr(self, "_prof_cap", 0))
        rows = [(self._lib.fdmt_kernel_name(ids[i]).decode(), int(lv[i]), float(ms[i])) for i in range(have)]
        return cnt.value, rows

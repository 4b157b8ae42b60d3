"""STFT filterbank in front of the transform (``fdmt_filterbank``):
argument marshalling only.  Section 2: blocks of Nf complex voltages,
Fourier transform, squared magnitude, optional binning of nbin spectra;
channels in ascending frequency."""
from __future__ import annotations

from . import _native as N
from .plan import _ptr, _stream_handle


def filterbank(volts, nf: int, nbin: int = 1, out=None, nt: int | None = None, stream=None):
    """Spectra [nf, nt] (float32) of complex64 voltages `volts` (1-D, on the
    device); nt defaults to len(volts) // (nf * nbin)."""
    import torch
    if volts.dim() != 1 or volts.dtype != torch.complex64 or not volts.is_contiguous():
        raise ValueError("volts must be a contiguous 1-D complex64 tensor")
    n = volts.numel()
    if nt is None:
        nt = n // (nf * nbin)
    if out is None:
        out = torch.empty((nf, nt), dtype=torch.float32, device=volts.device)
    N.check(N.load().fdmt_filterbank(_ptr(volts), n, nf, nbin, _ptr(out), nt, _stream_handle(stream)),
            "fdmt_filterbank")
    return out

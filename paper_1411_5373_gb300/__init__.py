"""GB300 (sm_103a) Fast Dispersion Measure Transform (Zackay & Ofek, arXiv:1411.5373).

The compute path is the CUDA library ``libfdmt_gb300.so`` behind the C ABI
of include/fdmt.h; this package only marshals arguments to it.  Build the
library with ``python -m paper_1411_5373_gb300.build``.
"""
from . import _native
from ._native import FdmtError, load
from .batch import BatchPlan
from .plan import Plan
from .search import search, search_workspace_bytes
from .stream import Stream
from .filterbank import filterbank
from .pipeline import Pipeline
from .fft_fdmt import FFTPlan

__all__ = ["Plan", "BatchPlan", "Stream", "Pipeline", "FFTPlan", "FdmtError", "load", "search", "search_workspace_bytes", "filterbank",
           "fdmt", "FDMTFunction"]


def __getattr__(name):
    # torch is only needed for the differentiable wrapper.
    if name in ("fdmt", "FDMTFunction"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)

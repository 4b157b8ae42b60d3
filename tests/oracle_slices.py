"""Oracle column slices of seeded batch beams, computed by worker processes
(test infrastructure only).

An output column t of the transform depends only on input columns
t - (Nd - 1) .. t (section 4: every curve spans at most Nd - 1 samples), so
output columns [T0, T0 + S) of a beam equal the oracle run on input columns
[T0 - Nd + 1, T0 + S), from its column Nd - 1 on (for T0 = 0 the input simply
starts at 0).  The workers draw the input window themselves from the seeded
generator, so nothing large crosses process boundaries.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

import filterbank_synth as fs
import oracle


def beam_slice(args):
    """(beam, T0, S, f_min, f_max) -> the oracle's int32 output columns [T0, T0 + S)."""
    b, t0, s, f_min, f_max = args
    a = max(0, t0 - (b.nd - 1))
    x = fs.beam_u8(b, f_min, f_max, t_begin=a, t_end=t0 + s)
    T = oracle.build_tables(f_min, f_max, b.nf, b.nd)
    return oracle.fdmt(x, T, "i64")[:, t0 - a:].astype(np.int32)


def beam_slices(tasks, procs=None):
    """Oracle slices for a list of beam_slice tasks, on every host core
    (spawned workers)."""
    procs = procs or max(1, min(len(tasks), len(os.sched_getaffinity(0))))
    if procs == 1:
        return [beam_slice(t) for t in tasks]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(beam_slice, tasks)

"""Seeded synthetic filterbanks (frequency x time intensity matrices).

This module only draws inputs; it holds none of the transform's arithmetic, so
the CPU oracle and the CUDA path can both be fed the same bytes from here.

Noise is drawn in column blocks of BLOCK samples, each block from its own
numpy PCG64 stream keyed by (seed, block index).  Any column slice of a large
input can therefore be regenerated on the host without drawing the rest,
which is how slices of the largest workload are checked.

Pulses follow the dispersion law of the paper (Eq. DtD with the constants
absorbed): a pulse of total delay D (samples across the band) that reaches the
lowest frequency f_min at t0 reaches frequency f at t0 - D * r(f), with
r(f) = (f_min^-2 - f^-2) / (f_min^-2 - f_max^-2).  Channel k covers frequencies
[e_k, e_{k+1}], so a pulse of width W samples lights samples
t0 - round(D r(e_{k+1})) .. t0 - round(D r(e_k)) + W - 1 of that channel.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BLOCK = 1 << 16
SEED_BASE = 1411537300


@dataclass(frozen=True)
class Pulse:
    delay: int          # total delay D across the band, in samples
    t0: int             # arrival time at f_min
    width: int          # boxcar width W in samples
    amp: np.ndarray = field(compare=False)  # per-channel amplitude (sigma units)


@dataclass(frozen=True)
class Workload:
    name: str
    nf: int
    nt: int
    nd: int
    f_min: float
    f_max: float
    seed: int
    n_pulses: int
    width_range: tuple
    amp_range: tuple
    fixed_pulse: tuple | None = None   # (D, t0, W, amp) instead of drawn pulses


def _edge(f_min, f_max, nf, k):
    return f_min + (f_max - f_min) * k / nf


def _delay_fraction(f_min, f_max, f):
    return (f_min ** -2 - f ** -2) / (f_min ** -2 - f_max ** -2)


# Workloads of the benchmark suite (sizes in samples / channels / delay rows).
SINGLE_SMALL = Workload("single beam Nf=64 Nt=1024 Nd=64", 64, 1024, 64,
                        1200.0, 1600.0, SEED_BASE + 1, 1, (2, 2), (3.0, 3.0),
                        fixed_pulse=(40, 500, 2, 3.0))
SINGLE_1K = Workload("single beam Nf=1024 Nt=65536 Nd=1024", 1024, 1 << 16, 1024,
                     1200.0, 1600.0, SEED_BASE + 2, 16, (1, 16), (0.5, 2.0))
DIFF_1K = Workload("differentiable Nf=1024 Nt=65536 Nd=1024", 1024, 1 << 16, 1024,
                   1200.0, 1600.0, SEED_BASE + 4, 8, (1, 16), (0.5, 2.0))
LARGE_4K = Workload("large beam Nf=4096 Nt=2^20 Nd=4096", 4096, 1 << 20, 4096,
                    1100.0, 1700.0, SEED_BASE + 5, 32, (1, 64), (0.5, 2.0))


def noise_f32(seed: int, nf: int, t_begin: int, t_end: int) -> np.ndarray:
    """N(0,1) float32 noise for columns [t_begin, t_end) of an nf-row input."""
    if t_end <= t_begin:
        return np.zeros((nf, 0), dtype=np.float32)
    out = np.empty((nf, t_end - t_begin), dtype=np.float32)
    b0 = t_begin // BLOCK
    b1 = (t_end - 1) // BLOCK
    for blk in range(b0, b1 + 1):
        rng = np.random.Generator(np.random.PCG64([seed, nf, blk]))
        z = rng.standard_normal((nf, BLOCK), dtype=np.float32)
        lo = max(t_begin, blk * BLOCK)
        hi = min(t_end, (blk + 1) * BLOCK)
        out[:, lo - t_begin:hi - t_begin] = z[:, lo - blk * BLOCK:hi - blk * BLOCK]
    return out


def draw_pulses(w: Workload) -> list:
    """Pulse parameters of a workload, drawn from its seed.

    Delays uniform in [0, Nd), widths uniform in width_range, one arrival per
    equal slot of [Nd, Nt - max width) so pulses are spaced by more than Nd.
    """
    rng = np.random.Generator(np.random.PCG64([w.seed, 7]))
    pulses = []
    if w.n_pulses == 0:
        return pulses
    if w.fixed_pulse is not None:
        d, t0, width, a = w.fixed_pulse
        return [Pulse(d, t0, width, np.full(w.nf, a, dtype=np.float32))]
    lo_t = w.nd + 32
    hi_t = w.nt - w.width_range[1] - 1
    slot = (hi_t - lo_t) // w.n_pulses
    for i in range(w.n_pulses):
        d = int(rng.integers(0, w.nd))
        width = int(rng.integers(w.width_range[0], w.width_range[1] + 1))
        t0 = lo_t + i * slot + int(rng.integers(0, max(1, slot - w.nd - 32)))
        amp = rng.uniform(w.amp_range[0], w.amp_range[1], size=w.nf).astype(np.float32)
        pulses.append(Pulse(d, t0, width, amp))
    return pulses


def pulse_mask_rows(w: Workload, p: Pulse, k: int):
    """Sample range [s0, s1] of channel k lit by pulse p (inclusive)."""
    lo_edge = _edge(w.f_min, w.f_max, w.nf, k)
    hi_edge = _edge(w.f_min, w.f_max, w.nf, k + 1)
    s0 = p.t0 - int(np.floor(p.delay * _delay_fraction(w.f_min, w.f_max, hi_edge) + 0.5))
    s1 = p.t0 - int(np.floor(p.delay * _delay_fraction(w.f_min, w.f_max, lo_edge) + 0.5)) + p.width - 1
    return s0, s1


def add_pulses(x: np.ndarray, w: Workload, pulses, t_begin: int = 0, scale: float = 1.0):
    """Add pulses (amplitude * scale) into x, which holds columns
    [t_begin, t_begin + x.shape[1]) of the workload's input."""
    t_end = t_begin + x.shape[1]
    for p in pulses:
        for k in range(w.nf):
            s0, s1 = pulse_mask_rows(w, p, k)
            a = max(s0, t_begin)
            b = min(s1 + 1, t_end)
            if a < b:
                x[k, a - t_begin:b - t_begin] += np.float32(p.amp[k] * scale)
    return x


def filterbank_f32(w: Workload, t_begin: int = 0, t_end: int | None = None) -> np.ndarray:
    """float32 input I[f, t] (N(0,1) noise plus the workload's pulses) for
    columns [t_begin, t_end)."""
    t_end = w.nt if t_end is None else t_end
    x = noise_f32(w.seed, w.nf, t_begin, t_end)
    return add_pulses(x, w, draw_pulses(w), t_begin)


def filterbank_u8(w: Workload, t_begin: int = 0, t_end: int | None = None) -> np.ndarray:
    """uint8 variant: clip(round(128 + 16 * (noise + pulses)), 0, 255)."""
    x = filterbank_f32(w, t_begin, t_end)
    return np.clip(np.rint(128.0 + 16.0 * x), 0, 255).astype(np.uint8)


def random_u8(seed: int, nf: int, nt: int) -> np.ndarray:
    """Plain uniform uint8 matrix (edge cases and exhaustive parity)."""
    rng = np.random.Generator(np.random.PCG64([seed, nf, nt, 3]))
    return rng.integers(0, 256, size=(nf, nt), dtype=np.uint8)


def random_f32(seed: int, nf: int, nt: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64([seed, nf, nt, 5]))
    return rng.standard_normal((nf, nt), dtype=np.float32)


def small_ints(seed: int, shape, lo: int = -2, hi: int = 2) -> np.ndarray:
    """Integers in [lo, hi] as float32 (exact dot-product tests)."""
    rng = np.random.Generator(np.random.PCG64([seed, *shape, 11]))
    return rng.integers(lo, hi + 1, size=shape).astype(np.float32)


# ---- batched uneven beams ------------------------------------------------

@dataclass(frozen=True)
class Beam:
    nf: int
    nt: int
    nd: int
    seed: int


def batch_beams(n: int = 64, seed: int = SEED_BASE + 3) -> list:
    """Uneven beams: Nf in {256,512,1024,4096}, Nt in {2^14,2^16,2^18},
    Nd in {256,512,1024,2048} with Nd <= Nt, drawn i.i.d. from the seed."""
    rng = np.random.Generator(np.random.PCG64([seed, 13]))
    nfs = [256, 512, 1024, 4096]
    nts = [1 << 14, 1 << 16, 1 << 18]
    nds = [256, 512, 1024, 2048]
    beams = []
    for i in range(n):
        nf = nfs[int(rng.integers(0, 4))]
        nt = nts[int(rng.integers(0, 3))]
        nd = nds[int(rng.integers(0, 4))]
        beams.append(Beam(nf, nt, min(nd, nt), seed * 1000 + i))
    return beams


def beam_workload(b: Beam, f_min: float = 1200.0, f_max: float = 1600.0, n_pulses: int = 4) -> Workload:
    """The uint8 workload of one batch beam: noise as the single beam's
    uint8 variant plus n_pulses injected pulses."""
    return Workload("beam", b.nf, b.nt, b.nd, f_min, f_max, b.seed, n_pulses, (1, 16), (0.5, 2.0))


def beam_u8(b: Beam, f_min: float = 1200.0, f_max: float = 1600.0,
            n_pulses: int = 4, t_begin: int = 0, t_end: int | None = None) -> np.ndarray:
    return filterbank_u8(beam_workload(b, f_min, f_max, n_pulses), t_begin, t_end)


def _beam_u8_task(args):
    b, f_min, f_max, n_pulses = args
    return beam_u8(b, f_min, f_max, n_pulses)


def batch_inputs_u8(beams, f_min: float = 1200.0, f_max: float = 1600.0, n_pulses: int = 4,
                    procs: int | None = None):
    """Every beam's uint8 input (beam_u8), drawn by a pool of worker
    processes (started with spawn, so a caller that already uses a GPU can
    call it).  Yields (index, array) as beams complete, in order."""
    import multiprocessing as mp
    import os
    procs = procs or max(1, min(len(beams), len(os.sched_getaffinity(0))))
    if procs == 1:
        for i, b in enumerate(beams):
            yield i, beam_u8(b, f_min, f_max, n_pulses)
        return
    with mp.get_context("spawn").Pool(procs) as pool:
        for i, x in enumerate(pool.imap(_beam_u8_task, [(b, f_min, f_max, n_pulses) for b in beams])):
            yield i, x

"""Work division across ranks (one process per GPU), without any exchange of
transform data.

Two ways the transform shards (no collective on the data path):

* beams: independent problems; ``shard_beams`` assigns whole beams to ranks,
  largest first to the least-loaded rank (cells Nd x Nt as the load);
* time: output column t depends only on input columns [t - Nd + 1, t]
  (Algorithm 1 looks back in time only; samples before the first are zero by
  the copy rule of section 4), so rank r can produce output columns
  [t0, t1) from input columns [t0 - halo, t1) alone; ``time_shards`` gives
  each rank its columns and the halo it must read (duplicated, not
  exchanged).
"""
from __future__ import annotations

from dataclasses import dataclass


def shard_beams(beams, world: int):
    """Beam indices per rank: greedy by load (Nd x Nt, largest first), ties to
    the lower rank.  beams: sequence of (f_min, f_max, nf, nt, nd)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(beams)), key=lambda i: (-(beams[i][3] * beams[i][4]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += beams[i][3] * beams[i][4]
    return [sorted(o) for o in out]


@dataclass(frozen=True)
class TimeShard:
    t_in: int    # first input column this rank reads
    t0: int      # first output column it owns
    t1: int      # end of its output columns
    window: int  # columns the rank transforms (t1 - t_in rounded up to `align`)

    @property
    def skip(self) -> int:
        """Leading output columns of the window that belong to the halo."""
        return self.t0 - self.t_in


def time_shards(nt: int, nd: int, world: int, align: int = 16):
    """Output columns [t0, t1) per rank (contiguous, sizes multiples of
    `align` except the last) and the input each needs: columns
    [t0 - halo, t1), halo = nd - 1 rounded up to `align` (clipped at 0).  The
    window a rank transforms is t1 - t_in rounded up to `align` (zeros past
    the input's end do not change columns before it)."""
    if world < 1 or nt < 1 or nd < 1:
        raise ValueError("need world, nt, nd >= 1")
    per = -(-nt // world)
    per = -(-per // align) * align
    halo = -(-(nd - 1) // align) * align
    out = []
    for r in range(world):
        t0, t1 = min(nt, r * per), min(nt, (r + 1) * per)
        t_in = max(0, t0 - halo)
        out.append(TimeShard(t_in, t0, t1, -(-(t1 - t_in) // align) * align if t1 > t0 else 0))
    return out

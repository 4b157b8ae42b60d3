"""Work division across ranks on CPU: world_size-2 gloo process groups run
the multi-rank host logic (beam and time shards, the max-over-ranks timing
reduction) with the CPU oracle standing in for each rank's transform.
Time shards must reproduce one transform of the whole input bit for bit
(causality, no exchange of data); beam shards must cover every beam once."""
import os
import socket

import numpy as np
import pytest

import filterbank_synth as fs
import oracle
from paper_1411_5373_gb300.shard import shard_beams, time_shards

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # time shards of one beam: each rank transforms its window alone
        nf, nt, nd = 16, 400, 37
        x = fs.random_u8(5, nf, nt).astype(np.int64)
        T = oracle.build_tables(1200.0, 1600.0, nf, nd)
        sh = time_shards(nt, nd, world)[rank]
        win = np.zeros((nf, sh.window), dtype=np.int64)
        win[:, : sh.t1 - sh.t_in] = x[:, sh.t_in: sh.t1]
        part = oracle.fdmt(win, T, "i64")[:, sh.skip: sh.skip + (sh.t1 - sh.t0)]
        full = torch.zeros((nd, nt), dtype=torch.int64)
        full[:, sh.t0: sh.t1] = torch.from_numpy(part)
        dist.all_reduce(full)  # test-side gather only; the shards never exchange data
        # beam shards: each rank reports its beams
        beams = [(1200.0, 1600.0, 16, nt_, nd_) for nt_, nd_ in ((256, 20), (512, 64), (128, 9), (1024, 100),
                                                                 (256, 31))]
        mine = torch.zeros(len(beams), dtype=torch.int64)
        for i in shard_beams(beams, world)[rank]:
            mine[i] += 1
        dist.all_reduce(mine)
        # the bench's timing: the max over ranks
        t = torch.tensor([1.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            results["time_ok"] = bool(np.array_equal(full.numpy(), oracle.fdmt(x, T, "i64")))
            results["beams"] = mine.tolist()
            results["tmax"] = float(t.item())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shards():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), results), nprocs=2, join=True, start_method="spawn")
        assert results["time_ok"]
        assert results["beams"] == [1] * 5
        assert results["tmax"] == 2.0


@pytest.mark.parametrize("nt,nd,world", [(65536, 1024, 2), (65536, 1024, 8), (1000, 64, 3), (40, 64, 4),
                                         (17, 1, 5)])
def test_time_shards_cover_and_align(nt, nd, world):
    sh = time_shards(nt, nd, world)
    assert sh[0].t0 == 0 and sh[-1].t1 == nt
    for a, b in zip(sh, sh[1:]):
        assert a.t1 == b.t0
    for s in sh:
        if s.t1 == s.t0:  # more ranks than 16-column blocks: an empty shard
            assert s.window == 0
            continue
        assert s.t_in == max(0, s.t0 - (-(-(nd - 1) // 16) * 16))
        assert s.t0 % 16 == 0 and s.window % 16 == 0 and s.window >= s.t1 - s.t_in


def test_beam_shards_balance():
    beams = [(1200.0, 1600.0, 256, nt, nd) for nt, nd in ((1 << 18, 2048), (1 << 14, 256), (1 << 16, 1024),
                                                          (1 << 16, 512), (1 << 14, 2048), (1 << 18, 256))]
    for world in (1, 2, 3, 4, 8):
        sh = shard_beams(beams, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(beams)))
        loads = [sum(beams[i][3] * beams[i][4] for i in s) for s in sh]
        biggest = max(b[3] * b[4] for b in beams)
        assert max(loads) - min(loads) <= biggest  # greedy bound

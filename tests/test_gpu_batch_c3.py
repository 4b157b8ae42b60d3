"""The 64-beam uneven batch at full size (the batch benchmark's workload):
Nf in {256, 512, 1024, 4096}, Nt in {2^14, 2^16, 2^18}, Nd in {256, 512,
1024, 2048} drawn from the seed, band 1200-1600 MHz, uint8 noise with four
injected pulses per beam, int32 outputs.

Each batch schedule (one merge level per work item, every beam's fused cone
programme in one persistent launch, every beam's own fused launches) runs
the whole batch; every beam is then checked bit for bit on two column slices
against the oracle: the first S columns (where the copy rule matters) and a
seeded window [T0, T0 + S), computed from the input window
[T0 - Nd + 1, T0 + S) (an output column depends only on the Nd - 1 input
columns before it, section 4).
"""
import numpy as np
import pytest

import filterbank_synth as fs
import paper_1411_5373_gb300 as FD
from oracle_slices import beam_slices
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

F_MIN, F_MAX = 1200.0, 1600.0
S = 512


@pytest.fixture(scope="module")
def batch():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()
    beams = fs.batch_beams()
    rng = np.random.Generator(np.random.PCG64([fs.SEED_BASE, 31]))
    windows = [(0, int(rng.integers(b.nd, b.nt - S + 1) // 16 * 16)) for b in beams]
    tasks = [(b, t0, S, F_MIN, F_MAX) for b, w in zip(beams, windows) for t0 in w]
    want = beam_slices(tasks)
    ins = [None] * len(beams)
    for i, x in fs.batch_inputs_u8(beams, F_MIN, F_MAX):
        ins[i] = torch.from_numpy(x).cuda()
    return beams, windows, want, ins


@pytest.mark.parametrize("params", [{}, {"schedule": "fused"}, {"schedule": "launches"}])
def test_full_size_batch_slices_match_oracle(batch, params):
    beams, windows, want, ins = batch
    spec = [(F_MIN, F_MAX, b.nf, b.nt, b.nd) for b in beams]
    bp = FD.BatchPlan(spec, "u8", **params)
    ws = torch.empty(max(bp.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    outs = bp.outputs(torch.device("cuda"))
    bp.execute(ins, outs, workspace=ws)
    torch.cuda.synchronize()
    k = 0
    for i, b in enumerate(beams):
        for t0 in windows[i]:
            got = outs[i][:, t0:t0 + S].cpu().numpy()
            assert np.array_equal(got, want[k]), f"beam {i} ({b.nf}x{b.nt}x{b.nd}) columns [{t0}, {t0 + S})"
            k += 1
    bp.close()
    del outs, ws

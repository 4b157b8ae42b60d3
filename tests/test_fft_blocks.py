"""FFT-FDMT block decomposition on the CPU (no GPU): the block length, hop
and block pairs that ``fdmt_fft_plan`` chooses, run through a float64 numpy
model of the GPU data flow (overlapping blocks, two blocks per complex FFT,
level-0 rows formed as X_c(k) sum_{i<=j} w^{ik}, the merges per bin, the
inverse FFT keeping samples [Nd - 1, N) of each block), must give the
oracle's direct transform (Algorithm 1).  Checks the plan's host logic
(block, hop, pairs) and the overlap-save and packing arguments independently
of the kernels.
"""
import numpy as np
import pytest

import oracle
import paper_1411_5373_gb300 as F


def blocked_model(I, T, N, hop, pairs):
    nf, nt = I.shape
    G = T.nd - 1
    assert hop == N - G
    X = np.zeros((nf, pairs * N), dtype=np.complex128)
    n = np.arange(N)
    for p in range(pairs):
        ta = 2 * p * hop - G + n
        tb = ta + hop
        za = np.where((ta >= 0) & (ta < nt), I[:, np.clip(ta, 0, nt - 1)], 0.0)
        zb = np.where((tb >= 0) & (tb < nt), I[:, np.clip(tb, 0, nt - 1)], 0.0)
        X[:, p * N:(p + 1) * N] = np.fft.fft(za + 1j * zb, axis=1)
    k = np.arange(pairs * N) % N
    state = []
    for c in range(nf):
        rows, g = [], np.zeros(pairs * N, dtype=np.complex128)
        for j in range(T.rows[0][c]):
            g = g + np.exp(-2j * np.pi * ((j * k) % N) / N)
            rows.append(X[c] * g)
        state.append(rows)
    for l in range(1, T.levels + 1):
        nxt = []
        for b in range(len(T.rows[l])):
            if not T.has_upper(l, b):
                nxt.append(state[2 * b][:T.rows[l][b]])
                continue
            out = []
            for dt in range(T.rows[l][b]):
                j = int(T.dl[l][b][dt])
                out.append(state[2 * b][j] + state[2 * b + 1][dt - j] * np.exp(-2j * np.pi * ((j * k) % N) / N))
            nxt.append(out)
        state = nxt
    Y = np.array(state[0])
    A = np.zeros((T.nd, nt))
    for p in range(pairs):
        y = np.fft.ifft(Y[:, p * N:(p + 1) * N], axis=1)[:, G:]
        for part, t0 in ((y.real, 2 * p * hop), (y.imag, (2 * p + 1) * hop)):
            m = min(hop, max(0, nt - t0))
            A[:, t0:t0 + m] = part[:, :m]
    return A


@pytest.mark.parametrize("nf,nt,nd,block", [(16, 1000, 20, 256), (6, 700, 40, 256), (2, 77, 8, 256),
                                             (37, 2000, 200, 512), (64, 5000, 250, 0), (8, 1, 4, 0),
                                             (4, 600, 1, 256)])
def test_block_plan_reproduces_direct_transform(nf, nt, nd, block):
    p = F.FFTPlan(1200.0, 1600.0, nf, nt, nd, block=block, host_only=True)
    assert p.hop == p.block - (nd - 1) > 0
    assert 2 * p.pairs * p.hop >= nt > 2 * (p.pairs - 1) * p.hop
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    I = np.random.default_rng(nf * 1000 + nd).standard_normal((nf, nt))
    A = blocked_model(I, T, p.block, p.hop, p.pairs)
    ref = oracle.fdmt(I, T)
    assert np.max(np.abs(A - ref)) <= 1e-9 * (1 + np.max(np.abs(ref)))

"""STFT filterbank front end (``fdmt_filterbank``, section 2) against the
oracle's float64 ``stft_filterbank``, through the C ABI.

Bar: a float32 radix-2 FFT of Nf points errs by at most about
2 eps log2(Nf) ||X|| per bin (eps = 2^-24), so a squared magnitude errs by at
most about 4 eps log2(Nf) times the spectrum's total power (Parseval); the
tests allow twice that per output sample (binned spectra add their powers).
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def volts(seed, n):
    rng = np.random.Generator(np.random.PCG64([seed, n, 23]))
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)


def check(got, v, nf, nbin):
    ref = oracle.stft_filterbank(v.astype(np.complex128), nf, nbin)
    assert got.shape == ref.shape
    bound = 8 * EPS * max(1, int(np.log2(nf))) * ref.sum(axis=0)
    err = np.abs(got.astype(np.float64) - ref)
    bad = np.argwhere(err > bound[None, :])
    assert bad.size == 0, f"{bad[:4].tolist()}: {err[tuple(bad[0])]} > {bound[bad[0][1]]}"


@pytest.mark.parametrize("nf,nbin,nt", [(2, 1, 37), (16, 1, 100), (32, 1, 50), (64, 1, 33), (128, 1, 20),
                                        (64, 3, 41), (1024, 1, 70), (1024, 4, 9), (4096, 1, 5), (256, 2, 1),
                                        (2048, 1, 3)])
def test_filterbank_matches_oracle(nf, nbin, nt):
    v = volts(nf + nbin, nt * nf * nbin + 5)  # a few trailing samples are not read
    got = FD.filterbank(torch.from_numpy(v).cuda(), nf, nbin).cpu().numpy()
    check(got, v, nf, nbin)


def test_filterbank_tone_and_order():
    nf, nt = 256, 32
    n = np.arange(nf * nt)
    for q, a in ((7, 1.0), (-5, 0.5), (-128, 2.0)):
        v = (a * np.exp(2j * np.pi * q * n / nf)).astype(np.complex64)
        got = FD.filterbank(torch.from_numpy(v).cuda(), nf).cpu().numpy().astype(np.float64)
        c = (q + nf // 2) % nf
        assert np.allclose(got[c], a * a * nf * nf, rtol=1e-4)
        assert np.max(np.delete(got, c, axis=0)) <= 1e-4 * a * a * nf * nf


def test_filterbank_then_transform():
    """The front end feeding the transform (float32 plan) against the oracle
    chain in float64: within 1e-5 of each output row's RMS."""
    nf, nt, nd = 64, 1024, 64
    v = volts(7, nf * nt)
    x = FD.filterbank(torch.from_numpy(v).cuda(), nf)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32")
    got = p.execute(x).cpu().numpy().astype(np.float64)
    I = oracle.stft_filterbank(v.astype(np.complex128), nf)
    ref = oracle.fdmt(I, oracle.build_tables(1200.0, 1600.0, nf, nd), "f64")
    rms = np.sqrt(np.mean(ref ** 2, axis=1))
    assert np.all(np.max(np.abs(got - ref), axis=1) <= 1e-5 * rms)


def test_filterbank_full_size():
    """64 M complex samples into the Nf = 1024, Nt = 65536 input of the
    headline transform, compared in full."""
    nf, nt = 1024, 1 << 16
    v = volts(fs.SEED_BASE + 60, nf * nt)
    got = FD.filterbank(torch.from_numpy(v).cuda(), nf).cpu().numpy()
    check(got, v, nf, 1)

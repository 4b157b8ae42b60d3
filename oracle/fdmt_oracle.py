"""Plain CPU oracle for the Fast Dispersion Measure Transform (FDMT).

Zackay & Ofek, "An accurate and efficient algorithm for detection of radio
bursts with an unknown dispersion measure" (arXiv:1411.5373).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` use it.  It shares no code with the CUDA library (its own
table builder, its own loops) and is deliberately slow and literal: every loop
follows the paper's Algorithm 1 in the paper's order, with numpy vector row
additions as the only library primitive (the paper's Fig. 2 caption says the
rows add as vectors).

Notation (section 4 of the paper):
  Nf  number of frequency channels, channel 0 at f_min (ascending)
  Nt  number of time samples per channel, t contiguous
  Nd  number of output delay rows; row d is the curve whose total delay across
      the whole band is d samples (the paper's N_Delta)
  A[d][t] sum along the discretised curve of total delay d that arrives at the
      lowest frequency f_min at time t  (Eq. "parametrization")

Readings of the paper taken here (the paper is silent or inconsistent):
  * Edge model: channel k spans [e_k, e_{k+1}] with
    e_k = f_min + (f_max - f_min) * k / Nf  (delta_f of section 4).
    Band (l, b) spans channels [b 2^l, (b+1) 2^l); its merge point f1 is the
    border between its two halves (section 4.2, "N_f != 2^k" paragraph);
    the printed f1 = (f2 - f0)/2 is a typo.
  * Rounding: the lower sub-band row is dl = floor(C * Dt + 0.5) computed in
    FP64, C from Eq. (C_{f2,f0}); the upper sub-band is read at row Dt - dl
    and time t - dl (one C per merge).
  * Initialisation (Option 1 of section 4) sums backwards in time,
    A0[k][j][t] = sum_{i=0..j} I[k][t-i], the sign that Eq. "parametrization"
    and t1 = t0 - C Dt fix; the printed forward sum I(f, t+i) is read as a
    sign slip.
  * The copy rule (t1 < 0) equals treating every input and partial sum as
    zero before t = 0.
  * Exactly Nd output rows d = 0..Nd-1.  Sub-band row extents are sized top
    down: a band holds exactly the rows its parent reads.

Parity pins (tests/test_oracle_*.py): recursion == brute force along the
unrolled curves (exhaustive small sizes); hand-derived worked example
(tests/golden/); d = 0 row equals the channel sum; constant-input closed form;
impulse response; linearity; time-shift equivariance; weighted flux; curve
offsets within a rounding bound of the ideal f^-2 law; adjoint dot-product
identity and dense transpose; boxcar search; the d_min input map; FFT-FDMT
(Algorithm 2) against the direct transform, the cyclic brute force without
padding, and two packed instances.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "OracleTables",
    "band_edge",
    "merge_coefficient",
    "build_tables",
    "fdmt",
    "curve_offsets",
    "bruteforce",
    "fdmt_adjoint",
    "ideal_delay_fraction",
    "boxcar_search",
    "input_shifts",
    "map_input",
    "map_input_adjoint",
    "stft_filterbank",
    "shift_vector",
    "fft_fdmt",
]


def band_edge(f_min: float, f_max: float, nf: int, k: int) -> float:
    """Frequency of channel edge k (section 4: delta_f = (f_max - f_min)/N_f).

    Evaluated in FP64 as f_min + ((f_max - f_min) * k) / nf.
    """
    return f_min + (f_max - f_min) * k / nf


def _power(f: float, gamma: float) -> float:
    # f^gamma in FP64; the dispersion law's f^-2 as 1 / (f f)
    return 1.0 / (f * f) if gamma == -2.0 else f ** gamma


def merge_coefficient(f0: float, f1: float, f2: float, gamma: float = -2.0) -> float:
    """C_{f2,f0} of Eq. (C_{f2,f0}): where the curve crosses the merge point.

    C = (f0^-2 - f1^-2) / (f0^-2 - f2^-2), the fraction of the band's total
    delay spent in the lower sub-band.  FP64, evaluated in exactly this order.
    For other functional forms Dt ~ f^gamma (section 4.2, "Applying FDMT for
    other functional forms") the power -2 becomes gamma.
    """
    i0 = _power(f0, gamma)
    i1 = _power(f1, gamma)
    i2 = _power(f2, gamma)
    return (i0 - i1) / (i0 - i2)


def ideal_delay_fraction(f_min: float, f_max: float, f: float, gamma: float = -2.0) -> float:
    """Delay at frequency f relative to f_min, as a fraction of the band's
    total delay (Eq. DtD with the dispersion constants absorbed into d; the
    power -2 becomes gamma for other functional forms)."""
    return (_power(f_min, gamma) - _power(f, gamma)) / (_power(f_min, gamma) - _power(f_max, gamma))


@dataclass
class OracleTables:
    """Per-level, per-band row extents and lower-row tables.

    rows[l][b]  number of delay rows held by band b at level l
                (level 0: single channels; level L = ceil(log2 Nf): whole band)
    dl[l][b]    for l >= 1: int64 array of length rows[l][b]; dl[l][b][Dt] is
                the lower sub-band row (and the time shift of the upper one);
                for a band with no upper sub-band (Nf not a power of two,
                the band passes up unchanged) dl[l][b][Dt] = Dt
    coef[l][b]  the FP64 C of that merge (None for a band passed up)

    Band b of level l covers channels [b 2^l, min((b+1) 2^l, Nf)); it merges
    bands 2b and 2b+1 of level l-1 when the latter exists.
    """

    f_min: float
    f_max: float
    nf: int
    nd: int
    levels: int
    rows: list = field(default_factory=list)
    dl: list = field(default_factory=list)
    coef: list = field(default_factory=list)

    def level_rows(self, l: int) -> int:
        return int(sum(self.rows[l]))

    def has_upper(self, l: int, b: int) -> bool:
        """Band b of level l >= 1 merges two sub-bands (else it is passed up)."""
        return 2 * b + 1 < len(self.rows[l - 1])


def build_tables(f_min: float, f_max: float, nf: int, nd: int, gamma: float = -2.0) -> OracleTables:
    """Delay tables of Algorithm 1, built top-down in FP64.

    For each iteration i (paper) = level l here, each band f0 with
    f2 = f0 + 2^l delta_f and merge point f1 = f0 + 2^(l-1) delta_f,
    Dt runs over the rows the parent needs and the lower row is
    dl = floor(C Dt + 1/2) (section 4 addition rule, t1 = t0 - C Dt).
    gamma: the curves' power law Dt ~ f^gamma (-2: dispersion; section 4.2).

    Nf not a power of two (section 4.2: the split is unequal and f1 is the
    border frequency): the top band's upper edge is f_max = e_Nf, so a band
    starting at channel b 2^l ends at min((b+1) 2^l, Nf); its merge point is
    still the border after 2^(l-1) channels, and a band with no channel above
    that border holds its single sub-band's rows unchanged.
    """
    if not (0.0 < f_min < f_max):
        raise ValueError("need 0 < f_min < f_max")
    if not (math.isfinite(gamma) and gamma != 0.0):
        raise ValueError("gamma must be finite and nonzero")
    if nf < 2:
        raise ValueError("Nf must be >= 2")
    if nd < 1:
        raise ValueError("Nd must be >= 1")
    L = (nf - 1).bit_length()  # ceil(log2 Nf)
    rows = [None] * (L + 1)
    dl = [None] * (L + 1)
    coef = [None] * (L + 1)
    rows[L] = [nd]
    for l in range(L, 0, -1):
        nb = (nf + (1 << l) - 1) >> l
        nb_child = (nf + (1 << (l - 1)) - 1) >> (l - 1)
        rows[l - 1] = [0] * nb_child
        dl[l] = [None] * nb
        coef[l] = [None] * nb
        for b in range(nb):
            r = rows[l][b]
            k0, k1 = b << l, (b << l) + (1 << (l - 1))
            if k1 >= nf:  # no upper sub-band: the band passes up unchanged
                dl[l][b] = np.arange(r, dtype=np.int64)
                rows[l - 1][2 * b] = r
                continue
            f0 = band_edge(f_min, f_max, nf, k0)
            f1 = band_edge(f_min, f_max, nf, k1)
            f2 = band_edge(f_min, f_max, nf, min((b + 1) << l, nf))
            c = merge_coefficient(f0, f1, f2, gamma)
            lo = np.empty(r, dtype=np.int64)
            for dt in range(r):
                lo[dt] = math.floor(c * float(dt) + 0.5)
            dl[l][b] = lo
            coef[l][b] = c
            top = r - 1
            rows[l - 1][2 * b] = int(lo[top]) + 1
            rows[l - 1][2 * b + 1] = top - int(lo[top]) + 1
    return OracleTables(f_min, f_max, nf, nd, L, rows, dl, coef)


def _shifted(x: np.ndarray, s: int) -> np.ndarray:
    """y[t] = x[t - s] for t >= s, else 0 (the copy rule as zero padding)."""
    y = np.zeros_like(x)
    if s < x.shape[-1]:
        y[..., s:] = x[..., : x.shape[-1] - s]
    return y


_MODES = ("f64", "f32", "i64", "f16state")


def fdmt(I: np.ndarray, tables: OracleTables, mode: str = "f64",
         weights: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 1 of the paper, literally: Option-1 initialisation, then
    log2(Nf) iterations of the addition rule over bands, Dt and t0.

    mode:
      "f64"      all arithmetic in float64
      "f32"      float32 with this exact association: init row j = row j-1 +
                 I[t-j]; each merge is one add lo + hi.  With weights the
                 input is first multiplied by w[k] in float32.
      "i64"      integer input, int64 accumulation
      "f16state" float32 arithmetic as "f32" but every stored partial state
                 (level 0 .. L-1) is rounded to float16; the last level's
                 output is float32.
    Returns A with shape (Nd, Nt).
    """
    if mode not in _MODES:
        raise ValueError(mode)
    nf, nt = I.shape
    if nf != tables.nf:
        raise ValueError("input rows != Nf")
    acc = {"f64": np.float64, "f32": np.float32, "i64": np.int64,
           "f16state": np.float32}[mode]
    X = I.astype(acc)
    if weights is not None:
        if mode == "i64":
            raise ValueError("weights are for floating-point modes")
        X = X * np.asarray(weights, dtype=acc)[:, None]

    def store(a):
        if mode == "f16state":
            return a.astype(np.float16)
        return a

    def load(a):
        if mode == "f16state":
            return a.astype(np.float32)
        return a

    L = tables.levels
    # Initialisation, Option 1: A_f^{f+df}(t, Dt) = sum_{i=0..Dt} I(f, t-i).
    state = []
    for k in range(nf):
        w = tables.rows[0][k]
        rows_k = []
        run = X[k].copy()
        rows_k.append(store(run.copy()))
        for j in range(1, w):
            run = run + _shifted(X[k], j)
            rows_k.append(store(run.copy()))
        state.append(rows_k)
    # Iterations i = 1 .. ceil(log2 Nf).
    for l in range(1, L + 1):
        nxt = []
        for b in range(len(tables.rows[l])):
            lo_band = state[2 * b]
            out_rows = []
            if not tables.has_upper(l, b):  # passed up unchanged
                for dt in range(tables.rows[l][b]):
                    v = load(lo_band[dt])
                    out_rows.append(v if l == L else store(v))
                nxt.append(out_rows)
                continue
            hi_band = state[2 * b + 1]
            for dt in range(tables.rows[l][b]):
                j = int(tables.dl[l][b][dt])
                lo = load(lo_band[j])
                hi = load(hi_band[dt - j])
                # t0 >= C Dt: both halves; t0 < C Dt: copy the lower half.
                v = lo + _shifted(hi, j)
                out_rows.append(v if l == L else store(v))
            nxt.append(out_rows)
        state = nxt
    out = np.stack(state[0], axis=0)
    return out.astype(np.float32 if mode == "f16state" else acc)


def curve_offsets(tables: OracleTables, d: int) -> np.ndarray:
    """Unroll output row d into the channel-edge offsets o_0..o_Nf.

    The curve of row d enters channel k at time t - o_k and leaves it at
    t - o_{k+1}; it covers samples t - o for o in [o_k, o_{k+1}] of channel k.
    Follows the addition rule: the lower half keeps the arrival time, the
    upper half arrives dl samples earlier and carries row Dt - dl.
    """
    nf = tables.nf
    o = np.zeros(nf + 1, dtype=np.int64)
    stack = [(tables.levels, 0, d, 0)]
    while stack:
        l, b, dt, base = stack.pop()
        if l == 0:
            o[b] = base
            o[b + 1] = base + dt
            continue
        if not tables.has_upper(l, b):
            stack.append((l - 1, 2 * b, dt, base))
            continue
        j = int(tables.dl[l][b][dt])
        stack.append((l - 1, 2 * b, j, base))
        stack.append((l - 1, 2 * b + 1, dt - j, base + j))
    return o


def bruteforce(I: np.ndarray, tables: OracleTables, dtype=np.float64) -> np.ndarray:
    """Eq. "parametrization" evaluated directly along the discretised curves:
    A[d][t] = sum_k sum_{o = o_k(d)}^{o_{k+1}(d)} I[k][t - o], zero before t = 0.
    Cost Nd * Nf * Nt * (mean sweep): for tiny inputs only."""
    nf, nt = I.shape
    X = I.astype(dtype)
    A = np.zeros((tables.nd, nt), dtype=dtype)
    for d in range(tables.nd):
        o = curve_offsets(tables, d)
        for k in range(nf):
            for off in range(int(o[k]), int(o[k + 1]) + 1):
                A[d] += _shifted(X[k], off)
    return A


def _shifted_back(x: np.ndarray, s: int) -> np.ndarray:
    """Adjoint of _shifted: y[u] = x[u + s] for u + s < Nt, else 0."""
    y = np.zeros_like(x)
    n = x.shape[-1]
    if s < n:
        y[..., : n - s] = x[..., s:]
    return y


def fdmt_adjoint(G: np.ndarray, tables: OracleTables) -> np.ndarray:
    """Transpose of the FDMT linear map (not in the paper; derived from the
    addition rule and Option-1 initialisation), in float64, scatter form.

    Levels L..1: for each parent row Dt with lower row j = dl:
      gLo[j][t] += G[Dt][t];   gHi[Dt - j][u] += G[Dt][u + j]  (u + j < Nt).
    Initialisation: gI[k][s] += gA0[k][j][s + i] for 0 <= i <= j, s + i < Nt.
    Returns gI with shape (Nf, Nt).
    """
    nd, nt = G.shape
    if nd != tables.nd:
        raise ValueError("grad rows != Nd")
    L = tables.levels
    grad = [[G[d].astype(np.float64) for d in range(nd)]]
    for l in range(L, 0, -1):
        nb = len(tables.rows[l])
        child = []
        for b in range(nb):
            glo = [np.zeros(nt) for _ in range(tables.rows[l - 1][2 * b])]
            if not tables.has_upper(l, b):  # passed up unchanged
                for dt in range(tables.rows[l][b]):
                    glo[dt] += grad[b][dt]
                child.append(glo)
                continue
            ghi = [np.zeros(nt) for _ in range(tables.rows[l - 1][2 * b + 1])]
            for dt in range(tables.rows[l][b]):
                j = int(tables.dl[l][b][dt])
                g = grad[b][dt]
                glo[j] += g
                ghi[dt - j] += _shifted_back(g, j)
            child.append(glo)
            child.append(ghi)
        grad = child
    gI = np.zeros((tables.nf, nt))
    for k in range(tables.nf):
        for j, g in enumerate(grad[k]):
            for i in range(j + 1):
                gI[k] += _shifted_back(g, i)
    return gI


def boxcar_search(A: np.ndarray, n_widths: int):
    """Boxcar search of an FDMT output (section 4.2, "Pulse profile": a
    uniform pulse profile convolved with the time axis commutes with the
    whole transform, so several widths are tested on one output).

    For width w = 2^k, k < n_widths, and every row d:
        B_w[d][t] = sum_{i=0}^{w-1} A[d][t - i]   (A = 0 before t = 0),
    summed as a binary tree: float32 outputs in float32, integer outputs in
    int64 (an exact sum of integers, as the transform's own sums are):
    B_1 = A, B_{2w}[t] = B_w[t] + B_w[t - w].  Returns (peak, time), each
    [Nd][n_widths]: peak = max over t in [0, Nt) of B_w[d][t], time = the
    first t where it is reached.
    """
    if not 1 <= n_widths <= 16:
        raise ValueError("n_widths must be in 1..16")
    A = np.asarray(A)
    B = A.astype(np.int64) if np.issubdtype(A.dtype, np.integer) else A.copy()
    nd, nt = A.shape
    peak = np.zeros((nd, n_widths), dtype=B.dtype)
    time = np.zeros((nd, n_widths), dtype=np.int32)
    w = 1
    for k in range(n_widths):
        if k > 0:
            B = B + _shifted(B, w)
            w *= 2
        time[:, k] = np.argmax(B, axis=1)  # the first maximum
        peak[:, k] = B[np.arange(nd), time[:, k]]
    return peak, time


def input_shifts(f_min: float, f_max: float, nf: int, d_min: int, gamma: float = -2.0) -> np.ndarray:
    """Per-channel delay of the d_min pre-shift (section 4.2: to scan delays
    from d_min, the input is first shifted by the delay of d_min, so that row
    d of the transform follows total delay d_min + d).

    Reading: channel k is delayed by the ideal delay of its lower edge,
    s_k = floor(d_min r(e_k) + 1/2), r the delay fraction of the curve
    family; FP64, evaluated as written.
    """
    return np.array([int(math.floor(d_min * ideal_delay_fraction(f_min, f_max, band_edge(f_min, f_max, nf, k), gamma)
                                    + 0.5)) for k in range(nf)], dtype=np.int64)


def map_input(I: np.ndarray, shifts, descending: bool = False) -> np.ndarray:
    """The transform's input from the raw rows: I'[k][t] = I[src(k)][t - s_k]
    (zero for t < s_k, the copy rule), src(k) = k for ascending rows and
    Nf - 1 - k when row 0 holds the highest channel."""
    I = np.asarray(I)
    nf = I.shape[0]
    out = np.zeros_like(I)
    for k in range(nf):
        src = nf - 1 - k if descending else k
        out[k] = _shifted(I[src], int(shifts[k]))
    return out


def map_input_adjoint(G: np.ndarray, shifts, descending: bool = False) -> np.ndarray:
    """Transpose of map_input: raw[src(k)][u] = G[k][u + s_k] (zero past the
    last sample)."""
    G = np.asarray(G)
    nf = G.shape[0]
    out = np.zeros_like(G)
    for k in range(nf):
        src = nf - 1 - k if descending else k
        out[src] = _shifted_back(G[k], int(shifts[k]))
    return out


def stft_filterbank(v: np.ndarray, nf: int, nbin: int = 1) -> np.ndarray:
    """The front end of section 2: the voltage series is cut into blocks of
    Nf samples, each block is Fourier transformed (STFT) and the squared
    magnitude at each frequency kept; the footnote's optional binning sums
    nbin consecutive spectra.

    Reading: complex (baseband) voltages, so a block gives Nf channels;
    channels are returned in ascending frequency, negative offsets first
    (channel c holds DFT bin (c + Nf/2) mod Nf).  Returns float64 [Nf][Nt]
    with Nt = len(v) // (Nf nbin); trailing samples are dropped.  The DFT is
    numpy's FFT in float64 (a library step).
    """
    v = np.asarray(v, dtype=np.complex128)
    nt = len(v) // (nf * nbin)
    blocks = v[: nt * nbin * nf].reshape(nt * nbin, nf)
    P = np.abs(np.fft.fft(blocks, axis=1)) ** 2
    P = np.concatenate([P[:, nf // 2:], P[:, : nf // 2]], axis=1)  # ascending frequency
    return P.reshape(nt, nbin, nf).sum(axis=1).T.copy()


def shift_vector(s: int, n: int) -> np.ndarray:
    """Algorithm 2's shift vector V(., s): the Fourier transform (length n) of
    a vector holding one at position s and zeros elsewhere (numpy's FFT, a
    library step).  Multiplying a transformed row by it delays the row by s
    samples, cyclically."""
    delta = np.zeros(n, dtype=np.complex128)
    delta[s % n] = 1.0
    return np.fft.fft(delta)


def fft_fdmt(I: np.ndarray, tables: OracleTables, n_fft: int | None = None) -> np.ndarray:
    """FFT-FDMT, Algorithm 2 (section 5), in complex128, step by step:

      1. Option-1 initialisation in time (backward sums, the same reading as
         ``fdmt``);
      2. shift vectors V(., s) = FFT(delta_s) for every shift s a merge uses;
      3. Fourier transform of every initial row along time, after zero
         padding to n_fft samples (the zero-padding paragraph: shifts become
         cyclic, so n_fft >= Nt + Nd - 1 keeps every sum off the wrap; the
         default is the next power of two of that);
      4. (transpose: a layout step, nothing to compute here);
      5. the iterations of Algorithm 1 with the shifted addition replaced by
         a product with the shift vector, the same for every Fourier bin:
         B_band[Dt] = B_lo[dl] + B_hi[Dt - dl] V(., dl)   (vectors over bins);
      6. (transpose back);
      7. inverse Fourier transform along time, first Nt samples.

    Complex input packs two instances (the machine-word paragraph): the
    transform is real-linear, so real and imaginary parts of the result are
    the transforms of the real and imaginary parts of I.  Returns complex128
    [Nd][Nt] for complex input, float64 (the real part) for real input.
    With n_fft < Nt + Nd - 1 the result is the cyclic transform of the first
    n_fft samples (inputs past n_fft are not read)."""
    nf, nt = I.shape
    if nf != tables.nf:
        raise ValueError("input rows != Nf")
    complex_in = np.iscomplexobj(I)
    if n_fft is None:
        need = nt + tables.nd - 1
        n_fft = 1 << (need - 1).bit_length()
    if n_fft < 1:
        raise ValueError("n_fft must be >= 1")
    X = np.zeros((nf, n_fft), dtype=np.complex128)
    m = min(nt, n_fft)
    X[:, :m] = I[:, :m]
    L = tables.levels
    # Step 1: A_f(t, Dt) = sum_{i=0..Dt} I(f, t - i), cyclic in the n_fft frame
    # (zeros before t = 0 come from the padding).
    init = []
    for k in range(nf):
        rows_k, run = [], X[k].copy()
        rows_k.append(run.copy())
        for j in range(1, tables.rows[0][k]):
            run = run + np.roll(X[k], j)
            rows_k.append(run.copy())
        init.append(rows_k)
    # Step 2: shift vectors, one per distinct shift.
    V = {}

    def vec(s):
        if s not in V:
            V[s] = shift_vector(s, n_fft)
        return V[s]

    # Step 3: transform every initial row along time.
    state = [[np.fft.fft(r) for r in rows_k] for rows_k in init]
    # Step 5: the merges, bin-wise.
    for l in range(1, L + 1):
        nxt = []
        for b in range(len(tables.rows[l])):
            lo_band = state[2 * b]
            if not tables.has_upper(l, b):
                nxt.append([lo_band[dt] for dt in range(tables.rows[l][b])])
                continue
            hi_band = state[2 * b + 1]
            out_rows = []
            for dt in range(tables.rows[l][b]):
                j = int(tables.dl[l][b][dt])
                out_rows.append(lo_band[j] + hi_band[dt - j] * vec(j))
            nxt.append(out_rows)
        state = nxt
    # Step 7: back to time.
    A = np.stack([np.fft.ifft(r) for r in state[0]], axis=0)[:, :m]
    if m < nt:
        A = np.concatenate([A, np.zeros((A.shape[0], nt - m), dtype=A.dtype)], axis=1)
    return A if complex_in else A.real.copy()

"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pin suite catches every one: a dropped term, a wrong sign, an off-by-one
index, a transposed operand, the paper's printed typos.

Each mutation is a textual replacement in the oracle's source; the mutated
copy is loaded as a fresh module and must fail at least one pin.
"""
import importlib.util
import os
import sys
import types

import pytest

import oracle.fdmt_oracle as real
from oracle_pins import ALL_PINS

SRC_PATH = real.__file__

MUTATIONS = [
    ("fft_shift_vector_advances",
     "delta[s % n] = 1.0", "delta[-s % n] = 1.0"),
    ("fft_no_zero_padding",
     "n_fft = 1 << (need - 1).bit_length()", "n_fft = nt"),
    ("fft_lower_band_shifted",
     "out_rows.append(lo_band[j] + hi_band[dt - j] * vec(j))",
     "out_rows.append(lo_band[j] * vec(j) + hi_band[dt - j])"),
    ("fft_upper_row_index",
     "out_rows.append(lo_band[j] + hi_band[dt - j] * vec(j))",
     "out_rows.append(lo_band[j] + hi_band[max(dt - j - 1, 0)] * vec(j))"),
    ("fft_init_forward_sum",
     "run = run + np.roll(X[k], j)", "run = run + np.roll(X[k], -j)"),
    ("fft_packed_real_only",
     "return A if complex_in else A.real.copy()", "return A.real.copy()"),
    ("stft_not_ascending",
     "P = np.concatenate([P[:, nf // 2:], P[:, : nf // 2]], axis=1)  # ascending frequency", "P = P"),
    ("stft_bins_averaged",
     "return P.reshape(nt, nbin, nf).sum(axis=1).T.copy()", "return P.reshape(nt, nbin, nf).mean(axis=1).T.copy()"),
    ("stft_magnitude_not_squared",
     "P = np.abs(np.fft.fft(blocks, axis=1)) ** 2", "P = np.abs(np.fft.fft(blocks, axis=1))"),
    ("unequal_split_at_midpoint",
     "k0, k1 = b << l, (b << l) + (1 << (l - 1))",
     "k0, k1 = b << l, (b << l) + (min((b + 1) << l, nf) - (b << l)) // 2"),
    ("unequal_split_ignores_nf_edge",
     "f2 = band_edge(f_min, f_max, nf, min((b + 1) << l, nf))", "f2 = band_edge(f_min, f_max, nf, (b + 1) << l)"),
    ("input_shift_wrong_direction",
     "out[k] = _shifted(I[src], int(shifts[k]))", "out[k] = _shifted_back(I[src], int(shifts[k]))"),
    ("input_shift_upper_edge",
     "ideal_delay_fraction(f_min, f_max, band_edge(f_min, f_max, nf, k), gamma)",
     "ideal_delay_fraction(f_min, f_max, band_edge(f_min, f_max, nf, k + 1), gamma)"),
    ("descending_not_reversed",
     "src = nf - 1 - k if descending else k", "src = k"),
    ("input_map_adjoint_unshifted",
     "out[src] = _shifted_back(G[k], int(shifts[k]))", "out[src] = G[k]"),
    ("boxcar_window_one_short",
     "B = B + _shifted(B, w)", "B = B + _shifted(B, w - 1 if w > 1 else 1)"),
    ("boxcar_last_maximum",
     "time[:, k] = np.argmax(B, axis=1)  # the first maximum",
     "time[:, k] = nt - 1 - np.argmax(B[:, ::-1], axis=1)"),
    ("boxcar_adds_input_not_partial",
     "B = B + _shifted(B, w)", "B = B + _shifted(A, w)"),
    ("gamma_ignored",
     "return 1.0 / (f * f) if gamma == -2.0 else f ** gamma", "return 1.0 / (f * f)"),
    ("gamma_sign_flipped",
     "return 1.0 / (f * f) if gamma == -2.0 else f ** gamma", "return 1.0 / (f * f) if gamma == -2.0 else f ** -gamma"),
    ("round_down_not_half_up",
     "math.floor(c * float(dt) + 0.5)", "math.floor(c * float(dt))"),
    ("coefficient_upper_subband",
     "return (i0 - i1) / (i0 - i2)", "return (i1 - i2) / (i0 - i2)"),
    ("printed_midpoint_typo",
     "f1 = band_edge(f_min, f_max, nf, k1)",
     "f1 = (band_edge(f_min, f_max, nf, min((b + 1) << l, nf)) - band_edge(f_min, f_max, nf, k0)) / 2 + 1e-9"),
    ("point_model_upper_edge",
     "f2 = band_edge(f_min, f_max, nf, min((b + 1) << l, nf))",
     "f2 = band_edge(f_min, f_max, nf, min((b + 1) << l, nf) - 1)"),
    ("upper_shift_off_by_one",
     "v = lo + _shifted(hi, j)", "v = lo + _shifted(hi, j + 1)"),
    ("upper_term_dropped",
     "v = lo + _shifted(hi, j)", "v = lo + 0 * hi"),
    ("upper_not_shifted",
     "v = lo + _shifted(hi, j)", "v = lo + hi"),
    ("subbands_transposed",
     "hi_band = state[2 * b + 1]",
     "hi_band, lo_band = state[2 * b], state[2 * b + 1]"),
    ("init_forward_sum_as_printed",
     "run = run + _shifted(X[k], j)", "run = run + _shifted_back(X[k], j)"),
    ("init_row_missing_sample",
     "for j in range(1, w):\n            run = run + _shifted(X[k], j)",
     "for j in range(1, w):\n            run = run + _shifted(X[k], j) * (j < w - 1)"),
    ("upper_row_index",
     "hi = load(hi_band[dt - j])", "hi = load(hi_band[max(dt - j - 1, 0)])"),
    ("f32_mode_in_f64",
     '"f32": np.float32, "i64"', '"f32": np.float64, "i64"'),
    ("f16_state_not_rounded",
     "            return a.astype(np.float16)\n", "            return a\n"),
    ("unroll_upper_base",
     "stack.append((l - 1, 2 * b + 1, dt - j, base + j))",
     "stack.append((l - 1, 2 * b + 1, dt - j, base + j + 1))"),
    ("adjoint_shift_off_by_one",
     "ghi[dt - j] += _shifted_back(g, j)", "ghi[dt - j] += _shifted_back(g, j + 1)"),
    ("adjoint_upper_unshifted",
     "ghi[dt - j] += _shifted_back(g, j)", "ghi[dt - j] += g"),
    ("adjoint_init_short",
     "for i in range(j + 1):", "for i in range(j):"),
    ("weights_ignored",
     "X = X * np.asarray(weights, dtype=acc)[:, None]", "X = X"),
]


def _load_mutant(old, new):
    src = open(SRC_PATH).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    src = src.replace(old, new, 1)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = SRC_PATH
    sys.modules["oracle_mutant"] = mod
    try:
        exec(compile(src, SRC_PATH + "<mutant>", "exec"), mod.__dict__)
    finally:
        sys.modules.pop("oracle_mutant", None)
    return mod


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, old, new):
    mutant = _load_mutant(old, new)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(mutant)
        except Exception as exc:  # AssertionError, or the mutant crashing
            caught.append((pin.__name__, type(exc).__name__))
    assert caught, f"no pin caught mutation {name}"

"""CPU oracle for the FDMT (test infrastructure only; never on the product path).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline and
reference legs may import this package.
"""
from .fdmt_oracle import (  # noqa: F401
    OracleTables,
    band_edge,
    boxcar_search,
    bruteforce,
    build_tables,
    curve_offsets,
    fdmt,
    fdmt_adjoint,
    fft_fdmt,
    ideal_delay_fraction,
    input_shifts,
    map_input,
    map_input_adjoint,
    merge_coefficient,
    shift_vector,
    stft_filterbank,
)

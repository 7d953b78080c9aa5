"""FP64 CPU oracle for ATSFFT -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product library (paper_1908_02461_gb300) never imports it and
shares no code with it.
"""

from .oracle import (  # noqa: F401
    OracleParams,
    OracleResult,
    build,
    lib,
    default_params,
    splitmix64_stream,
    hash_params,
    inv_mod,
    filter_taps,
    filter_response,
    fft,
    hash_spectrum_1d,
    hash_spectrum_2d,
    local_maxima,
    controller_branch,
    top_num,
    median_componentwise,
    atsfft_1d,
    atsfft_2d,
    atsfft_log,
    estimates_1d,
    local_maxima_log,
    location_select_log,
    bucket_of,
    Decision,
    DEC_KIND,
)

"""CPU oracle for the SGM hot path (test infrastructure only).

The oracle is the plain C program in ``sgm_oracle.c``.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may use it; the product path
never imports it.  Build it with ``build()`` (gcc, no GPU needed).
"""
from .oracle import (  # noqa: F401
    build,
    load,
    csct,
    csct_at,
    bitcount,
    cost,
    ct62,
    ct62_at,
    bitcount64,
    cost64,
    aggregate,
    directions,
    wta,
    median3x3,
    sgm,
    sgm_threads,
    sgm_ex,
    aggregate_ex,
    subpixel,
    median3x3_u16,
    POST_SUBPIXEL,
    POST_LR_CHECK,
    POST_ADAPTIVE_P2,
    DISP16_INVALID,
    pixel,
    disp_at,
)

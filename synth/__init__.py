"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package only *makes inputs*: original fields f, decompressed stand-ins
f_hat and the absolute error bound xi.  It holds none of the correction's
arithmetic (no neighbour search, no classification, no edits), so the oracle
and the CUDA library can both be fed from it without sharing method code.
"""
from .fields import (  # noqa: F401
    gaussian_bumps,
    multi_octave,
    xi_from_relative,
    fhat_quantised,
    fhat_uniform,
    clamp_into_bound,
    make_case,
    make_cases_cpu,
    batched_specs,
    serving_requests,
    WORKLOADS,
)

"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds only input data: the Potjans-Diesmann parameter tables as the
paper prints them (Tables params, params2, params3 of §2.2), the readings taken where
the paper is ambiguous, and named workload presets (scales, seeds, step counts).
It contains none of the method's arithmetic: propagators, pair counts, Poisson
tables, fixed-point conversion, network sampling and the step recurrence are each
implemented independently by the oracle (``oracle/``) and by the library.
"""

from .microcircuit import (  # noqa: F401
    POP_NAMES,
    Model,
    Workload,
    WORKLOADS,
    microcircuit_model,
    batched_workloads,
)

"""Seeded synthetic inputs shared by the tests, the bench and the oracle's tests.

This package holds workload parameter tables (domains, boundary kinds, sizes,
initial-condition names) and seeded random generators. It holds none of the
method's arithmetic: every initial condition, flux, ghost rule and mesh rule
is implemented separately by the oracle (``oracle/``) and by the CUDA library.
"""
from .workloads import WORKLOADS, workload, reduced  # noqa: F401
from .rng import seeded_normal, seeded_uniform, mlp_init  # noqa: F401

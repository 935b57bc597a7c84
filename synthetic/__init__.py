"""Seeded synthetic workloads for the multinomial-logit SPS.

This package only draws inputs: covariate matrices X, outcomes y, particle sets and random
numbers. It holds none of the simulator's arithmetic, so both the CPU oracle (``oracle/``) and
the CUDA library (``paper_1304_4333_b300/``) can be fed from it without sharing any code.
"""
from .configs import (  # noqa: F401
    Workload,
    CONFIG_NAMES,
    make_workload,
    make_c1,
    make_c2,
    make_c3,
    make_c4,
    make_c5,
    particles_around,
    prior_draws,
)

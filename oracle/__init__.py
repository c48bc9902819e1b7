"""FP64 CPU oracle of the lattice-Boltzmann Maxwell scheme (arXiv:1108.2651).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.
"""
from .oracle import (Oracle, medium, init_state, run, fields, diagnostics, adjoint, threads, set_threads,  # noqa: F401
                     time_fp32,
                     PERIODIC, PEC, PMC, pole_state)

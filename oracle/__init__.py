"""CPU oracle (FP64 numpy) for the spectral-element Poisson hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the CUDA library.
"""
from .sem_oracle import *  # noqa: F401,F403

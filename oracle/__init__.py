"""FP64 CPU oracle of the fixed-step cable-network engine.

TEST INFRASTRUCTURE ONLY.  Used by the tests, the smoke check and the
benchmark's CPU-baseline leg to produce expected results.  The CUDA engine
does not import, link or execute anything in this package.
"""
from .oracle import OracleModel, simulate, hines_solve, build_oracle, adjoint, KIND

__all__ = ["OracleModel", "simulate", "hines_solve", "build_oracle", "adjoint", "KIND"]

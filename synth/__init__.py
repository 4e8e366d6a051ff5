"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the oracle.

This package holds input construction only (operators, right-hand sides, start vectors,
random fields): none of the Gram-Schmidt, Arnoldi, GMRES or Krylov-Schur arithmetic lives
here, so both sides can import it without sharing any of the method's code.
"""
from .operators import (CSR, convdiff_csr, manteuffel_csr, config1_operator,
                        config2_operator, config3_operator, config5_operator,
                        varcoef_fields_2d)
from .vectors import gaussian_vector

__all__ = ["CSR", "convdiff_csr", "manteuffel_csr", "config1_operator", "config2_operator",
           "config3_operator", "config5_operator", "varcoef_fields_2d", "gaussian_vector"]

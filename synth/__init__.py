"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the oracle.

This package holds input construction only (operators, right-hand sides, start vectors,
random fields): none of the Gram-Schmidt, Arnoldi, GMRES or Krylov-Schur arithmetic lives
here, so both sides can import it without sharing any of the method's code.
"""
from .operators import (CSR, Stencil7, convdiff_csr, convdiff_stencil7, manteuffel_csr,
                        manteuffel_stencil7, config1_operator, config1_stencil,
                        config2_operator, config2_stencil, config3_operator,
                        config5_operator, varcoef_fields_2d)
from .vectors import gaussian_vector, graded_factors, graded_matrix

__all__ = ["CSR", "Stencil7", "convdiff_csr", "convdiff_stencil7", "manteuffel_csr",
           "manteuffel_stencil7", "config1_operator", "config1_stencil", "config2_operator",
           "config2_stencil", "config3_operator", "config5_operator", "varcoef_fields_2d",
           "gaussian_vector", "graded_factors", "graded_matrix"]

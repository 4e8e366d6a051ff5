"""FP64 CPU oracle for the DCGS2 Arnoldi-QR hot path (test infrastructure only).

Plain, slow, readable numpy/scipy code that follows the paper step by step, used to check
the CUDA library.  Only the tests, the package smoke check and the benchmark's CPU baseline
may import it; the library never does, and the two share no code (only the seeded input
generators in ``synth`` serve both).

Modules
  arnoldi       DCGS2-Arnoldi (Algorithm 4), CGS2-Arnoldi (Algorithm 3), MGS-Arnoldi,
                DCGS2-QR (Algorithm 2), CGS2-QR (Algorithm 1)
  metrics       loss of orthogonality and Arnoldi representation error (Section 6.1)
  gmres         restarted GMRES / FGMRES on DCGS2-Arnoldi, FP32 / BF16-basis inner solves
                inside FP64 iterative refinement
  krylov_schur  Krylov-Schur eigenvalues (Stewart) on DCGS2-Arnoldi, Arnoldi residual test
  cnn           the 6-layer 3x3 convolutional preconditioner, forward and backward in FP64
  stencil       the matrix-free 7-point stencil operator (padded shifts; Kronecker assembly)
  partitioned   DCGS2-Arnoldi on row blocks of simulated ranks (one all-reduce per step)

Parity status per function is listed in each module header; the learned preconditioner's
benefit (an empirical quantity) is the one "parity unpinned" item.
"""

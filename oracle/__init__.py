"""FP64 CPU oracle for the QTT-accelerated PDIP Newton solve (test infrastructure).

This package is the slow, plain reference that the CUDA path is checked
against.  It is test infrastructure only: the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the library itself never
does, and it shares no code with the CUDA kernels.

Modules
  contacts : active set, contact frames, Morton ordering       (Sec. 2.2, 3.3)
  qp       : D, N = D^T M^-1 D, r, Schur blocks, padded layout  (Sec. 2.3, 2.4, 3.3)
  pdip     : primal-dual interior point iteration               (Sec. 2.4)
  krylov   : Jacobi-preconditioned CG                           (Sec. 3.3, 4.2)
  tt       : TT-SVD, rounding, QTT tensorisation and mat-vec    (Sec. 3.1, 3.2)
  timestep : velocity/position update, warm start of the PDIP   (Sec. 2.3, 3.3)
  mpnn     : message-passing network of the learned warm start (extension)

Parity status per function is stated in each module header; functions with no
independent pin say "parity unpinned" there.
"""

"""Plain, slow, FP64 CPU oracle for the curvilinear PIC hot path (test infrastructure).

This package is test infrastructure, not product code: only the test suite, the smoke
check and the CPU-baseline leg of the benchmark may import it. It shares no code with the
CUDA path. It follows the paper's steps in its order and notation (Sec. II): metric from
the discrete map (Sec. II.A), b2 charge assignment (Sec. II.B.1), b1 field interpolation
(Sec. II.B.2), conservative finite-volume Poisson with ghost cells (Sec. II.B.3) and the
hybrid predictor-corrector mover (Sec. II.B.4, eqs. (hybridx), (step1)-(step4)).

Modules:
  geometry  - spec M: Jacobi matrix, inverse, Jacobian, face metric coefficients
  poisson   - spec P: finite-volume operator, right-hand side, direct solve
  gradient  - spec G: logical field at vertices
  deposit   - spec Q: b2 weights, fixed-point charge deposit
  mover     - spec R/B: hybrid mover in FP64 (and the FP32 replay in replay32.c)
  philox    - Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  inject    - spec I: Maxwellian flux injection
  pic       - the PIC cycle composed from the above

Parity status of every function is pinned by tests/test_oracle_*.py; no function here is
"parity unpinned".
"""

"""CPU oracle for the multilevel spectral domain decomposition hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import or run anything in this
package.  The CUDA library (paper_2106_06404_gb300) never imports, links or
calls it, and this package shares no code with the library: the only module
both sides use is `synthetic_inputs`, which generates seeded coefficient
fields and holds none of the method's arithmetic.

Plain FP64: Q1 assembly (fem.py), box decomposition and partition of unity
(decomposition.py), LAPACK-free dense Cholesky and cyclic Jacobi (linalg.c,
linalg.py), exact local GEVPs, coarse spaces, the additive multilevel
preconditioner and PCG (method.py).

Pins: every function is checked in tests/test_oracle_*.py against closed forms,
invariants and brute force, never against the CUDA path.  Parity pinned for
all functions except where a test module says "parity unpinned", and except
method.normalise_sign: parity unpinned (a sign convention for exported
eigenvectors; every comparison goes through spans or Ritz values).
"""
from . import fem, linalg, decomposition, method  # noqa: F401

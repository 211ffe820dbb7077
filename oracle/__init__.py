"""FP64 CPU oracle for IHS-BIN (Wang & Pilanci, "Sketching the Krylov Subspace").

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
definition that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import it.  The product library never imports,
links or executes anything in here, and nothing in here imports the product
package: the two share no code.  The one thing both sides consume is the data
made by the separate ``synthetic`` module, which holds no IHS-BIN arithmetic.

Every routine is FP64 and follows the paper's steps in its own notation; each
cites the section / equation / algorithm it restates.  Library primitives
(numpy matmul, Cholesky, triangular solve, SVD) serve as single steps.

Parity status: all routines are pinned by ``tests/test_oracle_pins.py``
(closed forms, textbook routines on tiny inputs, brute force, invariants and
the published Philox known-answer vectors); none is "parity unpinned".
"""
from . import philox, sketch, ihsbin, precision  # noqa: F401,E402

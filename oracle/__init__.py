"""FP64 CPU oracle for covariance-free EM on clustered multi-task compressive sensing.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import anything from this package; the CUDA library never does and
shares no code with it.  ``philox`` draws the method's random numbers (alpha initialisation
and Rademacher probes) from the published Philox-4x32-10 definition; ``cofem`` holds exact
EM and CoFEM written from the paper's equations and algorithms.

Parity pins: every function here is checked by ``tests/test_oracle_*.py`` against values
fixed by the paper or by mathematics (published Philox known-answer vectors, closed forms,
the matrix-determinant lemma, brute force over assignments and over all Rademacher probes,
Lanczos identities, EM monotonicity).  The paper prints no worked numeric example of the
method itself, so no output is pinned to a number printed in the paper.
"""
from . import philox, cofem  # noqa: F401

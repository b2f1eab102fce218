"""CPU oracle for 3P-ADMM-PC2 (arXiv 2601.14980).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, independent
reference that the CUDA library is checked against.  Only ``tests/``, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
import it; the library (``paper_2601_14980_b300``) never does, and the oracle
never imports the library.

* ``oracle.paillier`` -- big-integer Paillier (plain C, schoolbook arithmetic)
  following Sec. III-B/III-C and Definitions 1-2 of the paper.
* ``oracle.admm`` -- FP64 LASSO ADMM (centralised, distributed, and the
  private 3P-ADMM-PC2 loop of Algorithm 1) with the quantizers of Eq. (et21)
  and Theorem 1, in numpy / Python integers.

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
something other than itself (Python's built-in three-argument ``pow``, brute
force on tiny keys, closed forms, published test vectors).  Functions with no
such pin are marked "parity unpinned" in their docstring.
"""

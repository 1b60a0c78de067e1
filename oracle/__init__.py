"""Test oracle for C = A^t A and C = X^t Y (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything under ``oracle/``.  The product library never
does: it shares no code, header, table or helper with this package, and this
package imports nothing from the product.

Contents
--------
``ata_oracle.c``      the plain definition C[i][j] = sum_k A[k][i] A[k][j]
                      (Section 3, Eq. "Cij" summed back), FP64, packed upper;
                      and the general product C[i][j] = sum_k X[k][i] Y[k][j]
                      (the HASA step of Section 4.2.2 on two operands), dense.
``core.py``           build + ctypes wrapper of the C file, packed-index maps,
                      error metrics (componentwise and normwise).
``ata_recursive.py``  Algorithm 1 (ATA) with the Strassen products of Section
                      4.2.2, restated step by step in numpy FP64.  It reaches
                      the same product up to rounding and pins the reading of
                      the recursion and of the (corrected) Strassen formulas.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(brute force against exact rationals, exact-integer identities against
integer arithmetic, closed forms, invariants, and LAPACK/BLAS special cases).
"""
from .core import (  # noqa: F401
    build, ata_packed, abs_gram_packed, ata_entries, ata_rows, num_threads, gemm_tn, gemm_entries,
    packed_index, packed_size, unpack_full, pack_upper, componentwise_error,
    normwise_error, classical_mults,
)

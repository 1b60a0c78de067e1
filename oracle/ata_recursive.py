"""Algorithm 1 (ATA, serial) with HASA realised as Strassen's algorithm,
restated in numpy FP64.  Test infrastructure only (see ``oracle/__init__.py``).

This is a second oracle: it follows the paper's steps in the paper's order
and notation, so it reaches A^t A up to rounding.  It pins three readings of
the paper that the plain definition cannot see:

* Section 3, Eq. "submatrices": m1 = ceil(m/2), m2 = floor(m/2),
  n1 = ceil(n/2), n2 = floor(n/2); A11 is m1 x n1, A12 m1 x n2, A21 m2 x n1,
  A22 m2 x n2.
* Algorithm 1: S1..S4 are recursive ATA calls on A11, A21, A12, A22;
  S5 = HASA(A12^t, A11), S6 = HASA(A22^t, A21); the result is the lower
  triangle [[S1+S2, .], [S5+S6, S3+S4]].  The base case, printed as
  "m or n <= 32", is read as min(m, n) <= cutoff (cutoff replaces 32).
* Section 4.2.2 (communication in HASA-P) prints the seven Strassen products
  and the four output blocks.  Two products are misprinted there: the
  product the paper calls M1 must be (A11 + A22)(B11 + B22) and M7 must be
  (A12 - A22)(B21 + B22) (Strassen 1969) for the printed D11 and D22 to hold;
  the other five products and all four D blocks are used as printed.
  Winograd's variant (mentioned in Section 1: 7 products, 15 additions) is
  provided as ``variant="winograd"``.

HASA's own splitting is not printed (the paper defers to d'Alberto and
Nicolau).  Reading used here: the base case is min(p, q, r) <= cutoff; odd
dimensions split into ceil/floor halves, the smaller blocks are padded with
zeros up to the ceil size, and the padded rows/columns of the product are
dropped.  This is exact algebra, so only rounding changes.

Every multiplication is counted in ``MultCounter`` (base-case products count
p*q*r scalar multiplications each, on the padded sizes), which gives the
exact value of the recurrence of Section 3.1 for the tree actually run.
"""
from __future__ import annotations

import numpy as np


class MultCounter:
    def __init__(self):
        self.mults = 0


def _ceil_half(x: int) -> int:
    return (x + 1) // 2


def mult(A: np.ndarray, counter: MultCounter | None = None) -> np.ndarray:
    """Base case of Algorithm 1: the classical product, lower triangle of
    A^t A (the strictly upper part is left zero, as only one triangle is
    returned).  Counts the n(n+1)/2 * m multiplications of the triangle."""
    m, n = A.shape
    if counter is not None:
        counter.mults += m * n * (n + 1) // 2
    return np.tril(A.T @ A)


def _pad(X: np.ndarray, rows: int, cols: int) -> np.ndarray:
    if X.shape == (rows, cols):
        return X
    P = np.zeros((rows, cols), dtype=np.float64)
    P[: X.shape[0], : X.shape[1]] = X
    return P


def hasa(X: np.ndarray, Y: np.ndarray, cutoff: int, counter: MultCounter | None = None,
         variant: str = "strassen") -> np.ndarray:
    """X (p x q) times Y (q x r) by Strassen recursion with ceil/floor
    splitting and implicit zero padding (HASA, Section 3 and Section 4.2.2)."""
    p, q = X.shape
    q2, r = Y.shape
    assert q == q2
    if min(p, q, r) <= cutoff:
        if counter is not None:
            counter.mults += p * q * r
        return X @ Y
    p1, q1, r1 = _ceil_half(p), _ceil_half(q), _ceil_half(r)
    Xp = _pad(X, 2 * p1, 2 * q1)
    Yp = _pad(Y, 2 * q1, 2 * r1)
    A11, A12 = Xp[:p1, :q1], Xp[:p1, q1:]
    A21, A22 = Xp[p1:, :q1], Xp[p1:, q1:]
    B11, B12 = Yp[:q1, :r1], Yp[:q1, r1:]
    B21, B22 = Yp[q1:, :r1], Yp[q1:, r1:]

    def rec(U, V):
        return hasa(U, V, cutoff, counter, variant)

    if variant in ("strassen", "as_printed"):
        # the seven products (Section 4.2.2, M1 and M7 corrected); the
        # "as_printed" variant keeps the two misprinted products and exists
        # only so a test can show that the exact-integer pins reject them
        M3 = rec(A11, B12 - B22)
        M6 = rec(A21 - A11, B11 + B12)
        M2 = rec(A21 + A22, B11)
        if variant == "strassen":
            M1 = rec(A11 + A22, B11 + B22)
            M7 = rec(A12 - A22, B21 + B22)
        else:
            M1 = rec(A11 + A12, B11 + B22)
            M7 = rec(A11 - A22, B21 - B22)
        M5 = rec(A11 + A12, B22)
        M4 = rec(A22, B21 - B11)
        # the four blocks of D = X Y, additions in the printed order
        D11 = M1 - M5 + M7 + M4
        D12 = M3 + M5
        D21 = M2 + M4
        D22 = M3 + M6 - M2 + M1
    elif variant == "winograd":
        # Winograd's form: 7 products, 8 operand sums, 7 output sums
        S1 = A21 + A22
        S2 = S1 - A11
        S3 = A11 - A21
        S4 = A12 - S2
        T1 = B12 - B11
        T2 = B22 - T1
        T3 = B22 - B12
        T4 = T2 - B21
        M1 = rec(A11, B11)
        M2 = rec(A12, B21)
        M3 = rec(S4, B22)
        M4 = rec(A22, T4)
        M5 = rec(S1, T1)
        M6 = rec(S2, T2)
        M7 = rec(S3, T3)
        U2 = M1 + M6
        U3 = U2 + M7
        U4 = U2 + M5
        D11 = M1 + M2
        D12 = U4 + M3
        D21 = U3 - M4
        D22 = U3 + M5
    else:
        raise ValueError(f"unknown variant {variant!r}")
    D = np.empty((2 * p1, 2 * r1), dtype=np.float64)
    D[:p1, :r1] = D11
    D[:p1, r1:] = D12
    D[p1:, :r1] = D21
    D[p1:, r1:] = D22
    return D[:p, :r]


def ata(A: np.ndarray, cutoff: int = 32, counter: MultCounter | None = None,
        variant: str = "strassen") -> np.ndarray:
    """Algorithm 1: lower triangle of C = A^t A (full n x n array, strictly
    upper part zero)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if min(m, n) <= cutoff:
        return mult(A, counter)
    m1, m2 = _ceil_half(m), m // 2
    n1, n2 = _ceil_half(n), n // 2
    A11, A12 = A[:m1, :n1], A[:m1, n1:]
    A21, A22 = A[m1:, :n1], A[m1:, n1:]
    S1 = ata(A11, cutoff, counter, variant)
    S2 = ata(A21, cutoff, counter, variant)
    S3 = ata(A12, cutoff, counter, variant)
    S4 = ata(A22, cutoff, counter, variant)
    S5 = hasa(A12.T, A11, cutoff, counter, variant)
    S6 = hasa(A22.T, A21, cutoff, counter, variant)
    C = np.zeros((n, n), dtype=np.float64)
    C[:n1, :n1] = S1 + S2
    C[n1:, :n1] = S5 + S6
    C[n1:, n1:] = S3 + S4
    return C


def ata_packed_upper(A: np.ndarray, cutoff: int = 32, variant: str = "strassen",
                     counter: MultCounter | None = None) -> np.ndarray:
    """Algorithm 1's lower triangle, returned in the row-major packed upper
    order (the same numbers: C_upper[i][j] = C_lower[j][i])."""
    L = ata(A, cutoff, counter, variant)
    n = L.shape[0]
    return np.ascontiguousarray(L.T[np.triu_indices(n)])

"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/) against something other than itself:
exact rational arithmetic, integer arithmetic, closed forms, invariants,
BLAS routines, and the paper's own recurrence (Section 3.1).  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import oracle
from oracle import ata_recursive as R
from paper_1902_02104_gb300 import inputs

U = np.finfo(np.float64).eps / 2  # unit roundoff


def exact_gram(A):
    """A^t A over the rationals (every double is an exact rational)."""
    m, n = A.shape
    F = [[Fraction(float(A[k, i])) for i in range(n)] for k in range(m)]
    C = [[sum((F[k][i] * F[k][j] for k in range(m)), Fraction(0)) for j in range(n)] for i in range(n)]
    return C


def test_brute_force_tiny_against_rationals():
    rng = np.random.default_rng(11)
    for m, n in itertools.product(range(0, 7), range(1, 7)):
        A = rng.standard_normal((m, n))
        C = oracle.ata_packed(A)
        G = oracle.abs_gram_packed(A)
        E = exact_gram(A)
        idx = 0
        for i in range(n):
            for j in range(i, n):
                err = abs(Fraction(C[idx]) - E[i][j])
                # recursive summation bound: |fl(s) - s| <= gamma_m * sum |a_k b_k|
                gamma = m * U / (1 - m * U)
                assert err <= Fraction(gamma) * Fraction(G[idx]) + Fraction(0), (m, n, i, j)
                idx += 1


def test_tiny_integers_equal_rationals_bitwise():
    rng = np.random.default_rng(12)
    for m, n in itertools.product(range(0, 7), range(1, 7)):
        A = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
        C = oracle.ata_packed(A)
        E = exact_gram(A)
        iu = np.triu_indices(n)
        want = np.array([float(E[i][j]) for i, j in zip(*iu)])
        assert np.array_equal(C, want)


@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (3, 7), (64, 48), (129, 65), (1024, 37), (200, 200)])
def test_exact_integers_against_int64(m, n):
    A = inputs.integers(m, n, seed=m * 1000 + n)
    Ai = A.astype(np.int64)
    want = (Ai.T @ Ai)[np.triu_indices(n)].astype(np.float64)
    assert np.array_equal(oracle.ata_packed(A), want)


def test_transposed_operand_is_caught():
    # A A^t differs from A^t A; the int64 pin above would reject an oracle
    # that multiplied the wrong way round.
    A = inputs.integers(5, 5, seed=3)
    Ai = A.astype(np.int64)
    wrong = (Ai @ Ai.T)[np.triu_indices(5)]
    assert not np.array_equal(oracle.ata_packed(A), wrong.astype(np.float64))


def test_closed_form_identity_block():
    n = 17
    A = np.vstack([np.eye(n), np.zeros((9, n))])
    C = oracle.unpack_full(oracle.ata_packed(A), n)
    assert np.array_equal(C, np.eye(n))


def test_closed_form_rank_one():
    rng = np.random.default_rng(2)
    u = rng.integers(-5, 6, size=40).astype(np.float64)
    v = rng.integers(-5, 6, size=13).astype(np.float64)
    A = np.outer(u, v)
    want = (u @ u) * np.outer(v, v)
    assert np.array_equal(oracle.unpack_full(oracle.ata_packed(A), 13), want)


def test_closed_form_single_column():
    a = np.arange(1, 101, dtype=np.float64).reshape(-1, 1)
    assert oracle.ata_packed(a)[0] == 100 * 101 * 201 / 6  # sum of squares


def test_closed_form_orthonormal_columns():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((300, 60)))
    C = oracle.unpack_full(oracle.ata_packed(Q), 60)
    assert np.max(np.abs(C - np.eye(60))) < 1e-13


def test_entries_symmetric_and_equal_to_packed():
    A = inputs.normal(120, 40, seed=7)
    C = oracle.ata_packed(A)
    I, J = np.triu_indices(40)
    e_ij = oracle.ata_entries(A, I, J)
    e_ji = oracle.ata_entries(A, J, I)
    assert np.array_equal(e_ij, C)
    assert np.array_equal(e_ji, C)


def test_diagonal_is_column_norms_squared():
    A = inputs.normal(333, 21, seed=8)
    acc = np.zeros(21)
    for k in range(A.shape[0]):  # same k order, separately coded
        acc = acc + A[k] * A[k]
    C = oracle.ata_packed(A)
    diag = C[oracle.packed_index(np.arange(21), np.arange(21), 21)]
    assert np.array_equal(diag, acc)


@pytest.mark.parametrize("m,n", [(50, 30), (30, 50), (200, 200)])
def test_positive_semidefinite_and_rank(m, n):
    A = inputs.normal(m, n, seed=m + n)
    C = oracle.unpack_full(oracle.ata_packed(A), n)
    w = np.linalg.eigvalsh(C)
    assert w.min() >= -n * U * np.abs(w).max() * 10
    if m < n:
        # rank <= m: the n - m smallest eigenvalues vanish to rounding
        assert np.all(np.abs(w[: n - m]) <= n * 1e-12 * w.max())


def test_matches_blas_dsyrk():
    blas = pytest.importorskip("scipy.linalg.blas")
    A = inputs.normal(257, 71, seed=9)
    C_full = blas.dsyrk(1.0, A, trans=1, lower=0)  # upper triangle of A^t A
    want = C_full[np.triu_indices(71)]
    G = oracle.abs_gram_packed(A)
    got = oracle.ata_packed(A)
    assert np.all(np.abs(got - want) <= 2 * 257 * U * G)


def test_packed_layout_matches_lapack_lower_packed():
    # row-major packed upper == column-major packed lower (LAPACK 'L');
    # dspr builds A^t A as a sum of rank-one updates into that layout
    blas = pytest.importorskip("scipy.linalg.blas")
    A = inputs.integers(23, 9, seed=10)
    ap = np.zeros(9 * 10 // 2)
    for k in range(A.shape[0]):
        ap = blas.dspr(9, 1.0, A[k], ap, lower=1)
    assert np.array_equal(oracle.ata_packed(A), ap)


def test_packed_index_map():
    n = 11
    I, J = np.triu_indices(n)
    assert np.array_equal(oracle.packed_index(I, J, n), np.arange(n * (n + 1) // 2))
    F = np.arange(n * n, dtype=float).reshape(n, n)
    F = F + F.T
    assert np.array_equal(oracle.unpack_full(oracle.pack_upper(F), n), F)


def test_rows_and_abs_gram():
    A = inputs.normal(90, 31, seed=12)
    C = oracle.ata_packed(A)
    s0 = int(oracle.packed_index(5, 5, 31))
    s1 = int(oracle.packed_index(12, 12, 31))
    assert np.array_equal(oracle.ata_rows(A, 5, 12), C[s0:s1])
    assert np.array_equal(oracle.ata_rows(A, 25, 31), C[int(oracle.packed_index(25, 25, 31)):])
    assert np.array_equal(oracle.abs_gram_packed(A), oracle.ata_packed(np.abs(A)))


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.ata_entries(np.ones((3, 3)), [0, 5], [0, 1])


def test_error_metrics():
    C_ref = np.array([4.0, 1.0, 9.0])  # n = 2: (0,0), (0,1), (1,1)
    G = np.array([4.0, 2.0, 9.0])
    C = C_ref + np.array([0.0, 1e-3, 0.0])
    assert oracle.componentwise_error(C, C_ref, G) == pytest.approx(5e-4)
    # full matrix: off-diagonal counted twice
    want = np.sqrt(2 * 1e-6) / np.sqrt(16 + 2 * 1 + 81)
    assert oracle.normwise_error(C, C_ref, 2) == pytest.approx(want)
    # a zero column pair must give an exactly zero entry
    assert oracle.componentwise_error([1e-30], [0.0], [0.0]) == float("inf")


# ---------------------------------------------------------------------------
# The recursive restatement of Algorithm 1 (oracle/ata_recursive.py)

@pytest.mark.parametrize("variant", ["strassen", "winograd"])
@pytest.mark.parametrize("m,n,cutoff", [(64, 64, 8), (100, 37, 5), (37, 100, 5), (129, 127, 16), (512, 384, 64),
                                        (33, 17, 4), (1, 50, 4), (50, 1, 4)])
def test_recursion_exact_on_integers(m, n, cutoff, variant):
    A = inputs.integers(m, n, seed=m * 7 + n)
    got = R.ata_packed_upper(A, cutoff, variant)
    assert np.array_equal(got, oracle.ata_packed(A))


def test_misprinted_products_are_rejected():
    # Section 4.2.2 prints M1 = (A11 + A12)(B11 + B22) and
    # M7 = (A11 - A22)(B21 - B22); with the printed D blocks these give a
    # wrong product, which the exact-integer pin detects.
    A = inputs.integers(64, 64, seed=1)
    assert not np.array_equal(R.ata_packed_upper(A, 8, "as_printed"), oracle.ata_packed(A))
    X, Y = inputs.integers(40, 40, seed=2), inputs.integers(40, 40, seed=3)
    assert not np.array_equal(R.hasa(X, Y, 8, variant="as_printed"), X @ Y)
    assert np.array_equal(R.hasa(X, Y, 8), X @ Y)


@pytest.mark.parametrize("p,q,r", [(17, 33, 9), (40, 40, 40), (31, 64, 63), (100, 20, 100)])
def test_hasa_exact_on_integers(p, q, r):
    rng = np.random.default_rng(p * q * r)
    X = rng.integers(-4, 5, size=(p, q)).astype(float)
    Y = rng.integers(-4, 5, size=(q, r)).astype(float)
    for v in ("strassen", "winograd"):
        assert np.array_equal(R.hasa(X, Y, 4, variant=v), X @ Y)


def test_recursion_float_accuracy():
    A = inputs.normal(300, 220, seed=1)
    got = R.ata_packed_upper(A, 16)
    err = oracle.componentwise_error(got, oracle.ata_packed(A), oracle.abs_gram_packed(A))
    assert err < 1e-12


def paper_recurrence(N, c):
    """Section 3.1, T(N) = 4 T(N/2) + 2 * H(N/2), for N a power of two and a
    power-of-two cutoff c: the base case costs N * N(N+1)/2 multiplications,
    a HASA product of order h costs 7^s c^3 with h / 2^s = c."""
    if N <= c:
        return N * N * (N + 1) // 2
    h = N // 2
    s = 0
    while h > c:
        h //= 2
        s += 1
    return 4 * paper_recurrence(N // 2, c) + 2 * 7 ** s * h ** 3


@pytest.mark.parametrize("N,c", [(64, 8), (128, 16), (256, 32), (512, 64), (256, 16)])
def test_multiplication_count_matches_recurrence(N, c):
    cnt = R.MultCounter()
    R.ata(np.zeros((N, N)), c, cnt)
    assert cnt.mults == paper_recurrence(N, c)
    assert cnt.mults < oracle.classical_mults(N, N)


def test_cost_constant_reading():
    # The recurrence solves to (2/3) n^log2(7) multiplications for full
    # recursion (cutoff 1), not the (2/7) n^log2(7) of Section 3.1's claim:
    # sum_l 4^l * (2/7) (n/2^l)^log2(7) = (2/7) n^log2(7) / (1 - 4/7).
    lg7 = np.log2(7)
    n = 2.0 ** 20
    total = sum(4 ** l * (2 / 7) * (n / 2 ** l) ** lg7 for l in range(60))
    assert total / n ** lg7 == pytest.approx(2 / 3, rel=1e-9)


# ---------------------------------------------------------------------------
# General product C = X^t Y (the HASA step of Section 4.2.2 on two operands)

def exact_gemm_tn(X, Y):
    m, p = X.shape
    r = Y.shape[1]
    FX = [[Fraction(float(X[k, i])) for i in range(p)] for k in range(m)]
    FY = [[Fraction(float(Y[k, j])) for j in range(r)] for k in range(m)]
    return [[sum((FX[k][i] * FY[k][j] for k in range(m)), Fraction(0)) for j in range(r)] for i in range(p)]


def test_gemm_brute_force_tiny_against_rationals():
    rng = np.random.default_rng(31)
    for m, p, r in itertools.product(range(0, 5), range(1, 5), range(1, 5)):
        X = rng.standard_normal((m, p))
        Y = rng.standard_normal((m, r))
        C = oracle.gemm_tn(X, Y)
        G = oracle.gemm_tn(X, Y, absval=True)
        E = exact_gemm_tn(X, Y)
        gamma = m * U / (1 - m * U)
        for i in range(p):
            for j in range(r):
                assert abs(Fraction(C[i, j]) - E[i][j]) <= Fraction(gamma) * Fraction(G[i, j]), (m, p, r, i, j)


def test_gemm_tiny_integers_equal_rationals_bitwise():
    rng = np.random.default_rng(32)
    for m, p, r in itertools.product(range(0, 6), range(1, 5), range(1, 5)):
        X = rng.integers(-9, 10, size=(m, p)).astype(np.float64)
        Y = rng.integers(-9, 10, size=(m, r)).astype(np.float64)
        E = exact_gemm_tn(X, Y)
        want = np.array([[float(E[i][j]) for j in range(r)] for i in range(p)]).reshape(p, r)
        assert np.array_equal(oracle.gemm_tn(X, Y), want)


@pytest.mark.parametrize("m,p,r", [(1, 1, 1), (7, 3, 5), (3, 7, 2), (64, 48, 80), (129, 65, 33), (1024, 37, 50)])
def test_gemm_exact_integers_against_int64(m, p, r):
    X = inputs.integers(m, p, seed=m + p)
    Y = inputs.integers(m, r, seed=m + r + 1)
    want = (X.astype(np.int64).T @ Y.astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.gemm_tn(X, Y), want)


def test_gemm_with_itself_is_the_gram_bitwise():
    # X = Y = A: the same k-ascending sums as the A^t A oracle
    A = inputs.normal(300, 70, seed=5)
    C = oracle.gemm_tn(A, A)
    assert np.array_equal(C[np.triu_indices(70)], oracle.ata_packed(A))
    G = oracle.gemm_tn(A, A, absval=True)
    assert np.array_equal(G[np.triu_indices(70)], oracle.abs_gram_packed(A))


def test_gemm_closed_forms():
    # X = [I_p; 0]: C = the first p rows of Y
    Y = inputs.normal(50, 30, seed=6)
    X = np.zeros((50, 20))
    X[:20, :20] = np.eye(20)
    assert np.array_equal(oracle.gemm_tn(X, Y), Y[:20])
    # X = a b^t, Y = a c^t (integers): X^t Y = (a.a) b c^t exactly
    rng = np.random.default_rng(7)
    a = rng.integers(-5, 6, size=40).astype(float)
    b = rng.integers(-5, 6, size=9).astype(float)
    c = rng.integers(-5, 6, size=11).astype(float)
    assert np.array_equal(oracle.gemm_tn(np.outer(a, b), np.outer(a, c)), float(a @ a) * np.outer(b, c))


def test_gemm_matches_strassen_restatement_on_integers():
    rng = np.random.default_rng(8)
    X = rng.integers(-4, 5, size=(70, 45)).astype(float)
    Y = rng.integers(-4, 5, size=(70, 38)).astype(float)
    for v in ("strassen", "winograd"):
        assert np.array_equal(R.hasa(X.T, Y, 8, variant=v), oracle.gemm_tn(X, Y))


def test_gemm_entries_and_degenerate_shapes():
    X = inputs.normal(90, 25, seed=9)
    Y = inputs.normal(90, 31, seed=10)
    C = oracle.gemm_tn(X, Y)
    I = np.array([0, 24, 3, 11])
    J = np.array([30, 0, 3, 17])
    assert np.array_equal(oracle.gemm_entries(X, Y, I, J), C[I, J])
    assert np.array_equal(oracle.gemm_entries(X, Y, I, J, absval=True),
                          oracle.gemm_tn(np.abs(X), np.abs(Y))[I, J])
    assert np.array_equal(oracle.gemm_tn(np.zeros((0, 4)), np.zeros((0, 3))), np.zeros((4, 3)))
    assert oracle.gemm_tn(np.zeros((5, 0)), np.zeros((5, 3))).shape == (0, 3)
    with pytest.raises(Exception):
        oracle.gemm_tn(np.zeros((5, 2)), np.zeros((4, 3)))

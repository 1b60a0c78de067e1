"""Build and call the C oracle; packed layout maps; error metrics.

Test infrastructure only (see ``oracle/__init__.py``).

The packed layout is the row-major packed upper triangle of the symmetric
n x n product (Section 3: only one triangle of A^t A is stored, n(n+1)/2
entries):  idx(i, j) = i*n - i*(i-1)/2 + (j - i) for i <= j.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ata_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``ata_oracle.c`` with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dp = ctypes.c_int64, ctypes.c_void_p
            lib.oracle_ata_packed.argtypes = [dp, i64, i64, i64, dp]
            lib.oracle_abs_gram_packed.argtypes = [dp, i64, i64, i64, dp]
            lib.oracle_ata_entries.argtypes = [dp, i64, i64, i64, dp, dp, i64, ctypes.c_int, dp]
            lib.oracle_ata_rows.argtypes = [dp, i64, i64, i64, i64, i64, dp]
            lib.oracle_gemm_tn.argtypes = [dp, i64, i64, i64, dp, i64, i64, dp, i64, ctypes.c_int]
            lib.oracle_gemm_entries.argtypes = [dp, i64, i64, i64, dp, i64, i64, dp, dp, i64, ctypes.c_int, dp]
            for f in (lib.oracle_ata_packed, lib.oracle_abs_gram_packed,
                      lib.oracle_ata_entries, lib.oracle_ata_rows, lib.oracle_gemm_tn,
                      lib.oracle_gemm_entries):
                f.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _as_f64(A) -> np.ndarray:
    """FP64 copy of A.  FP32 inputs are widened exactly, so the oracle is the
    exact-input product of the FP32-rounded matrix."""
    A = np.asarray(A)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    return np.ascontiguousarray(A, dtype=np.float64)


def packed_size(n: int) -> int:
    return n * (n + 1) // 2


def packed_index(i, j, n):
    """Position of (i, j), i <= j, in the row-major packed upper triangle."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * n - i * (i - 1) // 2 + (j - i)


def _check(rc: int, what: str):
    if rc == -1:
        raise ValueError(f"{what}: bad arguments")
    if rc == -2:
        raise MemoryError(f"{what}: out of host memory")
    if rc != 0:
        raise RuntimeError(f"{what}: status {rc}")


def ata_packed(A) -> np.ndarray:
    """Packed upper triangle of A^t A in FP64 (the plain definition)."""
    A = _as_f64(A)
    m, n = A.shape
    C = np.empty(packed_size(n), dtype=np.float64)
    _check(_load().oracle_ata_packed(A.ctypes.data, m, n, n, C.ctypes.data), "oracle_ata_packed")
    return C


def abs_gram_packed(A) -> np.ndarray:
    """Packed upper triangle of |A|^t |A| (denominator of the componentwise error)."""
    A = _as_f64(A)
    m, n = A.shape
    G = np.empty(packed_size(n), dtype=np.float64)
    _check(_load().oracle_abs_gram_packed(A.ctypes.data, m, n, n, G.ctypes.data), "oracle_abs_gram_packed")
    return G


def ata_entries(A, I, J, absval: bool = False) -> np.ndarray:
    """Selected entries (I[t], J[t]) of A^t A (or |A|^t|A|), bitwise equal to
    the same entries of :func:`ata_packed`."""
    A = _as_f64(A)
    m, n = A.shape
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    if I.shape != J.shape:
        raise ValueError("I and J differ in shape")
    out = np.empty(I.size, dtype=np.float64)
    _check(_load().oracle_ata_entries(A.ctypes.data, m, n, n, I.ctypes.data, J.ctypes.data,
                                      I.size, int(absval), out.ctypes.data), "oracle_ata_entries")
    return out


def ata_rows(A, i0: int, i1: int) -> np.ndarray:
    """Rows [i0, i1) of the packed upper triangle of A^t A."""
    A = _as_f64(A)
    m, n = A.shape
    cnt = int(packed_index(i1, i1, n) - packed_index(i0, i0, n)) if i1 < n else \
        packed_size(n) - int(packed_index(i0, i0, n)) if i0 < n else 0
    out = np.empty(max(cnt, 0), dtype=np.float64)
    _check(_load().oracle_ata_rows(A.ctypes.data, m, n, n, i0, i1, out.ctypes.data), "oracle_ata_rows")
    return out


def gemm_tn(X, Y, absval: bool = False) -> np.ndarray:
    """C = X^t Y (p x r, FP64) for X: m x p and Y: m x r, k ascending, one
    accumulator per entry; with absval, |X|^t |Y|."""
    X = _as_f64(X)
    Y = _as_f64(Y)
    if X.shape[0] != Y.shape[0]:
        raise ValueError("X and Y must have the same number of rows")
    m, p = X.shape
    r = Y.shape[1]
    C = np.zeros((p, r), dtype=np.float64)
    _check(_load().oracle_gemm_tn(X.ctypes.data, m, p, p, Y.ctypes.data, r, r, C.ctypes.data, r, int(absval)),
           "oracle_gemm_tn")
    return C


def gemm_entries(X, Y, I, J, absval: bool = False) -> np.ndarray:
    """Entries (I[t], J[t]) of X^t Y (or |X|^t|Y|), bitwise equal to the same
    entries of :func:`gemm_tn`."""
    X = _as_f64(X)
    Y = _as_f64(Y)
    m, p = X.shape
    r = Y.shape[1]
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.empty(I.size, dtype=np.float64)
    _check(_load().oracle_gemm_entries(X.ctypes.data, m, p, p, Y.ctypes.data, r, r, I.ctypes.data, J.ctypes.data,
                                       I.size, int(absval), out.ctypes.data), "oracle_gemm_entries")
    return out


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def unpack_full(Cp: np.ndarray, n: int) -> np.ndarray:
    """Full symmetric n x n matrix from the packed upper triangle."""
    Cp = np.asarray(Cp, dtype=np.float64)
    if Cp.size != packed_size(n):
        raise ValueError("packed size mismatch")
    F = np.zeros((n, n), dtype=np.float64)
    iu = np.triu_indices(n)
    F[iu] = Cp  # row-major order of triu_indices matches the packed order
    F.T[iu] = Cp
    return F


def pack_upper(F: np.ndarray) -> np.ndarray:
    """Packed upper triangle (row-major) of a square matrix."""
    F = np.asarray(F)
    n = F.shape[0]
    return np.ascontiguousarray(F[np.triu_indices(n)])


def componentwise_error(C, C_ref, G) -> float:
    """max_{i<=j} |C - C_ref| / G with G = (|A|^t|A|)_ij.  Where G == 0 the
    column pair is all zero and C must be exactly 0 there (else +inf)."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    d = np.abs(C - C_ref)
    if d.size == 0:
        return 0.0
    zero = G == 0
    if np.any(d[zero] != 0) or np.any(~np.isfinite(d)):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float(np.max(d[~zero] / G[~zero]))


def normwise_error(C, C_ref, n: int, I=None) -> float:
    """||C - C_ref||_F / ||C_ref||_F over the full symmetric matrix, from
    packed entries (off-diagonal entries count twice in the squared sums).
    With row indices ``I`` of a sample of entries, the same weighting is
    applied to the sample (diagonal where I == J)."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    if I is None:
        w = np.full(C.size, 2.0)
        w[packed_index(np.arange(n), np.arange(n), n)] = 1.0
    else:
        I, J = I
        w = np.where(np.asarray(I) == np.asarray(J), 1.0, 2.0)
    num = np.sqrt(np.sum(w * (C - C_ref) ** 2))
    den = np.sqrt(np.sum(w * C_ref ** 2))
    if den == 0:
        return 0.0 if num == 0 else float("inf")
    return float(num / den)


def classical_mults(m: int, n: int) -> int:
    """Scalar multiplications of the classical symmetric product: m*n(n+1)/2
    (Section 6 gives n^2(n+1)/2 for the square case m = n)."""
    return m * n * (n + 1) // 2

"""Non-finite inputs (the paper is silent; the library propagates them).

With classical leaves every entry C[i][j] reads only columns i and j, so an
Inf or NaN in column c makes exactly the entries of row and column c of C
non-finite, and every other entry is what the oracle gives.  The sliced modes
(bf16x3, FP64 emulation) mark a column holding a non-finite value through its
column maximum and write NaN for its entries; plain FP64 and TF32 follow IEEE
arithmetic (Inf or NaN).  Strassen operand sums mix columns, so with Strassen
levels a non-finite value may spread to more entries; the entries of its own
row and column are still never finite.
"""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = [ata.ATA_F64, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]


def run(A_np, dtype, cutoff, **opts):
    import torch
    m, n = A_np.shape
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    C = plan(torch.from_numpy(np.ascontiguousarray(A_np)).cuda())
    torch.cuda.synchronize()
    return oracle.unpack_full(C.cpu().numpy(), n)


def poisoned(dtype, m=300, n=200, seed=4):
    dt = np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32
    A = inputs.integers(m, n, seed=seed).astype(dt)
    bad = [3, 77, 150]
    A[10, 3] = np.inf
    A[200, 77] = -np.inf
    A[5, 150] = np.nan
    return A, bad


@pytest.mark.parametrize("dtype", ALL)
def test_classical_leaves_keep_nonfinite_local(gpu, dtype):
    A, bad = poisoned(dtype)
    n = A.shape[1]
    F = run(A, dtype, 4096)  # one diagonal leaf, no Strassen
    mask = np.zeros((n, n), dtype=bool)
    mask[bad, :] = True
    mask[:, bad] = True
    assert not np.any(np.isfinite(F[mask]))
    good = A.copy()
    good[:, bad] = 0
    ref = oracle.unpack_full(oracle.ata_packed(good), n)
    assert np.array_equal(F[~mask], ref[~mask])


@pytest.mark.parametrize("dtype", ALL)
def test_strassen_keeps_own_entries_nonfinite(gpu, dtype):
    A, bad = poisoned(dtype, m=600, n=520)
    n = A.shape[1]
    F = run(A, dtype, 64 if dtype == ata.ATA_F64 else 128)
    mask = np.zeros((n, n), dtype=bool)
    mask[bad, :] = True
    mask[:, bad] = True
    assert not np.any(np.isfinite(F[mask]))

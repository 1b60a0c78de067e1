"""Maximum sizes: indices past 2^31 on the device, on exact integers.

* A of 600000 x 4000 (2.4e9 entries): A itself and every operand's part
  buffers hold more than 2^31 elements, and the leaves run 600000 deep in K.
* A of 256 x 70000: the packed output holds 2.45e9 entries, written by the
  149 878 upper tiles of one diagonal leaf.
* X^t Y with X 256 x 50000 and Y 256 x 45000: a dense output of 2.25e9
  entries.

Entries are integers in [-4, 4], so every mode is exact here (bf16 and
TF32 hold them, chunk sums stay below 2^24, |C_ij| <= 16 m < 2^24; the
plain FP64 path runs these sizes in a few seconds): sampled entries, with the first and last rows and columns, are
compared bitwise with the oracle's entries.  A case holds 20-50 GB on the
device; the plans' index arithmetic was checked on the host first
(ata_plan_check, test_planner.py)."""
import functools

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [(ata.ATA_F32_BF16X3, "float32"), (ata.ATA_F32_TF32, "float32"), (ata.ATA_F64_OZAKI, "float64"),
         (ata.ATA_F64, "float64")]


@functools.lru_cache(maxsize=2)
def _input(m, n, seed):
    return inputs.small_integers(m, n, seed=seed)


def _pairs(n, count, seed):
    rng = np.random.default_rng(seed)
    I, J = rng.integers(0, n, count), rng.integers(0, n, count)
    I, J = np.minimum(I, J), np.maximum(I, J)
    corner_i = np.array([0, 0, n // 2, n - 2, n - 1])
    corner_j = np.array([0, n - 1, n - 1, n - 1, n - 1])
    return np.concatenate([I, corner_i]), np.concatenate([J, corner_j])


def _run_and_sample(A8, dtype, tname, I, J):
    import torch
    m, n = A8.shape
    A = torch.from_numpy(A8).cuda().to(getattr(torch, tname))
    plan = ata.Plan(m, n, dtype, 0)
    C = plan(A)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    got = C[torch.from_numpy(oracle.packed_index(I, J, n)).cuda()].cpu().numpy()
    del A, C, plan
    torch.cuda.empty_cache()
    return got


@pytest.mark.parametrize("dtype,tname", MODES)
def test_input_past_2e31_entries(gpu, dtype, tname):
    m, n = 600000, 4000
    A8 = _input(m, n, 61)
    I, J = _pairs(n, 400, seed=62)
    got = _run_and_sample(A8, dtype, tname, I, J)
    # the oracle's entries on the sampled columns only (C_ij depends on
    # columns i and j alone)
    cols, inv = np.unique(np.concatenate([I, J]), return_inverse=True)
    ref = oracle.ata_entries(A8[:, cols], inv[:I.size], inv[I.size:])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype,tname", MODES)
def test_packed_output_past_2e31_entries(gpu, dtype, tname):
    m, n = 256, 70000
    assert n * (n + 1) // 2 > 2 ** 31
    A8 = _input(m, n, 63)
    I, J = _pairs(n, 2000, seed=64)
    got = _run_and_sample(A8, dtype, tname, I, J)
    assert np.array_equal(got, oracle.ata_entries(A8, I, J))


@pytest.mark.parametrize("dtype,tname", MODES)
def test_general_product_output_past_2e31_entries(gpu, dtype, tname):
    import torch
    m, p, r = 256, 50000, 45000
    assert p * r > 2 ** 31
    X8, Y8 = _input(m, p, 65), _input(m, r, 66)
    rng = np.random.default_rng(67)
    I = np.concatenate([rng.integers(0, p, 2000), [0, p - 1, p - 1]])
    J = np.concatenate([rng.integers(0, r, 2000), [r - 1, 0, r - 1]])
    tdt = getattr(torch, tname)
    X, Y = torch.from_numpy(X8).cuda().to(tdt), torch.from_numpy(Y8).cuda().to(tdt)
    plan = ata.GemmPlan(m, p, r, dtype, 0)
    C = plan(X, Y)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    got = C.reshape(-1)[torch.from_numpy(I * r + J).cuda()].cpu().numpy()
    del X, Y, C, plan
    torch.cuda.empty_cache()
    assert np.array_equal(got, oracle.gemm_entries(X8, Y8, I, J))

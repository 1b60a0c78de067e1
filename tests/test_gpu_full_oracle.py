"""Every entry of paper-scale products against the oracle (no sampling).

The plain FP64 path and the FP64 emulation at 5000 x 5000 and 10000 x 10000
(componentwise, 1e-11; the FP64 emulation also at 20000 x 8000), and both
FP32 leaf modes on the precision form's full input, A 16384 x 8192 FP32 with
every 8th column scaled by 1e3 (normwise over the whole symmetric matrix:
1e-6 bf16x3, 1e-3 TF32).  Each plan runs at the bench's launch
configuration (cutoff chosen by the planner).  The oracle takes a few
seconds at 5000^2 and 20-40 s for the larger inputs on the GPU machine's host
cores; each reference is computed once per module."""
import functools

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=1)
def _paper_scale(m, n):
    A = inputs.normal(m, n, seed=1)
    return A, oracle.ata_packed(A), oracle.abs_gram_packed(A)


@functools.lru_cache(maxsize=1)
def _precision_form():
    A = inputs.scaled_cols(16384, 8192, seed=2)
    return A, oracle.ata_packed(A)


def _run(A_np, dtype):
    import torch
    m, n = A_np.shape
    plan = ata.Plan(m, n, dtype, 0)
    C = plan(torch.from_numpy(A_np).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    out = C.cpu().numpy()
    del C, plan
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("m,n,dtype", [(5000, 5000, ata.ATA_F64), (5000, 5000, ata.ATA_F64_OZAKI),
                                       (10000, 10000, ata.ATA_F64_OZAKI), (10000, 10000, ata.ATA_F64),
                                       (20000, 8000, ata.ATA_F64_OZAKI)])
def test_paper_scale_every_entry(gpu, m, n, dtype):
    A, ref, G = _paper_scale(m, n)
    C = _run(A, dtype)
    err = oracle.componentwise_error(C, ref, G)
    assert err <= 1e-11, err


@pytest.mark.parametrize("dtype,tol", [(ata.ATA_F32_BF16X3, 1e-6), (ata.ATA_F32_TF32, 1e-3)])
def test_precision_form_every_entry(gpu, dtype, tol):
    A, ref = _precision_form()
    C = _run(A, dtype)
    err = oracle.normwise_error(C, ref, 8192)
    assert err <= tol, err

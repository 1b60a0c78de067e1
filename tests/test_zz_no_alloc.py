"""ata_execute_static_scratch: the FP64 product for callers that may not
allocate device memory (graph-capture preparation, fixed-footprint services,
memory owned by another allocator).  Its scratch is a 64 MiB array inside
the library, so its output is checked here against ata_execute on the same
input, on two calls in a row (the second reuses what the first left in the
array).  This file sorts last so that a run stopping at the first failure has
run every other test first; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _call(A, C, cutoff):
    import torch
    m, n = A.shape
    st = ata.load().ata_execute_static_scratch(m, n, ctypes.c_void_p(A.data_ptr()), n,
                                               ctypes.c_void_p(C.data_ptr()), cutoff,
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("m,n,cutoff", [(512, 384, 64), (700, 500, 64)])
def test_static_scratch_matches_execute(gpu, m, n, cutoff):
    import torch
    A_np = inputs.normal(m, n, seed=m + n)
    A = torch.from_numpy(A_np).cuda()
    plan = ata.Plan(m, n, ata.ATA_F64, cutoff, fuse_levels=0)
    ref = plan(A)
    G = oracle.abs_gram_packed(A_np)
    for _ in range(2):
        C = torch.full((n * (n + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(A, C, cutoff) == ata.ATA_OK, ata.load().ata_last_error_message()
        torch.cuda.synchronize()
        err = oracle.componentwise_error(C.cpu().numpy(), ref.cpu().numpy(), G)
        assert err <= TOL


def test_static_scratch_rejects_oversize(gpu):
    import torch
    A = torch.zeros((2000, 1000), dtype=torch.float64, device="cuda")
    C = torch.zeros(1000 * 1001 // 2, dtype=torch.float64, device="cuda")
    assert _call(A, C, 64) == ata.ATA_EINVAL
    assert b"scratch" in ata.load().ata_last_error_message()

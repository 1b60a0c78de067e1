"""ata_execute_static_scratch: the FP64 product for callers that may not
allocate device memory while they run (code about to capture a CUDA graph,
services that fix their device-memory footprint at start-up, hosts whose
device memory belongs to another allocator).  Its scratch is a 64 MiB array
inside the library that every call shares, so the tests call it several times
in a row with different shapes and cutoffs (each call must overwrite the
tables, tile counter and status word the previous call left there) and check
every result against the oracle and, bit for bit, against ata_execute with
the same plan options (same tables, same kernels).

This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _call(A, C, cutoff, stream=None):
    import torch
    m, n = A.shape
    s = torch.cuda.current_stream() if stream is None else stream
    return ata.load().ata_execute_static_scratch(m, n, ctypes.c_void_p(A.data_ptr()), n,
                                                 ctypes.c_void_p(C.data_ptr()), cutoff,
                                                 ctypes.c_void_p(s.cuda_stream))


def _case(m, n, cutoff, seed):
    import torch
    A_np = inputs.normal(m, n, seed=seed)
    A = torch.from_numpy(A_np).cuda()
    ref = ata.Plan(m, n, ata.ATA_F64, cutoff, fuse_levels=0, variant=ata.ATA_STRASSEN)(A)
    torch.cuda.synchronize()
    return A_np, A, ref


def _check(A_np, A, ref, cutoff):
    import torch
    n = A_np.shape[1]
    C = torch.full((n * (n + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert _call(A, C, cutoff) == ata.ATA_OK, ata.load().ata_last_error_message()
    torch.cuda.synchronize()
    assert torch.equal(C, ref)  # same plan, same kernels: the same bits
    got = C.cpu().numpy()
    err = oracle.componentwise_error(got, oracle.ata_packed(A_np), oracle.abs_gram_packed(A_np))
    assert err <= TOL, err


@pytest.mark.parametrize("m,n,cutoff", [(512, 384, 64), (700, 500, 64)])
def test_static_scratch_twice(gpu, m, n, cutoff):
    case = _case(m, n, cutoff, seed=m + n)
    for _ in range(2):
        _check(*case, cutoff)


def test_static_scratch_larger_then_smaller(gpu):
    # a larger product (41 MiB of scratch), then a smaller one with another
    # cutoff and a deeper tree, then the larger again: stale tables, counter
    # or status words left by the previous call would show in the results
    big, small = (1200, 800, 128), (300, 257, 32)
    cb = _case(*big, seed=5)
    cs = _case(*small, seed=6)
    _check(*cb, big[2])
    _check(*cs, small[2])
    _check(*cb, big[2])


def test_static_scratch_rejects_oversize(gpu):
    import torch
    A = torch.zeros((2000, 1000), dtype=torch.float64, device="cuda")
    C = torch.zeros(1000 * 1001 // 2, dtype=torch.float64, device="cuda")
    assert _call(A, C, 64) == ata.ATA_EINVAL
    assert b"scratch" in ata.load().ata_last_error_message()


def test_static_scratch_refuses_a_capturing_stream(gpu):
    import torch
    A = torch.from_numpy(inputs.normal(64, 48, seed=1)).cuda()
    C = torch.zeros(48 * 49 // 2, dtype=torch.float64, device="cuda")
    x = torch.zeros(16, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        x.add_(1.0)
        st = _call(A, C, 16, stream=s)
    assert st == ata.ATA_EINVAL
    assert b"capturing" in ata.load().ata_last_error_message()
    assert bool((C == 0).all())  # nothing was queued

"""Pipelined end-to-end execution (ata_execute_host_async / ata_plan_wait):
copies of one call overlap the executions of its neighbours, on two device
staging sets used alternately.  Every queued call must give exactly the
result of the synchronous host call on its own input."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("dtype,m,n,cutoff", [
    (ata.ATA_F64, 700, 500, 128),
    (ata.ATA_F64_OZAKI, 1200, 900, 256),
    (ata.ATA_F32_BF16X3, 1100, 700, 256),
])
def test_pipelined_calls_equal_synchronous(gpu, dtype, m, n, cutoff):
    f32 = dtype in (ata.ATA_F32_BF16X3, ata.ATA_F32_TF32)
    mats = [inputs.normal(m, n, seed=40 + i).astype(np.float32 if f32 else np.float64) for i in range(5)]
    plan = ata.Plan(m, n, dtype, cutoff)
    want = [ata.ata_execute_host(plan, a) for a in mats]
    As = [pinned(a) for a in mats]
    Cs = [pinned(np.full(ata.packed_size(n), np.nan)) for _ in mats]
    for a, c in zip(As, Cs):  # five calls over the two staging sets
        ata.ata_execute_host_async(plan, a, c)
    ata.ata_plan_wait(plan)
    for w, c in zip(want, Cs):
        assert np.array_equal(w, c)
    assert plan.device_status() == 0
    # against the oracle as well (FP64 path: componentwise bound)
    if dtype == ata.ATA_F64:
        err = oracle.componentwise_error(Cs[2], oracle.ata_packed(mats[2]), oracle.abs_gram_packed(mats[2]))
        assert err <= 1e-11


def test_pipelined_reuses_buffers_and_interleaves_with_device_calls(gpu):
    import torch
    m, n = 600, 400
    plan = ata.Plan(m, n, ata.ATA_F64, 64)
    A = pinned(inputs.normal(m, n, seed=7))
    C = pinned(np.zeros(ata.packed_size(n)))
    for _ in range(4):  # the same host buffers every call
        ata.ata_execute_host_async(plan, A, C)
    ata.ata_plan_wait(plan)
    Cd = plan(torch.from_numpy(A).cuda())  # a device call after the wait
    torch.cuda.synchronize()
    assert np.array_equal(C, Cd.cpu().numpy())
    ata.ata_plan_wait(plan)  # nothing queued: returns at once


def test_pipelined_empty_and_degenerate(gpu):
    plan = ata.Plan(0, 5, ata.ATA_F64, 32)  # m = 0: C = 0
    C = np.full(ata.packed_size(5), np.nan)
    ata.ata_execute_host_async(plan, np.zeros((0, 5)), C)
    ata.ata_plan_wait(plan)
    assert np.all(C == 0)
    plan0 = ata.Plan(4, 0, ata.ATA_F64, 32)  # n = 0: nothing to do
    ata.ata_execute_host_async(plan0, np.zeros((4, 0)), np.zeros(0))
    ata.ata_plan_wait(plan0)

"""Failure detection, exercised without a GPU fault.

* The tensor-core leaf kernel bounds every wait of its pipeline.  A plan
  option shortens that limit to 1 us, far below the time the first chunk of
  MMAs takes, so the waits run out on purpose: the kernel must record the
  code in the plan's status word and return (the call completes, the
  context stays usable, a later product is exact).  The waits for copies and
  MMAs still in flight before the kernel exits keep their full limit.
* Device allocations fail on request from the host (ATA_FAULT=alloc@N): the
  call must return ATA_ENOMEM and free what it had allocated.
* ata_poll's bounded wait (ATA_ETIMEOUT) is in test_gpu_server.py.
"""
import gc
import os

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

# status codes of the leaf kernel's waits (include/ata.h, ata_plan_device_status)
WAIT_CODES = {1, 2, 3}


@pytest.mark.parametrize("dtype,opts", [(ata.ATA_F64_OZAKI, {}), (ata.ATA_F32_BF16X3, {}),
                                        (ata.ATA_F32_TF32, {"cta_pair": 0})])
def test_pipeline_waits_run_out(gpu, dtype, opts):
    import torch
    f64 = dtype == ata.ATA_F64_OZAKI
    A_np = inputs.integers(2048, 640, seed=4).astype(np.float64 if f64 else np.float32)
    A = torch.from_numpy(A_np).cuda()
    # classical leaves (cutoff above n): one launch over 15 tiles of K = 2048
    bad = ata.Plan(2048, 640, dtype, 4096, wait_limit_us=1, **opts)
    C = torch.zeros(640 * 641 // 2, dtype=torch.float64, device="cuda")
    bad(A, C)
    torch.cuda.synchronize()  # the kernel returned
    assert bad.device_status() in WAIT_CODES
    del bad
    # the context is usable and the default limit computes the exact product
    good = ata.Plan(2048, 640, dtype, 4096, **opts)
    C2 = good(A)
    torch.cuda.synchronize()
    assert good.device_status() == 0
    assert np.array_equal(C2.cpu().numpy(), oracle.ata_packed(A_np))


def test_wait_limit_option_is_checked(gpu):
    with pytest.raises(ata.AtaError) as e:
        ata.Plan(256, 128, ata.ATA_F32_BF16X3, 4096, wait_limit_us=2_000_000)
    assert e.value.status == ata.ATA_EINVAL


def _held():
    gc.collect()
    return ata.ata_device_bytes_held()


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F64_OZAKI])
def test_allocation_faults_return_enomem_and_leak_nothing(gpu, dtype):
    import torch
    torch.cuda.synchronize()
    base = _held()
    failures = 0
    try:
        for n_fail in range(1, 12):
            os.environ["ATA_FAULT"] = f"alloc@{n_fail}"
            try:
                p = ata.Plan(3000, 1500, dtype, 256)
            except ata.AtaError as e:
                assert e.status == ata.ATA_ENOMEM
                failures += 1
                assert _held() == base
                continue
            # every allocation of the plan succeeded: it runs, and frees all
            A_np = inputs.integers(3000, 1500, seed=2).astype(np.float64)
            C = p(torch.from_numpy(A_np).cuda())
            torch.cuda.synchronize()
            assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(A_np))
            assert _held() > base
            del p
            assert _held() == base
            break
        else:
            pytest.fail("plan creation never succeeded")
    finally:
        os.environ.pop("ATA_FAULT", None)
    assert failures >= 2  # the workspace and the task tables at least


def test_allocation_fault_in_host_staging(gpu):
    import torch
    base = _held()
    A_np = inputs.integers(500, 300, seed=3).astype(np.float64)
    p = ata.Plan(500, 300, ata.ATA_F64, 64)
    C_host = np.zeros(300 * 301 // 2)
    try:
        os.environ["ATA_FAULT"] = "alloc@1"  # the staging buffer for A
        with pytest.raises(ata.AtaError) as e:
            ata.ata_execute_host(p, A_np, C_host)
        assert e.value.status == ata.ATA_ENOMEM
        os.environ["ATA_FAULT"] = "alloc@2"  # A's succeeds, C's fails
        with pytest.raises(ata.AtaError) as e:
            ata.ata_execute_host(p, A_np, C_host)
        assert e.value.status == ata.ATA_ENOMEM
        del e  # its traceback holds the plan
    finally:
        os.environ.pop("ATA_FAULT", None)
    ata.ata_execute_host(p, A_np, C_host)  # no injection: runs
    assert np.array_equal(C_host, oracle.ata_packed(A_np))
    del p
    torch.cuda.synchronize()
    assert _held() == base

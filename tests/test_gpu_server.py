"""Serving form: continuous batching through ata_server_create / ata_submit /
ata_poll.  Each result must be bitwise equal to the same request run alone
(same plan, same kernels), whatever else is in flight, and within the mode's
stated bound of the oracle.

The server's streams do not wait for the caller's streams, so every input is
complete (the current stream synchronised) before it is submitted.  No test here
offers the server more work than it completes: plain-FP64 serving under
overload is kept off the GPU (an unexplained illegal-address fault)."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

NORM_TOL = {ata.ATA_F32_BF16X3: 1e-6, ata.ATA_F32_TF32: 1e-3}


@pytest.mark.parametrize("dtype", [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
def test_mix_equals_alone_and_oracle(gpu, dtype):
    import torch
    shapes = [(300, 200), (1000, 129), (129, 400), (777, 333), (2048, 64), (500, 500)]
    f64 = dtype == ata.ATA_F64_OZAKI
    mats_np = [inputs.normal(m, n, seed=i, dtype=np.float64 if f64 else np.float32) for i, (m, n) in enumerate(shapes)]
    mats = [torch.from_numpy(a).cuda() for a in mats_np]
    alone = []
    for (m, n), A in zip(shapes, mats):
        p = ata.Plan(m, n, dtype, 0)
        alone.append(p(A).clone())
    torch.cuda.synchronize()
    srv = ata.Server(8 << 30, dtype, max_inflight=4)
    try:
        reqs = []
        for rep in range(5):
            for i, (m, n) in enumerate(shapes):
                C = torch.full((n * (n + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
                torch.cuda.current_stream().synchronize()  # the fill is done before the server writes C
                reqs.append((i, C, srv.submit(mats[i], C)))
        for i, C, t in reqs:
            assert srv.poll(t, 10_000_000) == ata.ATA_OK
            assert torch.equal(C, alone[i])
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["p99_us"] >= st["p50_us"] > 0
        assert srv.kernels() > 0
    finally:
        srv.close()
    # every served result against the oracle (each request of a shape is
    # bitwise equal to the alone run, so one comparison per shape covers all)
    for i, a in enumerate(mats_np):
        if f64:  # the FP64 emulation: componentwise, as the FP64 path
            err = oracle.componentwise_error(alone[i].cpu().numpy(), oracle.ata_packed(a), oracle.abs_gram_packed(a))
            assert err <= 1e-11, (shapes[i], err)
        else:
            err = oracle.normwise_error(alone[i].cpu().numpy(), oracle.ata_packed(a), a.shape[1])
            assert err <= NORM_TOL[dtype], (shapes[i], err)


def test_budget_too_small_fails_the_request(gpu):
    import torch
    srv = ata.Server(1 << 20, ata.ATA_F32_BF16X3, max_inflight=2)  # 1 MiB: no plan fits
    A = torch.zeros((4096, 1024), dtype=torch.float32, device="cuda")
    C = torch.zeros(1024 * 1025 // 2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    try:
        t = srv.submit(A, C)
        with pytest.raises(ata.AtaError) as e:
            srv.poll(t, 10_000_000)
        assert e.value.status == ata.ATA_EBUSY
    finally:
        srv.close()


def test_poll_pending_and_unknown_ticket(gpu):
    import torch
    srv = ata.Server(8 << 30, ata.ATA_F64, max_inflight=1)
    A = torch.from_numpy(inputs.normal(4000, 2000, seed=1)).cuda()
    C = torch.empty(2000 * 2001 // 2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    try:
        t = srv.submit(A, C)
        st = srv.poll(t, 0)
        assert st in (ata.ATA_OK, ata.ATA_PENDING)
        if st == ata.ATA_PENDING:
            assert srv.poll(t, 30_000_000) == ata.ATA_OK
        with pytest.raises(ata.AtaError):
            srv.poll(t + 1000, 0)
    finally:
        srv.close()


def test_poll_times_out_then_completes(gpu):
    """A bounded wait on a request that needs longer returns ATA_ETIMEOUT and
    keeps the ticket; a later wait sees it complete.  The first request
    (FP64, 8192 x 2048: about 30 ms of DFMA work, plus plan creation) is
    still running 200 us after submission."""
    import torch
    m, n = 8192, 2048
    A_np = inputs.normal(m, n, seed=3)
    A = torch.from_numpy(A_np).cuda()
    C = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    srv = ata.Server(8 << 30, ata.ATA_F64, max_inflight=1)
    try:
        t = srv.submit(A, C)
        assert srv.poll(t, 200) == ata.ATA_ETIMEOUT
        assert srv.poll(t, 60_000_000) == ata.ATA_OK
    finally:
        srv.close()
    I = np.arange(0, n, 97)
    J = np.minimum(I + 5, n - 1)
    got = C[torch.from_numpy(oracle.packed_index(I, J, n)).cuda()].cpu().numpy()
    err = oracle.componentwise_error(got, oracle.ata_entries(A_np, I, J), oracle.ata_entries(A_np, I, J, absval=True))
    assert err <= 1e-11

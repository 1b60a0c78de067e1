"""Serving form: continuous batching through ata_server_create / ata_submit /
ata_poll.  Each result must be bitwise equal to the same request run alone
(same plan, same kernels), whatever else is in flight."""
import numpy as np
import pytest

import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_mix_equals_alone(gpu):
    import torch
    shapes = [(300, 200), (1000, 129), (129, 400), (777, 333), (2048, 64), (500, 500)]
    mats = [torch.from_numpy(inputs.normal(m, n, seed=i, dtype=np.float32)).cuda() for i, (m, n) in enumerate(shapes)]
    alone = []
    for (m, n), A in zip(shapes, mats):
        p = ata.Plan(m, n, ata.ATA_F32_BF16X3, 0)
        alone.append(p(A).clone())
    torch.cuda.synchronize()
    srv = ata.Server(8 << 30, ata.ATA_F32_BF16X3, max_inflight=4)
    reqs = []
    for rep in range(5):
        for i, (m, n) in enumerate(shapes):
            C = torch.full((n * (n + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
            reqs.append((i, C, srv.submit(mats[i], C)))
    for i, C, t in reqs:
        assert srv.poll(t, 10_000_000) == ata.ATA_OK
        assert torch.equal(C, alone[i])
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_us"] >= st["p50_us"] > 0
    srv.close()


def test_budget_too_small_fails_the_request(gpu):
    import torch
    srv = ata.Server(1 << 20, ata.ATA_F32_BF16X3, max_inflight=2)  # 1 MiB: no plan fits
    A = torch.zeros((4096, 1024), dtype=torch.float32, device="cuda")
    C = torch.zeros(1024 * 1025 // 2, dtype=torch.float64, device="cuda")
    t = srv.submit(A, C)
    with pytest.raises(ata.AtaError) as e:
        srv.poll(t, 10_000_000)
    assert e.value.status == ata.ATA_EBUSY
    srv.close()


def test_poll_pending_and_unknown_ticket(gpu):
    import torch
    srv = ata.Server(8 << 30, ata.ATA_F64, max_inflight=1)
    A = torch.from_numpy(inputs.normal(4000, 2000, seed=1)).cuda()
    C = torch.empty(2000 * 2001 // 2, dtype=torch.float64, device="cuda")
    t = srv.submit(A, C)
    st = srv.poll(t, 0)
    assert st in (ata.ATA_OK, ata.ATA_PENDING)
    if st == ata.ATA_PENDING:
        assert srv.poll(t, 30_000_000) == ata.ATA_OK
    with pytest.raises(ata.AtaError):
        srv.poll(t + 1000, 0)
    srv.close()


def test_f64_concurrent_plans_and_evictions(gpu, monkeypatch):
    """Many FP64 plans of different shapes on concurrent streams, with a
    budget small enough to force evictions; kernels self-check every global
    access (ATA_CHECK_BOUNDS=1) and each result must equal the alone run."""
    import torch
    monkeypatch.setenv("ATA_CHECK_BOUNDS", "1")
    rng = np.random.default_rng(7)
    shapes = [(int(m), int(n)) for m, n in zip(rng.integers(128, 3000, 24), rng.integers(64, 900, 24))]
    mats = [torch.from_numpy(inputs.normal(m, n, seed=i)).cuda() for i, (m, n) in enumerate(shapes)]
    alone = []
    for (m, n), A in zip(shapes, mats):
        p = ata.Plan(m, n, ata.ATA_F64, 0)
        alone.append(p(A).clone())
        assert p.device_status() == 0
    torch.cuda.synchronize()
    budget = 3 * max(ata.ata_plan_query(m, n, ata.ATA_F64, 0)["workspace_bytes"] for m, n in shapes) + (64 << 20)
    srv = ata.Server(budget, ata.ATA_F64, max_inflight=8)
    reqs = []
    for rep in range(2):
        for i in range(len(shapes)):
            m, n = shapes[i]
            C = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device="cuda")
            reqs.append((i, C, srv.submit(mats[i], C)))
    for i, C, t in reqs:
        assert srv.poll(t, 60_000_000) == ata.ATA_OK
        assert torch.equal(C, alone[i])
    srv.close()

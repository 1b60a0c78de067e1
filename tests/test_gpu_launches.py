"""The launch counts that bench.py reports: the planner's count of kernels
per execution (ata_plan_info.n_launches) must equal the kernel nodes of the
captured graph, for single plans, batches and served requests."""
import numpy as np
import pytest

import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,m,n,cutoff,opts", [
    (ata.ATA_F64, 700, 600, 64, {}),
    (ata.ATA_F64, 700, 600, 64, {"variant": ata.ATA_WINOGRAD}),
    (ata.ATA_F64, 100, 30, 64, {}),  # a single leaf
    (ata.ATA_F64_OZAKI, 1500, 1300, 256, {}),
    (ata.ATA_F64_OZAKI, 1500, 1300, 256, {"variant": ata.ATA_WINOGRAD}),
    (ata.ATA_F64_OZAKI, 1500, 1300, 256, {"fuse_levels": 0}),
    (ata.ATA_F32_BF16X3, 1500, 1300, 256, {}),
    (ata.ATA_F32_BF16X3, 1500, 1300, 256, {"fuse_levels": 2}),
    (ata.ATA_F32_TF32, 1500, 1300, 256, {}),
])
def test_graph_kernels_equal_planned_launches(gpu, dtype, m, n, cutoff, opts):
    import torch
    f32 = dtype in (ata.ATA_F32_BF16X3, ata.ATA_F32_TF32)
    A = torch.from_numpy(inputs.normal(m, n, seed=5).astype(np.float32 if f32 else np.float64)).cuda()
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    with pytest.raises(ata.AtaError):
        plan.graph_kernels()  # nothing captured yet
    plan(A)
    torch.cuda.synchronize()
    assert plan.graph_kernels() == plan.info["n_launches"] > 0


def test_batched_graph_kernels(gpu):
    import torch
    shapes = [(300, 200), (64, 33), (1000, 129)]
    plans = [ata.Plan(m, n, ata.ATA_F32_BF16X3, 0) for m, n in shapes]
    As = [torch.from_numpy(inputs.normal(m, n, seed=i).astype(np.float32)).cuda() for i, (m, n) in enumerate(shapes)]
    with pytest.raises(ata.AtaError):
        ata.ata_batched_graph_kernels(plans, As)  # not executed yet
    ata.ata_execute_batched(plans[:1], As[:1])
    ata.ata_execute_batched(plans, As)
    torch.cuda.synchronize()
    # one instance: the plan's own launches; several: one split / combine
    # launch per level and one set of leaf kernels for all of them
    assert ata.ata_batched_graph_kernels(plans[:1], As[:1]) == plans[0].info["n_launches"]
    k = ata.ata_batched_graph_kernels(plans, As)
    assert 0 < k <= sum(p.info["n_launches"] for p in plans)
    assert k >= max(p.info["n_launches"] for p in plans)


def test_server_counts_kernels(gpu):
    import torch
    m, n = 500, 300
    A = torch.from_numpy(inputs.normal(m, n, seed=2).astype(np.float32)).cuda()
    C = torch.empty(ata.packed_size(n), dtype=torch.float64, device="cuda")
    srv = ata.Server(1 << 30, ata.ATA_F32_BF16X3, max_inflight=2)
    try:
        srv.poll(srv.submit(A, C), 600_000_000)
        srv.reset_stats()
        assert srv.kernels() == 0
        for _ in range(3):
            srv.poll(srv.submit(A, C), 600_000_000)
        per = ata.ata_plan_query(m, n, ata.ATA_F32_BF16X3, 0)["n_launches"]
        assert srv.kernels() == 3 * per
    finally:
        srv.close()

"""ata_execute and ata_gemm_tn inside a stream capture (torch.cuda.graph).

A graph launch cannot itself be captured, so on a capturing stream the
plan's kernels are enqueued into the caller's capture directly: the same
kernels and parameters a replay of the plan's own graph runs.  The captured
graph reads A and writes C at the capture's pointers.  The plan must outlive
it, and the caller orders its replays with the plan's other executions.  A
leading dimension that would need new tables is refused inside a capture
(ATA_EINVAL, nothing queued), and the capture stays valid."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = [ata.ATA_F64, ata.ATA_F64_OZAKI, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32]


def _dt(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


@pytest.mark.parametrize("dtype", ALL)
def test_execute_inside_a_capture(gpu, dtype):
    import torch
    m, n = 1500, 900
    A1, A2 = (inputs.integers(m, n, seed=s).astype(_dt(dtype)) for s in (101, 102))
    plan = ata.Plan(m, n, dtype, 64 if dtype == ata.ATA_F64 else 256)
    assert plan.info["max_strassen_levels"] >= 1
    A = torch.from_numpy(A1).cuda()
    C = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        plan(A, C, stream=s)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(A1))
    A.copy_(torch.from_numpy(A2))  # new contents at the captured pointer
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(A2))
    C2 = plan(A)  # an ordinary execution afterwards
    torch.cuda.synchronize()
    assert torch.equal(C2, C)
    assert plan.device_status() == 0


def test_capture_refuses_a_new_leading_dimension(gpu):
    import torch
    m, n = 400, 250
    wide = torch.from_numpy(inputs.integers(m, n + 6, seed=103).astype(np.float64)).cuda()
    A = wide[:, :n]  # lda = n + 6: the plan's tables are for lda = n
    plan = ata.Plan(m, n, ata.ATA_F64, 64)
    C = torch.zeros(n * (n + 1) // 2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        with pytest.raises(ata.AtaError) as e:
            plan(A, C, stream=s)
    assert e.value.status == ata.ATA_EINVAL
    assert "capturing" in str(e.value)
    g.replay()  # the (empty) capture ended normally
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0
    plan(A, C)  # outside a capture the new leading dimension is taken
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(wide[:, :n].cpu().numpy()))


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F64_OZAKI, ata.ATA_F32_BF16X3])
def test_general_product_inside_a_capture(gpu, dtype):
    import torch
    m, p, r = 1200, 700, 500
    X1, Y1 = inputs.integers(m, p, seed=104).astype(_dt(dtype)), inputs.integers(m, r, seed=105).astype(_dt(dtype))
    plan = ata.GemmPlan(m, p, r, dtype, 256)
    X, Y = torch.from_numpy(X1).cuda(), torch.from_numpy(Y1).cuda()
    C = torch.empty((p, r), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        plan(X, Y, C, stream=s)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm_tn(X1, Y1))


def test_batched_and_host_calls_refuse_a_capture(gpu):
    # batched executions launch the batch's graph (and may upload bindings
    # from host memory); host-buffer executions copy from host memory: none
    # can be recorded, so each refuses before any CUDA call
    import torch
    shapes = [(300, 200), (500, 129)]
    plans = [ata.Plan(m, n, ata.ATA_F32_BF16X3, 256) for m, n in shapes]
    mats = [torch.from_numpy(inputs.integers(m, n, seed=110 + i).astype(np.float32)).cuda()
            for i, (m, n) in enumerate(shapes)]
    Cs = [torch.zeros(n * (n + 1) // 2, dtype=torch.float64, device="cuda") for _, n in shapes]
    batch = ata.Batch(plans)
    A_all = torch.zeros(batch.a_numel, dtype=torch.float32, device="cuda")
    host_plan = ata.Plan(200, 100, ata.ATA_F64, 64)
    A_host = inputs.integers(200, 100, seed=112)
    C_host = np.zeros(100 * 101 // 2)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        for call in (lambda: ata.ata_execute_batched(plans, mats, Cs, stream=s),
                     lambda: batch(A_all, stream=s),
                     lambda: ata.ata_execute_host(host_plan, A_host, C_host, stream=s)):
            with pytest.raises(ata.AtaError) as e:
                call()
            assert e.value.status == ata.ATA_EINVAL and "capturing" in str(e.value)
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.count_nonzero(c).item() == 0 for c in Cs)
    # outside the capture every call runs
    ata.ata_execute_batched(plans, mats, Cs)
    ata.ata_execute_host(host_plan, A_host, C_host)
    torch.cuda.synchronize()
    for c, a in zip(Cs, mats):
        assert np.array_equal(c.cpu().numpy(), oracle.ata_packed(a.cpu().numpy()))
    assert np.array_equal(C_host, oracle.ata_packed(A_host))

"""Executions of one plan queued on different streams run one at a time.

A plan's executions share its workspace (operand sums, slices, Strassen
products), its leaf tile counter and its status word.  An execution queued
on another stream than the plan's latest one waits for it (an event), in
single-plan, batched and prepared-batch calls alike.  Back-to-back calls on
two streams, with no host synchronisation between them, must therefore
each give their own exact product (integer inputs: exact in every mode)."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dt(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F64_OZAKI, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32])
def test_one_plan_on_alternating_streams(gpu, dtype):
    import torch
    m, n = (1200, 700) if dtype == ata.ATA_F64 else (2000, 1200)
    mats = [inputs.integers(m, n, seed=70 + i).astype(_dt(dtype)) for i in range(4)]
    refs = [oracle.ata_packed(a) for a in mats]
    # Strassen levels: every execution rewrites the plan's workspace
    plan = ata.Plan(m, n, dtype, 64 if dtype == ata.ATA_F64 else 256)
    assert plan.info["max_strassen_levels"] >= 1
    dev = [torch.from_numpy(a).cuda() for a in mats]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.empty(n * (n + 1) // 2, dtype=torch.float64, device="cuda") for _ in range(8)]
    torch.cuda.synchronize()
    for i in range(8):
        plan(dev[i % 4], outs[i], stream=streams[i % 2])
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    for i in range(8):
        assert np.array_equal(outs[i].cpu().numpy(), refs[i % 4]), i


@pytest.mark.parametrize("dtype", [ata.ATA_F64_OZAKI, ata.ATA_F32_BF16X3])
def test_batched_and_single_calls_on_two_streams(gpu, dtype):
    import torch
    shapes = [(1500, 700), (900, 513), (1200, 300)]
    plans = [ata.Plan(m, n, dtype, 256) for m, n in shapes]
    A1 = [inputs.integers(m, n, seed=80 + i).astype(_dt(dtype)) for i, (m, n) in enumerate(shapes)]
    A2 = inputs.integers(*shapes[0], seed=90).astype(_dt(dtype))
    d1 = [torch.from_numpy(a).cuda() for a in A1]
    d2 = torch.from_numpy(A2).cuda()
    C2 = torch.empty(shapes[0][1] * (shapes[0][1] + 1) // 2, dtype=torch.float64, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    Cs = [torch.empty(n * (n + 1) // 2, dtype=torch.float64, device="cuda") for _, n in shapes]
    torch.cuda.synchronize()
    for _ in range(3):
        ata.ata_execute_batched(plans, d1, Cs, stream=s1)  # uses the workspaces of all three plans
        plans[0](d2, C2, stream=s2)                        # the first plan again, on another stream
    torch.cuda.synchronize()
    for c, a in zip(Cs, A1):
        assert np.array_equal(c.cpu().numpy(), oracle.ata_packed(a))
    assert np.array_equal(C2.cpu().numpy(), oracle.ata_packed(A2))

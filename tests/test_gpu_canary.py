"""Canary guard bands (ATA_CANARY=1 at plan creation): 64 KiB of a known
byte before and after every plan workspace.  ata_plan_device_status reads
them back and reports 90 (before) or 91 (after) if any byte changed, so a
kernel that wrote past its workspace would show here.  Every mode, with
Strassen levels (materialised and fused operand sums, combines into the
workspace), batched and general products: the bands must be intact and the
results correct."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [(ata.ATA_F64, 64), (ata.ATA_F64_OZAKI, 256), (ata.ATA_F32_BF16X3, 256), (ata.ATA_F32_TF32, 256)]


def _dt(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


@pytest.mark.parametrize("dtype,cutoff", MODES)
@pytest.mark.parametrize("variant", [ata.ATA_STRASSEN, ata.ATA_WINOGRAD])
def test_workspace_canaries_intact(gpu, monkeypatch, dtype, cutoff, variant):
    import torch
    monkeypatch.setenv("ATA_CANARY", "1")
    m, n = 1100, 777
    A_np = inputs.integers(m, n, seed=51).astype(_dt(dtype))
    held0 = ata.ata_device_bytes_held()
    plan = ata.Plan(m, n, dtype, cutoff, variant=variant)
    ws = plan.info["workspace_bytes"]
    assert ws > 0 and plan.info["max_strassen_levels"] >= 1
    assert ata.ata_device_bytes_held() - held0 >= ws + 2 * 65536
    C = plan(torch.from_numpy(A_np).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(A_np))


@pytest.mark.parametrize("dtype,cutoff", MODES)
def test_canaries_batched_and_general_product(gpu, monkeypatch, dtype, cutoff):
    import torch
    monkeypatch.setenv("ATA_CANARY", "1")
    shapes = [(700, 300), (300, 520), (900, 260)]
    mats = [inputs.integers(m, n, seed=60 + i).astype(_dt(dtype)) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, dtype, cutoff) for m, n in shapes]
    Cs = ata.ata_execute_batched(plans, [torch.from_numpy(a).cuda() for a in mats])
    torch.cuda.synchronize()
    for p, a, c in zip(plans, mats, Cs):
        assert p.device_status() == 0
        assert np.array_equal(c.cpu().numpy(), oracle.ata_packed(a))
    X = inputs.integers(800, 500, seed=70).astype(_dt(dtype))
    Y = inputs.integers(800, 330, seed=71).astype(_dt(dtype))
    g = ata.GemmPlan(800, 500, 330, dtype, cutoff)
    C = torch.empty((500, 330), dtype=torch.float64, device="cuda")
    g(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), C)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    assert np.array_equal(C.cpu().numpy(), oracle.gemm_tn(X, Y))

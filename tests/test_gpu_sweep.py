"""Seeded sweep of random shapes and plan options in every mode against the
oracle.  Exact-integer inputs (entries in -4..4, every partial sum an
integer below 2^24) must match bit for bit in every mode, whatever the
shape, cutoff, Strassen variant, fused levels, tile form or batch; the
shapes are drawn to cross tile edges (multiples of 128 plus or minus a few),
to be tall, wide, tiny and ragged."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [ata.ATA_F64, ata.ATA_F64_OZAKI, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32]


def _dt(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


def _dim(rng, hi):
    kind = rng.integers(0, 4)
    if kind == 0:
        return int(rng.integers(1, 40))                        # tiny
    if kind == 1:
        return int(128 * rng.integers(1, hi // 128 + 1) + rng.integers(-3, 4))  # near a tile edge
    return int(rng.integers(40, hi))                           # ragged


def _cases(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m, n = max(1, _dim(rng, 1100)), max(1, _dim(rng, 900))
        out.append((m, n, int(rng.choice([16, 32, 64, 128, 256, 512])), int(rng.integers(0, 2)),
                    int(rng.integers(0, 3)), int(rng.integers(0, 2))))
    return out


@pytest.mark.parametrize("dtype", MODES)
@pytest.mark.parametrize("case", range(10))
def test_sweep_exact(gpu, dtype, case):
    import torch
    m, n, cutoff, variant, fuse, pair = _cases(1000 + int(dtype), 10)[case]
    if dtype != ata.ATA_F64 and cutoff < 128:
        cutoff = 128 + cutoff  # tensor-core leaves: keep the tile count of a test modest
    if dtype == ata.ATA_F64_OZAKI and variant == ata.ATA_WINOGRAD:
        fuse = 0  # Winograd's chained sums stay materialised in this mode
    A_np = inputs.integers(m, n, seed=m * 7 + n).astype(_dt(dtype))
    opts = dict(variant=variant, fuse_levels=fuse)
    if dtype != ata.ATA_F64:
        opts["cta_pair"] = pair
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    C = plan(torch.from_numpy(A_np).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert np.array_equal(C.cpu().numpy(), oracle.ata_packed(A_np)), (m, n, cutoff, opts)


@pytest.mark.parametrize("dtype", MODES)
def test_sweep_general_products_exact(gpu, dtype):
    import torch
    rng = np.random.default_rng(77 + int(dtype))
    for _ in range(6):
        m, p, r = max(1, _dim(rng, 900)), max(1, _dim(rng, 700)), max(1, _dim(rng, 700))
        cutoff = int(rng.choice([64, 128, 256])) if dtype == ata.ATA_F64 else int(rng.choice([128, 256, 512]))
        X = inputs.integers(m, p, seed=int(rng.integers(1 << 30))).astype(_dt(dtype))
        Y = inputs.integers(m, r, seed=int(rng.integers(1 << 30))).astype(_dt(dtype))
        g = ata.GemmPlan(m, p, r, dtype, cutoff, variant=int(rng.integers(0, 2)) if dtype != ata.ATA_F64_OZAKI else 0)
        C = torch.empty((p, r), dtype=torch.float64, device="cuda")
        g(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), C)
        torch.cuda.synchronize()
        assert g.device_status() == 0
        assert np.array_equal(C.cpu().numpy(), oracle.gemm_tn(X, Y)), (m, p, r, cutoff)


@pytest.mark.parametrize("dtype", MODES)
def test_sweep_batch_exact(gpu, dtype):
    import torch
    rng = np.random.default_rng(91 + int(dtype))
    shapes = [(max(1, _dim(rng, 800)), max(1, _dim(rng, 600))) for _ in range(24)]
    mats = [inputs.integers(m, n, seed=i + 5).astype(_dt(dtype)) for i, (m, n) in enumerate(shapes)]
    cut = 64 if dtype == ata.ATA_F64 else 256
    plans = [ata.Plan(m, n, dtype, cut, cta_pair=0) if dtype != ata.ATA_F64 else ata.Plan(m, n, dtype, cut)
             for m, n in shapes]
    batch = ata.Batch(plans)
    A_all = torch.zeros(batch.a_numel, dtype=batch.in_dtype)
    for v, a in zip(batch.input_views(A_all), mats):
        v.copy_(torch.from_numpy(a))
    C_all = batch(A_all.cuda())
    torch.cuda.synchronize()
    for c, a in zip(batch.output_views(C_all), mats):
        assert np.array_equal(c.cpu().numpy(), oracle.ata_packed(a))

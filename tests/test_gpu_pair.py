"""The CTA-pair leaf kernel (tcgen05 cta_group::2 on two SMs: 256 x 128
output tiles, 256 x 256 for TF32) against the oracle and against the
single-CTA kernel.

With the plan option cta_pair=1 (the default for TF32), a plan whose leaves
are all wider than one 128-row tile pads its X operands to whole 256-row
tiles and runs the pair kernel when its tiles add at most 1/8 to the tile
area; `leaf_tile_rows` and `leaf_tile_cols` in the plan info say which
kernel runs.
"""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]


def run(A_np, dtype, cutoff, **opts):
    import torch
    m, n = A_np.shape
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    C = plan(A)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return C.cpu().numpy(), plan


def in_dtype(dtype):
    return np.float64 if dtype == ata.ATA_F64_OZAKI else np.float32


def tile_cols(dtype):
    return 256 if dtype == ata.ATA_F32_TF32 else 128


@pytest.mark.parametrize("p,r", [(1024, 1100), (1000, 1030)])
def test_tf32_wide_pair_ragged_general_product(gpu, p, r):
    # C = X^t Y on 256 x 256 pair tiles whose last tile column reaches past
    # Y's padding to 128 rows (r_pad = 1152: the odd CTA's half of that tile
    # lies wholly outside it and reads TMA's zero fill), exact integers:
    # bitwise against the oracle and against single-CTA tiles
    import torch
    m = 500
    X = inputs.integers(m, p, seed=p).astype(np.float32)
    Y = inputs.integers(m, r, seed=r + 1).astype(np.float32)
    out = {}
    for pair in (1, 0):
        plan = ata.GemmPlan(m, p, r, ata.ATA_F32_TF32, 512, cta_pair=pair)
        info = plan.info
        want = (256, 256) if pair else (128, 128)
        assert (info["leaf_tile_rows"], info["leaf_tile_cols"]) == want, info
        C = plan(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        out[pair] = C.cpu().numpy()
    assert np.array_equal(out[1], oracle.gemm_tn(X, Y))
    assert np.array_equal(out[1], out[0])


@pytest.mark.parametrize("dtype", MODES)
@pytest.mark.parametrize("m,n,cutoff,fuse", [(700, 999, 512, 1), (1030, 1000, 512, 0), (300, 1537, 768, 1),
                                             (257, 1000, 1024, 1)])
def test_pair_exact_integers(gpu, dtype, m, n, cutoff, fuse):
    # leaves of 250..600 columns: several 256-row pair tiles, ragged edges,
    # SYRK diagonal leaves and Strassen products
    A = inputs.integers(m, n, seed=m * 7 + n).astype(in_dtype(dtype))
    C, plan = run(A, dtype, cutoff, fuse_levels=fuse, cta_pair=1)
    info = plan.info
    if dtype == ata.ATA_F32_TF32 and (m, n, cutoff) == (300, 1537, 768):
        # 256 x 256 tiles would add more than 1/8 to these leaves' tile area
        assert (info["leaf_tile_rows"], info["leaf_tile_cols"]) == (128, 128), info
    else:
        assert (info["leaf_tile_rows"], info["leaf_tile_cols"]) == (256, tile_cols(dtype)), info
    assert np.array_equal(C, oracle.ata_packed(A))


@pytest.mark.parametrize("dtype", MODES)
def test_pair_matches_single_cta(gpu, dtype):
    m, n, cutoff = 1500, 2000, 1024
    A = (inputs.normal(m, n, seed=21) if dtype == ata.ATA_F64_OZAKI
         else inputs.scaled_cols(m, n, seed=21)).astype(in_dtype(dtype))
    C2, plan2 = run(A, dtype, cutoff, cta_pair=1)
    C1, plan1 = run(A, dtype, cutoff, cta_pair=0)
    assert (plan2.info["leaf_tile_rows"], plan2.info["leaf_tile_cols"]) == (256, tile_cols(dtype))
    assert (plan1.info["leaf_tile_rows"], plan1.info["leaf_tile_cols"]) == (128, 128)
    # the same dot products in the same K order: identical results
    assert np.array_equal(C1, C2), float(np.max(np.abs(C1 - C2)))
    ref = oracle.ata_packed(A)
    if dtype == ata.ATA_F64_OZAKI:
        assert oracle.componentwise_error(C2, ref, oracle.abs_gram_packed(A)) <= 1e-11
    else:
        tol = 1e-6 if dtype == ata.ATA_F32_BF16X3 else 1e-3
        assert oracle.normwise_error(C2, ref, n) <= tol


def test_pair_small_leaves_use_single_cta(gpu):
    # leaves of at most 128 rows gain nothing from pair tiles
    A = inputs.integers(400, 500, seed=3).astype(np.float32)
    C, plan = run(A, ata.ATA_F32_BF16X3, 64, cta_pair=1)
    assert plan.info["leaf_tile_rows"] == 128
    assert np.array_equal(C, oracle.ata_packed(A))

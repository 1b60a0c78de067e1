"""The CTA-pair leaf kernel (tcgen05 cta_group::2, 256 x 128 output tiles
on two SMs) against the oracle and against the single-CTA kernel.

A plan whose leaves are all wider than one 128-row tile pads its X operands
to whole 256-row tiles and runs the pair kernel; `leaf_tile_rows` in the
plan info says which kernel runs.  The single-CTA kernel is selected for a
whole process by ATA_NO_CTA_PAIR=1, so the comparison runs it in a child
process on the same input.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


@pytest.mark.parametrize("dtype", MODES)
@pytest.mark.parametrize("m,n,cutoff,fuse", [(700, 999, 512, 1), (1030, 1000, 512, 0), (300, 1537, 768, 1),
                                             (257, 1000, 1024, 1)])
def test_pair_exact_integers(gpu, dtype, m, n, cutoff, fuse):
    # leaves of 250..600 columns: several 256-row pair tiles, ragged edges,
    # SYRK diagonal leaves and Strassen products
    A = inputs.integers(m, n, seed=m * 7 + n).astype(in_dtype(dtype))
    C, plan = run(A, dtype, cutoff, fuse_levels=fuse)
    assert plan.info["leaf_tile_rows"] == 256, plan.info
    assert np.array_equal(C, oracle.ata_packed(A))


@pytest.mark.parametrize("dtype", MODES)
def test_pair_matches_single_cta(gpu, dtype, tmp_path):
    m, n, cutoff = 1500, 2000, 1024
    A = (inputs.normal(m, n, seed=21) if dtype == ata.ATA_F64_OZAKI
         else inputs.scaled_cols(m, n, seed=21)).astype(in_dtype(dtype))
    C2, plan = run(A, dtype, cutoff)
    assert plan.info["leaf_tile_rows"] == 256
    src = tmp_path / "A.npy"
    out = tmp_path / "C1.npy"
    np.save(src, A)
    child = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import paper_1902_02104_gb300 as ata\n"
        f"A = np.load({str(src)!r})\n"
        f"plan = ata.Plan({m}, {n}, {dtype}, {cutoff})\n"
        "assert plan.info['leaf_tile_rows'] == 128, plan.info\n"
        "C = plan(torch.from_numpy(A).cuda()); torch.cuda.synchronize()\n"
        "assert plan.device_status() == 0\n"
        f"np.save({str(out)!r}, C.cpu().numpy())\n")
    env = dict(os.environ, ATA_NO_CTA_PAIR="1")
    r = subprocess.run([sys.executable, "-c", child], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    C1 = np.load(out)
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
    C, plan = run(A, ata.ATA_F32_BF16X3, 64)
    assert plan.info["leaf_tile_rows"] == 128
    assert np.array_equal(C, oracle.ata_packed(A))

"""Parity of the tensor-core leaves (bf16x3, TF32, FP64 emulation) with the
oracle, through the C ABI.

Tolerances (FP32 accuracy): normwise ||C - C_ref||_F / ||C_ref||_F <=
1e-6 for bf16x3 and <= 1e-3 for TF32, where C_ref is the FP64 product of the
FP32-rounded input; the FP64-emulation leaf (ATA_F64_OZAKI) keeps the FP64
componentwise bound max |C - C_ref| / (|A|^t|A|) <= 1e-11.
Exact-integer inputs must match bitwise in every mode: bf16 holds integers
up to 256 exactly, TF32 up to 2048, and all partial sums stay below 2^24.
"""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

NORM_TOL = {ata.ATA_F32_BF16X3: 1e-6, ata.ATA_F32_TF32: 1e-3}
MODES32 = [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32]


def run(A_np, dtype, cutoff, **opts):
    import torch
    m, n = A_np.shape
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    C = plan(A)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return C.cpu().numpy(), plan


@pytest.mark.parametrize("dtype", [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
def test_single_tile_integers(gpu, dtype):
    # one diagonal leaf of 100 columns, K = 200: one 128 x 128 tile
    A = inputs.integers(200, 100, seed=1).astype(np.float64 if dtype == ata.ATA_F64_OZAKI else np.float32)
    C, _ = run(A, dtype, 4096)
    assert np.array_equal(C, oracle.ata_packed(A))


@pytest.mark.parametrize("dtype", [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
@pytest.mark.parametrize("m,n,cutoff,fuse", [(700, 300, 64, 0), (700, 300, 64, 1), (1000, 520, 128, 1),
                                             (129, 400, 32, 0), (1500, 257, 64, 0)])
def test_exact_integers_bitwise(gpu, dtype, m, n, cutoff, fuse):
    dt = np.float64 if dtype == ata.ATA_F64_OZAKI else np.float32
    A = inputs.integers(m, n, seed=m + n).astype(dt)
    C, _ = run(A, dtype, cutoff, fuse_levels=fuse)
    assert np.array_equal(C, oracle.ata_packed(A))


@pytest.mark.parametrize("dtype", MODES32)
@pytest.mark.parametrize("m,n,cutoff", [(1500, 700, 256), (3000, 1030, 512), (333, 1111, 128)])
def test_fp32_modes_normwise(gpu, dtype, m, n, cutoff):
    A = inputs.normal(m, n, seed=7, dtype=np.float32)
    C, _ = run(A, dtype, cutoff)
    err = oracle.normwise_error(C, oracle.ata_packed(A), n)
    assert err <= NORM_TOL[dtype], err


@pytest.mark.parametrize("dtype", MODES32)
def test_scaled_columns(gpu, dtype):
    # config-3 recipe at a small size: every 8th column scaled by 1e3
    A = inputs.scaled_cols(2048, 1024, seed=2)
    C, _ = run(A, dtype, 256)
    err = oracle.normwise_error(C, oracle.ata_packed(A), 1024)
    assert err <= NORM_TOL[dtype], err


@pytest.mark.parametrize("m,n,cutoff", [(1200, 800, 128), (257, 513, 64), (2000, 1000, 256)])
def test_ozaki_componentwise(gpu, m, n, cutoff):
    A = inputs.normal(m, n, seed=11)
    C, _ = run(A, ata.ATA_F64_OZAKI, cutoff)
    err = oracle.componentwise_error(C, oracle.ata_packed(A), oracle.abs_gram_packed(A))
    assert err <= 1e-11, err


@pytest.mark.parametrize("m,n,cutoff", [(1600, 900, 128), (1000, 1000, 200)])
def test_ozaki_row_bands_exact(gpu, m, n, cutoff):
    # integers whose row bands differ by powers of two: the blocks that the
    # Strassen operands sum (quadrants at several depths, column blocks) have
    # column maxima that differ block to block, and the maxima of a block are
    # assembled from its disjoint row segments.  Too small a column scale
    # would overflow the fixed point; the result must be exact.
    rng = np.random.default_rng(21)
    A = rng.integers(-4, 5, size=(m, n)).astype(np.float64)
    A *= np.exp2((np.arange(m) // 150 * 3) % 10)[:, None]  # |C| < 2^33: exact in every mode
    C, plan = run(A, ata.ATA_F64_OZAKI, cutoff)
    assert plan.info["max_strassen_levels"] >= 1
    assert np.array_equal(C, oracle.ata_packed(A))


def test_ozaki_wide_exponent_range(gpu):
    # columns spanning 2^-200 .. 2^200: the per-column scaling keeps each
    # classical leaf within the componentwise bound.  (Strassen sums mix
    # columns of different scale, so its error is bounded only normwise;
    # this case therefore runs the classical products.)
    rng = np.random.default_rng(5)
    A = inputs.normal(600, 300, seed=12)
    A *= np.exp2(rng.integers(-200, 200, size=300))[None, :]
    C, _ = run(A, ata.ATA_F64_OZAKI, 128, max_strassen_levels=0)
    err = oracle.componentwise_error(C, oracle.ata_packed(A), oracle.abs_gram_packed(A))
    assert err <= 1e-11, err


@pytest.mark.parametrize("dtype", [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
def test_tc_batched_equals_single(gpu, dtype):
    # batched launches run their own kernel layout (and, for the FP64
    # emulation, merged column-maxima segments across instances): the same
    # bits as the single-plan launches
    import torch
    shapes = [(300, 200), (1000, 129), (129, 400), (777, 333)]
    f64 = dtype == ata.ATA_F64_OZAKI
    mats = [inputs.normal(m, n, seed=i, dtype=np.float64 if f64 else np.float32) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, dtype, 128) for m, n in shapes]
    dev = [torch.from_numpy(a).cuda() for a in mats]
    singles = [p(d).clone() for p, d in zip(plans, dev)]
    Cs = ata.ata_execute_batched(plans, dev)
    torch.cuda.synchronize()
    for s, c in zip(singles, Cs):
        assert torch.equal(s, c)


def sampled_normwise(A_np, C, n, count, seed):
    """Normwise error estimated from every diagonal entry plus a uniform
    sample of off-diagonal entries (weighted up to the full triangle)."""
    import torch
    rng = np.random.default_rng(seed)
    I = rng.integers(0, n, size=count)
    J = rng.integers(0, n, size=count)
    keep = I != J
    I, J = np.minimum(I, J)[keep], np.maximum(I, J)[keep]
    d = np.arange(n)
    idx_d = torch.from_numpy(oracle.packed_index(d, d, n)).cuda()
    idx_o = torch.from_numpy(oracle.packed_index(I, J, n)).cuda()
    got_d, got_o = C[idx_d].cpu().numpy(), C[idx_o].cpu().numpy()
    ref_d = oracle.ata_entries(A_np, d, d)
    ref_o = oracle.ata_entries(A_np, I, J)
    w = (n * (n - 1) / 2) / I.size * 2.0
    num = np.sum((got_d - ref_d) ** 2) + w * np.sum((got_o - ref_o) ** 2)
    den = np.sum(ref_d ** 2) + w * np.sum(ref_o ** 2)
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("dtype", MODES32)
def test_fp32_workload_full_size_sampled(gpu, dtype):
    """16384 x 8192 FP32, every 8th column x 1e3 (the FP32 workload), at the
    bench's cutoff: sampled normwise error within the stated bound."""
    import torch
    A_np = inputs.scaled_cols(16384, 8192, seed=2)
    plan = ata.Plan(16384, 8192, dtype, 0)
    C = plan(torch.from_numpy(A_np).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    err = sampled_normwise(A_np, C, 8192, 20000, seed=3)
    assert err <= NORM_TOL[dtype], err
    del C, plan
    torch.cuda.empty_cache()


def test_ozaki_paper_scale_sampled(gpu):
    import torch
    from tests.test_gpu_f64 import sample_indices
    n = 10000
    A_np = inputs.normal(n, n, seed=1)
    plan = ata.Plan(n, n, ata.ATA_F64_OZAKI, 0)
    C = plan(torch.from_numpy(A_np).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    I, J = sample_indices(n, 3000, seed=9, cuts=[n // 2, n // 4])
    got = C[torch.from_numpy(oracle.packed_index(I, J, n)).cuda()].cpu().numpy()
    err = oracle.componentwise_error(got, oracle.ata_entries(A_np, I, J), oracle.ata_entries(A_np, I, J, absval=True))
    assert err <= 1e-11, err
    del C, plan
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# The FP64 emulation's accuracy across dynamic range.  Each column of a leaf
# operand is held in 48-bit fixed point below the column's largest entry and
# the low-order part products accumulate in FP32, so the bound that holds for
# every input is |dC_ij| <= 2^-35 K max_k|a_ki| max_k|a_kj| (K = m for
# classical leaves).  The componentwise 1e-11 is a property of inputs whose
# columns keep their weight within a bounded range of the column maximum
# (i.i.d., row- or column-scaled); a column with a few entries far above its
# others, in rows where another column is small, falls outside it.

def _ozaki_classical(A):
    C, _ = run(A, ata.ATA_F64_OZAKI, 4096, max_strassen_levels=0)
    return C


def _column_bound(A):
    """2^-35 m M_i M_j (packed), the worst-case bound of classical leaves."""
    m, n = A.shape
    M = np.max(np.abs(A), axis=0)
    return oracle.pack_upper(np.exp2(-35.0) * m * np.outer(M, M))


def test_ozaki_row_bands_2e20_componentwise(gpu):
    # row bands of 128 rows scaled by 2^+20 and 2^-20 alternately, inside
    # every column: inside the class
    A = inputs.normal(1536, 640, seed=31)
    A *= np.exp2(np.where((np.arange(1536) // 128) % 2 == 0, 20.0, -20.0))[:, None]
    C = _ozaki_classical(A)
    err = oracle.componentwise_error(C, oracle.ata_packed(A), oracle.abs_gram_packed(A))
    assert err <= 1e-11, err


@pytest.mark.parametrize("big", [30, 40])
def test_ozaki_column_outlier_outside_the_class(gpu, big):
    # column 0 holds one entry 2^big above its others; column 1 is zero in
    # that row.  C_01 is then a sum of ordinary products that column 0 holds
    # with only 48 - big - 2 bits: the componentwise 1e-11 does not hold for
    # it (plain FP64 meets it), while the worst-case bound holds everywhere
    # and the entries away from column 0 keep 1e-11.
    A = inputs.normal(1024, 256, seed=32)
    A[7, 0] = np.exp2(big)
    A[7, 1] = 0.0
    C = _ozaki_classical(A)
    ref, G = oracle.ata_packed(A), oracle.abs_gram_packed(A)
    n = A.shape[1]
    assert np.all(np.abs(C - ref) <= _column_bound(A))
    i01 = oracle.packed_index(0, 1, n)
    assert abs(C[i01] - ref[i01]) / G[i01] > 1e-11
    rest = np.ones(C.size, bool)
    rest[oracle.packed_index(np.zeros(n, int), np.arange(n), n)] = False  # row 0 of C
    assert oracle.componentwise_error(C[rest], ref[rest], G[rest]) <= 1e-11
    C64, _ = run(A, ata.ATA_F64, 4096)
    assert oracle.componentwise_error(C64, ref, G) <= 1e-11


@pytest.mark.parametrize("gen", ["normal", "uniform", "scaled", "sparse"])
def test_ozaki_worst_case_bound(gpu, gen):
    rng = np.random.default_rng(33)
    if gen == "normal":
        A = inputs.normal(1200, 400, seed=34)
    elif gen == "uniform":
        A = inputs.uniform(1200, 400, seed=35)
    elif gen == "scaled":
        A = inputs.normal(1200, 400, seed=36) * np.exp2(rng.integers(-60, 60, size=400))[None, :]
    else:  # most entries zero, a few far above the rest
        A = inputs.normal(1200, 400, seed=37) * (rng.random((1200, 400)) < 0.05)
        A[rng.integers(0, 1200, 40), rng.integers(0, 400, 40)] = np.exp2(30.0)
    C = _ozaki_classical(A)
    assert np.all(np.abs(C - oracle.ata_packed(A)) <= _column_bound(A))


# ---------------------------------------------------------------------------
# The bf16x3 running sum: every 256-deep chunk's order-0 sum joins hi
# exactly (TwoSum) and its orders-1-2 sum goes straight into the low part.
# Over K = 2^17 (512 chunks) with every product positive, that low part and
# its rounding grow the most; each entry must still be within a few units of
# 2^-24 (FP32 accuracy) of the exact product.

def test_bf16x3_long_k_same_sign_componentwise(gpu):
    A = np.abs(inputs.uniform(131072, 96, seed=11, dtype=np.float32))
    C, _ = run(A, ata.ATA_F32_BF16X3, 4096)
    err = oracle.componentwise_error(C, oracle.ata_packed(A), oracle.abs_gram_packed(A))
    assert err <= 2.5e-7, err


# Winograd's variant in the FP32 modes, at the precision form's bounds

@pytest.mark.parametrize("dtype", MODES32)
def test_fp32_modes_winograd_normwise(gpu, dtype):
    A = inputs.scaled_cols(4096, 2048, seed=2)
    C, plan = run(A, dtype, 256, variant=ata.ATA_WINOGRAD)
    assert plan.info["max_strassen_levels"] == 2
    err = oracle.normwise_error(C, oracle.ata_packed(A), 2048)
    assert err <= NORM_TOL[dtype], err


# ---------------------------------------------------------------------------
# Degenerate shapes in the tensor-core modes

@pytest.mark.parametrize("dtype", [ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
def test_tc_degenerate_shapes(gpu, dtype):
    import torch
    tdt = torch.float64 if dtype == ata.ATA_F64_OZAKI else torch.float32
    ndt = np.float64 if dtype == ata.ATA_F64_OZAKI else np.float32
    # m = 0: every entry of C is an empty sum
    plan = ata.Plan(0, 50, dtype, 256)
    C = torch.full((50 * 51 // 2,), 7.0, dtype=torch.float64, device="cuda")
    plan(torch.empty((0, 50), dtype=tdt, device="cuda"), C)
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0
    # n = 0: nothing to write
    plan = ata.Plan(10, 0, dtype, 256)
    plan(torch.empty((10, 0), dtype=tdt, device="cuda"), torch.empty((0,), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    # one column, one row, and a single entry: one partial tile each
    for m, n in [(5000, 1), (1, 700), (1, 1)]:
        A = inputs.integers(m, n, seed=m + 3 * n).astype(ndt)
        C, p = run(A, dtype, 256)
        assert p.device_status() == 0
        assert np.array_equal(C, oracle.ata_packed(A))

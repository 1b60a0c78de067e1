"""Parity of the FP64 path (ATA_F64) with the oracle, through the C ABI.

Tolerance (FP64 accuracy): max_ij |C - C_ref| / (|A|^t|A|)_ij <= 1e-11.
Exact-integer inputs must match bitwise (every product and partial sum is an
integer below 2^53, so any summation order gives the same doubles).
"""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-11


def run(A_np, cutoff=64, dtype=ata.ATA_F64, **opts):
    import torch
    m, n = A_np.shape
    plan = ata.Plan(m, n, dtype, cutoff, **opts)
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    C = plan(A)
    torch.cuda.synchronize()
    return C.cpu().numpy(), plan


def err_c(A_np, C):
    return oracle.componentwise_error(C, oracle.ata_packed(A_np), oracle.abs_gram_packed(A_np))


def test_uniform_512x384_cutoff64(gpu):
    A = inputs.uniform(512, 384, seed=0)
    C, plan = run(A, 64)
    assert plan.info["max_strassen_levels"] == 2
    assert err_c(A, C) <= TOL


@pytest.mark.parametrize("variant", [ata.ATA_STRASSEN, ata.ATA_WINOGRAD])
@pytest.mark.parametrize("fuse", [0, 1, 2])
@pytest.mark.parametrize("m,n,cutoff", [(512, 384, 64), (300, 257, 16), (129, 130, 32), (1000, 211, 16),
                                        (77, 300, 16), (700, 700, 64)])
def test_exact_integers_bitwise(gpu, m, n, cutoff, variant, fuse):
    A = inputs.integers(m, n, seed=m + 3 * n)
    C, _ = run(A, cutoff, variant=variant, fuse_levels=fuse)
    assert np.array_equal(C, oracle.ata_packed(A))


@pytest.mark.parametrize("m,n,cutoff", [(1, 1, 16), (2, 3, 16), (17, 5, 16), (100, 37, 16), (37, 100, 16),
                                        (129, 130, 16), (1025, 513, 64), (513, 1025, 64), (2000, 999, 128)])
def test_ragged_shapes_random(gpu, m, n, cutoff):
    A = inputs.normal(m, n, seed=m * n)
    C, _ = run(A, cutoff)
    assert err_c(A, C) <= TOL


def test_zero_rows_gives_zeros(gpu):
    import torch
    plan = ata.Plan(0, 50, ata.ATA_F64, 64)
    C = torch.full((50 * 51 // 2,), 7.0, dtype=torch.float64, device="cuda")
    A = torch.empty((0, 50), dtype=torch.float64, device="cuda")
    plan(A, C)
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0


def test_zero_columns_is_a_no_op(gpu):
    import torch
    plan = ata.Plan(10, 0, ata.ATA_F64, 64)
    A = torch.empty((10, 0), dtype=torch.float64, device="cuda")
    C = torch.empty((0,), dtype=torch.float64, device="cuda")
    plan(A, C)
    torch.cuda.synchronize()


def test_leading_dimension_and_repointing(gpu):
    import torch
    m, n = 400, 150
    A1 = inputs.normal(m, n, seed=1)
    A2 = inputs.normal(m, n, seed=2)
    plan = ata.Plan(m, n, ata.ATA_F64, 32)
    big = torch.zeros((m, n + 13), dtype=torch.float64, device="cuda")
    big[:, :n] = torch.from_numpy(A1).cuda()
    C1 = plan(big[:, :n])  # lda = n + 13
    d2 = torch.from_numpy(A2).cuda()
    C2 = plan(d2)  # lda = n, new pointers
    C1b = plan(big[:, :n])  # back to the first binding
    torch.cuda.synchronize()
    assert err_c(A1, C1.cpu().numpy()) <= TOL
    assert err_c(A2, C2.cpu().numpy()) <= TOL
    assert torch.equal(C1, C1b)


def test_deterministic(gpu):
    import torch
    A = inputs.normal(900, 700, seed=3)
    plan = ata.Plan(900, 700, ata.ATA_F64, 64)
    d = torch.from_numpy(A).cuda()
    C1 = plan(d).clone()
    C2 = plan(d)
    torch.cuda.synchronize()
    assert torch.equal(C1, C2)


def test_host_entry_point_matches_device(gpu):
    import torch
    A = inputs.normal(333, 222, seed=4)
    plan = ata.Plan(333, 222, ata.ATA_F64, 32)
    Ch = ata.ata_execute_host(plan, A)
    Cd = plan(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(Ch, Cd.cpu().numpy())


def test_batched_equals_single(gpu):
    import torch
    shapes = [(300, 200), (64, 33), (1000, 129), (129, 400), (50, 50)]
    mats = [inputs.normal(m, n, seed=i) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, ata.ATA_F64, 32) for m, n in shapes]
    dev = [torch.from_numpy(a).cuda() for a in mats]
    singles = [p(d).clone() for p, d in zip(plans, dev)]
    Cs = ata.ata_execute_batched(plans, dev)
    Cs2 = ata.ata_execute_batched(plans, dev)  # graph replay
    torch.cuda.synchronize()
    for s, c, c2, a in zip(singles, Cs, Cs2, mats):
        assert torch.equal(s, c)
        assert torch.equal(c, c2)
        assert err_c(a, c.cpu().numpy()) <= TOL


def test_stage_timing(gpu):
    import torch
    A = torch.from_numpy(inputs.normal(2000, 1500, seed=5)).cuda()
    plan = ata.Plan(2000, 1500, ata.ATA_F64, 128)
    plan.enable_stage_timing(True)
    plan(A)
    torch.cuda.synchronize()
    t = plan.stage_times()
    assert t["leaf_ms"] > 0 and t["split_ms"] >= 0 and t["combine_ms"] >= 0 and t["prep_ms"] >= 0


def sample_indices(n, count, seed, cuts=()):
    """Random upper-triangle entries plus the first/last rows and columns and
    entries straddling the given split points."""
    rng = np.random.default_rng(seed)
    I = rng.integers(0, n, size=count)
    J = rng.integers(0, n, size=count)
    I, J = np.minimum(I, J), np.maximum(I, J)
    extra = [(0, 0), (0, n - 1), (n - 1, n - 1)]
    for c in cuts:
        for a in (c - 1, c):
            for b in (c - 1, c, n - 1):
                if 0 <= a <= b < n:
                    extra.append((a, b))
    I = np.concatenate([I, [e[0] for e in extra]])
    J = np.concatenate([J, [e[1] for e in extra]])
    return I, J


@pytest.mark.parametrize("m,n", [(5000, 5000), (10000, 10000), (20000, 8000)])
def test_paper_scale_sampled(gpu, m, n):
    """Paper-scale square and tall inputs at the bench's launch configuration
    (autotuned cutoff): sampled entries against the oracle, plus invariants."""
    import torch
    A_np = inputs.normal(m, n, seed=1)
    plan = ata.Plan(m, n, ata.ATA_F64, 0)
    A = torch.from_numpy(A_np).cuda()
    C = plan(A)
    torch.cuda.synchronize()
    cuts = [n // 2, (n + 1) // 2, n // 4, (n + 3) // 4]
    I, J = sample_indices(n, 3000, seed=m + n, cuts=cuts)
    idx = torch.from_numpy(oracle.packed_index(I, J, n)).cuda()
    got = C[idx].cpu().numpy()
    ref = oracle.ata_entries(A_np, I, J)
    G = oracle.ata_entries(A_np, I, J, absval=True)
    assert oracle.componentwise_error(got, ref, G) <= TOL
    # diagonal entries are squared column norms: positive
    diag = C[torch.from_numpy(oracle.packed_index(np.arange(n), np.arange(n), n)).cuda()]
    assert bool((diag > 0).all())
    assert bool(torch.isfinite(C).all())
    del C, A, plan
    torch.cuda.empty_cache()

"""Prepared batches (ata_batch_create / ata_batch_execute): plans bound once
to one packed input buffer and one packed output buffer.  They run the same
merged task tables as ata_execute_batched, so their results must be the same
bits; they must follow their buffers when these move, honour caller-chosen
offsets and leading dimensions, and refuse to run once one of their plans is
destroyed."""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL_MODES = [ata.ATA_F64, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]


def _np_dtype(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


def _fill(batch, mats):
    import torch
    A = torch.zeros(batch.a_numel, dtype=batch.in_dtype, device="cuda")
    for v, a in zip(batch.input_views(A), mats):
        v.copy_(torch.from_numpy(a))
    return A


@pytest.mark.parametrize("dtype", ALL_MODES)
def test_prepared_batch_equals_list_api(gpu, dtype):
    import torch
    shapes = [(300, 200), (1000, 129), (129, 400), (777, 333), (5, 3)]
    if dtype == ata.ATA_F64:
        shapes.append((0, 7))  # m = 0: C = 0
    mats = [inputs.normal(m, n, seed=10 + i, dtype=_np_dtype(dtype)) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, dtype, 128) for m, n in shapes]
    dev = [torch.from_numpy(a).cuda() for a in mats]
    ref = ata.ata_execute_batched(plans, dev)
    batch = ata.Batch(plans)
    A = _fill(batch, mats)
    C = torch.full((batch.c_numel,), float("nan"), dtype=torch.float64, device="cuda")
    batch(A, C)
    torch.cuda.synchronize()
    for r, c in zip(ref, batch.output_views(C)):
        assert torch.equal(r, c)
    # and against the oracle (the FP64 modes componentwise, FP32 normwise)
    for a, c in zip(mats, batch.output_views(C)):
        got, want = c.cpu().numpy(), oracle.ata_packed(a.astype(np.float64))
        if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI):
            assert oracle.componentwise_error(got, want, oracle.abs_gram_packed(a)) <= 1e-11
        else:
            tol = 1e-6 if dtype == ata.ATA_F32_BF16X3 else 1e-3
            assert oracle.normwise_error(got, want, a.shape[1]) <= tol


def test_prepared_batch_many_instances(gpu):
    # more instances (300) than kernel parameters could hold: one launch
    # sequence reading the bindings from a device array
    import torch
    rng = np.random.default_rng(7)
    shapes = [(int(rng.integers(1, 200)), int(rng.integers(1, 150))) for _ in range(300)]
    mats = [inputs.uniform(m, n, seed=100 + i).astype(np.float32) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, ata.ATA_F32_BF16X3, 64) for m, n in shapes]
    batch = ata.Batch(plans)
    A = _fill(batch, mats)
    C = batch(A)
    torch.cuda.synchronize()
    dev = [torch.from_numpy(a).cuda() for a in mats]
    ref = ata.ata_execute_batched(plans, dev)
    torch.cuda.synchronize()
    for r, c in zip(ref, batch.output_views(C)):
        assert torch.equal(r, c)
    assert batch.graph_kernels() == ata.ata_batched_graph_kernels(plans, dev) > 0


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F32_BF16X3])
def test_prepared_batch_custom_layout(gpu, dtype):
    # caller-chosen offsets (reverse order, gaps) and leading dimensions
    # larger than n: the same bits as single-plan executions on those views
    import torch
    shapes = [(333, 150), (64, 257), (500, 40)]
    ldas = [160, 300, 41]
    mats = [inputs.normal(m, n, seed=20 + i, dtype=_np_dtype(dtype)) for i, (m, n) in enumerate(shapes)]
    plans = [ata.Plan(m, n, dtype, 64) for m, n in shapes]
    a_sizes = [(m - 1) * l + n for (m, n), l in zip(shapes, ldas)]
    c_sizes = [ata.packed_size(n) for _, n in shapes]
    a_off = [a_sizes[1] + a_sizes[2] + 96, a_sizes[2] + 32, 0]
    c_off = [0, c_sizes[0] + 8, c_sizes[0] + c_sizes[1] + 24]
    batch = ata.Batch(plans, a_offsets=a_off, c_offsets=c_off, lda=ldas)
    A = _fill(batch, mats)
    C = batch(A)
    torch.cuda.synchronize()
    for p, v, c in zip(plans, batch.input_views(A), batch.output_views(C)):
        assert v.stride(0) > v.shape[1]
        single = p(v)
        torch.cuda.synchronize()
        assert torch.equal(single, c)


def test_prepared_batch_follows_moved_buffers(gpu):
    import torch
    shapes = [(200, 100), (90, 130)]
    plans = [ata.Plan(m, n, ata.ATA_F64, 64) for m, n in shapes]
    batch = ata.Batch(plans)
    m1 = [inputs.normal(m, n, seed=30 + i) for i, (m, n) in enumerate(shapes)]
    m2 = [inputs.uniform(m, n, seed=40 + i) for i, (m, n) in enumerate(shapes)]
    A1, A2 = _fill(batch, m1), _fill(batch, m2)
    C1 = batch(A1)
    C2 = batch(A2)
    C3 = torch.empty_like(C1)
    batch(A1, C3)  # back to the first input, into a third output
    torch.cuda.synchronize()
    for mats, C in ((m1, C1), (m2, C2), (m1, C3)):
        for a, c in zip(mats, batch.output_views(C)):
            assert oracle.componentwise_error(c.cpu().numpy(), oracle.ata_packed(a), oracle.abs_gram_packed(a)) <= 1e-11
    for c1, c3 in zip(batch.output_views(C1), batch.output_views(C3)):
        assert torch.equal(c1, c3)  # the gaps between instances are not written


def test_prepared_batch_retired_when_a_plan_is_destroyed(gpu):
    import torch
    plans = [ata.Plan(100, 50, ata.ATA_F64, 64), ata.Plan(80, 30, ata.ATA_F64, 64)]
    batch = ata.Batch(plans)
    A = _fill(batch, [inputs.normal(100, 50, seed=1), inputs.normal(80, 30, seed=2)])
    batch(A)
    torch.cuda.synchronize()
    assert batch.graph_kernels() > 0
    plans[1].close()
    with pytest.raises(ata.AtaError):
        batch(A)
    with pytest.raises(ata.AtaError):
        batch.graph_kernels()
    batch.close()


def test_prepared_batch_rejects_bad_arguments(gpu):
    import torch
    p = ata.Plan(100, 50, ata.ATA_F64, 64)
    with pytest.raises(ata.AtaError):
        ata.Batch([p, p])  # a plan twice
    q = ata.Plan(100, 50, ata.ATA_F32_BF16X3, 64)
    with pytest.raises(ata.AtaError):
        ata.Batch([p, q])  # mixed dtype families
    with pytest.raises(ata.AtaError):
        ata.Batch([p], lda=[49])  # lda < n
    with pytest.raises(ata.AtaError):
        ata.Batch([p], a_offsets=[-1], c_offsets=[0])
    batch = ata.Batch([p])
    with pytest.raises(ValueError):
        batch(torch.zeros(10, dtype=torch.float64, device="cuda"))  # too small
    with pytest.raises(ValueError):
        batch(torch.zeros(batch.a_numel, dtype=torch.float32, device="cuda"))  # wrong dtype


def test_list_api_follows_new_pointers(gpu):
    # ata_execute_batched with the same plans on other tensors: the graph is
    # kept and the bindings array is uploaded again before the next launch
    import torch
    shapes = [(150, 70), (260, 129), (64, 64)]
    plans = [ata.Plan(m, n, ata.ATA_F32_BF16X3, 64) for m, n in shapes]
    sets = []
    for seed in (50, 60, 70):
        mats = [inputs.integers(m, n, seed=seed + i).astype(np.float32) for i, (m, n) in enumerate(shapes)]
        dev = [torch.from_numpy(a).cuda() for a in mats]
        sets.append((mats, dev, ata.ata_execute_batched(plans, dev)))
    kernels = ata.ata_batched_graph_kernels(plans, sets[0][1])
    torch.cuda.synchronize()
    for mats, _, Cs in sets:
        for a, c in zip(mats, Cs):
            assert np.array_equal(c.cpu().numpy(), oracle.ata_packed(a))
    assert kernels == ata.ata_batched_graph_kernels(plans, sets[2][1]) > 0

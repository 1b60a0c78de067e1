"""Measured tuning (ata_tune): the cost model's best cutoffs, and single-CTA
against CTA-pair tiles, timed on the device; the winner is cached per shape.
The chosen plan must not be slower than the cost model's own choice (beyond
timing noise) and must compute the product within the mode's bound."""
import time

import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu


def _time_plan(plan, A, reps=5):
    import torch
    C = plan(A)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        plan(A, C)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), C


@pytest.mark.parametrize("dtype,m,n", [(ata.ATA_F64_OZAKI, 3000, 3000), (ata.ATA_F32_BF16X3, 4096, 3072)])
def test_tuned_plan_is_not_slower_and_correct(gpu, dtype, m, n):
    import torch
    f64 = dtype == ata.ATA_F64_OZAKI
    A_np = inputs.normal(m, n, seed=41, dtype=np.float64 if f64 else np.float32)
    A = torch.from_numpy(A_np).cuda()
    opts = ata.ata_tune(m, n, dtype, candidates=3)
    best_ms = opts.pop("best_ms")
    assert best_ms > 0 and opts["cutoff"] >= 256 and opts["cta_pair"] in (0, 1)
    t0 = time.perf_counter()
    again = ata.ata_tune(m, n, dtype, candidates=3)
    assert time.perf_counter() - t0 < 0.05  # cached
    assert again.pop("best_ms") == best_ms and again == opts
    t_tuned, C = _time_plan(ata.Plan(m, n, dtype, **opts), A)
    t_model, _ = _time_plan(ata.Plan(m, n, dtype, 0), A)
    assert t_tuned <= 1.10 * t_model, (t_tuned, t_model, opts)
    got = C.cpu().numpy()
    if f64:
        I = np.arange(0, n, 37)
        J = np.minimum(I + 11, n - 1)
        sel = got[oracle.packed_index(I, J, n)]
        err = oracle.componentwise_error(sel, oracle.ata_entries(A_np, I, J), oracle.ata_entries(A_np, I, J, absval=True))
        assert err <= 1e-11
    else:
        assert oracle.normwise_error(got, oracle.ata_packed(A_np), n) <= 1e-6


def test_tune_keeps_fixed_options(gpu):
    opts = ata.ata_tune(1500, 700, ata.ATA_F32_TF32, candidates=2, cta_pair=0, variant=ata.ATA_WINOGRAD)
    assert opts["cta_pair"] == 0 and opts["variant"] == ata.ATA_WINOGRAD


def test_tune_rejects_bad_arguments(gpu):
    with pytest.raises(ata.AtaError) as e:
        ata.ata_tune(100, 100, ata.ATA_F64, candidates=0)
    assert e.value.status == ata.ATA_EINVAL
    with pytest.raises(ata.AtaError) as e:
        ata.ata_tune(-1, 100, ata.ATA_F64)
    assert e.value.status == ata.ATA_EINVAL

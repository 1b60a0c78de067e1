"""Property tests of the host planner (no GPU): random shapes, cutoffs,
variants, fused levels, level caps and modes.  For each, the host checker
(ata_plan_check / ata_gemm_plan_check) proves that every read and write of
every task stays inside A (or X and Y), the workspace and C, and that the
tasks write every entry of C exactly once; the multiplication count never
exceeds the classical count and equals it without Strassen levels.
Examples are derandomised (a fixed sequence), so the suite is
deterministic."""
import pytest

import paper_1902_02104_gb300 as ata

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

MODES = [ata.ATA_F64, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]
SETTINGS = settings(max_examples=80, deadline=None, derandomize=True, database=None)


def _opts(dtype, cutoff, variant, fuse, levels, pair):
    if dtype != ata.ATA_F64:
        cutoff = max(cutoff, 128)  # tensor-core tiles are 128 wide: keep the tile count modest
    if dtype == ata.ATA_F64_OZAKI and variant == ata.ATA_WINOGRAD:
        fuse = 0  # Winograd's chained sums stay materialised in this mode
    o = dict(variant=variant, fuse_levels=fuse, max_strassen_levels=levels)
    if dtype != ata.ATA_F64:
        o["cta_pair"] = pair
    return cutoff, o


@SETTINGS
@given(m=st.integers(1, 2500), n=st.integers(1, 1200), cutoff=st.sampled_from([16, 24, 32, 48, 64, 128, 200, 256]),
       variant=st.sampled_from([ata.ATA_STRASSEN, ata.ATA_WINOGRAD]), fuse=st.integers(0, 2),
       levels=st.sampled_from([-1, 0, 1, 2]), pair=st.sampled_from([-1, 0, 1]), dtype=st.sampled_from(MODES))
def test_random_ata_plans_are_in_bounds_and_cover_c_once(m, n, cutoff, variant, fuse, levels, pair, dtype):
    cutoff, o = _opts(dtype, cutoff, variant, fuse, levels, pair)
    ata.ata_plan_check(m, n, dtype, cutoff, **o)
    info = ata.ata_plan_query(m, n, dtype, cutoff, **o)
    assert info["classical_mults"] == m * n * (n + 1) // 2
    assert info["mults"] <= info["classical_mults"]
    if info["max_strassen_levels"] == 0:
        assert info["mults"] == info["classical_mults"]
    if levels >= 0:
        assert info["max_strassen_levels"] <= levels


@SETTINGS
@given(m=st.integers(1, 2000), p=st.integers(1, 900), r=st.integers(1, 900),
       cutoff=st.sampled_from([16, 32, 64, 128, 256]), variant=st.sampled_from([ata.ATA_STRASSEN, ata.ATA_WINOGRAD]),
       fuse=st.integers(0, 2), levels=st.sampled_from([-1, 0, 1, 2]), pair=st.sampled_from([-1, 0, 1]),
       dtype=st.sampled_from(MODES))
def test_random_gemm_plans_are_in_bounds_and_cover_c_once(m, p, r, cutoff, variant, fuse, levels, pair, dtype):
    cutoff, o = _opts(dtype, cutoff, variant, fuse, levels, pair)
    ata.ata_gemm_plan_check(m, p, r, dtype, cutoff, **o)
    info = ata.ata_gemm_query(m, p, r, dtype, cutoff, **o)
    assert info["mults"] <= m * p * r
    if info["max_strassen_levels"] == 0:
        assert info["mults"] == m * p * r

"""Host-side planner checks (no GPU): tree shapes, multiplication counts,
workspace, argument validation -- through the C ABI's ata_plan_query."""
import numpy as np
import pytest

import paper_1902_02104_gb300 as ata
from oracle import ata_recursive as R
from tests.test_oracle import paper_recurrence


def q(m, n, cutoff, dtype=ata.ATA_F64, **kw):
    return ata.ata_plan_query(m, n, dtype, cutoff, **kw)


def test_tree_512x384_cutoff64():
    # 512 x 384, cutoff 64: 512x384 -> 256x192 -> 128x96 -> 64x48 (Eq. "submatrices")
    i = q(512, 384, 64)
    assert i["depth"] == 3
    assert i["n_diag_leaves"] == 8
    assert i["n_nodes"] == 7
    assert i["max_strassen_levels"] == 2
    assert i["classical_mults"] == 512 * 384 * 385 // 2


@pytest.mark.parametrize("N,c", [(128, 16), (256, 32), (512, 64), (1024, 64), (2048, 256)])
def test_counts_match_paper_recurrence(N, c):
    assert q(N, N, c)["mults"] == paper_recurrence(N, c)


@pytest.mark.parametrize("m,n,c", [(512, 384, 64), (256, 256, 32), (100, 300, 32), (1024, 1024, 64)])
def test_counts_match_algorithm1_restatement(m, n, c):
    cnt = R.MultCounter()
    R.ata(np.zeros((m, n)), c, cnt)
    assert q(m, n, c)["mults"] == cnt.mults


@pytest.mark.parametrize("m,n", [(1, 1), (17, 5), (513, 385), (1000, 3000), (3000, 1000)])
def test_classical_when_strassen_disabled(m, n):
    i = q(m, n, 16, max_strassen_levels=0)
    assert i["mults"] == m * n * (n + 1) // 2
    # no Strassen workspace; a plan of fewer than 304 FP64 tiles holds only
    # the partial tiles of its tiles cut along K
    if i["n_leaf_tiles"] >= 304:
        assert i["workspace_bytes"] == 0
    else:
        assert i["workspace_bytes"] % (64 * 64 * 8) == 0
    assert i["n_leaf_products"] == i["n_diag_leaves"] + i["n_nodes"]


def test_strassen_saves_multiplications():
    for m, n, c in [(10000, 10000, 256), (20000, 8000, 256), (5000, 5000, 256)]:
        i = q(m, n, c)
        assert i["mults"] < 0.7 * i["classical_mults"]


def test_leaf_counts_and_fusion():
    a = q(1024, 1024, 64, fuse_levels=0)
    b = q(1024, 1024, 64, fuse_levels=1)
    assert a["mults"] == b["mults"]
    assert a["n_leaf_products"] == b["n_leaf_products"]
    assert a["n_sum_tasks"] > b["n_sum_tasks"]
    assert a["workspace_bytes"] > b["workspace_bytes"]


def test_degenerate_shapes():
    i = q(0, 10, 64)
    assert i["n_diag_leaves"] == 1 and i["mults"] == 0
    i = q(10, 0, 64)
    assert i["n_leaf_products"] == 0
    i = q(1000, 1, 64)
    assert i["n_diag_leaves"] == 1 and i["mults"] == 1000


@pytest.mark.parametrize("bad", [dict(m=-1, n=3, cutoff=64), dict(m=3, n=-1, cutoff=64),
                                 dict(m=3, n=3, cutoff=15), dict(m=3, n=3, cutoff=5000)])
def test_invalid_arguments(bad):
    with pytest.raises(ata.AtaError) as e:
        q(bad["m"], bad["n"], bad["cutoff"])
    assert e.value.status == ata.ATA_EINVAL


def test_invalid_cta_pair_option():
    for bad in (-2, 2):
        with pytest.raises(ata.AtaError) as e:
            q(100, 100, 64, ata.ATA_F32_BF16X3, cta_pair=bad)
        assert e.value.status == ata.ATA_EINVAL


def test_invalid_dtype_and_variant():
    with pytest.raises(ata.AtaError):
        ata.ata_plan_query(10, 10, 9, 64)
    with pytest.raises(ata.AtaError):
        ata.ata_plan_query(10, 10, 0, 64, variant=5)


def test_autotune_picks_a_listed_cutoff():
    i = q(10000, 10000, 0)
    assert 64 <= i["cutoff"] <= 2048
    assert i["workspace_bytes"] <= 48 << 30


def _upper_tiles(rows, tm, tn):
    # brute force: tiles (ti, tj) of a rows x rows SYRK block holding an entry j >= i
    a, b = -(-rows // tm), -(-rows // tn)
    return sum(1 for ti in range(a) for tj in range(b)
               if any(j >= i for i in range(ti * tm, min(rows, ti * tm + tm)) for j in (min(rows, tj * tn + tn) - 1,)))


@pytest.mark.parametrize("n", [100, 129, 256, 300, 511, 640, 1000, 1023, 1500, 2047])
def test_leaf_tile_shape_single_syrk_leaf(n):
    # one diagonal leaf (n <= cutoff): 128 x 128 tiles unless CTA pairs are
    # on (option 1, or the default -1 for TF32), every X operand is wider than
    # one tile and the pair tiles (256 x 128; 256 x 256 for TF32) cover at
    # most 1/8 more area
    for dtype in (ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI):
        pc = 256 if dtype == ata.ATA_F32_TF32 else 128
        t128 = _upper_tiles(n, 128, 128)
        tp = _upper_tiles(n, 256, pc)
        pair = n > 128 and tp * 256 * pc <= 1.125 * t128 * 128 * 128
        d = q(300, n, 4096, dtype, cta_pair=0)  # single-CTA 128 x 128 tiles
        assert (d["leaf_tile_rows"], d["leaf_tile_cols"], d["n_leaf_tiles"]) == (128, 128, t128)
        for opt in (1, -1):
            i = q(300, n, 4096, dtype, cta_pair=opt)
            on = opt == 1 or dtype == ata.ATA_F32_TF32
            shape = (256, pc, tp) if on and pair else (128, 128, t128)
            assert (i["leaf_tile_rows"], i["leaf_tile_cols"], i["n_leaf_tiles"]) == shape, (n, opt, dtype)
    f = q(300, n, 4096, ata.ATA_F64)
    assert (f["leaf_tile_rows"], f["leaf_tile_cols"]) == (64, 64)
    assert f["n_leaf_tiles"] == _upper_tiles(n, 64, 64)


# ---------------------------------------------------------------------------
# General product plans (X^t Y)

@pytest.mark.parametrize("m,p,r,c", [(512, 384, 300, 64), (700, 333, 517, 64), (300, 129, 1000, 32),
                                     (1030, 260, 260, 128), (100, 1, 7, 16), (64, 64, 64, 16)])
def test_gemm_counts_match_hasa_restatement(m, p, r, c):
    # the planner's multiplication count equals the Strassen restatement's
    # on the same (p, q = m, r) with the same cutoff
    cnt = R.MultCounter()
    R.hasa(np.zeros((p, m)), np.zeros((m, r)), c, cnt)
    i = ata.ata_gemm_query(m, p, r, ata.ATA_F64, c)
    assert i["mults"] == cnt.mults
    assert i["classical_mults"] == m * p * r
    assert (i["n"], i["r"]) == (p, r)


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI])
@pytest.mark.parametrize("variant", [ata.ATA_STRASSEN, ata.ATA_WINOGRAD])
@pytest.mark.parametrize("fuse", [0, 1, 2])
def test_gemm_plan_tables_cover_c_once(dtype, variant, fuse):
    for m, p, r, c in [(512, 384, 300, 64), (1000, 999, 777, 128), (257, 1025, 513, 64), (90, 700, 33, 16)]:
        ata.ata_gemm_plan_check(m, p, r, dtype, c, variant=variant, fuse_levels=fuse)


def test_gemm_classical_when_strassen_disabled():
    i = ata.ata_gemm_query(2000, 1500, 1700, ata.ATA_F64, 64, max_strassen_levels=0)
    assert i["max_strassen_levels"] == 0 and i["mults"] == 2000 * 1500 * 1700


def test_gemm_invalid_arguments():
    for args in [(-1, 3, 3), (3, -1, 3), (3, 3, -1)]:
        with pytest.raises(ata.AtaError) as e:
            ata.ata_gemm_query(*args, ata.ATA_F64, 64)
        assert e.value.status == ata.ATA_EINVAL
    with pytest.raises(ata.AtaError):
        ata.ata_gemm_query(10, 10, 10, ata.ATA_F64, 8)


@pytest.mark.parametrize("p,r", [(1024, 1100), (1000, 1030), (600, 300), (2048, 640), (300, 5000), (129, 129)])
def test_gemm_pair_tile_shape_follows_area_rule(p, r):
    # one classical general product (no Strassen level): pair tiles (256 x 256
    # for TF32, 256 x 128 otherwise) when X is wider than one 128-row tile and
    # the pair tiles add at most 1/8 to the area of 128 x 128 tiles
    m = 500
    for dtype in (ata.ATA_F32_TF32, ata.ATA_F32_BF16X3, ata.ATA_F64_OZAKI):
        pc = 256 if dtype == ata.ATA_F32_TF32 else 128
        t128 = -(-p // 128) * -(-r // 128)
        tp = -(-p // 256) * -(-r // pc)
        pair = p > 128 and tp * 256 * pc <= 1.125 * t128 * 128 * 128
        i = ata.ata_gemm_query(m, p, r, dtype, 4096, cta_pair=1)
        shape = (256, pc, tp) if pair else (128, 128, t128)
        assert (i["leaf_tile_rows"], i["leaf_tile_cols"], i["n_leaf_tiles"]) == shape, (p, r, dtype)
        i0 = ata.ata_gemm_query(m, p, r, dtype, 4096, cta_pair=0)
        assert (i0["leaf_tile_rows"], i0["leaf_tile_cols"], i0["n_leaf_tiles"]) == (128, 128, t128)


@pytest.mark.parametrize("dtype", [ata.ATA_F32_TF32, ata.ATA_F32_BF16X3, ata.ATA_F64_OZAKI])
@pytest.mark.parametrize("pair", [0, 1])
def test_plan_check_tile_grid(dtype, pair):
    # the host checker walks every product's tile grid for the planned tile
    # shape: X parts padded to whole tiles, Y rows past the padding only for
    # one-part operands (TF32's 256-column pair tiles) and by at most half a tile
    for m, n, c in [(300, 129, 256), (1000, 700, 512), (4097, 1537, 1024), (1000, 3000, 4096), (300, 2048, 512)]:
        ata.ata_plan_check(m, n, dtype, c, cta_pair=pair)
    for m, p, r in [(500, 1024, 1100), (500, 1000, 1030), (2000, 600, 300), (500, 2000, 2500), (500, 129, 100)]:
        ata.ata_gemm_plan_check(m, p, r, dtype, 512, cta_pair=pair)


# ---------------------------------------------------------------------------
# Automatic plan shape under the workspace cap.  Every Strassen level holds
# the operand sums and outputs of all its products at once, so the largest
# products fit the 48 GiB cap only with fewer levels.

CAP = 48 << 30
TC_CUTOFFS = (256, 320, 384, 512, 768, 1024, 1536, 2048, 3072, 4096)


def test_autotune_lowers_strassen_levels_to_fit_the_cap():
    m, n, dt = 50000, 30000, ata.ATA_F32_BF16X3
    free = [q(m, n, c, dt)["workspace_bytes"] for c in TC_CUTOFFS]
    assert min(free) > CAP  # with free depth no cutoff fits
    auto = q(m, n, 0, dt)
    assert auto["workspace_bytes"] <= CAP
    assert auto["max_strassen_levels"] >= 1  # the deepest cap that fits, not zero
    # a fixed level cap is the caller's: it is kept, not lowered, and the
    # smallest workspace under it is taken although it exceeds the cap
    fixed = q(m, n, 0, dt, max_strassen_levels=3)
    assert fixed["max_strassen_levels"] > auto["max_strassen_levels"]
    assert fixed["workspace_bytes"] == min(free) > CAP


def test_autotune_takes_the_smallest_workspace_when_nothing_fits():
    m, n, dt = 40000, 60000, ata.ATA_F32_BF16X3
    classical = [q(m, n, c, dt, max_strassen_levels=0)["workspace_bytes"] for c in TC_CUTOFFS]
    assert min(classical) > CAP
    auto = q(m, n, 0, dt)
    assert auto["max_strassen_levels"] == 0
    assert auto["workspace_bytes"] == min(classical)
    ata.ata_plan_check(m, n, dt, 0)


def test_autotune_unchanged_where_the_cap_holds():
    # paper-scale shapes keep the cost model's free-depth choice
    for m, n, dt in [(10000, 10000, ata.ATA_F64_OZAKI), (16384, 8192, ata.ATA_F32_BF16X3)]:
        auto = q(m, n, 0, dt)
        same = q(m, n, auto["cutoff"], dt)
        assert auto["workspace_bytes"] == same["workspace_bytes"] <= CAP
        assert auto["max_strassen_levels"] == same["max_strassen_levels"]


def test_small_fp64_plans_cut_their_tiles_along_k():
    # config 1 (512 x 384, cutoff 64): 75 FP64 tiles, fewer than two per SM,
    # so the tiles with enough K are cut into K ranges; the partial tiles sit
    # in the workspace (checked in bounds and disjoint by the host checker)
    # and one more kernel adds them; paper-scale plans are not cut
    small = q(512, 384, 64)
    assert small["n_leaf_tiles"] < 304
    # a split and a combine kernel per Strassen level (FP64 sums are not
    # fused), the leaf, and the partial sums
    assert small["n_launches"] == 2 * small["max_strassen_levels"] + 1 + 1
    ata.ata_plan_check(512, 384, ata.ATA_F64, 64)
    big = q(5000, 5000, 0)
    assert big["n_leaf_tiles"] >= 304
    assert big["n_launches"] == 2 * big["max_strassen_levels"] + 1

"""Host-side logic that needs no GPU: the packed layout of prepared batches
and the per-step statistics that bench.py reports."""
import numpy as np
import pytest

import paper_1902_02104_gb300 as ata


@pytest.mark.parametrize("elem", [4, 8])
def test_packed_layout_aligned_disjoint_and_tight(elem):
    rng = np.random.default_rng(11)
    shapes = [(int(rng.integers(0, 300)), int(rng.integers(0, 200))) for _ in range(200)] + [(0, 7), (5, 0), (1, 1)]
    lda, a_off, c_off, a_numel, c_numel = ata.packed_layout(shapes, elem=elem, align_bytes=256)
    a_sizes = [(m - 1) * l + n if m > 0 and n > 0 else 0 for (m, n), l in zip(shapes, lda)]
    c_sizes = [n * (n + 1) // 2 for _, n in shapes]
    assert lda == [max(n, 1) for _, n in shapes]
    for offs, sizes, e, numel in ((a_off, a_sizes, elem, a_numel), (c_off, c_sizes, 8, c_numel)):
        assert all((o * e) % 256 == 0 for o in offs)                      # every instance aligned
        ends = [o + s for o, s in zip(offs, sizes)]
        assert all(ends[i] <= offs[i + 1] for i in range(len(offs) - 1))  # in order, disjoint
        assert numel == max(ends)
        # no gap wider than the alignment padding
        assert all(offs[i + 1] - ends[i] < 256 // e for i in range(len(offs) - 1))


def test_packed_layout_leading_dimensions():
    lda, a_off, _, a_numel, _ = ata.packed_layout([(3, 4), (2, 5)], lda=[10, 6], elem=8, align_bytes=16)
    # A_0 spans (3 - 1) * 10 + 4 = 24 elements, padded to 24 (2 per 16 bytes)
    assert lda == [10, 6] and a_off == [0, 24] and a_numel == 24 + 6 + 5


def test_step_percentiles():
    import bench
    s = bench.step_percentiles([3.0, 1.0, 2.0])
    assert (s["median"], s["p99"], s["min"], s["max"], s["count"]) == (2.0, 3.0, 1.0, 3.0, 3)
    s = bench.step_percentiles([5.0] * 99 + [9.0])
    assert s["p99"] == 5.0 and s["max"] == 9.0       # nearest rank: the 99th of 100
    s = bench.step_percentiles([5.0] * 20 + [9.0])
    assert s["p99"] == 9.0                            # the 21st of 21

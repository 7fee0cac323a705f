"""Host-side arithmetic of the benchmark's roofline report (CPU only): the
algorithmic bytes of the vertex-quadruple kernel (16 B per disjoint
pair x pair entry, 24 entries per quadruple) and the scaling of the stored
DRAM capture by the number of quadruples."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

QUAD = "k_entries (pair x pair; closed: disjoint edges by vertex quadruple)"


def test_quadruple_kernel_bytes_and_fraction():
    N = 200
    M = N * N - 1
    peaks = {"hbm_gbs": 6769.4}
    r = bench.assembly_roofline("closed", QUAD, 10.0, N, M, None, 1.25, peaks)
    entries = 24 * math.comb(N, 4)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(16.0 * entries)
    assert r["achieved"] == pytest.approx(16.0 * entries / 0.010 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6769.4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_disjoint_entry_count_matches_edge_pairs():
    # ordered pairs of disjoint edges times 4 type pairs = 24 C(N, 4)
    for N in range(4, 12):
        edges = [(a, b) for a in range(N) for b in range(a + 1, N)]
        disjoint = sum(1 for e in edges for f in edges if not set(e) & set(f))
        assert 4 * disjoint == 24 * math.comb(N, 4)


def test_stored_traffic_scales_with_quadruples():
    t200, src = bench.ncu_traffic(QUAD, 200)
    t100, _ = bench.ncu_traffic(QUAD, 100)
    assert src and t200 > 0
    assert t100 / t200 == pytest.approx(math.comb(100, 4) / math.comb(200, 4))
    assert bench.ncu_traffic("k_pd (pair x diagonal)", 200) == (None, None)


def test_csr_step_bytes_by_stage():
    """The CSR RK4 step's algorithmic bytes, listed stage by stage."""
    for nnz, M in [(27978001, 3999999), (7, 3), (0, 5)]:
        for prec, val, x in [("fp32", 4, 4), ("fp64", 8, 8)]:
            total = 0
            for stage in (1, 2, 3, 4):
                total += nnz * (val + 4)          # values and int32 columns
                total += (M + 1) * 8              # int64 row pointers
                total += M * x                    # gathered stage vector
                total += M * 8 + M * 8            # Keff and v read
                total += M * x                    # next stage vector written
                total += M * {1: 8, 2: 16, 3: 16, 4: 8}[stage]  # acc
                if stage == 4:
                    total += M * 8                # v written
            assert bench.csr_step_bytes(prec, nnz, M) == total
    nnz, M = 27978001, 3999999
    assert bench.csr_step_bytes("fp32", nnz, M) == 32 * nnz + 32 * (M + 1) + 152 * M


def test_upload_bytes_cover_the_copied_region():
    """Page-locked a: exactly the upper triangle.  Pageable a: the row blocks
    of the copy engine, counted element by element on small cases."""
    for M in (3, 99, 2500):
        assert bench.upload_bytes(M, True) == 16 * M * (M + 1) // 2
    assert bench.upload_bytes(2000, False) == 16 * 2000 * 2000
    M = 4097
    h = max(256, (M + 63) // 64)
    count = sum((min(M, j0 + h) - j0) * (M - j0) for j0 in range(0, M, h))
    assert bench.upload_bytes(M, False) == 16 * count
    assert 16 * M * (M + 1) // 2 < bench.upload_bytes(M, False) < 16 * M * M

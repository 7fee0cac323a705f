"""lb_structure_export_noalloc (kernel (a) with its scratch in a static device
array) against lb_structure_export, through the C ABI (needs a GPU).

Bars are those of the structure-list tests: indices bit-exact, values within
1e-14.  Calls come in pairs on the same input, and the sequence changes N and
f/d between pairs, so a result that depended on what an earlier call left in
the shared scratch would differ from the allocating export.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_01491_gb300 import build
    build.build()


def lbm():
    import paper_1912_01491_gb300 as lb
    return lb


def _noalloc(B, which, n, pad=5):
    idx = torch.full((n + pad, 3), -7, dtype=torch.int32, device="cuda")
    val = torch.full((n + pad,), np.nan, dtype=torch.float64, device="cuda")
    got = B.structure_into(which, idx, val)
    return got, idx, val


@pytest.mark.parametrize("seq", [[(12, "f"), (7, "d"), (40, "f"), (3, "d"), (2, "f"), (21, "d")]])
def test_noalloc_matches_export_two_calls_in_a_row(seq):
    lb = lbm()
    for N, which in seq:
        with lb.Basis(N) as B:
            ref_idx, ref_val = B.structure(which)
            n = ref_idx.shape[0]
            for _ in range(2):
                got, idx, val = _noalloc(B, which, n)
                torch.cuda.synchronize()
                assert got == n
                assert torch.equal(idx[:n], ref_idx), (N, which)
                if n:
                    assert (val[:n] - ref_val).abs().max().item() < 1e-14, (N, which)
                # nothing written past nnz
                assert bool((idx[n:] == -7).all()) and bool(torch.isnan(val[n:]).all())


def test_noalloc_at_maximum_size():
    """N = 256 (M = 65535, the scratch limit): f count and contents."""
    lb = lbm()
    N = 256
    with lb.Basis(N) as B:
        ref_idx, ref_val = B.structure("f")
        n = ref_idx.shape[0]
        assert 6 * n == 5 * N**3 - 9 * N**2 - 2 * N + 6
        for _ in range(2):
            got, idx, val = _noalloc(B, "f", n, pad=0)
            torch.cuda.synchronize()
            assert got == n
            assert torch.equal(idx, ref_idx)
            assert (val - ref_val).abs().max().item() < 1e-14


def test_noalloc_rejects_oversize_and_small_capacity():
    lb = lbm()
    with lb.Basis(257) as B:
        idx = torch.zeros((8, 3), dtype=torch.int32, device="cuda")
        val = torch.zeros(8, dtype=torch.float64, device="cuda")
        with pytest.raises(lb.LBError, match="65535"):
            B.structure_into("f", idx, val)
    with lb.Basis(5) as B:
        n = B.structure_count("d")
        idx = torch.full((n - 1, 3), -7, dtype=torch.int32, device="cuda")
        val = torch.zeros(n - 1, dtype=torch.float64, device="cuda")
        with pytest.raises(lb.LBError, match="capacity"):
            B.structure_into("d", idx, val)
        torch.cuda.synchronize()
        assert bool((idx == -7).all())
        # a correct call right after the rejected one
        ref_idx, _ = B.structure("d")
        got, idx2, _ = _noalloc(B, "d", n)
        torch.cuda.synchronize()
        assert got == n and torch.equal(idx2[:n], ref_idx)

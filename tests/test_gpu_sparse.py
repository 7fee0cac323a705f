"""Sparse (CSR) path against the oracle, through the C ABI (needs a GPU).

Bars: the CSR pattern (row pointers, sorted columns) bit-exact against the
oracle's; values within 1e-12 of the sum of the magnitudes of each entry's
terms; K within 1e-12 of its scale; FP64 trajectories within 1e-12 ||v||.
At N = 2000 (M = 3,999,999): the pattern size 7N^2 - 11N + 1 of the ladder
model, and the exact death process of its populations when H is diagonal.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import Oracle, lowrank_csr, rk4_csr as ora_rk4_csr

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


def _channels_ladder(B, L, g):
    l = B.expand(torch.tensor(L, device="cuda"))
    nz = torch.nonzero(l.abs() > 0).flatten()
    return [(g, nz, l[nz].contiguous())], l


def _gpu_csr(B, H, channels):
    h = B.expand(torch.tensor(H, device="cuda")).real.contiguous() if H is not None else None
    c = lbm().Csr(B, h=h, channels=channels)
    return c, c.to_host()


def _oracle_csr(o, H, gammas, lps):
    h = o.expand(H)[0].real if H is not None else None
    return lowrank_csr(o, h, gammas, lps, with_mag=True)


def _assert_csr(g, r):
    rp, col, val, K = g
    orp, ocol, oval, oK, omag = r
    assert np.array_equal(rp, orp), "row pointers differ"
    assert np.array_equal(col, ocol), "columns differ"
    err = np.abs(val - oval)
    assert np.all(err <= 1e-12 * np.maximum(np.abs(oval), omag)), err.max()
    ks = max(np.abs(oK).max(), 1e-300)
    assert np.abs(K - oK).max() <= 1e-12 * ks + 1e-18


@pytest.mark.parametrize("N", [2, 3, 4, 6, 9, 12])
def test_ladder_csr_parity(N):
    H, L, g = wl.ladder_model(N, 300 + N)
    with lbm().Basis(N) as B, Oracle(N) as o:
        ch, l = _channels_ladder(B, L, g)
        c, got = _gpu_csr(B, H, ch)
        lo, _ = o.expand(L)
        nz = np.nonzero(np.abs(lo) > 0)[0]
        ref = _oracle_csr(o, H, [g], [(nz, lo[nz])])
        assert np.array_equal(torch.nonzero(l.abs() > 0).flatten().cpu().numpy(), nz)
    _assert_csr(got, ref)


@pytest.mark.parametrize("N", [5, 7])
def test_random_multichannel_csr_parity(N):
    """Two channels with random sparse complex l_p (pair and diagonal
    components) and a random sparse H."""
    M = N * N - 1
    rng = np.random.default_rng(N)
    Hd = np.zeros((N, N), complex)
    for _ in range(2 * N):
        i, j = rng.integers(0, N, 2)
        x = rng.normal() + 1j * rng.normal() * (i != j)
        Hd[i, j] += x
        Hd[j, i] += np.conj(x)
    lps, gam, chans = [], [0.3, 0.7], []
    with lbm().Basis(N) as B, Oracle(N) as o:
        for p in range(2):
            idx = np.sort(rng.choice(M, size=min(M, 3 * N), replace=False)).astype(np.int64)
            vals = rng.normal(size=len(idx)) + 1j * rng.normal(size=len(idx))
            lps.append((idx, vals))
            chans.append((gam[p], torch.tensor(idx, device="cuda"), torch.tensor(vals, device="cuda")))
        c, got = _gpu_csr(B, Hd, chans)
        ref = _oracle_csr(o, Hd, gam, lps)
    _assert_csr(got, ref)


@pytest.mark.parametrize("N", [40, 80])
def test_ladder_csr_parity_larger(N):
    H, L, g = wl.ladder_model(N, 9)
    with lbm().Basis(N) as B, Oracle(N) as o:
        ch, _ = _channels_ladder(B, L, g)
        c, got = _gpu_csr(B, H, ch)
        lo, _ = o.expand(L)
        nz = np.nonzero(np.abs(lo) > 0)[0]
        ref = _oracle_csr(o, H, [g], [(nz, lo[nz])])
    _assert_csr(got, ref)
    assert got[0][-1] == 7 * N * N - 11 * N + 1


def test_ladder_rk4_csr_matches_oracle():
    N, dt, steps = 30, 1e-3, 500
    H, L, g = wl.ladder_model(N, 31)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        ch, _ = _channels_ladder(B, L, g)
        c, (rp, col, val, K) = _gpu_csr(B, H, ch)
        lo, _ = o.expand(L)
        nz = np.nonzero(np.abs(lo) > 0)[0]
        orp, ocol, oval, oK, _ = _oracle_csr(o, H, [g], [(nz, lo[nz])])
        v0 = o.expand(wl.pure_state(N, N - 1))[0].real
        ref = ora_rk4_csr(orp, ocol, oval, oK, v0, dt, steps)
        v = torch.tensor(v0, device="cuda")
        c.rk4(v, dt, steps, precision="fp64")
        vg = v.cpu().numpy()
        assert np.linalg.norm(vg - ref) <= 1e-12 * np.linalg.norm(ref)
        v32 = torch.tensor(v0, device="cuda")
        c.rk4(v32, dt, steps, precision="fp32", correct_every=50)
        err32 = np.linalg.norm(v32.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err32 < 1e-6, err32


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pipelined_stage_equals_block_staged(precision):
    """N = 800 (M = 639,999: about three chunks of 256 rows per resident
    block, so both staging buffers are reused and the phase parity flips):
    the bulk-copy pipelined stage (16-byte aligned v) and the block-staged
    stage (v one element off that alignment) sum in the same order and give
    the same bits."""
    N, dt, steps = 800, 2e-4, 12
    H, L, g = wl.ladder_model(N, 801)
    lb = lbm()
    with lb.Basis(N) as B:
        ch, _ = _channels_ladder(B, L, g)
        h = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
        c = lb.Csr(B, h=h, channels=ch)
        v0 = B.expand(torch.tensor(wl.pure_state(N, N // 2), device="cuda")).real.contiguous()
        va = v0.clone()
        assert va.data_ptr() % 16 == 0
        raw = torch.empty(B.M + 1, dtype=torch.float64, device="cuda")
        vb = raw[1:]
        assert vb.data_ptr() % 16 == 8
        vb.copy_(v0)
        c.rk4(va, dt, steps, precision=precision, correct_every=5 if precision == "fp32" else 0)
        c.rk4(vb, dt, steps, precision=precision, correct_every=5 if precision == "fp32" else 0)
        torch.cuda.synchronize()
        assert torch.isfinite(va).all()
        assert torch.equal(va, vb)
        assert not torch.equal(va, v0)
        c.close()


def test_ladder_n2000_pattern_size_and_death_process():
    """M = 3,999,999: nnz(Q + R) = 7N^2 - 11N + 1; with H diagonal the
    populations follow p_n(t) = C(n0,n) e^{-g n t}(1 - e^{-g t})^{n0-n}."""
    N = 2000
    lb = lbm()
    H, L, g = wl.ladder_model(N, 2000)
    with lb.Basis(N) as B:
        ch, _ = _channels_ladder(B, L, g)
        h = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
        c = lb.Csr(B, h=h, channels=ch)
        assert c.nnz == 7 * N * N - 11 * N + 1
        c.close()
        Hd = np.diag(np.diag(H))
        hd = B.expand(torch.tensor(Hd, device="cuda")).real.contiguous()
        c = lb.Csr(B, h=hd, channels=ch)
        n0 = N - 1
        rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
        rho0[n0, n0] = 1.0
        v = B.expand(rho0).real.contiguous()
        T, steps = 0.5, 5000
        c.rk4(v, T / steps, steps, precision="fp64")
        p = torch.diagonal(B.rho(v)).real.cpu().numpy()
    e = math.exp(-g * T)
    n = np.arange(N)
    logc = np.array([math.lgamma(n0 + 1) - math.lgamma(k + 1) - math.lgamma(n0 - k + 1) for k in n])
    with np.errstate(divide="ignore"):
        ref = np.exp(logc + n * math.log(e) + (n0 - n) * math.log(1 - e))
    assert abs(p.sum() - 1.0) < 1e-12
    assert np.abs(p - ref).max() < 1e-6   # RK4 at h*gamma*N = 0.02: global error ~1e-7 at most


def _dimer_gpu(B, N):
    """CSR A0 = Q0 + R, the CSR Q1 of H1, and the drive of the rocked dimer."""
    H0, H1, L, rate, eps = wl.dimer_model(N)
    ch, _ = _channels_ladder(B, L, rate)
    A0 = lbm().Csr(B, h=B.expand(torch.tensor(H0, device="cuda")).real.contiguous(), channels=ch)
    Q1 = lbm().Csr(B, h=B.expand(torch.tensor(H1, device="cuda")).real.contiguous(), channels=())
    return A0, Q1, eps


@pytest.mark.parametrize("N", [6, 11])
def test_dimer_time_dependent_rk4_vs_oracle(N):
    """The periodically rocked dimer (Sec. 3, Eqs. (10)-(11)): Q(t) = Q0 +
    eps(t) Q1 with eps = E + A Theta(t) switching at T/2, one period T = 2 pi
    in 4000 steps, against the oracle's time-dependent RK4 on its own dense
    A0 = Q0 + R, Q1 and K, within 1e-12 ||v|| at every quarter period."""
    from oracle import rk4_dense_td
    T = 2.0 * math.pi
    steps = 4000
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        H0, H1, L, rate, eps = wl.dimer_model(N)
        h0, _ = o.expand(H0)
        h1, _ = o.expand(H1)
        l, _ = o.expand(L)
        a = rate * np.outer(l, l.conj())
        A0o = o.Q(h0.real) + o.R(a)
        Q1o = o.Q(h1.real)
        Ko = o.K(a)
        v0 = o.expand(wl.pure_state(N, N - 1))[0].real
        A0, Q1, eps_g = _dimer_gpu(B, N)
        assert tuple(eps_g) == tuple(eps)
        v = torch.tensor(v0, device="cuda")
        ref = v0.copy()
        for q in range(4):
            t0 = q * T / 4
            ref = rk4_dense_td(A0o, Q1o, Ko, ref, T / steps, steps // 4, [0.0, T / 2], list(eps), T, t0=t0)
            A0.rk4_td(Q1, v, T / steps, steps // 4, [0.0, T / 2], list(eps), T, t0=t0)
            torch.cuda.synchronize()
            got = v.cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), q
        A0.close()
        Q1.close()


def test_dimer_constant_drive_equals_autonomous():
    """With one segment the time-dependent RK4 is the autonomous CSR RK4 of
    A0 + eps Q1 (here eps = 0: the same system, the same bits)."""
    N = 9
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A0, Q1, _ = _dimer_gpu(B, N)
        v0 = torch.tensor(o.expand(wl.pure_state(N, 3))[0].real, device="cuda")
        v1, v2 = v0.clone(), v0.clone()
        A0.rk4_td(Q1, v1, 1e-3, 300, [0.0], [0.0], 1.0)
        A0.rk4(v2, 1e-3, 300)
        torch.cuda.synchronize()
        assert torch.equal(v1, v2)
        with pytest.raises(lb.LBError):
            A0.rk4_td(Q1, v1, 1e-3, 10, [0.5], [1.0], 1.0)  # seg_start[0] must be 0
        A0.close()
        Q1.close()

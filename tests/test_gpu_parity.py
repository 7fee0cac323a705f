"""GPU-versus-oracle parity through the C ABI (needs an sm_103a GPU).

Bars: index lists bit-exact; values within the per-entry tolerance
|x_gpu - x_ora| <= 1e-12 max(|x_ora|, S) with S = 1/4 sum |terms| the
oracle's absolute-sum scale of the entry (summation order is free, so an
entry with heavy cancellation is judged against its condition); FP64
trajectories within 1e-12 ||v|| of the oracle's RK4.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import Oracle, rk4_dense as ora_rk4

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_01491_gb300 import build
    build.build()


def lbm():
    import paper_1912_01491_gb300 as lbm
    return lbm


def _canonical_d_count(N):
    pd = sum(N - max(a, 1) for a in range(N) for b in range(a + 1, N))
    return 4 * math.comb(N, 3) + 2 * pd - (2 if N >= 2 else 0) + (N - 1) * (N - 2) // 2 + (N - 2)


@pytest.mark.parametrize("N", list(range(2, 13)) + [16, 21, 32])
def test_structure_lists_bit_exact(N):
    with lbm().Basis(N) as B, Oracle(N) as o:
        for w in "fd":
            idx, val = B.structure(w)
            oi, ov = o.structure(w)
            assert idx.shape[0] == oi.shape[0]
            assert np.array_equal(idx.cpu().numpy(), oi)
            if len(ov):
                assert np.abs(val.cpu().numpy() - ov).max() < 1e-14


@pytest.mark.parametrize("N", [50, 200, 1000, 2000])
def test_structure_counts_large_n(N):
    with lbm().Basis(N) as B:
        assert 6 * B.structure_count("f") == 5 * N**3 - 9 * N**2 - 2 * N + 6
        assert B.structure_count("d") == _canonical_d_count(N)


def test_labels():
    with lbm().Basis(5) as B, Oracle(5) as o:
        for i in range(B.M):
            assert B.label(i) == o.label(i)


@pytest.mark.parametrize("N", [3, 7, 17])
def test_expand_and_rho(N):
    g = np.random.default_rng(N)
    A = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    v = g.standard_normal(N * N - 1)
    with lbm().Basis(N) as B, Oracle(N) as o:
        coef = B.expand(torch.tensor(A, device="cuda")).cpu().numpy()
        ref, _ = o.expand(A)
        assert np.abs(coef - ref).max() < 1e-13
        rho = B.rho(torch.tensor(v, device="cuda")).cpu().numpy()
        assert np.abs(rho - o.rho(v)).max() < 1e-13


def _case(N, seed):
    return wl.gue_hamiltonian(N, seed), wl.wishart_kossakowski(N, seed + 1)


def _assert_entries(x, ref, scale, what):
    err = np.abs(x - ref)
    tol = 1e-12 * np.maximum(np.abs(ref), scale) + 1e-300
    bad = np.argwhere(err > tol)
    assert len(bad) == 0, "%s: %d entries out of tolerance, first %s (err %g, tol %g)" % (
        what, len(bad), bad[:3].tolist(), err[tuple(bad[0])], tol[tuple(bad[0])])


def _gpu_system(B, H, a, algorithm="join"):
    h = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
    out = B.assemble_dense(torch.tensor(a, device="cuda"), h=h, A=True, Q=True, R=True, K=True,
                           algorithm=algorithm)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("algorithm", ["join", "closed"])
@pytest.mark.parametrize("N", list(range(2, 13)) + [16, 23])
def test_dense_assembly_parity(N, algorithm):
    H, a = _case(N, 1000 + N)
    with lbm().Basis(N) as B, Oracle(N) as o:
        g = _gpu_system(B, H, a, algorithm)
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
        W = o.join_terms()
        assert B.join_terms() == W
    _assert_entries(g["R"], R, S, "R")
    qs = np.abs(Q).max()
    assert np.abs(g["Q"] - Q).max() <= 1e-12 * qs
    _assert_entries(g["A"], Q + R, S + np.abs(Q), "A")
    assert np.abs(g["K"] - K).max() <= 1e-12 * max(np.abs(K).max(), 1e-300) + 1e-17


@pytest.mark.parametrize("algorithm", ["join", "closed"])
def test_dense_assembly_n50_random_lindbladian(algorithm):
    """The 50-level random Lindbladian (M = 2499): full R, Q, K parity."""
    N = 50
    H, a = _case(N, 1050)
    with lbm().Basis(N) as B, Oracle(N) as o:
        g = _gpu_system(B, H, a, algorithm)
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
        assert B.join_terms() == o.join_terms()
    _assert_entries(g["R"], R, S, "R")
    assert np.abs(g["Q"] - Q).max() <= 1e-12 * np.abs(Q).max()
    assert np.abs(g["K"] - K).max() <= 1e-12 * np.abs(K).max()


def test_identity_and_amplitude_damping_closed_forms():
    g = 0.3
    for N in (2, 4):
        M = N * N - 1
        with lbm().Basis(N) as B:
            out = B.assemble_dense(torch.eye(M, dtype=torch.complex128, device="cuda") * g, R=True)
            assert torch.allclose(out["R"], -g * N * torch.eye(M, dtype=torch.float64, device="cuda"), atol=1e-14)
            assert out["K"].abs().max().item() < 1e-15
    with lbm().Basis(2) as B:
        L = torch.tensor([[0, 1], [0, 0]], dtype=torch.complex128, device="cuda")
        l = B.expand(L)
        a = g * torch.outer(l, l.conj())
        out = B.assemble_dense(a.contiguous(), R=True)
        ref = torch.tensor(np.diag([-g / 2, -g / 2, -g]), device="cuda")
        assert torch.allclose(out["R"], ref, atol=1e-15)
        assert torch.allclose(out["K"], torch.tensor([0, 0, g / math.sqrt(2)], device="cuda",
                                                     dtype=torch.float64), atol=1e-15)


def _oracle_system(o, H, a):
    h, _ = o.expand(H)
    return o.Q(h.real) + o.R(a), o.K(a)


def test_rk4_fp64_n10_full_trajectory():
    """Dense N = 10 random Lindbladian, rho0 = |0><0|, t = 10, dt = 1e-3 (10^4 steps)."""
    N, dt, steps, every = 10, 1e-3, 10_000, 1000
    H, a = _case(N, 1010)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 0))[0].real
        ref_v, ref_snaps = ora_rk4(A, K, v0, dt, steps, snap_every=every)
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous())
        v = torch.tensor(v0, device="cuda")
        snaps = lb.rk4_dense(g["A"], g["K"], v, dt, steps, precision="fp64", snap_every=every)
        torch.cuda.synchronize()
    snaps = snaps.cpu().numpy()
    for t in range(len(ref_snaps)):
        assert np.linalg.norm(snaps[t] - ref_snaps[t]) <= 1e-12 * np.linalg.norm(ref_snaps[t])
    assert np.linalg.norm(v.cpu().numpy() - ref_v) <= 1e-12 * np.linalg.norm(ref_v)


@pytest.mark.parametrize("precision,tol_plain,tol_corr", [("fp32", 1e-5, 2e-6), ("bf16", 2e-2, 1e-3)])
def test_rk4_low_precision_with_correction(precision, tol_plain, tol_corr):
    """FP32 / BF16-with-row-scale storage: stated trajectory error against the
    FP64 oracle, and the FP64 defect correction every 50 steps reduces it."""
    N, dt, steps = 12, 1e-3, 2000
    H, a = _case(N, 1212)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 0))[0].real
        ref_v, _ = ora_rk4(A, K, v0, dt, steps)
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous())
        if precision == "fp32":
            Ap, sc = lb.pack_fp32(g["A"]), None
        else:
            Ap, sc = lb.pack_bf16(g["A"])
        errs = []
        for corr in (0, 50):
            v = torch.tensor(v0, device="cuda")
            lb.rk4_dense(Ap, g["K"], v, dt, steps, precision=precision, scale=sc, A64=g["A"],
                         correct_every=corr)
            torch.cuda.synchronize()
            errs.append(np.linalg.norm(v.cpu().numpy() - ref_v) / np.linalg.norm(ref_v))
    assert errs[0] < tol_plain, errs
    assert errs[1] < tol_corr, errs
    assert errs[1] < 0.5 * errs[0], errs


def test_host_buffer_api():
    N = 6
    H, a = _case(N, 606)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        sysm = lb.System(B, a, H=H, keep_parts=True)
        A, K = _oracle_system(o, H, a)
        R, S = o.R(a, return_scale=True)
        _assert_entries(sysm.get("R"), R, S, "R")
        assert np.abs(sysm.get("A") - A).max() < 1e-12 * np.abs(A).max()
        v0 = o.expand(wl.pure_state(N, 1))[0].real
        ref, _ = ora_rk4(A, K, v0, 1e-3, 500)
        v = sysm.integrate(v0, 0.5, 1e-3)
        assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)
        with pytest.raises(lb.LBError) as e:
            sysm.integrate(v0, 0.5, 0.3)
        assert e.value.code == lb.native.LB_EINVAL
        sysm.close()


@pytest.mark.parametrize("N", [46, 51])
def test_host_buffer_upper_triangle_upload(N):
    """Above M = 2048 only the upper triangle of the host a is read (a is
    Hermitian): a host a whose strict lower triangle is NaN assembles to the
    same bits as the full Hermitian a assembled from device memory."""
    H, a = _case(N, 4600 + N)
    M = N * N - 1
    lb = lbm()
    a_half = a.copy()
    a_half[np.tril_indices(M, -1)] = np.nan
    with lb.Basis(N) as B:
        ref = _gpu_system(B, H, a, "closed")
        for alg in ("closed", "join"):
            sysm = lb.System(B, a_half, H=H, keep_parts=True, algorithm=alg)
            got = sysm.get("A")
            K = sysm.get("K")
            sysm.close()
            assert np.isfinite(got).all() and np.isfinite(K).all()
            if alg == "closed":
                assert np.array_equal(got, ref["A"]) and np.array_equal(K, ref["K"])
            else:
                _assert_entries(got, ref["A"], np.abs(ref["A"]).max(), "A (join)")


@pytest.mark.parametrize("N", [6, 46])
def test_host_buffer_pinned_upload(N):
    """A page-locked host a is read by the upload kernel over the host link,
    upper triangle only, at every M: with the strict lower triangle NaN it
    assembles to the bits of the device-resident a."""
    H, a = _case(N, 4700 + N)
    M = N * N - 1
    lb = lbm()
    pinned = torch.empty((M, M), dtype=torch.complex128, pin_memory=True)
    pinned.copy_(torch.from_numpy(a))
    pinned.numpy()[np.tril_indices(M, -1)] = np.nan
    with lb.Basis(N) as B:
        ref = _gpu_system(B, H, a, "closed")
        sysm = lb.System(B, pinned.numpy(), H=H, keep_parts=True, algorithm="closed")
        got, K = sysm.get("A"), sysm.get("K")
        sysm.close()
    assert np.array_equal(got, ref["A"]) and np.array_equal(K, ref["K"])
    del pinned


def test_empty_and_degenerate_inputs():
    lb = lbm()
    # a = 0, H = 0: everything vanishes
    with lb.Basis(3) as B:
        out = B.assemble_dense(torch.zeros((8, 8), dtype=torch.complex128, device="cuda"), A=True, K=True)
        assert out["A"].abs().max().item() == 0 and out["K"].abs().max().item() == 0
        # zero steps leave v untouched
        v = torch.arange(8, dtype=torch.float64, device="cuda")
        lb.rk4_dense(out["A"], out["K"], v, 1e-3, 0)
        assert torch.equal(v, torch.arange(8, dtype=torch.float64, device="cuda"))
    with pytest.raises(lb.LBError):
        lb.Basis(1)


def test_system_save_load_and_resume(tmp_path):
    """A saved and reloaded system is bit-identical; an integration split at
    multiples of the correction period gives the bits of one run."""
    N = 7
    H, a = _case(N, 707)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        sysm = lb.System(B, a, H=H, keep_parts=True, algorithm="closed")
        path = str(tmp_path / "sys.lbs")
        sysm.save(path)
        back = lb.System.load(B, path)
        for part in "AKQR":
            assert np.array_equal(back.get(part), sysm.get(part)), part
        v0 = o.expand(wl.pure_state(N, 1))[0].real
        for prec, corr in (("fp64", 0), ("fp32", 50), ("bf16", 25)):
            one = sysm.integrate(v0, 300 * 1e-3, 1e-3, precision=prec, correct_every=corr)
            v = v0.copy()
            back.integrate_resume(v, 1e-3, 100, precision=prec, correct_every=corr)
            back.integrate_resume(v, 1e-3, 150, precision=prec, correct_every=corr)
            back.integrate_resume(v, 1e-3, 50, precision=prec, correct_every=corr)
            assert np.array_equal(v, one), prec
        with lb.Basis(N + 1) as B2:
            with pytest.raises(lb.LBError):
                lb.System.load(B2, path)
        with pytest.raises(lb.LBError):
            lb.System.load(B, str(tmp_path / "missing.lbs"))
        with open(path, "r+b") as f:  # truncate: the loader reports it, the GPU is untouched
            f.truncate(1000)
        with pytest.raises(lb.LBError):
            lb.System.load(B, path)
        back.close()
        sysm.close()


def test_dense_assembly_n200_sampled_entries():
    """Dense random Lindbladian N = 200 (M = 39,999) in the launch the benchmark
    times: closed algorithm, A = Q + R written in place, K beside it.  Two full
    rows of A and 3000 random entries in each of four more rows (S, J and D
    rows) against the oracle's entry-by-entry Eq. (07) + Eq. (09); K in full
    against the oracle's Eq. (08) over the pairs f reads."""
    N = 200
    M, P = N * N - 1, N * (N - 1) // 2
    lb = lbm()
    a = wl.wishart_kossakowski_device(N, 20200)
    H = wl.gue_hamiltonian(N, 20201)
    with lb.Basis(N) as B:
        h = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
        A = torch.empty((M, M), dtype=torch.float64, device="cuda")
        K = torch.empty(M, dtype=torch.float64, device="cuda")
        B.assemble_dense_timed(a, h=h, A=A, K=K, algorithm="closed")
        torch.cuda.synchronize()
    g = np.random.default_rng(200)
    full = [P // 3, 2 * P + N // 2]
    part = [0, P + P // 2, 2 * P - 1, M - 1]
    s = np.concatenate([np.repeat(full, M), np.repeat(part, 3000)]).astype(np.int64)
    n = np.concatenate([np.tile(np.arange(M), len(full)), g.integers(0, M, 3000 * len(part))]).astype(np.int64)
    got = A[torch.as_tensor(s, device="cuda"), torch.as_tensor(n, device="cuda")].cpu().numpy()
    Kg = K.cpu().numpy()
    assert np.isfinite(Kg).all()
    del A
    # K (Eq. (08)) in full: the oracle reads a only where f touches it
    with Oracle(N) as o:
        fi, _ = o.structure("f", ordered=True)
        j = torch.as_tensor(fi[:, 0].astype(np.int64), device="cuda")
        k = torch.as_tensor(fi[:, 1].astype(np.int64), device="cuda")
        del fi
        ima = a.imag[j, k].cpu().numpy()
        del j, k
        Kref = o.K_on_f(ima)
        del ima
    assert np.abs(Kg - Kref).max() <= 1e-12 * np.abs(Kref).max()
    with Oracle(N) as o:
        need = o.rows_needed(np.unique(s))
        rows = a[torch.as_tensor(need, device="cuda")].cpu().numpy()
        del a
        R, S = o.R_entries_rows(need, rows, s, n)
        hh, _ = o.expand(H)
        Q = o.Q_entries(hh.real, s, n)
    ref = Q + R
    err = np.abs(got - ref)
    tol = 1e-12 * np.maximum(np.abs(ref), S + np.abs(Q)) + 1e-300
    bad = np.flatnonzero(err > tol)
    assert len(bad) == 0, "%d of %d sampled entries out of tolerance, first (s, n) = (%d, %d)" % (
        len(bad), len(s), s[bad[0]], n[bad[0]])


def _edge_scaled_kossakowski(N, seed, exps, zero_frac):
    """Wishart a = D W D with D diagonal: every basis element of edge (x, y)
    (its S and J index) is scaled by 2^e(x, y), every D_l by 2^e_l, e drawn
    from `exps`, and a fraction of the edges and of the D_l by 0.  The three
    matchings of a vertex quadruple then read a-blocks whose magnitudes
    differ by up to 2 (max - min) binades, some of them vanish, and the
    D-section sums mix magnitudes the same way."""
    W = wl.wishart_kossakowski(N, seed)
    g = np.random.default_rng(seed + 1)
    P = N * (N - 1) // 2
    M = N * N - 1
    e = g.choice(exps, P).astype(float)
    eD = g.choice(exps, N - 1).astype(float)
    d = np.concatenate([2.0 ** e, 2.0 ** e, 2.0 ** eD])
    zero = g.random(M) < zero_frac
    d[:P][zero[:P]] = 0.0
    d[P:2 * P][zero[:P]] = 0.0
    d[2 * P:][zero[2 * P:]] = 0.0
    return (d[:, None] * W) * d[None, :]


@pytest.mark.parametrize("N,exps,zero_frac", [
    (12, [-4, 0, 4], 0.0),           # spreads up to 8 binades: fixed-point sums near their limit
    (13, [-5, 0, 5], 0.0),           # up to 10
    (12, [-14, 0, 14], 0.0),         # far beyond: the FP64 form
    (17, [-14, -8, 0, 8, 14], 0.15), # mostly beyond 10 binades, and zero blocks
    (23, [-8, 0, 8], 0.3),
    (12, [0], 0.3),                  # equal magnitudes, many zero blocks: entries whose terms all vanish
])
def test_closed_assembly_mixed_magnitude_kossakowski(N, exps, zero_frac):
    """The closed form's disjoint-edge sums take an exact fixed-point path
    when the values of a vertex quadruple lie within 10 binades of its
    largest, and FP64 otherwise (and for zero blocks).  Both paths, and the
    switch between them inside one launch, against the oracle at the
    per-entry tolerance.  The diagonal rows sum only terms whose Eq. (09)
    coefficient is not zero, so an entry whose terms all vanish is exactly
    zero and a small entry beside large ones keeps its relative accuracy."""
    H = wl.gue_hamiltonian(N, 3300 + N)
    a = _edge_scaled_kossakowski(N, 3400 + N, exps, zero_frac)
    with lbm().Basis(N) as B, Oracle(N) as o:
        g = _gpu_system(B, H, a, "closed")
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
    _assert_entries(g["R"], R, S, "R")
    _assert_entries(g["A"], Q + R, S + np.abs(Q), "A")
    assert np.abs(g["K"] - K).max() <= 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("N,seed", [(12, 0), (16, 1), (21, 2)])
def test_pair_diagonal_entries_own_terms_only(N, seed):
    """Pair x diagonal rows (s, D_nu): their D-section sums run over the
    D_x of a window of x set by s and nu.  A Kossakowski matrix whose
    pair x D blocks are scaled by 2^eD(x) with eD = +-14 per D_x, and whose
    pair x pair block is 2^-40 (so the D-section terms dominate every
    entry's scale S), puts terms 2^28 apart inside and outside each window:
    the closed form must not form a window sum as a difference of two wider
    sums, whose rounding would be relative to the terms outside."""
    W = wl.wishart_kossakowski(N, 3500 + seed)
    g = np.random.default_rng(3600 + seed)
    P = N * (N - 1) // 2
    eD = g.choice([-14.0, 14.0], N - 1)
    d = np.concatenate([np.full(2 * P, 2.0 ** -20), 2.0 ** eD])
    a = (d[:, None] * W) * d[None, :]
    H = wl.gue_hamiltonian(N, 3700 + seed)
    with lbm().Basis(N) as B, Oracle(N) as o:
        gsys = _gpu_system(B, H, a, "closed")
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
    _assert_entries(gsys["R"], R, S, "R")
    _assert_entries(gsys["A"], Q + R, S + np.abs(Q), "A")
    assert np.abs(gsys["K"] - K).max() <= 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("N", [12, 19])
def test_closed_assembly_dense_ladder_kossakowski(N):
    """The ladder model's rank-one a = g l l^dagger given as a dense matrix:
    most vertex quadruples read zero blocks beside nonzero ones."""
    H, L, gam = wl.ladder_model(N, 50 + N)
    with lbm().Basis(N) as B, Oracle(N) as o:
        l, _ = o.expand(L)
        a = gam * np.outer(l, l.conj())
        g = _gpu_system(B, H, a, "closed")
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
    _assert_entries(g["R"], R, S, "R")
    _assert_entries(g["A"], Q + R, S + np.abs(Q), "A")
    assert np.abs(g["K"] - K).max() <= 1e-12 * np.abs(K).max()


def test_rk4_fp64_n50_full_trajectory():
    """Dense N = 50 random Lindbladian (M = 2499), rho0 = |0><0|, 10^4 FP64
    RK4 steps of dt = 1e-3: every 1000-step snapshot within 1e-12 ||v|| of the
    oracle's RK4 on the oracle's own A and K."""
    N, dt, steps, every = 50, 1e-3, 10_000, 1000
    H, a = _case(N, 1050)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 0))[0].real
        ref_v, ref_snaps = ora_rk4(A, K, v0, dt, steps, snap_every=every)
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous(), algorithm="closed")
        v = torch.tensor(v0, device="cuda")
        snaps = lb.rk4_dense(g["A"], g["K"], v, dt, steps, precision="fp64", snap_every=every)
        torch.cuda.synchronize()
    snaps = snaps.cpu().numpy()
    for t in range(len(ref_snaps)):
        assert np.linalg.norm(snaps[t] - ref_snaps[t]) <= 1e-12 * np.linalg.norm(ref_snaps[t]), t
    assert np.linalg.norm(v.cpu().numpy() - ref_v) <= 1e-12 * np.linalg.norm(ref_v)


def _ladder_channels(o, N, seed):
    H, L, g = wl.ladder_model(N, seed)
    l, _ = o.expand(L)
    nz = np.nonzero(np.abs(l) > 0)[0]
    return H, g, nz, l[nz], g * np.outer(l, l.conj())


@pytest.mark.parametrize("N", [5, 8])
def test_host_api_lowrank_dense_and_csr_systems(N):
    """lb_assemble with a low-rank Kossakowski matrix (one channel, the ladder
    operator; Sec. 2's sum over jump operators) into a dense and into a CSR
    system: dense A against the oracle's Q + R at the per-entry tolerance; the
    CSR pattern bit-exact and its values against the oracle's sparse route;
    snapshots of lb_integrate on both systems within 1e-12 ||v|| of the
    oracle's RK4."""
    from oracle import lowrank_csr
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        H, g, nz, lv, a = _ladder_channels(o, N, 900 + N)
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        R, S = o.R(a, return_scale=True)
        K = o.K(a)
        rp_o, col_o, val_o, K_o = lowrank_csr(o, h.real, [g], [(nz, lv)])
        v0 = o.expand(wl.pure_state(N, N - 1))[0].real
        ref_v, ref_snaps = ora_rk4(Q + R, K, v0, 1e-3, 600, snap_every=200)
        ch = [(g, nz, lv)]
        dense = lb.System(B, None, H=H, channels=ch, format="dense", keep_parts=True)
        assert dense.info() == {"format": "dense", "M": B.M, "nnz": B.M * B.M}
        _assert_entries(dense.get("R"), R, S, "R (low-rank a, dense system)")
        _assert_entries(dense.get("A"), Q + R, S + np.abs(Q), "A (low-rank a, dense system)")
        assert np.abs(dense.get("K") - K).max() <= 1e-12 * np.abs(K).max()
        tm = dense.timings()
        assert set(tm) == {"alloc", "h2d", "kernels", "d2h", "free"} and min(tm.values()) >= 0.0
        csr = lb.System(B, None, H=H, channels=ch, format="csr")
        rp, col, val = csr.get_csr()
        assert csr.info()["format"] == "csr" and csr.info()["nnz"] == len(col)
        assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
        assert np.abs(val - val_o).max() <= 1e-12 * np.abs(val_o).max()
        assert np.abs(csr.get("K") - K_o).max() <= 1e-12 * max(np.abs(K_o).max(), 1e-300) + 1e-18
        for sysm, prec in ((dense, "fp64"), (csr, "fp64")):
            snaps = sysm.integrate(v0, 0.6, 1e-3, precision=prec, snap_every=200)
            assert snaps.shape == ref_snaps.shape
            for t in range(len(ref_snaps)):
                assert np.linalg.norm(snaps[t] - ref_snaps[t]) <= 1e-12 * np.linalg.norm(ref_snaps[t])
            fin = sysm.integrate(v0, 0.6, 1e-3, precision=prec)
            assert np.array_equal(fin, snaps[-1])
        with pytest.raises(lb.LBError) as e:
            dense.integrate(v0, 0.6, 1e-3, snap_every=250)          # 600 steps, not a multiple
        assert e.value.code == lb.native.LB_EINVAL
        with pytest.raises(lb.LBError) as e:
            csr.get("A")
        assert e.value.code == lb.native.LB_EINVAL
        dense.close()
        csr.close()
        with pytest.raises(lb.LBError) as e:                       # dense a into CSR
            lb.System(B, a, H=H, format="csr")
        assert e.value.code == lb.native.LB_EUNSUPPORTED
        with pytest.raises(lb.LBError) as e:                       # Q, R not kept in CSR
            lb.System(B, None, channels=ch, format="csr", keep_parts=True)
        assert e.value.code == lb.native.LB_EUNSUPPORTED
        lb.native.host_release()


def test_host_api_expand_and_rho():
    N = 9
    g = np.random.default_rng(9)
    A = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    v = g.standard_normal(N * N - 1)
    with lbm().Basis(N) as B, Oracle(N) as o:
        assert np.abs(B.expand_host(A) - o.expand(A)[0]).max() < 1e-13
        assert np.abs(B.rho_host(v) - o.rho(v)).max() < 1e-13


def test_host_api_repeated_calls_reuse_memory():
    """Repeated host-buffer assemblies of one size give the same bits (the
    pool hands back the same reservation), and their allocation phase is
    short once the size has been seen."""
    N = 30
    H, a = _case(N, 3030)
    lb = lbm()
    with lb.Basis(N) as B:
        outs, allocs = [], []
        for _ in range(3):
            s = lb.System(B, a, H=H)
            outs.append(s.get("A"))
            allocs.append(s.timings()["alloc"])
            s.close()
        assert all(np.array_equal(outs[0], x) for x in outs[1:])
        assert allocs[2] < 50.0


@pytest.mark.parametrize("N,R", [(6, 5), (10, 1)])
def test_propagator_multistate_fp64_vs_oracle(N, R):
    """lb_propagator_form / lb_propagate in FP64: R initial states stepped
    together (one product of D' = (P(hA) - 1)/h with the block of states per
    step) stay within 1e-12 ||v|| of the oracle's stage-by-stage RK4 for
    every state, over 3000 steps with snapshots every 1000."""
    dt, steps, every = 1e-3, 3000, 1000
    H, a = _case(N, 1300 + N)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0s = [o.expand(wl.pure_state(N, k % N))[0].real for k in range(R)]
        refs = [ora_rk4(A, K, v0, dt, steps, snap_every=every)[1] for v0 in v0s]
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous())
    P = lb.Propagator(g["A"], g["K"], dt, precision="fp64", nrhs=R)
    V = torch.tensor(np.stack(v0s), device="cuda")
    snaps = P.step(V, steps, snap_every=every)
    torch.cuda.synchronize()
    snaps = snaps.cpu().numpy()
    for r in range(R):
        for t in range(steps // every):
            ref = refs[r][t]
            assert np.linalg.norm(snaps[t, r] - ref) <= 1e-12 * np.linalg.norm(ref), (r, t)
    assert np.array_equal(V.cpu().numpy(), snaps[-1])


def test_propagator_multistate_fp32_corrected():
    """FP32 propagator, 4 states of a 12-level system, 2000 steps: within the
    FP32 bars (1e-5 plain, 2e-6 with the FP64 defect every 50 steps) of the
    oracle's RK4, and the correction lowers the error."""
    N, R, dt, steps = 12, 4, 1e-3, 2000
    H, a = _case(N, 1212)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0s = [o.expand(wl.pure_state(N, 3 * k))[0].real for k in range(R)]
        refs = [ora_rk4(A, K, v0, dt, steps)[0] for v0 in v0s]
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous())
    P = lb.Propagator(g["A"], g["K"], dt, precision="fp32", nrhs=R)
    errs = {}
    for corr in (0, 50):
        V = torch.tensor(np.stack(v0s), device="cuda")
        P.step(V, steps, correct_every=corr)
        torch.cuda.synchronize()
        Vh = V.cpu().numpy()
        errs[corr] = max(np.linalg.norm(Vh[r] - refs[r]) / np.linalg.norm(refs[r]) for r in range(R))
    assert errs[0] < 1e-5, errs
    assert errs[50] < 2e-6, errs
    assert errs[50] < 0.5 * errs[0], errs
    with pytest.raises(lb.LBError):
        lb.Propagator(g["A"], g["K"], dt, precision="fp64", nrhs=65)


@pytest.mark.parametrize("N", [5, 12, 30])
def test_steady_state_against_oracle_solve(N):
    """FP64 GMRES on the device for (Q + R) v* = -K (Sec. 2: the steady
    state of the real system) against numpy's dense solve of the oracle's
    A and K: true relative residual <= 1e-11, solution within 1e-8, and the
    rebuilt rho* is a density matrix (trace 1, Hermitian, PSD within 1e-10)."""
    H, a = _case(N, 1400 + N)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        ref = np.linalg.solve(A, -K)
        g = B.assemble_dense(torch.tensor(a, device="cuda"),
                             h=B.expand(torch.tensor(H, device="cuda")).real.contiguous())
        v, res, it = lb.steady_state(g["A"], g["K"], tol=1e-13, max_iter=5000)
        torch.cuda.synchronize()
        assert res <= 1e-11, (res, it)
        vh = v.cpu().numpy()
        assert np.linalg.norm(vh - ref) <= 1e-8 * np.linalg.norm(ref), (res, it)
        chk = lb.rho_checks(B, v.contiguous(), psd_shift=1e-10)[0]
        rho = o.rho(vh)
    assert abs(chk[0]) < 1e-13 and chk[1] < 1e-13 and chk[2] > 0.0, chk
    assert abs(np.trace(rho) - 1) < 1e-13 and np.linalg.eigvalsh(rho).min() > -1e-10


@pytest.mark.parametrize("N", [4, 23, 40])
def test_dense_assembly_deterministic(N):
    """The CLOSED assembly writes every entry once, with no atomics: two
    calls (lb_assemble_dense and the event-timed lb_assemble_dense_timed)
    write the same bits into buffers prefilled with NaN."""
    H, a = _case(N, 4800 + N)
    lb = lbm()
    with lb.Basis(N) as B:
        ad = torch.tensor(a, device="cuda")
        h = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
        M = B.M
        A1 = torch.full((M, M), float("nan"), dtype=torch.float64, device="cuda")
        A2 = torch.full((M, M), float("nan"), dtype=torch.float64, device="cuda")
        K1, K2 = (torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(2))
        B.assemble_dense(ad, h=h, A=A1, K=K1, algorithm="closed")
        ms = B.assemble_dense_timed(ad, h=h, A=A2, K=K2, algorithm="closed")
        torch.cuda.synchronize()
    assert torch.isfinite(A1).all()
    assert torch.equal(A1, A2) and torch.equal(K1, K2)
    assert all(t >= 0.0 for t in ms.values())


@pytest.mark.parametrize("N", [5, 12, 30])
def test_steady_state_preconditioned_against_oracle_solve(N):
    """The same solve preconditioned from H's eigenbasis (P = Q - sigma 1,
    sigma = -Tr(A)/M): the same bars, in far fewer iterations than the plain
    GMRES takes on the same system."""
    H, a = _case(N, 1400 + N)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        ref = np.linalg.solve(A, -K)
        Hd = torch.tensor(H, device="cuda")
        g = B.assemble_dense(torch.tensor(a, device="cuda"), h=B.expand(Hd).real.contiguous())
        v, res, it = lb.steady_state(g["A"], g["K"], tol=1e-13, max_iter=500, basis=B, H=Hd)
        _, res0, it0 = lb.steady_state(g["A"], g["K"], tol=1e-13, max_iter=5000)
        torch.cuda.synchronize()
        assert res <= 1e-11, (res, it)
        assert np.linalg.norm(v.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref), (res, it)
        assert it <= max(10, it0 // 4), (it, it0)
        # an explicit shift gives the same solution
        v2, res2, _ = lb.steady_state(g["A"], g["K"], tol=1e-13, max_iter=500, basis=B, H=Hd,
                                      sigma=-float(np.trace(A)) / B.M)
        assert res2 <= 1e-11 and np.linalg.norm(v2.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_steady_state_degenerate_inputs():
    """K = 0 (a = gamma 1): v* = 0 with zero residual and no iteration."""
    N = 4
    M = N * N - 1
    lb = lbm()
    with lb.Basis(N) as B:
        g = B.assemble_dense(torch.eye(M, dtype=torch.complex128, device="cuda") * 0.3)
        v = torch.ones(M, dtype=torch.float64, device="cuda")
        v, res, it = lb.steady_state(g["A"], g["K"], v=v)
        torch.cuda.synchronize()
        assert res == 0.0 and it == 0 and v.abs().max().item() == 0.0


def test_rho_checks_against_oracle():
    """Trace, Hermiticity and the shifted-Cholesky PSD test of rho on the
    device, on states with known answers: snapshots of an RK4 trajectory
    (density matrices), a pure state (PSD, eigenvalue 0 present) and a
    state scaled out of the PSD cone."""
    N = 6
    H, a = _case(N, 606)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        A, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 2))[0].real
        _, snaps = ora_rk4(A, K, v0, 1e-2, 400, snap_every=100)
        states = np.concatenate([snaps, v0[None, :], -3.0 * v0[None, :]])
        out = lb.rho_checks(B, torch.tensor(states, device="cuda"), psd_shift=1e-10)
        for k in range(len(states)):
            rho = o.rho(states[k])
            assert abs(out[k, 0] - (np.trace(rho).real - 1.0)) < 1e-14
            assert out[k, 1] < 1e-15
        lam_min = [np.linalg.eigvalsh(o.rho(x)).min() for x in states]
    assert all(out[k, 2] > 0.0 for k in range(len(snaps) + 1)), out
    assert lam_min[-1] < -1e-3 and out[-1, 2] <= 0.0, (lam_min[-1], out[-1])

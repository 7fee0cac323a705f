"""Batched form: many realizations of mixed N through lb_batch_* (needs a GPU).

Bars: each realization's assembled A and K bit-identical to the single-system
assembly; FP32 trajectories within the single-system FP32 bars of the FP64
trajectory (1e-5 relative without correction, 2e-6 with the FP64 defect
correction every 50 steps) at every cluster size; the FP64 trajectory itself
within 1e-12 of the oracle's for small N; a realization gives the same bits
alone as inside a mixed batch.
"""
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
    import paper_1912_01491_gb300 as lb
    return lb


def _inputs(N, seed):
    H = wl.gue_hamiltonian(N, seed)
    a = wl.wishart_kossakowski(N, seed + 1)
    return H, a


class _Ens:
    """Device inputs and FP64 single-system references for a list of N."""

    def __init__(self, Ns, seed, dt, steps):
        lb = lbm()
        self.Ns, self.dt, self.steps = list(Ns), dt, steps
        self.a, self.h, self.v0, self.A, self.K, self.ref = [], [], [], [], [], []
        for r, N in enumerate(self.Ns):
            H, a = _inputs(N, seed + 10 * r)
            with lb.Basis(N) as B:
                ad = torch.tensor(a, device="cuda")
                hd = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
                g = B.assemble_dense(ad, h=hd, algorithm="closed")
                rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
                rho0[r % N, r % N] = 1.0
                v0 = B.expand(rho0).real.contiguous()
            v = v0.clone()
            lb.rk4_dense(g["A"], g["K"], v, dt, steps, precision="fp64")
            self.a.append(ad)
            self.h.append(hd)
            self.v0.append(v0)
            self.A.append(g["A"])
            self.K.append(g["K"])
            self.ref.append(v)
        torch.cuda.synchronize()

    def batch(self):
        b = lbm().Batch(self.Ns)
        self.v = [x.clone() for x in self.v0]
        for r in range(len(self.Ns)):
            b.set(r, self.a[r], self.h[r], self.v[r])
        b.assemble("closed")
        return b

    def errors(self):
        torch.cuda.synchronize()
        return [float(torch.linalg.norm(self.v[r] - self.ref[r]) / torch.linalg.norm(self.ref[r]))
                for r in range(len(self.Ns))]


def test_batch_assembly_bit_identical_to_single():
    ens = _Ens([4, 7, 12, 5, 20, 9, 2], 7000, 1e-3, 1)
    b = ens.batch()
    for r in range(len(ens.Ns)):
        A, K = b.system(r)
        assert np.array_equal(A, ens.A[r].cpu().numpy()), r
        assert np.array_equal(K, ens.K[r].cpu().numpy()), r
    b.close()


def test_fp64_reference_matches_oracle():
    """The FP64 single-system trajectories used as the batch's reference agree
    with the oracle's RK4 (small N)."""
    ens = _Ens([3, 6, 9], 7100, 1e-3, 300)
    for r, N in enumerate(ens.Ns):
        H, a = _inputs(N, 7100 + 10 * r)
        with Oracle(N) as o:
            h, _ = o.expand(H)
            A = o.Q(h.real) + o.R(a)
            K = o.K(a)
            ref, _ = ora_rk4(A, K, ens.v0[r].cpu().numpy(), ens.dt, ens.steps)
        got = ens.ref[r].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_batch_fp32_every_cluster_size(C):
    ens = _Ens([4, 11, 17, 23, 30, 6, 40, 13], 7200, 1e-3, 400)
    for corr, tol in ((0, 1e-5), (50, 2e-6)):
        b = ens.batch()
        for r in range(len(ens.Ns)):
            b.set_cluster(r, C)
        b.integrate(ens.dt, ens.steps, correct_every=corr)
        errs = ens.errors()
        b.close()
        assert max(errs) < tol, (corr, errs)


def test_batch_tune_keeps_state_and_integrates():
    Ns = [int(n) for n in wl.batch_sizes(24, 7300)]
    ens = _Ens(Ns, 7300, 1e-3, 300)
    b = ens.batch()
    choice = b.tune(width=6, probe_steps=10, dt=ens.dt)
    assert set(int(c) for c in choice) <= {1, 2, 4, 8, 16}
    for r in range(len(Ns)):
        assert torch.equal(ens.v[r], ens.v0[r]), "tune must restore the states"
    b.integrate(ens.dt, ens.steps, correct_every=50)
    errs = ens.errors()
    b.close()
    assert max(errs) < 2e-6, errs


def test_alone_equals_in_mix():
    """One realization integrated in a batch of one gives the same bits as the
    same realization inside a mixed batch (same cluster size)."""
    ens = _Ens([9, 31, 5, 17, 38], 7400, 1e-3, 200)
    for C in (1, 4):
        b = ens.batch()
        for r in range(len(ens.Ns)):
            b.set_cluster(r, C)
        b.integrate(ens.dt, ens.steps, correct_every=25)
        torch.cuda.synchronize()
        mixed = [x.clone() for x in ens.v]
        b.close()
        for r in (0, 1, 4):
            lb = lbm()
            one = lb.Batch([ens.Ns[r]])
            v = ens.v0[r].clone()
            one.set(0, ens.a[r], ens.h[r], v)
            one.assemble("closed")
            one.set_cluster(0, C)
            one.integrate(ens.dt, ens.steps, correct_every=25)
            torch.cuda.synchronize()
            assert torch.equal(v, mixed[r]), (C, r)
            one.close()


def test_batch_degenerate_and_errors():
    lb = lbm()
    with pytest.raises(lb.LBError):
        lb.Batch([1, 4])
    with pytest.raises(lb.LBError):
        lb.Batch([65])
    ens = _Ens([2, 3], 7500, 1e-3, 5)
    b = ens.batch()
    with pytest.raises(lb.LBError):
        b.set_cluster(0, 3)
    b.integrate(ens.dt, 0)   # zero steps leave the state unchanged
    torch.cuda.synchronize()
    for r in range(2):
        assert torch.equal(ens.v[r], ens.v0[r])
    b.close()


@pytest.mark.parametrize("C", [1, 4, 16])
def test_batch_fp64_matches_single_system(C):
    """FP64 persistent form: same RK4 in FP64 arithmetic, against the FP64
    single-system trajectory within 1e-12 (summation order differs)."""
    ens = _Ens([3, 6, 10, 17, 29], 7600, 1e-3, 300)
    b = ens.batch()
    b.set_precision("fp64")
    for r in range(len(ens.Ns)):
        b.set_cluster(r, C)
    b.integrate(ens.dt, ens.steps)
    errs = ens.errors()
    b.close()
    assert max(errs) < 1e-12, errs


def test_batch_fp64_n10_full_trajectory_vs_oracle():
    """Dense N = 10, rho0 = |0><0|, t = 10, dt = 1e-3 (10^4 steps) in one
    persistent FP64 launch, against the oracle's RK4 within 1e-12 ||v||."""
    N, dt, steps = 10, 1e-3, 10_000
    H, a = _inputs(N, 1010)
    lb = lbm()
    with Oracle(N) as o:
        h, _ = o.expand(H)
        A = o.Q(h.real) + o.R(a)
        K = o.K(a)
        v0 = o.expand(wl.pure_state(N, 0))[0].real
        ref, _ = ora_rk4(A, K, v0, dt, steps)
    with lb.Basis(N) as B:
        hd = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
    ad = torch.tensor(a, device="cuda")
    v = torch.tensor(v0, device="cuda")
    b = lb.Batch([N])
    b.set(0, ad, hd, v)
    b.assemble("closed")
    b.set_precision("fp64")
    choice = b.tune(width=4, probe_steps=20, dt=dt)
    b.integrate(dt, steps)
    torch.cuda.synchronize()
    b.close()
    got = v.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), choice


# ---------------------------------------------------------------- propagator form

@pytest.mark.parametrize("N", [4, 7, 10])
def test_propagator_fp64_full_trajectory_vs_oracle(N):
    """The propagator form v <- v + h (D' v + c'), D' = (P(hA) - 1)/h, is one
    classical RK4 step (Sec. 4 item 3) written as one product: in FP64 it
    stays within 1e-12 ||v|| of the oracle's stage-by-stage RK4 over 10^4
    steps of dt = 1e-3."""
    dt, steps = 1e-3, 10_000
    H, a = _inputs(N, 1100 + N)
    lb = lbm()
    with Oracle(N) as o:
        h, _ = o.expand(H)
        A = o.Q(h.real) + o.R(a)
        K = o.K(a)
        v0 = o.expand(wl.pure_state(N, N // 2))[0].real
        ref, _ = ora_rk4(A, K, v0, dt, steps)
    with lb.Basis(N) as B:
        hd = B.expand(torch.tensor(H, device="cuda")).real.contiguous()
    ad = torch.tensor(a, device="cuda")
    v = torch.tensor(v0, device="cuda")
    b = lb.Batch([N])
    b.set(0, ad, hd, v)
    b.assemble("closed")
    b.set_precision("fp64")
    b.set_form("propagator")
    assert b.form_propagator(dt) >= 0.0
    b.integrate(dt, steps)
    torch.cuda.synchronize()
    b.close()
    got = v.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("C", [1, 4, 16])
def test_propagator_fp32_corrected_every_cluster_size(C):
    """FP32 propagator with the FP64 defect every 50 steps: within the FP32
    bar of the corrected stage-by-stage form (2e-6 of the FP64 trajectory,
    2000 steps), and the correction lowers the error."""
    ens = _Ens([12, 9, 20, 5], 2200, 1e-3, 2000)
    errs = {}
    for corr in (0, 50):
        b = ens.batch()
        b.set_form("propagator")
        for r in range(len(ens.Ns)):
            b.set_cluster(r, C)
        b.integrate(ens.dt, ens.steps, correct_every=corr)
        errs[corr] = ens.errors()
        b.close()
    assert max(errs[0]) < 1e-5, errs
    assert max(errs[50]) < 2e-6, errs
    assert max(errs[50]) < 0.5 * max(errs[0]), errs


def test_propagator_alone_equals_in_mix():
    """A realization integrated by the propagator form gives the same bits
    alone as inside a batch of mixed N (the clusters share nothing)."""
    ens = _Ens([11, 6, 17, 30, 11], 2300, 1e-3, 300)
    b = ens.batch()
    b.set_form("propagator")
    b.integrate(ens.dt, ens.steps, correct_every=50)
    torch.cuda.synchronize()
    mix = [x.clone() for x in ens.v]
    b.close()
    for r in (0, 3):
        lb = lbm()
        v = ens.v0[r].clone()
        one = lb.Batch([ens.Ns[r]])
        one.set(0, ens.a[r], ens.h[r], v)
        one.assemble("closed")
        one.set_form("propagator")
        one.set_cluster(0, 1)
        one.integrate(ens.dt, ens.steps, correct_every=50)
        torch.cuda.synchronize()
        one.close()
        # the cluster size of the batch run is the default (1) for every realization
        assert torch.equal(v, mix[r]), r


def test_propagator_reformed_when_dt_changes():
    """D' depends on h: integrating with another dt forms it again, and the
    result equals a batch formed for that dt from the start."""
    ens = _Ens([8, 13], 2400, 2e-3, 400)
    b = ens.batch()
    b.set_form("propagator")
    b.set_precision("fp64")
    b.form_propagator(1e-3)
    b.integrate(2e-3, 400)
    torch.cuda.synchronize()
    errs = ens.errors()
    b.close()
    assert max(errs) < 1e-12, errs

"""Serving form through lb_server_* (needs a GPU).

Bars: a request's result is bit-identical alone and inside a mix of
concurrent requests of other sizes, precisions and engines; stream-engine
results are bit-identical to lb_rk4_dense with the same parameters (the CUDA
graph replays the same kernels), cluster-engine results to lb_batch with the
same cluster size; against the FP64 trajectory the FP32 + correction results
are within 2e-6 and BF16 + correction within 1e-3 (the single-system bars).
Admission, bounded waits and input release are checked on the host side.
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


class Job:
    def __init__(self, N, seed, precision, corr, nsteps=300, dt=1e-3):
        self.N, self.M = N, N * N - 1
        self.precision, self.corr, self.nsteps, self.dt = precision, corr, nsteps, dt
        self.Hd = torch.tensor(wl.gue_hamiltonian(N, seed), device="cuda")
        if N < 40:
            self.ad = torch.tensor(wl.wishart_kossakowski(N, seed + 1), device="cuda")
        else:
            self.ad = wl.wishart_kossakowski_device(N, seed + 1)
        rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
        rho0[seed % N, seed % N] = 1.0
        with lbm().Basis(N) as B:
            self.v0 = B.expand(rho0).real.contiguous()
            self.h = B.expand(self.Hd).real.contiguous()
            g = B.assemble_dense(self.ad, h=self.h, algorithm="closed")
        self.A, self.K = g["A"], g["K"]
        v = self.v0.clone()
        lbm().rk4_dense(self.A, self.K, v, dt, nsteps, precision="fp64")
        self.ref64 = v

    def submit(self, srv):
        out = torch.full_like(self.v0, float("nan"))
        rid = srv.submit(self.ad, self.v0, out, self.dt, self.nsteps, H=self.Hd, precision=self.precision,
                         correct_every=self.corr)
        return rid, out

    def single(self):
        """Same request through the single-system entry point."""
        lb = lbm()
        v = self.v0.clone()
        if self.precision == "fp64":
            lb.rk4_dense(self.A, self.K, v, self.dt, self.nsteps, precision="fp64")
        elif self.precision == "fp32":
            lb.rk4_dense(lb.pack_fp32(self.A), self.K, v, self.dt, self.nsteps, precision="fp32", A64=self.A,
                         correct_every=self.corr)
        else:
            Ab, sc = lb.pack_bf16(self.A)
            lb.rk4_dense(Ab, self.K, v, self.dt, self.nsteps, precision="bf16", scale=sc, A64=self.A,
                         correct_every=self.corr)
        return v

    def err64(self, v):
        return float(torch.linalg.norm(v - self.ref64) / torch.linalg.norm(self.ref64))


def _jobs():
    return [Job(5, 11, "fp32", 50), Job(12, 12, "fp32", 25), Job(20, 13, "fp32", 50), Job(33, 14, "fp32", 0),
            Job(70, 15, "bf16", 50), Job(90, 16, "fp32", 50), Job(8, 17, "fp64", 0), Job(30, 18, "bf16", 50),
            Job(66, 19, "fp64", 0)]


TOL = {"fp64": 1e-12, "fp32": 2e-6, "bf16": 1e-3}


def test_alone_equals_in_mix_and_matches_single_system():
    lb = lbm()
    jobs = _jobs()
    budget = 8 << 30
    alone = []
    with lb.Server(budget, slots=8, bypass_ms=50.0) as srv:
        for j in jobs:
            rid, out = j.submit(srv)
            res = srv.wait(rid, 120_000)
            assert res["state"] == 3
            alone.append((out, res))
        # everything at once, in another order, each job twice
        order = [8, 3, 0, 5, 1, 7, 2, 6, 4] * 2
        subs = [(k, *jobs[k].submit(srv)) for k in order]
        for k, rid, out in subs:
            res = srv.wait(rid, 120_000)
            assert res["engine"] == alone[k][1]["engine"]
            assert torch.equal(out, alone[k][0]), (jobs[k].N, jobs[k].precision)
        st = srv.stats()
        assert st["completed"] == len(jobs) * 3
        assert 0 < st["p50_ms"] <= st["p99_ms"]
    for k, j in enumerate(jobs):
        out, res = alone[k]
        e = j.err64(out)
        assert e < TOL[j.precision], (j.N, j.precision, e)
        if res["engine"] == 1:   # stream engine: same kernels as the single-system path
            assert torch.equal(out, j.single()), (j.N, j.precision)
        else:                    # cluster engine: same as lb_batch at the same cluster size
            b = lb.Batch([j.N])
            v = j.v0.clone()
            b.set(0, j.ad, j.h, v)
            b.assemble("closed")
            b.set_cluster(0, res["cluster"])
            b.integrate(j.dt, j.nsteps, correct_every=j.corr)
            torch.cuda.synchronize()
            b.close()
            assert torch.equal(out, v), (j.N, res["cluster"])


def test_fp64_request_matches_oracle():
    j = Job(6, 40, "fp64", 0, nsteps=200)
    H, a = wl.gue_hamiltonian(6, 40), wl.wishart_kossakowski(6, 41)
    with Oracle(6) as o:
        h, _ = o.expand(H)
        ref, _ = ora_rk4(o.Q(h.real) + o.R(a), o.K(a), j.v0.cpu().numpy(), j.dt, j.nsteps)
    with lbm().Server(1 << 30) as srv:
        rid, out = j.submit(srv)
        srv.wait(rid, 60_000)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_admission_by_memory_and_refusal():
    lb = lbm()
    j = Job(60, 50, "bf16", 50, nsteps=400)
    need = lb.request_bytes(60, "bf16", True)
    # room for exactly one at a time
    with lb.Server(need + need // 2, slots=8, bypass_ms=0.0) as srv:
        subs = [j.submit(srv) for _ in range(3)]
        res = [srv.wait(rid, 120_000) for rid, _ in subs]
        for (_, out), r in zip(subs, res):
            assert torch.equal(out, subs[0][1])
        # the later ones waited for memory
        assert res[1]["queue_ms"] > 0.5 * res[0]["gpu_ms"]
        assert res[2]["queue_ms"] > res[1]["queue_ms"]
        big = Job(70, 51, "fp32", 50, nsteps=1)
        with pytest.raises(lb.LBError) as ei:
            big.submit(srv)
        assert ei.value.code == 2   # LB_ENOMEM: can never fit


def test_wait_is_bounded_and_inputs_are_released():
    lb = lbm()
    j = Job(90, 60, "fp32", 50, nsteps=3000)
    with lb.Server(8 << 30) as srv:
        rid, out = j.submit(srv)
        with pytest.raises(lb.LBError) as ei:
            srv.wait(rid, 0.01)
        assert ei.value.code == 4   # LB_ETIMEOUT
        # once assembled, the caller may overwrite its inputs
        import time
        t0 = time.time()
        while srv.state(rid) < 2 and time.time() - t0 < 60:
            time.sleep(0.001)
        assert srv.state(rid) >= 2
        j.ad.fill_(float("nan"))
        j.Hd.fill_(float("nan"))
        j.v0.fill_(float("nan"))
        srv.wait(rid, 120_000)
    assert bool(torch.isfinite(out).all())
    assert j.err64(out) < TOL["fp32"]


def test_bad_requests():
    lb = lbm()
    with lb.Server(1 << 30) as srv:
        v = torch.zeros(3, dtype=torch.float64, device="cuda")
        with pytest.raises(lb.LBError):
            srv.submit(None, v, v, 1e-3, 10)
        with pytest.raises(lb.LBError):
            srv.poll(12345)

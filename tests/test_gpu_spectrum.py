"""Spectrum of the generator (Sec. 6, Fig. 5) through the C ABI (needs a GPU).

The eigenvalues of A = Q + R against numpy's eigenvalues of the oracle's A
(LAPACK's dense nonsymmetric solver on the CPU), matched one to one; the
properties every generator's spectrum has (conjugate pairs, sum = Tr A, no
eigenvalue in the right half plane); and the density grid against counts
that are known exactly (a block-diagonal matrix of 2 x 2 blocks a I + b J,
eigenvalues a +- i b).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import Oracle

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


def _match(got, ref):
    """Largest distance of a one-to-one matching of two eigenvalue lists."""
    sp = pytest.importorskip("scipy.optimize")
    cost = np.abs(got[:, None] - ref[None, :])
    r, c = sp.linear_sum_assignment(cost)
    return cost[r, c].max()


@pytest.mark.parametrize("N", [3, 6, 9])
def test_spectrum_against_oracle_eigenvalues(N):
    H, a = wl.gue_hamiltonian(N, 500 + N), wl.wishart_kossakowski(N, 501 + N)
    lb = lbm()
    with lb.Basis(N) as B, Oracle(N) as o:
        h, _ = o.expand(H)
        A = o.Q(h.real) + o.R(a)
        ref = np.linalg.eigvals(A)
        sysm = lb.System(B, a, H=H)
        got = sysm.spectrum()
        sysm.close()
        dev = lb.spectrum(torch.tensor(A, device="cuda")).cpu().numpy()
    scale = np.abs(ref).max()
    assert _match(got, ref) <= 1e-9 * scale
    assert _match(dev, ref) <= 1e-9 * scale
    # properties of the spectrum of a real generator of a CPTP semigroup
    assert got.real.max() <= 1e-9 * scale
    assert abs(got.sum() - np.trace(A)) <= 1e-9 * scale * len(got)
    assert _match(got, np.conj(got)) <= 1e-9 * scale


def test_spectrum_density_exact_counts():
    """Blocks [[a, -b], [b, a]] have eigenvalues a +- i b; the grid counts
    them cell by cell, divided by the cell area."""
    rng = np.random.default_rng(5)
    nb = 64
    pts = rng.uniform([-4.0, 0.1], [-0.1, 3.0], size=(nb, 2))
    M = 2 * nb
    A = np.zeros((M, M))
    for k, (x, y) in enumerate(pts):
        A[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[x, -y], [y, x]]
    lb = lbm()
    eig = lb.spectrum(torch.tensor(A, device="cuda"))
    e = eig.cpu().numpy()
    ref = np.concatenate([pts[:, 0] + 1j * pts[:, 1], pts[:, 0] - 1j * pts[:, 1]])
    assert _match(e, ref) <= 1e-12 * np.abs(ref).max()
    box, nre, nim = (-4.0, 0.0, -3.0, 3.0), 8, 12
    dens = lb.spectrum_density(eig, box, nre, nim).cpu().numpy()
    area = (box[1] - box[0]) / nre * (box[3] - box[2]) / nim
    # the same counts from the matched reference values
    cnt = np.zeros((nre, nim))
    for z in ref:
        i = min(int((z.real - box[0]) / (box[1] - box[0]) * nre), nre - 1)
        j = min(int((z.imag - box[2]) / (box[3] - box[2]) * nim), nim - 1)
        cnt[i, j] += 1
    assert np.array_equal(np.rint(dens * area), cnt)
    assert np.rint(dens.sum() * area) == M
    # eigenvalues outside the box are not counted
    dens2 = lb.spectrum_density(eig, (-2.0, 0.0, 0.0, 3.0), 4, 4).cpu().numpy()
    inside = np.sum((ref.real >= -2.0) & (ref.imag >= 0.0) & (ref.imag < 3.0))
    assert np.rint(dens2.sum() * (2.0 / 4) * (3.0 / 4)) == inside


def test_spectrum_arguments():
    lb = lbm()
    with pytest.raises(lb.LBError):
        lb.spectrum_density(torch.zeros(4, dtype=torch.complex128, device="cuda"), (0.0, 0.0, 0.0, 1.0))
    with lb.Basis(4) as B:
        N = 4
        H, L, g = wl.ladder_model(N, 3)
        l = B.expand(torch.tensor(L, device="cuda"))
        nz = torch.nonzero(l.abs() > 0).flatten()
        csr = lb.System(B, None, H=H, channels=[(g, nz.cpu().numpy(), l[nz].cpu().numpy())], format="csr")
        with pytest.raises(lb.LBError) as e:
            csr.spectrum()
        assert e.value.code == lb.native.LB_EINVAL
        csr.close()

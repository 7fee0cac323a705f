"""The seeded input recipe (CPU only): exact Hermiticity and normalisation of
the random-Lindbladian inputs (the host-buffer assembly reads only the upper
triangle of a, and K's diagonal rows use a = a^dagger), the GUE second moment,
the ladder model's operators, and the batch / serving draws."""
import numpy as np
import pytest

import workloads as wl


@pytest.mark.parametrize("N", [3, 6, 10])
def test_wishart_is_exactly_hermitian_psd_unit_trace(N):
    a = wl.wishart_kossakowski(N, 100 + N)
    M = N * N - 1
    assert a.shape == (M, M) and a.dtype == np.complex128
    assert np.array_equal(a, a.conj().T)  # bit for bit
    assert abs(np.trace(a).real - 1.0) < 1e-13
    assert np.linalg.eigvalsh(a).min() > -1e-15
    assert np.array_equal(a, wl.wishart_kossakowski(N, 100 + N))  # seeded
    assert not np.array_equal(a, wl.wishart_kossakowski(N, 101 + N))
    assert np.allclose(wl.wishart_kossakowski(N, 100 + N, scale=N), N * a, rtol=1e-14, atol=0)


def test_gue_hermitian_and_second_moment():
    H = wl.gue_hamiltonian(400, 5)
    assert np.array_equal(H, H.conj().T)
    off = H[np.triu_indices(400, 1)]
    assert abs(np.mean(np.abs(off) ** 2) - 1.0) < 0.02   # E|H_ij|^2 = 1
    d = np.diag(H)
    assert np.abs(d.imag).max() == 0.0
    assert abs(np.var(d.real) - 1.0) < 0.15             # H_ii ~ N(0, 1)


def test_ladder_model_operators():
    N = 9
    H, L, gamma = wl.ladder_model(N, 3)
    assert gamma == 0.1
    assert np.array_equal(H, H.conj().T) and np.abs(H.imag).max() == 0.0
    assert np.all(np.abs(np.diag(H).real) <= 1.0)
    assert np.array_equal(np.diag(H, 1), np.ones(N - 1)) and np.array_equal(np.diag(H, -1), np.ones(N - 1))
    assert np.count_nonzero(H) == N + 2 * (N - 1)
    # L = sum_n sqrt(n) |n-1><n|: the lowering operator, traceless
    assert np.allclose(np.diag(L, 1), np.sqrt(np.arange(1, N))) and np.count_nonzero(L) == N - 1
    assert np.trace(L) == 0


def test_batch_and_serving_draws():
    Ns = wl.batch_sizes(5000, 7)
    assert Ns.min() == 4 and Ns.max() == 40 and abs(Ns.mean() - 22.0) < 0.5
    t, NN = wl.serving_trace(4000, 8, rate=2.0)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.5) < 0.03           # Poisson gaps, mean 1 / rate
    assert set(np.unique(NN)) == {20, 50, 100, 150, 200}
    rho = wl.pure_state(5, 2)
    assert rho[2, 2] == 1.0 and np.count_nonzero(rho) == 1

"""Pins for the oracle's Q, K, R (Eqs. (07)-(09)) and RK4 (CPU only).

Independent references: brute-force traces of the literal Lindbladian (O1),
the matrix-unit superoperator (O2), textbook Bloch equations for N = 2,
the completeness relation of an orthonormal operator basis (a = gamma 1),
the exact propagator (expm), the exact death process of the ladder model.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import Oracle, brute, rk4_dense, superop


def _random_case(N, seed):
    H = wl.gue_hamiltonian(N, seed)
    a = wl.wishart_kossakowski(N, seed + 1)
    return H, a


def _oracle_system(o, H, a):
    h, _ = o.expand(H)
    Q = o.Q(h.real)
    K = o.K(a)
    R = o.R(a)
    return Q, R, K


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_equals_brute_force(N):
    H, a = _random_case(N, 100 + N)
    Qb, Rb, Kb = brute.split_generator(N, H, a)
    with Oracle(N) as o:
        Q, R, K = _oracle_system(o, H, a)
        Rr, Ri = o.R(a, return_imag=True)
        Kr, Ki = o.K(a, return_imag=True)
    assert np.abs(Q - Qb).max() < 1e-13
    assert np.abs(R - Rb).max() < 1e-14
    assert np.abs(K - Kb).max() < 1e-14
    assert np.abs(Ri).max() < 1e-15 and np.abs(Ki).max() < 1e-15


@pytest.mark.parametrize("N", [2, 3, 6, 8])
def test_equals_superoperator_route(N):
    H, a = _random_case(N, 200 + N)
    Qs, Rs, Ks, imag = superop.generator(N, H, a)
    assert imag < 1e-13
    with Oracle(N) as o:
        Q, R, K = _oracle_system(o, H, a)
    scale = max(1.0, np.abs(Rs).max())
    assert np.abs(Q - Qs).max() < 1e-12 * max(1.0, np.abs(Qs).max())
    assert np.abs(R - Rs).max() < 1e-13 * scale
    assert np.abs(K - Ks).max() < 1e-13 * scale


def test_q_antisymmetric_and_k_r_real():
    N = 7
    H, a = _random_case(N, 7)
    with Oracle(N) as o:
        h, a0 = o.expand(H)
        assert np.abs(h.imag).max() < 1e-14          # Hermitian H -> real h (Eq. (02))
        Q = o.Q(h.real)
        assert np.abs(Q + Q.T).max() < 1e-14 * np.abs(Q).max()   # up to summation order
        _, Ri = o.R(a, return_imag=True)
        _, Ki = o.K(a, return_imag=True)
    assert np.abs(Ri).max() < 1e-15 and np.abs(Ki).max() < 1e-15


@pytest.mark.parametrize("N", [3, 6, 9])
def test_k_diagonal_rows_closed_form(N):
    """Eq. (08) on the diagonal rows: the only nonzero f_{j k D_nu} with pair
    j, k are f(S_xy, J_xy, D_nu) = delta_x(nu) - delta_y(nu) = -f(J_xy, S_xy,
    D_nu), so for Hermitian a, K_{D_nu} = -(1/N) sum_k delta_k(nu) G_k with
    G_k = sum_{y>k} g_ky - sum_{x<k} g_xk and g_xy = 2 Im a_{S_xy, J_xy}; the
    diagonal elements delta_k(nu) of D_nu come from the basis matrices."""
    _, a = _random_case(N, 900 + N)
    M, P = N * N - 1, N * (N - 1) // 2
    pairs = [(x, y) for x in range(N) for y in range(x + 1, N)]
    G = np.zeros(N)
    for p_, (x, y) in enumerate(pairs):
        g = 2.0 * a[p_, P + p_].imag
        G[x] += g
        G[y] -= g
    with Oracle(N) as o:
        K = o.K(a)
        for nu in range(1, N):
            delta = np.diag(o.basis_matrix(2 * P + nu - 1)).real
            ref = -(delta @ G) / N
            assert abs(K[2 * P + nu - 1] - ref) <= 1e-14 * max(np.abs(K).max(), 1e-300)


def test_n2_bloch_precession():
    """H = (w/2) sigma_z: d<sx>/dt = -w <sy>, d<sy>/dt = w <sx>."""
    w = 1.7
    H = np.diag([w / 2, -w / 2]).astype(complex)
    with Oracle(2) as o:
        h, _ = o.expand(H)
        Q = o.Q(h.real)
    assert np.allclose(Q, [[0, -w, 0], [w, 0, 0], [0, 0, 0]], atol=1e-15)


def test_n2_amplitude_damping():
    """L = sqrt(gamma) |0><1|: rho_11' = -gamma rho_11, rho_01' = -gamma/2 rho_01.
    In Bloch components (S, J, D) = (<sx>, <sy>, <sz>)/sqrt 2:
    R = diag(-g/2, -g/2, -g), K = (0, 0, g/sqrt 2)."""
    g = 0.37
    L = np.array([[0, 1], [0, 0]], complex)
    with Oracle(2) as o:
        l, l0 = o.expand(L)
        assert abs(l0) < 1e-15
        a = g * np.outer(l, l.conj())
        R = o.R(a)
        K = o.K(a)
        Rl, mask = o.R_lowrank([g], [(np.arange(3), l)])
    assert np.allclose(R, np.diag([-g / 2, -g / 2, -g]), atol=1e-15)
    assert np.allclose(K, [0, 0, g / math.sqrt(2)], atol=1e-15)
    assert np.allclose(Rl, R, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_identity_kossakowski(N):
    """a = gamma 1: sum_j F_j X F_j = Tr(X) 1 - X/N gives L_D(X) = gamma(Tr X 1 - N X),
    so R = -gamma N 1 and K = 0."""
    g = 0.3
    M = N * N - 1
    with Oracle(N) as o:
        R = o.R(g * np.eye(M))
        K = o.K(g * np.eye(M))
    assert np.allclose(R, -g * N * np.eye(M), atol=1e-14)
    assert np.abs(K).max() < 1e-15


@pytest.mark.parametrize("N", [4, 9])
def test_entrywise_matches_full(N):
    H, a = _random_case(N, 300 + N)
    with Oracle(N) as o:
        R, S = o.R(a, return_scale=True)
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        g = np.random.default_rng(1)
        s = g.integers(0, o.M, 300)
        n = g.integers(0, o.M, 300)
        Re, Rim, Se = o.R_entries(a, s, n)
        Qe = o.Q_entries(h.real, s, n)
    assert np.abs(Re - R[s, n]).max() < 1e-15
    assert np.abs(Se - S[s, n]).max() < 1e-14
    assert np.abs(Rim).max() < 1e-15
    assert np.abs(Qe - Q[s, n]).max() == 0


def test_lowrank_equals_dense():
    N = 6
    H, L, g = wl.ladder_model(N, 5)
    with Oracle(N) as o:
        l, _ = o.expand(L)
        nz = np.nonzero(np.abs(l) > 0)[0]
        a = g * np.outer(l, l.conj())
        Rd = o.R(a)
        Rl, mask = o.R_lowrank([g], [(nz, l[nz])])
    assert np.abs(Rd - Rl).max() < 1e-15
    assert np.all(mask[np.abs(Rd) > 1e-14])


def _exact(A, K, v0, t):
    """exp of the augmented generator [[A, K], [0, 0]] applied to (v0, 1)."""
    M = len(v0)
    B = np.zeros((M + 1, M + 1))
    B[:M, :M] = A
    B[:M, M] = K
    x = scipy.linalg.expm(B * t) @ np.concatenate([v0, [1.0]])
    return x[:M]


def test_rk4_fourth_order_against_expm():
    N = 4
    H, a = _random_case(N, 11)
    with Oracle(N) as o:
        Q, R, K = _oracle_system(o, H, a)
        rho0 = wl.pure_state(N, 0)
        v0 = o.expand(rho0)[0].real
    A = Q + R
    T = 1.0
    ref = _exact(A, K, v0, T)
    errs = []
    for steps in (40, 80, 160):
        v, _ = rk4_dense(A, K, v0, T / steps, steps)
        errs.append(np.abs(v - ref).max())
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14


def test_rk4_trace_positivity_steady_state():
    N = 5
    H, a = _random_case(N, 21)
    with Oracle(N) as o:
        Q, R, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 2))[0].real
        A = Q + R
        v, snaps = rk4_dense(A, K, v0, 1e-2, 400, snap_every=100)
        for vv in snaps:
            rho = o.rho(vv)
            assert abs(np.trace(rho) - 1) < 1e-14
            assert np.allclose(rho, rho.conj().T, atol=1e-15)
            assert np.linalg.eigvalsh(rho).min() > -1e-10
        vs = np.linalg.solve(A, -K)             # steady state (Q+R) v* = -K
        rho = o.rho(vs)
        assert abs(np.trace(rho) - 1) < 1e-13
        assert np.linalg.eigvalsh(rho).min() > -1e-10


def test_unitary_norm_conserved():
    N = 4
    H, _ = _random_case(N, 31)
    with Oracle(N) as o:
        h, _ = o.expand(H)
        Q = o.Q(h.real)
        v0 = o.expand(wl.pure_state(N, 1))[0].real
    v, _ = rk4_dense(Q, np.zeros(len(v0)), v0, 1e-3, 2000)
    assert abs(np.linalg.norm(v) - np.linalg.norm(v0)) < 1e-10


def test_ladder_death_process():
    """H diagonal: populations follow p_n(t) = C(n0,n) e^{-g n t}(1-e^{-g t})^{n0-n}."""
    N = 6
    H, L, g = wl.ladder_model(N, 3)
    H = np.diag(np.diag(H))
    n0 = N - 1
    with Oracle(N) as o:
        h, _ = o.expand(H)
        l, _ = o.expand(L)
        a = g * np.outer(l, l.conj())
        A = o.Q(h.real) + o.R(a)
        K = o.K(a)
        v0 = o.expand(wl.pure_state(N, n0))[0].real
        T = 3.0
        v, _ = rk4_dense(A, K, v0, 1e-3, 3000)
        p = np.diag(o.rho(v)).real
    e = math.exp(-g * T)
    ref = np.array([math.comb(n0, n) * e**n * (1 - e) ** (n0 - n) for n in range(N)])
    assert np.abs(p - ref).max() < 1e-11


def test_entries_from_rows_match_full():
    N = 8
    H, a = _random_case(N, 808)
    with Oracle(N) as o:
        R, S = o.R(a, return_scale=True)
        g = np.random.default_rng(2)
        s = np.repeat([0, 5, o.P + 3, o.M - 1], 20)
        n = g.integers(0, o.M, len(s))
        rows = o.rows_needed(s)
        assert len(rows) < o.M
        out, sc = o.R_entries_rows(rows, a[rows], s, n)
        with pytest.raises(ValueError):
            o.R_entries_rows(rows[1:], a[rows[1:]], s, n)
    assert np.abs(out - R[s, n]).max() < 1e-15
    assert np.abs(sc - S[s, n]).max() < 1e-14


def _dense_from_csr(rowptr, col, val, M):
    D = np.zeros((M, M))
    mask = np.zeros((M, M), bool)
    for s in range(M):
        D[s, col[rowptr[s]:rowptr[s + 1]]] = val[rowptr[s]:rowptr[s + 1]]
        mask[s, col[rowptr[s]:rowptr[s + 1]]] = True
    return D, mask


@pytest.mark.parametrize("N", [3, 5, 8])
def test_lowrank_csr_equals_dense(N):
    """Sparse generator of the ladder model equals the dense Q + R; its pattern
    holds every entry that is nonzero beyond rounding and nothing else."""
    from oracle import lowrank_csr
    H, L, g = wl.ladder_model(N, 40 + N)
    with Oracle(N) as o:
        h, _ = o.expand(H)
        l, _ = o.expand(L)
        nz = np.nonzero(np.abs(l) > 0)[0]
        rp, col, val, K = lowrank_csr(o, h.real, [g], [(nz, l[nz])])
        a = g * np.outer(l, l.conj())
        A = o.Q(h.real) + o.R(a)
        Rl, mask_r = o.R_lowrank([g], [(nz, l[nz])])
        Kd = o.K(a)
    D, mask = _dense_from_csr(rp, col, val, o.M)
    assert np.abs(D - A).max() < 1e-14
    assert np.abs(K - Kd).max() < 1e-15
    assert np.array_equal(mask, np.abs(A) > 1e-13)   # no value here is near the cut
    assert np.all(np.diff(rp) >= 0)
    for s in range(o.M):                       # sorted, unique columns
        c = col[rp[s]:rp[s + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("N", list(range(6, 15)))
def test_ladder_pattern_counts(N):
    """nnz of Q + R for the ladder model (tridiagonal H): 7N^2 - 11N + 1."""
    from oracle import lowrank_csr
    H, L, g = wl.ladder_model(N, 7)
    with Oracle(N) as o:
        h, _ = o.expand(H)
        l, _ = o.expand(L)
        nz = np.nonzero(np.abs(l) > 0)[0]
        rp, col, val, K = lowrank_csr(o, h.real, [g], [(nz, l[nz])])
    assert rp[-1] == 7 * N * N - 11 * N + 1


def _csr_from_dense(A):
    """CSR arrays of the nonzero entries of a dense matrix (columns sorted)."""
    M = A.shape[0]
    rowptr = np.zeros(M + 1, np.int64)
    cols, vals = [], []
    for s in range(M):
        nz = np.nonzero(A[s])[0]
        rowptr[s + 1] = rowptr[s] + len(nz)
        cols.append(nz)
        vals.append(A[s, nz])
    return rowptr, np.concatenate(cols).astype(np.int32), np.concatenate(vals)


def test_rk4_csr_fourth_order_against_expm():
    """The CSR RK4 of the oracle converges to the exact affine propagator at
    order 4 (Sec. 4 item 3, classical RK4): a wrong stage weight or a dropped
    K lowers the order or leaves an O(1) error.  The system is a random
    Lindbladian with its zero entries removed (so K != 0 enters every stage)."""
    from oracle import rk4_csr
    N = 4
    H, a = _random_case(N, 13)
    with Oracle(N) as o:
        Q, R, K = _oracle_system(o, H, a)
        v0 = o.expand(wl.pure_state(N, 1))[0].real
    A = Q + R
    A[np.abs(A) < 1e-3 * np.abs(A).max()] = 0.0   # a genuinely sparse pattern
    assert np.abs(K).max() > 1e-3
    rp, col, val = _csr_from_dense(A)
    assert rp[-1] < A.size
    T = 1.0
    ref = _exact(A, K, v0, T)
    errs = []
    for steps in (40, 80, 160):
        v = rk4_csr(rp, col, val, K, v0, T / steps, steps)
        errs.append(np.abs(v - ref).max())
    assert errs[2] < 1e-7
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14
    # K = None means K = 0: the exact solution of v' = A v
    v = rk4_csr(rp, col, val, None, v0, T / 160, 160)
    assert np.abs(v - _exact(A, np.zeros_like(K), v0, T)).max() < 1e-7


def test_rk4_csr_ladder_death_process():
    """Ladder model with diagonal H, assembled as CSR by the oracle's sparse
    route and integrated by its CSR RK4: populations follow the exact binomial
    death process p_n(t) = C(n0,n) e^{-g n t} (1 - e^{-g t})^{n0-n}."""
    from oracle import lowrank_csr, rk4_csr
    N = 6
    H, L, g = wl.ladder_model(N, 3)
    H = np.diag(np.diag(H))
    n0 = N - 1
    with Oracle(N) as o:
        h, _ = o.expand(H)
        l, _ = o.expand(L)
        nz = np.nonzero(np.abs(l) > 0)[0]
        rp, col, val, K = lowrank_csr(o, h.real, [g], [(nz, l[nz])])
        v0 = o.expand(wl.pure_state(N, n0))[0].real
        T = 3.0
        v = rk4_csr(rp, col, val, K, v0, 1e-3, 3000)
        p = np.diag(o.rho(v)).real
    e = math.exp(-g * T)
    ref = np.array([math.comb(n0, n) * e**n * (1 - e) ** (n0 - n) for n in range(N)])
    assert np.abs(p - ref).max() < 1e-11


def test_rk4_csr_equals_rk4_dense():
    """Same system through the dense and the CSR RK4 of the oracle: the same
    sums in the same column order, so they agree to rounding."""
    from oracle import lowrank_csr, rk4_csr
    N = 6
    H, L, g = wl.ladder_model(N, 5)
    with Oracle(N) as o:
        h, _ = o.expand(H)
        l, _ = o.expand(L)
        nz = np.nonzero(np.abs(l) > 0)[0]
        rp, col, val, K = lowrank_csr(o, h.real, [g], [(nz, l[nz])])
        v0 = o.expand(wl.pure_state(N, 2))[0].real
    D, _ = _dense_from_csr(rp, col, val, len(v0))
    vd, _ = rk4_dense(D, K, v0, 1e-3, 500)
    vc = rk4_csr(rp, col, val, K, v0, 1e-3, 500)
    assert np.linalg.norm(vc - vd) <= 1e-14 * np.linalg.norm(vd)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_k_on_f_equals_k(N):
    """Eq. (08) from Im a on the pairs that f touches equals Eq. (08) from the
    full a (itself pinned by brute force above); a Hermitian a's real part
    does not enter."""
    H, a = _random_case(N, 70 + N)
    with Oracle(N) as o:
        idx, _ = o.structure("f", ordered=True)
        K = o.K(a)
        Kp = o.K_on_f(a.imag[idx[:, 0], idx[:, 1]])
        with pytest.raises(ValueError):
            o.K_on_f(np.zeros(3))
    assert np.abs(Kp - K).max() <= 1e-15 * max(np.abs(K).max(), 1.0)


def _dimer_system(o, N):
    H0, H1, L, rate, eps = wl.dimer_model(N)
    h0, _ = o.expand(H0)
    h1, _ = o.expand(H1)
    l, _ = o.expand(L)
    a = rate * np.outer(l, l.conj())
    A0 = o.Q(h0.real) + o.R(a)
    Q1 = o.Q(h1.real)
    K = o.K(a)
    return A0, Q1, K, eps


def _exact_piecewise(A0, Q1, K, v0, eps, T, t_end):
    """Exact solution of dv/dt = (A0 + eps(t) Q1) v + K for eps = eps[0] on
    [0, T/2) and eps[1] on [T/2, T) of each period: the affine propagators
    exp of the augmented matrix, segment by segment."""
    M = len(v0)
    x = np.concatenate([v0, [1.0]])
    t = 0.0
    while t < t_end - 1e-12:
        u = t % T
        k, end = (0, t - u + T / 2) if u < T / 2 - 1e-12 else (1, t - u + T)
        d = min(end, t_end) - t
        B = np.zeros((M + 1, M + 1))
        B[:M, :M] = A0 + eps[k] * Q1
        B[:M, M] = K
        x = scipy.linalg.expm(B * d) @ x
        t += d
    return x[:M]


def test_rk4_td_fourth_order_against_piecewise_exact():
    """The time-dependent RK4 of the oracle (Q(t) = Q0 + eps(t) Q1, each
    stage at its own time) on the rocked dimer (Sec. 3, Eqs. (10)-(11))
    converges at order 4 to the exact piecewise-affine propagation over one
    period, the switch of eps at T/2 falling on a step boundary."""
    from oracle import rk4_dense_td
    N = 4
    T = 2.0 * math.pi
    with Oracle(N) as o:
        A0, Q1, K, eps = _dimer_system(o, N)
        v0 = o.expand(wl.pure_state(N, 0))[0].real
    ref = _exact_piecewise(A0, Q1, K, v0, eps, T, T)
    errs = []
    for steps in (400, 800, 1600):
        v = rk4_dense_td(A0, Q1, K, v0, T / steps, steps, [0.0, T / 2], list(eps), T)
        errs.append(np.abs(v - ref).max())
    assert errs[2] < 1e-7
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14, errs


def test_rk4_td_constant_eps_is_rk4():
    """With eps constant the time-dependent RK4 is the autonomous RK4 of
    A0 + eps Q1 (same sums, same order)."""
    from oracle import rk4_dense_td
    N = 5
    with Oracle(N) as o:
        A0, Q1, K, eps = _dimer_system(o, N)
        v0 = o.expand(wl.pure_state(N, 2))[0].real
    v_td = rk4_dense_td(A0, Q1, K, v0, 1e-3, 500, [0.0], [0.7], 1.0)
    v, _ = rk4_dense(A0 + 0.7 * Q1, K, v0, 1e-3, 500)
    assert np.abs(v_td - v).max() <= 1e-15 * np.abs(v).max()


def test_dimer_trajectory_is_a_density_matrix():
    """Over one period of the rocked dimer the trace stays 1 and rho stays
    Hermitian and positive semidefinite (within 1e-10)."""
    from oracle import rk4_dense_td
    N = 6
    T = 2.0 * math.pi
    with Oracle(N) as o:
        A0, Q1, K, eps = _dimer_system(o, N)
        v = o.expand(wl.pure_state(N, N - 1))[0].real
        for k in range(4):  # quarter periods
            v = rk4_dense_td(A0, Q1, K, v, T / 4000, 1000, [0.0, T / 2], list(eps), T, t0=k * T / 4)
            rho = o.rho(v)
            assert abs(np.trace(rho) - 1) < 1e-13
            assert np.allclose(rho, rho.conj().T, atol=1e-15)
            assert np.linalg.eigvalsh(rho).min() > -1e-10

"""Pins for the oracle's basis and structure constants (CPU only).

Each check rests on something other than the oracle's own code: textbook
Gell-Mann matrices and su(3) constants (golden files), orthonormality
(Sec. 2), Lie-algebra identities (antisymmetry, Jacobi, Casimir sums),
brute-force traces, and nonzero counts derived by combinatorics.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import Oracle, brute


def _read_gellmann(golden_dir):
    lam = np.zeros((8, 3, 3), complex)
    for line in open(os.path.join(golden_dir, "gellmann_su3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, r, c, re, im = line.split()
        lam[int(a) - 1, int(r), int(c)] = float(re) + 1j * float(im)
    return lam


# Gell-Mann label (1-based) -> basis index in the order S(01,02,12), J(01,02,12), D1, D2
GM_TO_OURS = {1: 0, 2: 3, 3: 6, 4: 1, 5: 4, 6: 2, 7: 5, 8: 7}


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7])
def test_orthonormal_hermitian_traceless(N):
    with Oracle(N) as o:
        F = [o.basis_matrix(i) for i in range(o.M)]
    G = np.array([[np.trace(a @ b.conj().T) for b in F] for a in F])
    assert np.allclose(G, np.eye(len(F)), atol=1e-14)
    for X in F:
        assert np.allclose(X, X.conj().T, atol=0)
        assert abs(np.trace(X)) < 1e-14


def test_n2_is_pauli_over_sqrt2():
    sx = np.array([[0, 1], [1, 0]], complex)
    sy = np.array([[0, -1j], [1j, 0]])
    sz = np.array([[1, 0], [0, -1]], complex)
    with Oracle(2) as o:
        F = [o.basis_matrix(i) for i in range(3)]
    for X, P in zip(F, [sx, sy, sz]):
        assert np.allclose(X, P / np.sqrt(2), atol=1e-15)


def test_n3_is_gellmann_over_sqrt2(golden_dir):
    lam = _read_gellmann(golden_dir)
    with Oracle(3) as o:
        for a in range(1, 9):
            assert np.allclose(o.basis_matrix(GM_TO_OURS[a]), lam[a - 1] / np.sqrt(2), atol=1e-15)


def test_n3_structure_constants_match_textbook(golden_dir):
    """Paper's f, d (Eq. (05)) = sqrt(2) x textbook su(3) constants."""
    fT = np.zeros((8, 8, 8))
    dT = np.zeros((8, 8, 8))
    for line in open(os.path.join(golden_dir, "su3_structure_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, a, b, c, v = line.split()
        a, b, c = GM_TO_OURS[int(a)], GM_TO_OURS[int(b)], GM_TO_OURS[int(c)]
        for p in itertools.permutations((0, 1, 2)):
            idx = tuple((a, b, c)[q] for q in p)
            if kind == "f":
                sign = 1 if p in [(0, 1, 2), (1, 2, 0), (2, 0, 1)] else -1
                fT[idx] = sign * float(v)
            else:
                dT[idx] = float(v)
    with Oracle(3) as o:
        f = o.dense_structure("f")
        d = o.dense_structure("d")
    assert np.allclose(f, np.sqrt(2) * fT, atol=1e-14)
    assert np.allclose(d, np.sqrt(2) * dT, atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_structure_constants_equal_brute_force_traces(N):
    fb, db = brute.structure_constants(N)
    with Oracle(N) as o:
        f = o.dense_structure("f")
        d = o.dense_structure("d")
    assert np.abs(f - fb).max() < 1e-14
    assert np.abs(d - db).max() < 1e-14
    # nothing above the threshold was dropped
    thr = 1e-12 * max(np.abs(fb).max(), 1e-300)
    assert (np.abs(fb) > thr).sum() == (f != 0).sum()
    thr = 1e-12 * max(np.abs(db).max(), 1e-300)
    assert (np.abs(db) > thr).sum() == (d != 0).sum()


@pytest.mark.parametrize("N", [3, 4, 5])
def test_symmetries_jacobi_casimir(N):
    with Oracle(N) as o:
        f = o.dense_structure("f")
        d = o.dense_structure("d")
    for p in itertools.permutations((0, 1, 2)):
        sign = 1 if p in [(0, 1, 2), (1, 2, 0), (2, 0, 1)] else -1
        assert np.allclose(np.transpose(f, p), sign * f, atol=0)
        assert np.allclose(np.transpose(d, p), d, atol=0)
    # Jacobi: sum_e f_abe f_ecg + f_bce f_eag + f_cae f_ebg = 0
    J = (np.einsum("abe,ecg->abcg", f, f) + np.einsum("bce,eag->abcg", f, f)
         + np.einsum("cae,ebg->abcg", f, f))
    assert np.abs(J).max() < 1e-13
    # Casimir sums: textbook sum f f = N delta, sum d d = (N^2-4)/N delta; x2 here
    M = N * N - 1
    assert np.allclose(np.einsum("mns,mnt->st", f, f), 2 * N * np.eye(M), atol=1e-12)
    assert np.allclose(np.einsum("mns,mnt->st", d, d), 2 * (N * N - 4) / N * np.eye(M), atol=1e-12)
    # {F_m, F_n} = (2/N) delta_mn 1 + sum_s d_mns F_s (checks the anticommutator reading)
    with Oracle(N) as o:
        F = np.array([o.basis_matrix(i) for i in range(M)])
    for m, n in [(0, 0), (1, M - 1), (M - 1, M - 1), (2, 3)]:
        lhs = F[m] @ F[n] + F[n] @ F[m]
        rhs = (2.0 / N) * (m == n) * np.eye(N) + np.einsum("s,sab->ab", d[m, n], F)
        assert np.allclose(lhs, rhs, atol=1e-13)


def _count_by_combinatorics(N):
    """Ordered nonzero counts of f and d from the SU(N) multiplication rules:
    triangles of three distinct index pairs (4 of the 8 S/J type patterns
    give f, the other 4 give d), a pair with a diagonal generator, and three
    diagonal generators (the diagonal entries of D_l are
    1/sqrt(l(l+1)) below l, -l/sqrt(l(l+1)) at l, 0 above)."""
    tri = math.comb(N, 3)

    def dl(k, l):
        c = 1.0 / math.sqrt(l * (l + 1))
        return c if k < l else (-l * c if k == l else 0.0)

    nf = 24 * tri
    nd = 24 * tri
    for a in range(N):
        for b in range(a + 1, N):
            for l in range(1, N):
                if abs(dl(a, l) - dl(b, l)) > 1e-12:   # f(S_ab, J_ab, D_l)
                    nf += 6
                if abs(dl(a, l) + dl(b, l)) > 1e-12:   # d(S_ab,S_ab,D_l), d(J_ab,J_ab,D_l)
                    nd += 2 * 3
    for l, m, n in itertools.product(range(1, N), repeat=3):
        v = 2 * sum(dl(k, l) * dl(k, m) * dl(k, n) for k in range(N))
        if abs(v) > 1e-12:
            nd += 1
    return nf, nd


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_nonzero_counts(N):
    nf, nd = _count_by_combinatorics(N)
    with Oracle(N) as o:
        assert o.nnz("f", ordered=True) == nf
        assert o.nnz("d", ordered=True) == nd
    # closed forms of the same counts
    assert nf == 5 * N**3 - 9 * N**2 - 2 * N + 6
    assert 2 * nd == 12 * N**3 - 21 * N**2 - 7 * N + 2


def test_canonical_export_sorted_and_consistent():
    with Oracle(6) as o:
        for w in "fd":
            idx, val = o.structure(w)
            assert np.all(idx[:, 0] <= idx[:, 1]) and np.all(idx[:, 1] <= idx[:, 2])
            key = (idx[:, 0].astype(np.int64) * o.M + idx[:, 1]) * o.M + idx[:, 2]
            assert np.all(np.diff(key) > 0)
            T = o.dense_structure(w)
            assert np.array_equal(T[idx[:, 0], idx[:, 1], idx[:, 2]], val)
            assert (val != 0).all()


def test_join_term_count_n10():
    """W(10) = 376,508 join terms (sum over l of Z-section x F-section sizes)."""
    with Oracle(10) as o:
        W = o.join_terms()
        Zs = np.zeros(o.M, np.int64)
        Fs = np.zeros(o.M, np.int64)
        for w in "fd":
            idx, _ = o.structure(w, ordered=True)
            np.add.at(Zs, idx[:, 1], 1)
            if w == "f":
                np.add.at(Fs, idx[:, 1], 1)
        assert W == int((Zs * Fs).sum())
    assert W == 376508

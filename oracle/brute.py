"""O1: brute force from dense matrices (test infrastructure, tiny N).

Builds every basis matrix F_i of Sec. 2 densely, applies the Lindbladian of
Eqs. (L0)/(1) literally and takes traces:

    M_sn = Tr(F_s L(F_n)),   K_s = Tr(F_s L(1/N)),

with L(rho) = -i[H, rho] + sum_jk a_jk (F_j rho F_k - 1/2 {F_k F_j, rho})
(the dissipator of Eq. (1) with the Kossakowski matrix transposed,
a = K^T, which is the index convention of Eqs. (diss_new), (08), (09)).
Also f and d of Eq. (05) straight from their trace definitions.
"""
import numpy as np


def pairs(N):
    return [(a, b) for a in range(N) for b in range(a + 1, N)]


def basis(N):
    """List of M = N^2 - 1 dense Hermitian matrices, order S, J, D (0-based).

    D_l (l = 1..N-1) is (sum_{k<l} E_kk - l E_ll)/sqrt(l(l+1)): the Hermitian,
    orthonormal reading of the printed D^l (whose factor i would make it
    anti-Hermitian and break Tr(F_n F_m) = delta_nm)."""
    F = []
    pr = pairs(N)
    for a, b in pr:
        X = np.zeros((N, N), complex)
        X[a, b] = X[b, a] = 1 / np.sqrt(2)
        F.append(X)
    for a, b in pr:
        X = np.zeros((N, N), complex)
        X[a, b] = -1j / np.sqrt(2)
        X[b, a] = 1j / np.sqrt(2)
        F.append(X)
    for l in range(1, N):
        X = np.zeros((N, N), complex)
        for k in range(l):
            X[k, k] = 1
        X[l, l] = -l
        F.append(X / np.sqrt(l * (l + 1)))
    return F


def structure_constants(N):
    """Dense f[m,n,s] and d[m,n,s] from Eq. (05) by traces."""
    F = np.array(basis(N))
    # Tr(F_s F_m F_n) for all m, n, s
    T = np.einsum("sab,mbc,nca->mns", F, F, F)
    f = (-1j * (T - np.transpose(T, (1, 0, 2)))).real
    d = (T + np.transpose(T, (1, 0, 2))).real
    return f, d


def lindbladian(N, H, a):
    """Returns a function rho -> L(rho) (dense)."""
    F = np.array(basis(N))
    H = np.asarray(H, complex)
    a = np.asarray(a, complex)
    # Gamma = sum_jk a_jk F_k F_j
    G = np.einsum("jk,kab,jbc->ac", a, F, F)

    def L(rho):
        out = -1j * (H @ rho - rho @ H)
        out += np.einsum("jk,jab,bc,kcd->ad", a, F, rho, F)
        out -= 0.5 * (G @ rho + rho @ G)
        return out

    return L


def generator(N, H, a):
    """(M_full, K_full, imag_max): M_sn = Tr(F_s L(F_n)), K_s = Tr(F_s L(1/N))."""
    F = basis(N)
    M = len(F)
    L = lindbladian(N, H, a)
    LF = [L(F[n]) for n in range(M)]
    Mm = np.array([[np.trace(F[s] @ LF[n]) for n in range(M)] for s in range(M)])
    L0 = L(np.eye(N) / N)
    K = np.array([np.trace(F[s] @ L0) for s in range(M)])
    imag = max(np.abs(Mm.imag).max(), np.abs(K.imag).max())
    return Mm.real, K.real, imag


def split_generator(N, H, a):
    """Q (H only), R (a only), K -- each by brute force."""
    M = N * N - 1
    Q, _, _ = generator(N, H, np.zeros((M, M)))
    R, K, _ = generator(N, np.zeros((N, N)), a)
    return Q, R, K

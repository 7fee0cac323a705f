"""O2: the generator from the superoperator in the matrix-unit basis.

Test infrastructure.  Independent of the structure constants f and d: the
Lindbladian of Eqs. (L0)/(1) is written as an N^2 x N^2 matrix acting on
row-major vec(rho), using vec(A X B) = (A kron B^T) vec(X):

    L_H = -i (H kron 1 - 1 kron H^T)
    L_D = S - 1/2 (Gamma kron 1 + 1 kron Gamma^T),
    S[(p,q),(r,t)] = sum_jk a_jk (F_j)_pr (F_k)_tq    (reshuffled T a T^T)
    Gamma = sum_jk a_jk F_k F_j

and projected onto the SU(N) basis with T (columns vec(F_j)):
M = T^dagger L T, K = T^dagger L vec(1)/N, since Tr(F_s Y) = vec(F_s)^dagger vec(Y)
for Hermitian F_s.
"""
import numpy as np

from .brute import basis


def change_of_basis(N):
    """T: N^2 x M, column j = row-major vec(F_j)."""
    F = basis(N)
    return np.stack([X.reshape(-1) for X in F], axis=1)


def superoperator(N, H, a):
    T = change_of_basis(N)
    F = np.array(basis(N))
    I = np.eye(N)
    H = np.asarray(H, complex)
    a = np.asarray(a, complex)
    LH = -1j * (np.kron(H, I) - np.kron(I, H.T))
    Sp = T @ a @ T.T                                   # [(p,r),(t,q)]
    S = Sp.reshape(N, N, N, N).transpose(0, 3, 1, 2).reshape(N * N, N * N)  # [(p,q),(r,t)]
    G = np.einsum("jk,kab,jbc->ac", a, F, F)
    LD = S - 0.5 * (np.kron(G, I) + np.kron(I, G.T))
    return LH, LD, T


def generator(N, H, a):
    """(Q, R, K) from the superoperator route."""
    LH, LD, T = superoperator(N, H, a)
    Td = T.conj().T
    Q = Td @ LH @ T
    R = Td @ LD @ T
    K = Td @ LD @ (np.eye(N).reshape(-1) / N)
    return Q.real, R.real, K.real, max(abs(Q.imag).max(), abs(R.imag).max(), abs(K.imag).max())

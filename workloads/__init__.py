"""Seeded synthetic inputs shaped like the paper's two test-bed models.

This module holds only input synthesis (random matrices, model operators),
none of the transformation's arithmetic, so that the oracle and the CUDA
library can both consume the identical arrays.

* Random Lindbladian (Sec. 3): Kossakowski matrix from the complex Wishart
  ensemble, a = G G^dagger / Tr(G G^dagger) with G an (N^2-1) x (N^2-1)
  complex Ginibre matrix (entries (x + i y)/sqrt 2, x, y ~ N(0,1) iid).  The
  paper normalises Tr K = N; this workload normalises Tr a = 1 (``scale``
  restores any other trace).  A GUE Hamiltonian H = (X + X^dagger)/sqrt 2
  (X Ginibre as above) is added; the paper's random model has H = 0.
* Sparse ladder model: real tridiagonal H (diagonal ~ U[-1, 1], off-diagonal
  1) and one jump operator L = sum_{n=1}^{N-1} sqrt(n) |n-1><n| at rate
  gamma = 0.1 -- a stand-in for the paper's sparse rocked-dimer model of the
  same sparsity class (P = 1, sparse H and L).
* rho0 = |n0><n0|.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(np.random.PCG64(int(seed)))


def ginibre(n, seed, m=None):
    """n x m complex Ginibre, entries (x + i y)/sqrt(2)."""
    m = n if m is None else m
    g = rng(seed)
    return (g.standard_normal((n, m)) + 1j * g.standard_normal((n, m))) / np.sqrt(2.0)


def gue_hamiltonian(N, seed):
    """H = (X + X^dagger)/sqrt 2, E|H_ij|^2 = 1, H_ii ~ N(0, 1)."""
    X = ginibre(N, seed)
    H = (X + X.conj().T) / np.sqrt(2.0)
    return np.ascontiguousarray(H)


def wishart_kossakowski(N, seed, scale=1.0):
    """Dense Hermitian PSD M x M (M = N^2 - 1), a = scale G G^dagger / Tr(G G^dagger)."""
    M = N * N - 1
    G = ginibre(M, seed)
    a = G @ G.conj().T
    a = 0.5 * (a + a.conj().T)
    a *= scale / np.trace(a).real
    return np.ascontiguousarray(a)


def wishart_kossakowski_device(N, seed, device="cuda", scale=1.0, chunk=8192):
    """Large-N variant formed on a GPU with torch (input synthesis only).

    G is drawn with torch's counter-based generator on the device; the four
    real products of G G^dagger run as TF32 tensor-core GEMMs with FP32
    output, and the result is made exactly Hermitian and normalised in FP64.
    Returns a complex128 M x M tensor on ``device``."""
    import torch
    M = N * N - 1
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    s = 1.0 / np.sqrt(2.0)
    Gr = torch.randn((M, M), generator=gen, device=device, dtype=torch.float32) * s
    Gi = torch.randn((M, M), generator=gen, device=device, dtype=torch.float32) * s
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.empty((M, M), dtype=torch.complex128, device=device)
        av = torch.view_as_real(a)
        for r0 in range(0, M, chunk):
            r1 = min(M, r0 + chunk)
            re = Gr[r0:r1] @ Gr.T
            re += Gi[r0:r1] @ Gi.T
            im = Gi[r0:r1] @ Gr.T
            im -= Gr[r0:r1] @ Gi.T
            av[r0:r1, :, 0] = re
            av[r0:r1, :, 1] = im
            del re, im
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del Gr, Gi
    # exact Hermitian: a <- (a + a^H)/2, done blockwise to bound temporaries
    for r0 in range(0, M, chunk):
        r1 = min(M, r0 + chunk)
        for c0 in range(r0, M, chunk):
            c1 = min(M, c0 + chunk)
            blk = 0.5 * (a[r0:r1, c0:c1] + a[c0:c1, r0:r1].conj().T)
            a[r0:r1, c0:c1] = blk
            a[c0:c1, r0:r1] = blk.conj().T
    tr = torch.diagonal(a).real.sum().item()
    a.mul_(scale / tr)
    torch.cuda.synchronize(device)
    return a


def random_lindbladian_device(N, seed, device="cuda"):
    """(H, a) of one random Lindbladian formed on the GPU in FP64 (moderate N):
    GUE H from the host generator, a = G G^dagger / Tr with G from torch's
    counter-based generator on the device."""
    import torch
    M = N * N - 1
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    s = 1.0 / np.sqrt(2.0)
    G = torch.complex(torch.randn((M, M), generator=gen, device=device, dtype=torch.float64) * s,
                      torch.randn((M, M), generator=gen, device=device, dtype=torch.float64) * s)
    a = G @ G.conj().T
    a = 0.5 * (a + a.conj().T)
    a = a / torch.diagonal(a).real.sum()
    H = torch.tensor(gue_hamiltonian(N, seed + 1), device=device)
    return H, a.contiguous()


def random_lindbladian_paper_device(N, seed, device="cuda"):
    """The random Lindbladian of Sec. 3 as the paper defines it: H = 0 and the
    Kossakowski matrix N G G^dagger / Tr(G G^dagger) (Tr = N), G complex
    Ginibre, formed on the GPU in FP64.  Returns a (M x M complex128)."""
    _, a = random_lindbladian_device(N, seed, device=device)
    return a * float(N)


def ladder_model(N, seed, gamma=0.1):
    """(H real tridiagonal N x N complex128, L N x N complex128, gamma)."""
    g = rng(seed)
    H = np.zeros((N, N), np.complex128)
    H[np.arange(N), np.arange(N)] = g.uniform(-1.0, 1.0, N)
    H[np.arange(N - 1), np.arange(1, N)] = 1.0
    H[np.arange(1, N), np.arange(N - 1)] = 1.0
    L = np.zeros((N, N), np.complex128)
    n = np.arange(1, N)
    L[n - 1, n] = np.sqrt(n)
    return H, L, float(gamma)


def pure_state(N, n0=0):
    rho = np.zeros((N, N), np.complex128)
    rho[n0, n0] = 1.0
    return rho


def batch_sizes(count, seed, lo=4, hi=40):
    """N ~ uniform integers in [lo, hi]."""
    return rng(seed).integers(lo, hi + 1, size=count)


def serving_trace(count, seed, rate, Ns=(20, 50, 100, 150, 200)):
    """Poisson arrivals: (arrival times, N per request)."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    return np.cumsum(gaps), g.choice(np.asarray(Ns), size=count)


def dimer_model(N, J=-1.0, U=2.2, E=-1.0, A=-1.5, gamma=0.1):
    """The periodically rocked Bose-Hubbard dimer of Sec. 3 (Eqs. (10), (11))
    with N - 1 bosons: Hilbert-space dimension N, basis |n> with n bosons on
    site 1 and N - 1 - n on site 2.  Returns (H0, H1, L, rate, eps) with
    H(t) = H0 + eps(t) H1, H0 = -J (b1^+ b2 + b1 b2^+) + 2U/(N-1) sum_j
    n_j (n_j - 1), H1 = n2 - n1, the jump operator L = (b1^+ + b2^+)(b1 - b2)
    (the printed L is Hermitian, which contradicts the non-Hermitian L the
    text describes; this is the operator that recycles the out-of-phase mode
    into the in-phase one), rate = gamma / (N - 1), and eps = (E + A, E - A),
    the drive on the first and second half of the period T = 2 pi
    (Theta = +1 on [0, T/2), -1 on [T/2, T))."""
    n = np.arange(N, dtype=np.float64)
    c = np.sqrt((n[:-1] + 1.0) * (N - 1.0 - n[:-1]))  # <n+1| b1^+ b2 |n>
    hop = np.zeros((N, N))
    hop[np.arange(1, N), np.arange(N - 1)] = c          # b1^+ b2
    hop = hop + hop.T                                   # + b1 b2^+
    n1, n2 = n, N - 1.0 - n
    inter = 2.0 * U / (N - 1.0) * (n1 * (n1 - 1.0) + n2 * (n2 - 1.0))
    H0 = -J * hop + np.diag(inter)
    H1 = np.diag(n2 - n1)
    # (b1^+ + b2^+)(b1 - b2) = n1 - n2 - b1^+ b2 + b2^+ b1
    L = np.diag(n1 - n2) - np.tril(hop, -1) + np.triu(hop, 1)
    return (H0.astype(np.complex128), H1.astype(np.complex128), L.astype(np.complex128),
            gamma / (N - 1.0), (E + A, E - A))

// lb_steady.cu -- FP64 checks on the device: the steady state of the real
// linear system and the physical properties of rho.
//
// Steady state (Sec. 2: dv/dt = (Q + R) v + K with rho = 1/N + sum_i v_i F_i):
// v* solves (Q + R) v* = -K.  Q + R is a dense nonsymmetric M x M matrix
// whose spectrum (that of the Lindbladian on traceless operators) lies in
// the left half plane, far from the real axis when H is large; it is solved
// by restarted GMRES(m) in FP64: this file's row-per-warp matrix-vector
// product, the Krylov basis on the device, classical Gram-Schmidt with one
// reorthogonalisation pass (block dot products and one combined update per
// pass), and the small Hessenberg least-squares problem with Givens
// rotations on the host.
//
// Preconditioner (optional): the Hamiltonian part Q acts on rho as
// -i[H, rho], diagonal in the eigenbasis of H with -i(E_j - E_k); the
// dissipator of a random Lindbladian shifts the spectrum by about
// -sigma = Tr(A)/M (Tr Q = 0) with little spread.  P = Q - sigma 1 is
// therefore close to A, and P^-1 x is: rho(x) = sum_i x_i F_i, Y = U^dag
// rho U, Y_jk / (-i(E_j - E_k) - sigma), U Y U^dag, back to coordinates.
// GMRES runs on A P^-1 (right preconditioning, so the residual it
// minimises is that of A v = -K itself).
//
// rho checks (Eq. (rho)): from v, rho is rebuilt on the device and reduced
// to Tr rho - 1 and max |rho_jk - conj(rho_kj)|, and a Cholesky
// factorisation of rho + delta 1 in one block gives its smallest pivot
// (positive exactly when the smallest eigenvalue of rho exceeds -delta).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lb_internal.h"

namespace {

// y = A x (FP64), one warp per row; with b: y = b - A x.
__global__ void __launch_bounds__(256) k_gemv64(int64_t M, const double* __restrict__ A, const double* __restrict__ x,
                                                const double* __restrict__ b, double* __restrict__ y) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const double* row = A + s * M;
  double a = 0.0;
  for (int64_t n = lane; n < M; n += 32) a = fma(row[n], x[n], a);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) y[s] = b ? b[s] - a : a;
}

// h[i] = sum_e V[i][e] w[e] for i < nv: one block per i, fixed-order reduction.
__global__ void __launch_bounds__(256) k_basis_dots(int64_t n, int nv, const double* __restrict__ V,
                                                    const double* __restrict__ w, double* __restrict__ h) {
  __shared__ double red[8];
  const int i = blockIdx.x;
  if (i >= nv) return;
  const double* v = V + (int64_t)i * n;
  double a = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) a = fma(v[e], w[e], a);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    h[i] = s;
  }
}

// w[e] += sign * sum_{i < nv} c[i] V[i][e]
__global__ void k_basis_combo(int64_t n, int nv, const double* __restrict__ V, const double* __restrict__ c,
                              double sign, double* __restrict__ w) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(c[i], V[(int64_t)i * n + e], a);
    w[e] = fma(sign, a, w[e]);
  }
}

// y = x * s
__global__ void k_scale(int64_t n, const double* __restrict__ x, double s, double* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = x[e] * s;
}

// Tr rho - 1 and max |rho_jk - conj(rho_kj)| of one N x N complex rho, by
// one block (fixed-order reduction).
__global__ void __launch_bounds__(256) k_rho_trace_herm(int N, const double2* __restrict__ rho,
                                                        double* __restrict__ out) {
  __shared__ double st[8], sh[8];
  double tr = 0.0, her = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)N * N; e += blockDim.x) {
    const int j = (int)(e / N), k = (int)(e % N);
    const double2 a = rho[e], b = rho[(int64_t)k * N + j];
    if (j == k) tr += a.x;
    her = fmax(her, hypot(a.x - b.x, a.y + b.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    her = fmax(her, __shfl_xor_sync(0xffffffffu, her, o));
  }
  if ((threadIdx.x & 31) == 0) {
    st[threadIdx.x >> 5] = tr;
    sh[threadIdx.x >> 5] = her;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, h = 0.0;
    for (int w = 0; w < 8; ++w) {
      t += st[w];
      h = fmax(h, sh[w]);
    }
    out[0] = t - 1.0;
    out[1] = h;
  }
}

// Cholesky of the Hermitian matrix C = rho + delta 1 (lower triangle, in
// place, one block): out[2] = the smallest pivot d_k met (the first
// non-positive one stops the factorisation; positive for every k exactly
// when C is positive definite).
__global__ void __launch_bounds__(256) k_cholesky_pivot(int N, double2* __restrict__ C, double delta,
                                                        double* __restrict__ out) {
  __shared__ double piv, minpiv;
  if (threadIdx.x == 0) minpiv = 1e300;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x == 0) {
      piv = C[(int64_t)k * N + k].x + delta;
      minpiv = fmin(minpiv, piv);
    }
    __syncthreads();
    if (!(piv > 0.0)) break;
    const double sq = sqrt(piv);
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) {
      double2& c = C[(int64_t)i * N + k];
      c.x /= sq;
      c.y /= sq;
    }
    __syncthreads();
    // trailing update of the lower triangle: C_ij -= L_ik conj(L_jk), i >= j > k
    const int m = N - k - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      if (j > i) continue;
      const double2 li = C[(int64_t)i * N + k], lj = C[(int64_t)j * N + k];
      double2& c = C[(int64_t)i * N + j];
      c.x -= li.x * lj.x + li.y * lj.y;
      c.y -= li.y * lj.x - li.x * lj.y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[2] = minpiv;
}

inline unsigned vec_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 1024); }

// C = op_a(A) op_b(B) for N x N complex row-major matrices, op in
// {0: X, 1: X^T, 2: conj(X)}; 16 x 16 tiles in shared memory.
constexpr int kCT = 16;
template <int OPA, int OPB>
__global__ void __launch_bounds__(kCT * kCT) k_cgemm(int N, const double2* __restrict__ A,
                                                     const double2* __restrict__ B, double2* __restrict__ C) {
  __shared__ double2 ta[kCT][kCT + 1], tb[kCT][kCT + 1];
  const int i = blockIdx.y * kCT + threadIdx.y, j = blockIdx.x * kCT + threadIdx.x;
  double cr = 0.0, ci = 0.0;
  for (int k0 = 0; k0 < N; k0 += kCT) {
    {  // op_a(A)[i][k0 + tx]
      const int k = k0 + threadIdx.x;
      double2 x = make_double2(0.0, 0.0);
      if (i < N && k < N) x = OPA == 1 ? A[(int64_t)k * N + i] : A[(int64_t)i * N + k];
      if (OPA == 2) x.y = -x.y;
      ta[threadIdx.y][threadIdx.x] = x;
    }
    {  // op_b(B)[k0 + ty][j]
      const int k = k0 + threadIdx.y;
      double2 x = make_double2(0.0, 0.0);
      if (k < N && j < N) x = OPB == 1 ? B[(int64_t)j * N + k] : B[(int64_t)k * N + j];
      if (OPB == 2) x.y = -x.y;
      tb[threadIdx.y][threadIdx.x] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kCT; ++k) {
      const double2 a = ta[threadIdx.y][k], b = tb[k][threadIdx.x];
      cr = fma(a.x, b.x, fma(-a.y, b.y, cr));
      ci = fma(a.x, b.y, fma(a.y, b.x, ci));
    }
    __syncthreads();
  }
  if (i < N && j < N) C[(int64_t)i * N + j] = make_double2(cr, ci);
}

// Y_jk /= (-i (E_j - E_k) - sigma)
__global__ void k_pc_divide(int N, const double* __restrict__ E, double sigma, double2* __restrict__ Y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int j = (int)(t / N), k = (int)(t % N);
  const double dr = -sigma, di = -(E[j] - E[k]);  // d = dr + i di
  const double inv = 1.0 / (dr * dr + di * di);
  const double2 y = Y[t];
  Y[t] = make_double2((y.x * dr + y.y * di) * inv, (y.y * dr - y.x * di) * inv);
}

// y += x
__global__ void k_add_to(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

// y = Re(x)
__global__ void k_real(int64_t n, const double2* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i].x;
}

// out = Tr(A) (one block, fixed-order reduction)
__global__ void __launch_bounds__(256) k_trace(int64_t M, const double* __restrict__ A, double* __restrict__ out) {
  __shared__ double red[8];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) a += A[i * M + i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    out[0] = s;
  }
}

}  // namespace

namespace lbi {

constexpr int kRestart = 1024;  // default GMRES restart length m

int restart_len(int64_t M, int restart) {
  return (int)std::min<int64_t>(restart > 0 ? restart : kRestart, M);
}

size_t steady_workspace_bytes(int64_t M, int restart) {
  const int m = restart_len(M, restart);
  return 8 * ((size_t)(m + 1) * M + 2 * (size_t)M + 2 * (m + 2) + 16);
}

// The preconditioner's part of the workspace: E (N), Ub, X, T (N x N
// complex each), coef (M complex), z (M).
static size_t pc_offset(int64_t M, int restart) { return (steady_workspace_bytes(M, restart) + 255) & ~(size_t)255; }

size_t steady_pc_workspace_bytes(int N, int64_t M, int restart) {
  const size_t nn = (size_t)N * N;
  return pc_offset(M, restart) + 8 * ((size_t)N + 1 + 6 * nn + 3 * (size_t)M + 16);
}

// z = P^-1 x with P = Q - sigma 1 (Q = -i[H, .] on traceless coordinates).
static cudaError_t apply_pc(const PcView& pc, const double* x, double* z, cudaStream_t st) {
  const int N = pc.B.N;
  const dim3 tb(kCT, kCT), tg((N + kCT - 1) / kCT, (N + kCT - 1) / kCT);
  cudaError_t e = lbi::synth(pc.B, x, pc.X, st);                       // X = sum x_i F_i
  if (e != cudaSuccess) return e;
  k_cgemm<2, 0><<<tg, tb, 0, st>>>(N, pc.Ub, pc.X, pc.T);                // T = conj(Ub) X = U^dag X
  k_cgemm<0, 1><<<tg, tb, 0, st>>>(N, pc.T, pc.Ub, pc.X);                // Y = T Ub^T = U^dag X U
  k_pc_divide<<<(unsigned)(((int64_t)N * N + 255) / 256), 256, 0, st>>>(N, pc.E, pc.sigma, pc.X);
  k_cgemm<1, 0><<<tg, tb, 0, st>>>(N, pc.Ub, pc.X, pc.T);                // T = Ub^T Y = U Y
  k_cgemm<0, 2><<<tg, tb, 0, st>>>(N, pc.T, pc.Ub, pc.X);                // Z = T conj(Ub) = U Y U^dag
  note_launch(5);
  e = lbi::expand(pc.B, pc.X, pc.coef, st);                              // Tr(F_i Z)
  if (e != cudaSuccess) return e;
  k_real<<<(unsigned)((pc.B.M + 255) / 256), 256, 0, st>>>(pc.B.M, pc.coef, z);
  note_launch(1);
  return cudaGetLastError();
}

// Set up the preconditioner for H (device, N x N complex) in the tail of
// the workspace; sigma < 0 takes -Tr(A) / M.  Status as hermitian_eig.
int steady_pc_setup(const lb::BasisView& B, const double2* H, const double* A, double sigma, int restart,
                    void* work, PcView* pc, cudaStream_t st, cudaError_t* ce) {
  const int N = B.N;
  const int64_t M = B.M;
  const size_t nn = (size_t)N * N;
  char* p = static_cast<char*>(work) + pc_offset(M, restart);  // 256-byte aligned when work is
  pc->B = B;
  pc->E = reinterpret_cast<double*>(p);
  pc->Ub = reinterpret_cast<double2*>(pc->E + N + (N & 1));
  pc->X = pc->Ub + nn;
  pc->T = pc->X + nn;
  pc->coef = pc->T + nn;
  pc->z = reinterpret_cast<double*>(pc->coef + M);
  *ce = cudaSuccess;
  if (sigma < 0.0) {
    k_trace<<<1, 256, 0, st>>>(M, A, pc->z);
    note_launch(1);
    double tr = 0.0;
    *ce = cudaMemcpyAsync(&tr, pc->z, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (*ce == cudaSuccess) *ce = cudaStreamSynchronize(st);
    if (*ce != cudaSuccess) return 3;
    sigma = -tr / (double)M;
  }
  pc->sigma = sigma > 0.0 ? sigma : 1e-300;
  return hermitian_eig(H, N, pc->E, pc->Ub, st, ce);
}

// GMRES(m) for A v = -K from the initial v; returns the relative true
// residual ||K + A v|| / ||K|| and the total inner iterations.
cudaError_t steady_state(int64_t M, const double* A, const double* K, double* v, double tol, int max_iter,
                         int restart, double* rel_res, int* iters, void* work, cudaStream_t st, const PcView* pc) {
  const int m = restart_len(M, restart);
  double* V = static_cast<double*>(work);     // (m + 1) x M Krylov basis
  double* w = V + (size_t)(m + 1) * M;       // M
  double* b = w + M;                         // M: -K
  double* dh = b + M;                        // m + 2 coefficients
  double* dy = dh + (m + 2);                 // m + 2 solution weights
  const unsigned gg = (unsigned)((M * 32 + 255) / 256), vb = vec_blocks(M);
  cudaError_t e = cudaSuccess;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 2), y(m);
  auto sync_read = [&](double* host, const double* dev, int count) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  };
  auto norm = [&](const double* x) {
    k_basis_dots<<<1, 256, 0, st>>>(M, 1, x, x, dh);
    note_launch(1);
    double r = 0.0;
    sync_read(&r, dh, 1);
    return std::sqrt(r);
  };
  k_scale<<<vb, 256, 0, st>>>(M, K, -1.0, b);
  note_launch(1);
  const double bn = norm(b);
  *iters = 0;
  *rel_res = 0.0;
  if (e != cudaSuccess) return e;
  if (bn == 0.0) {  // K = 0: v = 0 solves it
    e = cudaMemsetAsync(v, 0, 8 * (size_t)M, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  int total = 0;
  double res = 0.0;
  while (e == cudaSuccess && total < max_iter) {
    // r = b - A v in V[0], beta = ||r||
    k_gemv64<<<gg, 256, 0, st>>>(M, A, v, b, V);
    note_launch(1);
    const double beta = norm(V);
    res = beta / bn;
    if (e != cudaSuccess || res <= tol || beta == 0.0) break;
    k_scale<<<vb, 256, 0, st>>>(M, V, 1.0 / beta, V);
    note_launch(1);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < m && total < max_iter && e == cudaSuccess; ++j) {
      ++total;
      if (pc) {  // w = A P^-1 V_j
        e = apply_pc(*pc, V + (size_t)j * M, pc->z, st);
        if (e != cudaSuccess) break;
        k_gemv64<<<gg, 256, 0, st>>>(M, A, pc->z, nullptr, w);
      } else {
        k_gemv64<<<gg, 256, 0, st>>>(M, A, V + (size_t)j * M, nullptr, w);
      }
      note_launch(1);
      // classical Gram-Schmidt, twice
      for (int k = 0; k < j + 1; ++k) H[(size_t)k * m + j] = 0.0;
      for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        k_basis_dots<<<j + 1, 256, 0, st>>>(M, j + 1, V, w, dh);
        k_basis_combo<<<vb, 256, 0, st>>>(M, j + 1, V, dh, -1.0, w);
        note_launch(2);
        sync_read(h.data(), dh, j + 1);
        for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] += h[k];
      }
      const double hn = norm(w);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        k_scale<<<vb, 256, 0, st>>>(M, w, 1.0 / hn, V + (size_t)(j + 1) * M);
        note_launch(1);
      }
      // apply the previous rotations to column j, then a new one
      for (int k = 0; k < j; ++k) {
        const double a0 = H[(size_t)k * m + j], a1 = H[(size_t)(k + 1) * m + j];
        H[(size_t)k * m + j] = cs[k] * a0 + sn[k] * a1;
        H[(size_t)(k + 1) * m + j] = -sn[k] * a0 + cs[k] * a1;
      }
      const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
      const double rr = std::hypot(a0, a1);
      cs[j] = rr > 0.0 ? a0 / rr : 1.0;
      sn[j] = rr > 0.0 ? a1 / rr : 0.0;
      H[(size_t)j * m + j] = rr;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (std::fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
        ++j;
        break;
      }
    }
    if (e != cudaSuccess) break;
    // y = H[0:j, 0:j]^-1 g[0:j], v += V y
    for (int k = j - 1; k >= 0; --k) {
      double t = g[k];
      for (int q = k + 1; q < j; ++q) t -= H[(size_t)k * m + q] * y[q];
      y[k] = H[(size_t)k * m + k] != 0.0 ? t / H[(size_t)k * m + k] : 0.0;
    }
    e = cudaMemcpyAsync(dy, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && pc) {  // v += P^-1 (V y)
      e = cudaMemsetAsync(w, 0, 8 * (size_t)M, st);
      if (e == cudaSuccess) {
        k_basis_combo<<<vb, 256, 0, st>>>(M, j, V, dy, 1.0, w);
        note_launch(1);
        e = apply_pc(*pc, w, pc->z, st);
      }
      if (e == cudaSuccess) {
        k_add_to<<<vb, 256, 0, st>>>(M, pc->z, v);
        note_launch(1);
        e = cudaStreamSynchronize(st);
      }
    } else if (e == cudaSuccess) {
      k_basis_combo<<<vb, 256, 0, st>>>(M, j, V, dy, 1.0, v);
      note_launch(1);
      e = cudaStreamSynchronize(st);  // y on the host is rewritten by the next cycle
    }
  }
  *iters = total;
  // true residual ||K + A v|| / ||K||
  if (e == cudaSuccess) {
    k_gemv64<<<gg, 256, 0, st>>>(M, A, v, b, w);
    note_launch(1);
    *rel_res = norm(w) / bn;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

size_t rho_checks_workspace_bytes(int N) { return 16 * (size_t)N * N + 64; }

cudaError_t rho_checks(const lb::BasisView& B, const double* V, int64_t nsnap, double delta, double* out_host,
                       void* work, cudaStream_t st) {
  double2* rho = static_cast<double2*>(work);
  double* res = reinterpret_cast<double*>(rho + (size_t)B.N * B.N);
  cudaError_t e = cudaSuccess;
  for (int64_t k = 0; k < nsnap && e == cudaSuccess; ++k) {
    e = lbi::rho(B, V + k * B.M, rho, st);
    if (e != cudaSuccess) break;
    k_rho_trace_herm<<<1, 256, 0, st>>>(B.N, rho, res);
    k_cholesky_pivot<<<1, 256, 0, st>>>(B.N, rho, delta, res);
    note_launch(2);
    if ((e = cudaMemcpyAsync(out_host + 3 * k, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      break;
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace lbi

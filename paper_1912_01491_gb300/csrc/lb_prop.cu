// lb_prop.cu -- the propagator form of classical RK4 (Sec. 4 item 3, Table 1
// step 3.1).  For the autonomous system dv/dt = A v + K one RK4 step of size
// h is, exactly in real arithmetic,
//     v <- v + h (D' v + c'),
//     D' = A + (h/2) A (A + (h/3) A (A + (h/4) A A))   [= (P(hA) - 1)/h,
//          P(x) = 1 + x + x^2/2 + x^3/6 + x^4/24],
//     c' = K + (h/2) A (K + (h/3) A (K + (h/4) A K)),
// since the four stages are k1 = f, k2 = (1 + hA/2) f, k3 = (1 + hA/2 +
// h^2A^2/4) f, k4 = (1 + hA + h^2A^2/2 + h^3A^3/4) f with f = A v + K, and
// h/6 (k1 + 2 k2 + 2 k3 + k4) = h (1 + hA/2 + h^2A^2/6 + h^3A^3/24) f.
// D' costs three matrix products once per (A, h); afterwards a step reads
// the matrix once instead of four times, with one exchange of the state
// instead of four.
//
// This file holds the building blocks: a batched tiled GEMM with the
// epilogue Y = B + alpha A G (FP32 or FP64, one launch over the tiles of
// every matrix of a batch), and a batched FP64 GEMV y = K + alpha A x.
#include <algorithm>
#include <vector>

#include "lb_internal.h"

namespace {

constexpr int kTile = 64, kBk = 16;

// Y[i][j] = B[i][j] + alpha sum_k A[i][k] G[k][j] on one 64 x 64 tile; 256
// threads as 16 x 16, 4 x 4 outputs each; B may be null (0).
template <class T>
__global__ void __launch_bounds__(256) k_batch_gemm(const lbi::GemmTile* __restrict__ tiles,
                                                    const lbi::GemmJob<T>* __restrict__ jobs) {
  __shared__ T As[kBk][kTile + 4];  // As[k][i]
  __shared__ T Gs[kBk][kTile + 4];  // Gs[k][j]
  const lbi::GemmTile tl = tiles[blockIdx.x];
  const lbi::GemmJob<T> jb = jobs[tl.job];
  const int64_t M = jb.M;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)tl.ti * kTile, j0 = (int64_t)tl.tj * kTile;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t k0 = 0; k0 < M; k0 += kBk) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;  // 0 .. 1023
      {  // A tile: 64 rows x 16 k, read along k
        const int i = e >> 4, k = e & 15;
        const int64_t gi = i0 + i, gk = k0 + k;
        As[k][i] = (gi < M && gk < M) ? jb.A[gi * M + gk] : T(0);
      }
      {  // G tile: 16 k x 64 columns, read along j
        const int k = e >> 6, j = e & 63;
        const int64_t gk = k0 + k, gj = j0 + j;
        Gs[k][j] = (gk < M && gj < M) ? jb.G[gk * M + gj] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBk; ++k) {
      T a[4], g[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty * 4 + q];
        g[q] = Gs[k][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], g[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gi = i0 + ty * 4 + p, gj = j0 + tx * 4 + q;
      if (gi < M && gj < M) {
        const T base = jb.B ? jb.B[gi * M + gj] : T(0);
        jb.Y[gi * M + gj] = fma(jb.alpha, acc[p][q], base);
      }
    }
}

// y = K + alpha A x for every job: one block per job, one warp per row.
__global__ void __launch_bounds__(256) k_batch_gemv64(const lbi::GemvJob* __restrict__ jobs) {
  const lbi::GemvJob jb = jobs[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t s = warp; s < jb.M; s += blockDim.x >> 5) {
    double a = 0.0;
    for (int64_t n = lane; n < jb.M; n += 32) a = fma(jb.A[s * jb.M + n], jb.x[n], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) jb.y[s] = fma(jb.alpha, a, jb.K[s]);
  }
}

// Y = A + R elementwise (FP32), one grid-stride launch per job list.
__global__ void k_add32(const float* __restrict__ A, const float* __restrict__ R, float* __restrict__ Y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = A[e] + R[e];
}

__global__ void k_add64(const double* __restrict__ A, const double* __restrict__ R, double* __restrict__ Y,
                        int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = A[e] + R[e];
}

}  // namespace

namespace lbi {

template <class T>
cudaError_t batch_gemm(const std::vector<GemmJob<T>>& jobs, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (jobs.empty()) return cudaSuccess;
  std::vector<GemmTile> tiles;
  for (int j = 0; j < (int)jobs.size(); ++j) {
    const int nt = (int)((jobs[j].M + kTile - 1) / kTile);
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) tiles.push_back(GemmTile{j, a, b});
  }
  const size_t bj = sizeof(GemmJob<T>) * jobs.size(), bt = sizeof(GemmTile) * tiles.size();
  const size_t off_t = (bj + 255) & ~size_t(255);
  if (off_t + bt > scratch_bytes) return cudaErrorInvalidValue;
  char* d = static_cast<char*>(scratch);
  cudaError_t e = cudaMemcpyAsync(d, jobs.data(), bj, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + off_t, tiles.data(), bt, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  // grids above 2^31 - 1 blocks do not occur: tiles <= jobs * 4096
  k_batch_gemm<T><<<(unsigned)tiles.size(), 256, 0, st>>>(reinterpret_cast<const GemmTile*>(d + off_t),
                                                           reinterpret_cast<const GemmJob<T>*>(d));
  note_launch(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the job and tile lists must stay until the kernel has read them
  return cudaStreamSynchronize(st);
}

size_t batch_gemm_scratch_bytes(const std::vector<int64_t>& Ms) {
  size_t tiles = 0;
  for (int64_t M : Ms) {
    const size_t nt = (size_t)((M + kTile - 1) / kTile);
    tiles += nt * nt;
  }
  return ((sizeof(GemmJob<double>) * Ms.size() + 255) & ~size_t(255)) + sizeof(GemmTile) * tiles + 256;
}

cudaError_t batch_gemv64(const std::vector<GemvJob>& jobs, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (jobs.empty()) return cudaSuccess;
  const size_t bj = sizeof(GemvJob) * jobs.size();
  if (bj > scratch_bytes) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(scratch, jobs.data(), bj, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  k_batch_gemv64<<<(unsigned)jobs.size(), 256, 0, st>>>(static_cast<const GemvJob*>(scratch));
  note_launch(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t add32(const float* A, const float* R, float* Y, int64_t n, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_add32<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(A, R, Y, n);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t add64(const double* A, const double* R, double* Y, int64_t n, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_add64<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(A, R, Y, n);
  note_launch(1);
  return cudaGetLastError();
}

template cudaError_t batch_gemm<float>(const std::vector<GemmJob<float>>&, void*, size_t, cudaStream_t);
template cudaError_t batch_gemm<double>(const std::vector<GemmJob<double>>&, void*, size_t, cudaStream_t);

}  // namespace lbi

// ---------------------------------------------------------------------------
// Single system, several initial states (the columns of V): one step is
// V_r <- V_r + h (D' V_r + c' + d_r) for every state r, i.e. a product of
// D' with the block of states, read once per step for all of them.
namespace {

// One warp per row s; lanes stride the columns, each keeping RS partial sums
// (states c0 .. c0 + RS - 1 of the block of states), D' read once per row
// and pass.  X (R x M, element type T) is the state rounded to T; V (R x M,
// FP64) the state; Xn receives the next X.
template <class T, int RS>
__global__ void __launch_bounds__(256) k_prop_rows(int64_t M, int R, const T* __restrict__ D,
                                                   const double* __restrict__ cp, const double* __restrict__ d,
                                                   const T* __restrict__ X, double* __restrict__ V,
                                                   T* __restrict__ Xn, double h) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const T* row = D + s * M;
  for (int c0 = 0; c0 < R; c0 += RS) {
    T acc[RS];
#pragma unroll
    for (int q = 0; q < RS; ++q) acc[q] = T(0);
    for (int64_t n = lane; n < M; n += 32) {
      const T a = row[n];
#pragma unroll
      for (int q = 0; q < RS; ++q)
        if (RS == 1 || c0 + q < R) acc[q] = fma(a, X[(int64_t)(c0 + q) * M + n], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < RS; ++q)
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    T mine = T(0);
#pragma unroll
    for (int q = 0; q < RS; ++q)
      if (lane == q) mine = acc[q];
    const int r = c0 + lane;
    if (lane < RS && r < R) {
      const int64_t o = (int64_t)r * M + s;
      const double k = (double)mine + cp[s] + (d ? d[o] : 0.0);
      const double nv = fma(h, k, V[o]);
      V[o] = nv;
      Xn[o] = (T)nv;
    }
  }
}

// FP64 defect of the FP32 form for every state: d_r = (A64 + R32 - D32) V_r.
// One warp per (row, state).
__global__ void __launch_bounds__(256) k_prop_defect(int64_t M, int R, const double* __restrict__ A64,
                                                     const float* __restrict__ R32, const float* __restrict__ D32,
                                                     const double* __restrict__ V, double* __restrict__ d) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= M * R) return;
  const int64_t s = w / R;
  const int r = (int)(w % R);
  double a = 0.0;
  for (int64_t n = lane; n < M; n += 32) {
    const int64_t q = s * M + n;
    a = fma((A64[q] + (double)R32[q]) - (double)D32[q], V[(int64_t)r * M + n], a);
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) d[(int64_t)r * M + s] = a;
}

template <class T>
__global__ void k_round_states(int64_t n, const double* __restrict__ V, T* __restrict__ X) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (T)V[e];
}

}  // namespace

namespace lbi {

size_t propagate_workspace_bytes(int64_t M, int R, int precision) {
  const size_t esz = precision == LB_FP64 ? 8 : 4;
  const size_t x = ((esz * (size_t)M * R + 255) & ~size_t(255));
  const size_t dd = ((8 * (size_t)M * R + 255) & ~size_t(255));
  return 2 * x + dd + 256;
}

cudaError_t propagator_form(int64_t M, int precision, const double* A64, const float* A32, const double* K, double h,
                            void* Dp, float* R32, double* cp, void* work, size_t work_bytes, cudaStream_t st) {
  // work: G0, G1 (M x M of the element type), two M-vectors, the job lists
  const size_t esz = precision == LB_FP64 ? 8 : 4, mm = (size_t)M * (size_t)M;
  const size_t gsz = (esz * mm + 255) & ~size_t(255), usz = (16 * (size_t)M + 255) & ~size_t(255);
  const size_t lsz = batch_gemm_scratch_bytes(std::vector<int64_t>{M});
  if (2 * gsz + usz + lsz > work_bytes) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  void* G0 = w;
  void* G1 = w + gsz;
  double* ua = reinterpret_cast<double*>(w + 2 * gsz);
  double* ub = ua + M;
  void* js = w + 2 * gsz + usz;
  cudaError_t e = cudaSuccess;
  for (int step = 0; step < 3 && e == cudaSuccess; ++step) {
    const double alpha = step == 0 ? h / 4.0 : step == 1 ? h / 3.0 : h / 2.0;
    if (precision == LB_FP64) {
      double* D = static_cast<double*>(Dp);
      const double* G = step == 0 ? A64 : step == 1 ? static_cast<double*>(G0) : static_cast<double*>(G1);
      double* Y = step == 0 ? static_cast<double*>(G0) : step == 1 ? static_cast<double*>(G1) : D;
      e = batch_gemm<double>({GemmJob<double>{M, A64, G, step == 2 ? nullptr : A64, Y, alpha}}, js, lsz, st);
    } else {
      const float* G = step == 0 ? A32 : step == 1 ? static_cast<float*>(G0) : static_cast<float*>(G1);
      float* Y = step == 0 ? static_cast<float*>(G0) : step == 1 ? static_cast<float*>(G1) : R32;
      e = batch_gemm<float>({GemmJob<float>{M, A32, G, step == 2 ? nullptr : A32, Y, (float)alpha}}, js, lsz, st);
    }
  }
  if (e == cudaSuccess)
    e = precision == LB_FP64 ? add64(A64, static_cast<double*>(Dp), static_cast<double*>(Dp), (int64_t)mm, st)
                             : add32(A32, R32, static_cast<float*>(Dp), (int64_t)mm, st);
  for (int step = 0; step < 3 && e == cudaSuccess; ++step) {
    const double alpha = step == 0 ? h / 4.0 : step == 1 ? h / 3.0 : h / 2.0;
    const double* x = step == 0 ? K : step == 1 ? ua : ub;
    double* y = step == 0 ? ua : step == 1 ? ub : cp;
    e = batch_gemv64({GemvJob{M, A64, x, K, y, alpha}}, js, lsz, st);
  }
  return e;
}

size_t propagator_form_workspace_bytes(int64_t M, int precision) {
  const size_t esz = precision == LB_FP64 ? 8 : 4, mm = (size_t)M * (size_t)M;
  const size_t gsz = (esz * mm + 255) & ~size_t(255), usz = (16 * (size_t)M + 255) & ~size_t(255);
  return 2 * gsz + usz + batch_gemm_scratch_bytes(std::vector<int64_t>{M});
}

cudaError_t propagate(int64_t M, int R, int precision, const void* Dp, const float* R32, const double* A64,
                      const double* cp, int correct_every, double* V, double h, int64_t nsteps, double* snaps,
                      int64_t snap_every, void* work, cudaStream_t st) {
  const bool f64 = precision == LB_FP64;
  const size_t esz = f64 ? 8 : 4;
  const size_t x = ((esz * (size_t)M * R + 255) & ~size_t(255));
  char* w = static_cast<char*>(work);
  void* X0 = w;
  void* X1 = w + x;
  double* dd = reinterpret_cast<double*>(w + 2 * x);
  const bool correct = !f64 && correct_every > 0 && A64 && R32;
  const int64_t n = M * R;
  const unsigned rb = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  if (f64)
    k_round_states<double><<<rb, 256, 0, st>>>(n, V, static_cast<double*>(X0));
  else
    k_round_states<float><<<rb, 256, 0, st>>>(n, V, static_cast<float*>(X0));
  note_launch(1);
  cudaError_t e = cudaGetLastError();
  const unsigned grid = (unsigned)((M * 32 + 255) / 256);
  const unsigned dgrid = (unsigned)((M * R * 32 + 255) / 256);
  auto step = [&](const void* Xc, void* Xn) {
    if (f64) {
      const double* D = static_cast<const double*>(Dp);
      const double* xc = static_cast<const double*>(Xc);
      double* xn = static_cast<double*>(Xn);
      if (R == 1) k_prop_rows<double, 1><<<grid, 256, 0, st>>>(M, R, D, cp, nullptr, xc, V, xn, h);
      else if (R <= 4) k_prop_rows<double, 4><<<grid, 256, 0, st>>>(M, R, D, cp, nullptr, xc, V, xn, h);
      else k_prop_rows<double, 16><<<grid, 256, 0, st>>>(M, R, D, cp, nullptr, xc, V, xn, h);
    } else {
      const float* D = static_cast<const float*>(Dp);
      const float* xc = static_cast<const float*>(Xc);
      float* xn = static_cast<float*>(Xn);
      const double* dd_ = correct ? dd : nullptr;
      if (R == 1) k_prop_rows<float, 1><<<grid, 256, 0, st>>>(M, R, D, cp, dd_, xc, V, xn, h);
      else if (R <= 4) k_prop_rows<float, 4><<<grid, 256, 0, st>>>(M, R, D, cp, dd_, xc, V, xn, h);
      else k_prop_rows<float, 16><<<grid, 256, 0, st>>>(M, R, D, cp, dd_, xc, V, xn, h);
    }
  };
  for (int64_t t = 0; t < nsteps && e == cudaSuccess; ++t) {
    if (correct && t % correct_every == 0) {
      k_prop_defect<<<dgrid, 256, 0, st>>>(M, R, A64, R32, static_cast<const float*>(Dp), V, dd);
      note_launch(1);
    }
    step((t & 1) ? X1 : X0, (t & 1) ? X0 : X1);
    note_launch(1);
    e = cudaGetLastError();
    if (e == cudaSuccess && snaps && snap_every > 0 && (t + 1) % snap_every == 0)
      e = cudaMemcpyAsync(snaps + (size_t)((t + 1) / snap_every - 1) * (size_t)n, V, 8 * (size_t)n,
                          cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

}  // namespace lbi

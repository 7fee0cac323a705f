// lb_spectrum.cu -- the spectrum of the generator and its density (Sec. 6,
// Fig. 5: the complex eigenvalues lambda_i, i = 2..N^2, of one random
// Lindbladian, histogrammed on a grid of cells and normalised by the cell
// area).
//
// The eigenvalues of the real M x M matrix A = Q + R (the generator on the
// traceless part; the remaining eigenvalue of the full N^2 x N^2 generator
// belongs to the steady state) come from the library's dense nonsymmetric
// eigensolver (Hessenberg reduction and shifted QR, eigenvalues only): a
// plain library routine, not on the integration path.  It is loaded at run
// time, so the rest of the library does not depend on it; a missing solver
// gives LB_EUNSUPPORTED.  The density grid is this file's own kernel.
#include <cusolverDn.h>
#include <dlfcn.h>

#include <mutex>

#include "lb_internal.h"

namespace {

// The entry points of the dense solver this file uses.
struct Solver {
  bool ok = false;
  decltype(&cusolverDnCreate) create = nullptr;
  decltype(&cusolverDnDestroy) destroy = nullptr;
  decltype(&cusolverDnSetStream) set_stream = nullptr;
  decltype(&cusolverDnCreateParams) create_params = nullptr;
  decltype(&cusolverDnDestroyParams) destroy_params = nullptr;
  decltype(&cusolverDnXgeev_bufferSize) geev_size = nullptr;
  decltype(&cusolverDnXgeev) geev = nullptr;
  decltype(&cusolverDnXsyevd_bufferSize) syevd_size = nullptr;
  decltype(&cusolverDnXsyevd) syevd = nullptr;
};

const Solver& solver() {
  static Solver s;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = dlopen("libcusolver.so.12", RTLD_NOW | RTLD_LOCAL);
    if (!h) h = dlopen("libcusolver.so", RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    s.create = reinterpret_cast<decltype(s.create)>(dlsym(h, "cusolverDnCreate"));
    s.destroy = reinterpret_cast<decltype(s.destroy)>(dlsym(h, "cusolverDnDestroy"));
    s.set_stream = reinterpret_cast<decltype(s.set_stream)>(dlsym(h, "cusolverDnSetStream"));
    s.create_params = reinterpret_cast<decltype(s.create_params)>(dlsym(h, "cusolverDnCreateParams"));
    s.destroy_params = reinterpret_cast<decltype(s.destroy_params)>(dlsym(h, "cusolverDnDestroyParams"));
    s.geev_size = reinterpret_cast<decltype(s.geev_size)>(dlsym(h, "cusolverDnXgeev_bufferSize"));
    s.geev = reinterpret_cast<decltype(s.geev)>(dlsym(h, "cusolverDnXgeev"));
    s.syevd_size = reinterpret_cast<decltype(s.syevd_size)>(dlsym(h, "cusolverDnXsyevd_bufferSize"));
    s.syevd = reinterpret_cast<decltype(s.syevd)>(dlsym(h, "cusolverDnXsyevd"));
    s.ok = s.create && s.destroy && s.set_stream && s.create_params && s.destroy_params && s.geev_size && s.geev &&
           s.syevd_size && s.syevd;
  });
  return s;
}

// Number of eigenvalues in each cell of an nre x nim grid over
// [re_lo, re_hi) x [im_lo, im_hi), divided by the cell area (row-major,
// real part along the rows); eigenvalues outside the box are not counted.
__global__ void k_density(const double2* __restrict__ w, int64_t n, double re_lo, double re_hi, double im_lo,
                          double im_hi, int nre, int nim, double inv_area, double* __restrict__ dens) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 z = w[i];
  if (!(z.x >= re_lo && z.x < re_hi && z.y >= im_lo && z.y < im_hi)) return;
  int a = (int)((z.x - re_lo) / (re_hi - re_lo) * nre), b = (int)((z.y - im_lo) / (im_hi - im_lo) * nim);
  a = a < nre ? a : nre - 1;
  b = b < nim ? b : nim - 1;
  atomicAdd(dens + (int64_t)a * nim + b, inv_area);
}

// y = conj(x) elementwise
__global__ void k_conj_copy(int64_t n, const double2* __restrict__ x, double2* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = make_double2(x[i].x, -x[i].y);
}

}  // namespace

namespace lbi {

// Status: 0 ok, 1 solver unavailable, 2 solver failure (info != 0), or a
// CUDA error through *ce.
int spectrum_dense(const double* A, int64_t M, double2* w, cudaStream_t st, cudaError_t* ce) {
  *ce = cudaSuccess;
  const Solver& s = solver();
  if (!s.ok) return 1;
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t prm = nullptr;
  double* a = nullptr;
  void* dwork = nullptr;
  int* dinfo = nullptr;
  int rc = 0;
  std::vector<char> hwork;
  size_t dbytes = 0, hbytes = 0;
  int info = 0;
  cudaError_t e = cudaSuccess;
  if (s.create(&h) != CUSOLVER_STATUS_SUCCESS || s.create_params(&prm) != CUSOLVER_STATUS_SUCCESS ||
      s.set_stream(h, st) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  // the solver overwrites its input: a copy of A (column-major A^T has the same spectrum)
  e = cudaMallocAsync(reinterpret_cast<void**>(&a), sizeof(double) * (size_t)M * M, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a, A, sizeof(double) * (size_t)M * M, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dinfo), sizeof(int), st);
  if (e != cudaSuccess) goto done;
  if (s.geev_size(h, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_NOVECTOR, M, CUDA_R_64F, a, M, CUDA_C_64F, w,
                  CUDA_R_64F, nullptr, 1, CUDA_R_64F, nullptr, 1, CUDA_R_64F, &dbytes,
                  &hbytes) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  e = cudaMallocAsync(&dwork, dbytes ? dbytes : 16, st);
  if (e != cudaSuccess) goto done;
  hwork.resize(hbytes ? hbytes : 16);
  if (s.geev(h, prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_NOVECTOR, M, CUDA_R_64F, a, M, CUDA_C_64F, w,
             CUDA_R_64F, nullptr, 1, CUDA_R_64F, nullptr, 1, CUDA_R_64F, dwork, dbytes, hwork.data(), hbytes,
             dinfo) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  e = cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && info != 0) rc = 2;
done:
  if (dwork) cudaFreeAsync(dwork, st);
  if (dinfo) cudaFreeAsync(dinfo, st);
  if (a) cudaFreeAsync(a, st);
  if (prm) s.destroy_params(prm);
  if (h) s.destroy(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *ce = e;
  return e != cudaSuccess ? 3 : rc;
}

// Eigenvalues E (ascending) and eigenvectors of the Hermitian row-major
// N x N matrix H (device): on return row j of Ub (device, N x N) is the
// eigenvector of E[j].  The solver takes column-major input, so it gets
// conj(H), which is H in column-major order for a Hermitian H; its
// column-major eigenvector matrix is then Ub in row-major order.  Status as
// spectrum_dense.
int hermitian_eig(const double2* H, int N, double* E, double2* Ub, cudaStream_t st, cudaError_t* ce) {
  *ce = cudaSuccess;
  const Solver& s = solver();
  if (!s.ok) return 1;
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t prm = nullptr;
  void* dwork = nullptr;
  int* dinfo = nullptr;
  int rc = 0, info = 0;
  std::vector<char> hwork;
  size_t dbytes = 0, hbytes = 0;
  const int64_t n = N;
  cudaError_t e = cudaSuccess;
  if (s.create(&h) != CUSOLVER_STATUS_SUCCESS || s.create_params(&prm) != CUSOLVER_STATUS_SUCCESS ||
      s.set_stream(h, st) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  k_conj_copy<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(n * n, H, Ub);
  note_launch(1);
  e = cudaMallocAsync(reinterpret_cast<void**>(&dinfo), sizeof(int), st);
  if (e != cudaSuccess) goto done;
  if (s.syevd_size(h, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, Ub, n, CUDA_R_64F, E,
                   CUDA_C_64F, &dbytes, &hbytes) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  e = cudaMallocAsync(&dwork, dbytes ? dbytes : 16, st);
  if (e != cudaSuccess) goto done;
  hwork.resize(hbytes ? hbytes : 16);
  if (s.syevd(h, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, Ub, n, CUDA_R_64F, E,
              CUDA_C_64F, dwork, dbytes, hwork.data(), hbytes, dinfo) != CUSOLVER_STATUS_SUCCESS) {
    rc = 2;
    goto done;
  }
  e = cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && info != 0) rc = 2;
done:
  if (dwork) cudaFreeAsync(dwork, st);
  if (dinfo) cudaFreeAsync(dinfo, st);
  if (prm) s.destroy_params(prm);
  if (h) s.destroy(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *ce = e;
  return e != cudaSuccess ? 3 : rc;
}

cudaError_t spectrum_density(const double2* w, int64_t n, const double* box, int nre, int nim, double* dens,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(dens, 0, sizeof(double) * (size_t)nre * nim, st);
  if (e != cudaSuccess || n == 0) return e;
  const double area = (box[1] - box[0]) / nre * ((box[3] - box[2]) / nim);
  k_density<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, n, box[0], box[1], box[2], box[3], nre, nim,
                                                         1.0 / area, dens);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace lbi

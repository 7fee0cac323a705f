// lb_api.cu -- the extern "C" boundary of liblindblad.so (declared in
// include/lindblad.h).  Argument checking, error codes, the thread-local
// error text, device memory for the host-buffer interface, and launches of
// the kernels in lb_basis.cu, lb_assemble.cu and lb_rk4.cu.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include <string>

#include "lb_internal.h"

namespace {

thread_local std::string g_err;

// Owning device buffer (freed on scope exit unless released).
struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, n ? n : 1);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
};

#define LB_TRY_CUDA(call, what)                          \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return lbi::cuda_fail(_e, what); \
  } while (0)

#define LB_REQUIRE(cond, ...)        \
  do {                               \
    if (!(cond)) {                   \
      lbi::set_error(__VA_ARGS__);   \
      return LB_EINVAL;              \
    }                                \
  } while (0)

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

int alloc_or_enomem(DevBuf& b, size_t n, const char* what) {
  cudaError_t e = b.alloc(n);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    lbi::set_error("device allocation of %zu bytes for %s refused", n, what);
    return LB_ENOMEM;
  }
  if (e != cudaSuccess) return lbi::cuda_fail(e, what);
  return LB_OK;
}

}  // namespace

namespace lbi {

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  // the library's kernels report a bounded wait that ran out as a launch timeout
  return e == cudaErrorLaunchTimeout ? LB_ETIMEOUT : LB_ECUDA;
}

}  // namespace lbi

// An assembled system of the host-buffer interface.  Dense systems hold A
// (and Q, R if kept) as M x M FP64 in memory of the library pool, returned
// to it (stream-ordered) on destruction; CSR systems hold A = Q + R in csr.
struct lb_system {
  const lb_basis* basis = nullptr;
  int64_t M = 0;
  int format = LB_DENSE;
  double* A = nullptr;
  double* Q = nullptr;
  double* R = nullptr;
  double* K = nullptr;
  float* A32 = nullptr;
  uint16_t* Abf = nullptr;
  float* scale = nullptr;
  lbi::CsrOut csr;               // LB_CSR: rowptr, col, val, K (K aliases csr.K)
  float* csr32 = nullptr;        // FP32 copy of csr.val, made on first use
  double ms[LB_PHASES] = {};     // phase times of the call that built it
};

extern "C" {

const char* lb_last_error(void) { return g_err.c_str(); }

int lb_version(void) { return 200; }

int lb_basis_create(int N, void* stream, lb_basis_t** out) {
  LB_REQUIRE(out != nullptr, "lb_basis_create: out is NULL");
  LB_REQUIRE(N >= 2 && N <= 4096, "lb_basis_create: N = %d outside [2, 4096]", N);
  *out = nullptr;
  const int64_t P = (int64_t)N * (N - 1) / 2;
  DevBuf pab, tab;
  int rc;
  if ((rc = alloc_or_enomem(pab, sizeof(int32_t) * P, "pair table")) != LB_OK) return rc;
  if ((rc = alloc_or_enomem(tab, sizeof(double) * (4 * (size_t)N + 1), "basis constants")) != LB_OK) return rc;
  LB_TRY_CUDA(lbi::build_tables(N, pab.as<int32_t>(), tab.as<double>(), S(stream)), "basis tables");
  LB_TRY_CUDA(cudaStreamSynchronize(S(stream)), "basis tables");
  lb_basis* b = new lb_basis;
  b->N = N;
  b->P = P;
  b->M = (int64_t)N * N - 1;
  b->d_pair_ab = static_cast<int32_t*>(pab.release());
  b->d_tab = static_cast<double*>(tab.release());
  *out = b;
  return LB_OK;
}

int lb_basis_destroy(lb_basis_t* b) {
  if (!b) return LB_OK;
  cudaFree(b->d_pair_ab);
  cudaFree(b->d_tab);
  delete b;
  return LB_OK;
}

int lb_basis_dims(const lb_basis_t* b, int* N, int64_t* M, int64_t* P) {
  LB_REQUIRE(b != nullptr, "lb_basis_dims: basis is NULL");
  if (N) *N = b->N;
  if (M) *M = b->M;
  if (P) *P = b->P;
  return LB_OK;
}

int lb_basis_label(const lb_basis_t* b, int64_t i, char* type, int* j, int* k) {
  LB_REQUIRE(b != nullptr, "lb_basis_label: basis is NULL");
  LB_REQUIRE(i >= 0 && i < b->M, "lb_basis_label: index %lld outside [0, %lld)", (long long)i,
             (long long)b->M);
  char t;
  int a, c;
  if (i < 2 * b->P) {
    int64_t p = i < b->P ? i : i - b->P;
    t = i < b->P ? 'S' : 'J';
    a = 0;
    while (p >= b->N - 1 - a) {
      p -= b->N - 1 - a;
      ++a;
    }
    c = a + 1 + (int)p;
  } else {
    t = 'D';
    a = c = (int)(i - 2 * b->P + 1);
  }
  if (type) *type = t;
  if (j) *j = a;
  if (k) *k = c;
  return LB_OK;
}

}  // extern "C"

namespace {

// count per m -> exclusive scan; offsets has M+1 entries, offsets[M] = total.
int count_and_scan(const lb_basis_t* b, int which, DevBuf& offsets, int64_t* total, cudaStream_t st) {
  const int64_t M = b->M;
  int rc;
  DevBuf per;
  if ((rc = alloc_or_enomem(per, sizeof(int64_t) * (M + 1), "structure counts")) != LB_OK) return rc;
  if ((rc = alloc_or_enomem(offsets, sizeof(int64_t) * (M + 1), "structure offsets")) != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemsetAsync(per.as<int64_t>() + M, 0, sizeof(int64_t), st), "structure counts");
  LB_TRY_CUDA(lbi::structure_count(b->view(), which, per.as<int64_t>(), st), "kernel (a) count");
  LB_TRY_CUDA(lbi::exclusive_scan(per.as<int64_t>(), offsets.as<int64_t>(), M, st), "scan");
  LB_TRY_CUDA(cudaMemcpyAsync(total, offsets.as<int64_t>() + M, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st),
              "structure total");
  LB_TRY_CUDA(cudaStreamSynchronize(st), "kernel (a)");
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_structure_count(const lb_basis_t* b, int which, int64_t* nnz) {
  LB_REQUIRE(b != nullptr && nnz != nullptr, "lb_structure_count: NULL argument");
  LB_REQUIRE(which == LB_F || which == LB_D, "lb_structure_count: which = %d", which);
  DevBuf off;
  return count_and_scan(b, which, off, nnz, nullptr);
}

int lb_structure_export(const lb_basis_t* b, int which, int32_t* idx3, double* val, int64_t capacity,
                        int64_t* nnz, void* stream) {
  LB_REQUIRE(b != nullptr && nnz != nullptr, "lb_structure_export: NULL argument");
  LB_REQUIRE(which == LB_F || which == LB_D, "lb_structure_export: which = %d", which);
  LB_REQUIRE(b->M <= 0x7fffffffLL, "lb_structure_export: M too large for int32 indices");
  DevBuf off;
  int64_t total = 0;
  int rc = count_and_scan(b, which, off, &total, S(stream));
  if (rc != LB_OK) return rc;
  *nnz = total;
  LB_REQUIRE(idx3 != nullptr && val != nullptr, "lb_structure_export: NULL output buffer");
  LB_REQUIRE(capacity >= total, "lb_structure_export: capacity %lld < %lld triples",
             (long long)capacity, (long long)total);
  LB_TRY_CUDA(lbi::structure_fill(b->view(), which, off.as<int64_t>(), idx3, val, S(stream)),
              "kernel (a) fill");
  // offsets are freed at scope exit: wait for the fill that reads them
  LB_TRY_CUDA(cudaStreamSynchronize(S(stream)), "kernel (a) fill");
  return LB_OK;
}

int lb_join_terms(const lb_basis_t* b, int64_t* W) {
  LB_REQUIRE(b != nullptr && W != nullptr, "lb_join_terms: NULL argument");
  DevBuf cnt;
  int rc;
  if ((rc = alloc_or_enomem(cnt, sizeof(unsigned long long), "term counter")) != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemset(cnt.p, 0, sizeof(unsigned long long)), "term counter");
  LB_TRY_CUDA(lbi::join_terms(b->view(), cnt.as<unsigned long long>(), nullptr), "join-term count");
  unsigned long long h = 0;
  LB_TRY_CUDA(cudaMemcpy(&h, cnt.p, sizeof h, cudaMemcpyDeviceToHost), "join-term count");
  *W = (int64_t)h;
  return LB_OK;
}

int lb_expand(const lb_basis_t* b, const double* A, double* coef, void* stream) {
  LB_REQUIRE(b && A && coef, "lb_expand: NULL argument");
  LB_TRY_CUDA(lbi::expand(b->view(), reinterpret_cast<const double2*>(A), reinterpret_cast<double2*>(coef),
                          S(stream)),
              "lb_expand");
  return LB_OK;
}

int lb_rho(const lb_basis_t* b, const double* v, double* rho, void* stream) {
  LB_REQUIRE(b && v && rho, "lb_rho: NULL argument");
  LB_TRY_CUDA(lbi::rho(b->view(), v, reinterpret_cast<double2*>(rho), S(stream)), "lb_rho");
  return LB_OK;
}

int lb_assemble_dense_ex(const lb_basis_t* b, const double* h, const double* a, double* A, double* Q,
                         double* R, double* K, int algorithm, void* stream) {
  LB_REQUIRE(b != nullptr && a != nullptr, "lb_assemble_dense: NULL basis or a");
  LB_REQUIRE(A || Q || R || K, "lb_assemble_dense: no output requested");
  LB_REQUIRE(b->N <= lbi::kMaxDenseN, "lb_assemble_dense: N = %d above %d", b->N, lbi::kMaxDenseN);
  LB_REQUIRE(algorithm == LB_ALG_JOIN || algorithm == LB_ALG_CLOSED, "lb_assemble_dense: algorithm = %d",
             algorithm);
  LB_TRY_CUDA(lbi::assemble_dense(b->view(), h, reinterpret_cast<const double2*>(a), A, Q, R, K, algorithm,
                                  S(stream)),
              "lb_assemble_dense");
  return LB_OK;
}

int lb_assemble_dense(const lb_basis_t* b, const double* h, const double* a, double* A, double* Q,
                      double* R, double* K, void* stream) {
  return lb_assemble_dense_ex(b, h, a, A, Q, R, K, LB_ALG_CLOSED, stream);
}

int lb_assemble_kernel_count(void) { return lbi::kAssembleKernels; }

const char* lb_assemble_kernel_name(int i) { return lbi::assemble_kernel_name(i); }

int lb_assemble_dense_timed(const lb_basis_t* b, const double* h, const double* a, double* A, double* Q,
                            double* R, double* K, int algorithm, void* stream, float* kernel_ms) {
  LB_REQUIRE(b != nullptr && a != nullptr && kernel_ms != nullptr, "lb_assemble_dense_timed: NULL argument");
  LB_REQUIRE(A || Q || R || K, "lb_assemble_dense_timed: no output requested");
  LB_REQUIRE(b->N <= lbi::kMaxDenseN, "lb_assemble_dense_timed: N = %d above %d", b->N, lbi::kMaxDenseN);
  LB_REQUIRE(algorithm == LB_ALG_JOIN || algorithm == LB_ALG_CLOSED, "lb_assemble_dense_timed: algorithm = %d",
             algorithm);
  cudaEvent_t ev[lbi::kAssembleKernels + 1] = {};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i <= lbi::kAssembleKernels && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess)
    e = lbi::assemble_dense(b->view(), h, reinterpret_cast<const double2*>(a), A, Q, R, K, algorithm, S(stream),
                            ev);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[lbi::kAssembleKernels]);
  for (int i = 0; i < lbi::kAssembleKernels && e == cudaSuccess; ++i)
    e = cudaEventElapsedTime(&kernel_ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i <= lbi::kAssembleKernels; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_assemble_dense_timed");
  return LB_OK;
}

int lb_pack_fp32(int64_t M, const double* A, float* A32, void* stream) {
  LB_REQUIRE(M > 0 && A && A32, "lb_pack_fp32: bad argument");
  LB_TRY_CUDA(lbi::pack_fp32(M, A, A32, S(stream)), "lb_pack_fp32");
  return LB_OK;
}

int lb_pack_bf16(int64_t M, const double* A, uint16_t* Abf, float* row_scale, void* stream) {
  LB_REQUIRE(M > 0 && A && Abf && row_scale, "lb_pack_bf16: bad argument");
  LB_TRY_CUDA(lbi::pack_bf16(M, A, Abf, row_scale, S(stream)), "lb_pack_bf16");
  return LB_OK;
}

size_t lb_rk4_workspace_bytes(int64_t M) { return M > 0 ? lbi::rk4_workspace_bytes(M) : 0; }

int lb_rk4_dense(int64_t M, int precision, const void* Ap, const float* row_scale, const double* A64,
                 int correct_every, const double* K, double* v, double dt, int64_t nsteps, double* snaps,
                 int64_t snap_every, void* work, void* stream) {
  LB_REQUIRE(M > 0 && Ap && K && v && work, "lb_rk4_dense: NULL argument or M <= 0");
  LB_REQUIRE(precision == LB_FP64 || precision == LB_FP32 || precision == LB_BF16,
             "lb_rk4_dense: precision = %d", precision);
  LB_REQUIRE(precision != LB_BF16 || row_scale, "lb_rk4_dense: BF16 needs row_scale");
  LB_REQUIRE(nsteps >= 0 && std::isfinite(dt), "lb_rk4_dense: bad step count or dt");
  LB_REQUIRE(!snaps || snap_every > 0, "lb_rk4_dense: snaps given without snap_every");
  LB_REQUIRE(correct_every >= 0, "lb_rk4_dense: correct_every < 0");
  LB_TRY_CUDA(lbi::rk4_dense(M, precision, Ap, row_scale, A64, correct_every, K, v, dt, nsteps, snaps,
                             snap_every, work, S(stream)),
              "lb_rk4_dense");
  return LB_OK;
}

// ------------------------------------------------------------------ propagator form

size_t lb_propagator_workspace_bytes(int64_t M, int nrhs, int precision) {
  if (M <= 0 || nrhs < 1 || nrhs > 64 || (precision != LB_FP64 && precision != LB_FP32)) return 0;
  return std::max(lbi::propagator_form_workspace_bytes(M, precision),
                  lbi::propagate_workspace_bytes(M, nrhs, precision));
}

int lb_propagator_form(int64_t M, int precision, const double* A64, const float* A32, const double* K, double dt,
                       void* Dp, float* R32, double* cp, void* work, void* stream) {
  LB_REQUIRE(M > 0 && A64 && K && Dp && cp && work, "lb_propagator_form: NULL argument or M <= 0");
  LB_REQUIRE(precision == LB_FP64 || (precision == LB_FP32 && A32 && R32),
             "lb_propagator_form: precision = %d (LB_FP32 needs A32 and R32)", precision);
  LB_REQUIRE(dt > 0 && std::isfinite(dt), "lb_propagator_form: bad dt");
  LB_TRY_CUDA(lbi::propagator_form(M, precision, A64, A32, K, dt, Dp, R32, cp, work,
                                   lbi::propagator_form_workspace_bytes(M, precision), S(stream)),
              "lb_propagator_form");
  return LB_OK;
}

int lb_propagate(int64_t M, int nrhs, int precision, const void* Dp, const float* R32, const double* A64,
                 const double* cp, int correct_every, double* V, double dt, int64_t nsteps, double* snaps,
                 int64_t snap_every, void* work, void* stream) {
  LB_REQUIRE(M > 0 && Dp && cp && V && work, "lb_propagate: NULL argument or M <= 0");
  LB_REQUIRE(nrhs >= 1 && nrhs <= 64, "lb_propagate: nrhs = %d outside [1, 64]", nrhs);
  LB_REQUIRE(precision == LB_FP64 || precision == LB_FP32, "lb_propagate: precision = %d", precision);
  LB_REQUIRE(nsteps >= 0 && dt > 0 && std::isfinite(dt) && correct_every >= 0, "lb_propagate: bad arguments");
  LB_REQUIRE(correct_every == 0 || precision == LB_FP64 || (R32 && A64),
             "lb_propagate: the correction needs A64 and R32");
  LB_REQUIRE(!snaps || snap_every > 0, "lb_propagate: snaps given without snap_every");
  LB_TRY_CUDA(lbi::propagate(M, nrhs, precision, Dp, R32, A64, cp, correct_every, V, dt, nsteps, snaps, snap_every,
                             work, S(stream)),
              "lb_propagate");
  return LB_OK;
}

// ------------------------------------------------------------------ FP64 checks

static int spectrum_status(int rc, cudaError_t ce, const char* what);

size_t lb_steady_workspace_bytes(int64_t M, int restart) {
  return M > 0 && restart >= 0 ? lbi::steady_workspace_bytes(M, restart) : 0;
}

int lb_steady_state(int64_t M, const double* A, const double* K, double* v, double tol, int max_iter, int restart,
                    double* rel_residual, int* iterations, void* work, void* stream) {
  LB_REQUIRE(M > 0 && A && K && v && work && rel_residual && iterations, "lb_steady_state: NULL argument");
  LB_REQUIRE(tol > 0 && std::isfinite(tol) && max_iter >= 1 && restart >= 0,
             "lb_steady_state: bad tol, max_iter or restart");
  LB_TRY_CUDA(lbi::steady_state(M, A, K, v, tol, max_iter, restart, rel_residual, iterations, work, S(stream)),
              "lb_steady_state");
  return LB_OK;
}

size_t lb_steady_pc_workspace_bytes(int N, int64_t M, int restart) {
  return N >= 2 && M == (int64_t)N * N - 1 && restart >= 0 ? lbi::steady_pc_workspace_bytes(N, M, restart) : 0;
}

int lb_steady_state_pc(const lb_basis_t* b, const double* A, const double* K, const double* H, double sigma,
                       double* v, double tol, int max_iter, int restart, double* rel_residual, int* iterations,
                       void* work, void* stream) {
  LB_REQUIRE(b && A && K && H && v && work && rel_residual && iterations, "lb_steady_state_pc: NULL argument");
  LB_REQUIRE(tol > 0 && std::isfinite(tol) && max_iter >= 1 && restart >= 0 && std::isfinite(sigma),
             "lb_steady_state_pc: bad tol, max_iter, restart or sigma");
  LB_REQUIRE((reinterpret_cast<uintptr_t>(work) & 255) == 0, "lb_steady_state_pc: work must be 256-byte aligned");
  lbi::PcView pc;
  cudaError_t ce = cudaSuccess;
  const int rc = lbi::steady_pc_setup(b->view(), reinterpret_cast<const double2*>(H), A, sigma, restart, work, &pc,
                                      S(stream), &ce);
  if (rc != 0) return spectrum_status(rc, ce, "lb_steady_state_pc");
  LB_TRY_CUDA(lbi::steady_state(b->M, A, K, v, tol, max_iter, restart, rel_residual, iterations, work, S(stream), &pc),
              "lb_steady_state_pc");
  return LB_OK;
}

size_t lb_rho_checks_workspace_bytes(int N) { return N >= 2 ? lbi::rho_checks_workspace_bytes(N) : 0; }

int lb_rho_checks(const lb_basis_t* b, const double* V, int64_t nsnap, double psd_shift, double* out, void* work,
                  void* stream) {
  LB_REQUIRE(b && V && out && work && nsnap >= 0, "lb_rho_checks: NULL argument or nsnap < 0");
  LB_REQUIRE(psd_shift >= 0 && std::isfinite(psd_shift), "lb_rho_checks: bad psd_shift");
  LB_REQUIRE(b->N <= 4096, "lb_rho_checks: N too large");
  LB_TRY_CUDA(lbi::rho_checks(b->view(), V, nsnap, psd_shift, out, work, S(stream)), "lb_rho_checks");
  return LB_OK;
}

// ------------------------------------------------------------------ sparse

}  // extern "C"

struct lb_csr {
  lbi::CsrOut m;
  float* val32 = nullptr;
};

extern "C" {

int lb_assemble_lowrank_csr(const lb_basis_t* b, const double* h, int nP, const double* gamma,
                            const int64_t* lp_ptr, const int64_t* lp_idx, const double* lp_val, lb_csr_t** out,
                            void* stream) {
  LB_REQUIRE(b && out && (nP == 0 || (gamma && lp_ptr)), "lb_assemble_lowrank_csr: NULL argument");
  LB_REQUIRE(nP >= 0 && nP <= 4096, "lb_assemble_lowrank_csr: nP = %d", nP);
  LB_REQUIRE(b->M <= 0x7fffffffLL, "lb_assemble_lowrank_csr: M too large for int32 columns");
  LB_REQUIRE(lp_ptr == nullptr || lp_ptr[0] == 0, "lb_assemble_lowrank_csr: lp_ptr[0] must be 0");
  for (int p = 0; p < nP; ++p) {
    LB_REQUIRE(lp_ptr[p + 1] >= lp_ptr[p], "lb_assemble_lowrank_csr: lp_ptr not monotone");
    LB_REQUIRE(std::isfinite(gamma[p]), "lb_assemble_lowrank_csr: gamma[%d] not finite", p);
  }
  LB_REQUIRE(nP == 0 || lp_ptr[nP] == 0 || (lp_idx && lp_val), "lb_assemble_lowrank_csr: NULL channel arrays");
  *out = nullptr;
  lb_csr* c = new lb_csr;
  static const int64_t zero_ptr[1] = {0};
  cudaError_t e = lbi::assemble_lowrank_csr(b->view(), h, nP, gamma, nP ? lp_ptr : zero_ptr, lp_idx,
                                            reinterpret_cast<const double2*>(lp_val), &c->m, S(stream));
  if (e != cudaSuccess) {
    delete c;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      lbi::set_error("lb_assemble_lowrank_csr: device memory exhausted");
      return LB_ENOMEM;
    }
    if (e == cudaErrorNotSupported) {
      lbi::set_error("lb_assemble_lowrank_csr: a row of A has more than 8192 distinct columns");
      return LB_EUNSUPPORTED;
    }
    return lbi::cuda_fail(e, "lb_assemble_lowrank_csr");
  }
  *out = c;
  return LB_OK;
}

int lb_csr_info(const lb_csr_t* c, int64_t* M, int64_t* nnz, int64_t* terms) {
  LB_REQUIRE(c != nullptr, "lb_csr_info: NULL handle");
  if (M) *M = c->m.M;
  if (nnz) *nnz = c->m.nnz;
  if (terms) *terms = c->m.terms;
  return LB_OK;
}

int lb_csr_arrays(const lb_csr_t* c, const int64_t** rowptr, const int32_t** col, const double** val,
                  const double** K) {
  LB_REQUIRE(c != nullptr, "lb_csr_arrays: NULL handle");
  if (rowptr) *rowptr = c->m.rowptr;
  if (col) *col = c->m.col;
  if (val) *val = c->m.val;
  if (K) *K = c->m.K;
  return LB_OK;
}

int lb_csr_copy(const lb_csr_t* c, int64_t* rowptr, int32_t* col, double* val, double* K, void* stream) {
  LB_REQUIRE(c != nullptr, "lb_csr_copy: NULL handle");
  const cudaStream_t st = S(stream);
  if (rowptr)
    LB_TRY_CUDA(cudaMemcpyAsync(rowptr, c->m.rowptr, sizeof(int64_t) * (c->m.M + 1), cudaMemcpyDefault, st), "copy");
  if (col) LB_TRY_CUDA(cudaMemcpyAsync(col, c->m.col, sizeof(int32_t) * c->m.nnz, cudaMemcpyDefault, st), "copy");
  if (val) LB_TRY_CUDA(cudaMemcpyAsync(val, c->m.val, sizeof(double) * c->m.nnz, cudaMemcpyDefault, st), "copy");
  if (K) LB_TRY_CUDA(cudaMemcpyAsync(K, c->m.K, sizeof(double) * c->m.M, cudaMemcpyDefault, st), "copy");
  LB_TRY_CUDA(cudaStreamSynchronize(st), "copy");
  return LB_OK;
}

int lb_csr_destroy(lb_csr_t* c) {
  if (!c) return LB_OK;
  cudaFree(c->m.rowptr);
  cudaFree(c->m.col);
  cudaFree(c->m.val);
  cudaFree(c->m.K);
  cudaFree(c->val32);
  delete c;
  return LB_OK;
}

int lb_rk4_csr(const lb_csr_t* c, int precision, int correct_every, double* v, double dt, int64_t nsteps,
               void* work, void* stream) {
  LB_REQUIRE(c && v && work, "lb_rk4_csr: NULL argument");
  LB_REQUIRE(precision == LB_FP64 || precision == LB_FP32, "lb_rk4_csr: precision = %d", precision);
  LB_REQUIRE(nsteps >= 0 && std::isfinite(dt) && correct_every >= 0, "lb_rk4_csr: bad arguments");
  lb_csr* cc = const_cast<lb_csr*>(c);
  const void* val = c->m.val;
  if (precision == LB_FP32) {
    if (!cc->val32) {
      DevBuf b32;
      int rc;
      if ((rc = alloc_or_enomem(b32, sizeof(float) * (size_t)(c->m.nnz + 1), "FP32 values")) != LB_OK) return rc;
      LB_TRY_CUDA(lbi::to_f32(c->m.nnz, c->m.val, b32.as<float>(), S(stream)), "pack FP32 values");
      cc->val32 = static_cast<float*>(b32.release());
    }
    val = cc->val32;
  }
  LB_TRY_CUDA(lbi::rk4_csr(c->m.M, precision, c->m.rowptr, c->m.col, val, c->m.val, correct_every, c->m.K, v, dt,
                           nsteps, work, S(stream)),
              "lb_rk4_csr");
  return LB_OK;
}

}  // extern "C"

extern "C" {

int lb_rk4_csr_td(const lb_csr_t* A0, const lb_csr_t* Q1, int nseg, const double* seg_start, const double* seg_eps,
                  double period, double t0, double* v, double dt, int64_t nsteps, void* work, void* stream) {
  LB_REQUIRE(A0 && Q1 && v && work && seg_start && seg_eps, "lb_rk4_csr_td: NULL argument");
  LB_REQUIRE(A0->m.M == Q1->m.M, "lb_rk4_csr_td: A0 and Q1 differ in size");
  LB_REQUIRE(nseg >= 1 && nseg <= 1024 && seg_start[0] == 0.0, "lb_rk4_csr_td: nseg = %d, seg_start[0] = %g", nseg,
             seg_start[0]);
  LB_REQUIRE(period > 0 && std::isfinite(period) && std::isfinite(t0), "lb_rk4_csr_td: bad period or t0");
  for (int k = 0; k < nseg; ++k) {
    LB_REQUIRE(std::isfinite(seg_eps[k]), "lb_rk4_csr_td: seg_eps[%d] not finite", k);
    LB_REQUIRE(k == 0 || (seg_start[k] > seg_start[k - 1] && seg_start[k] < period),
               "lb_rk4_csr_td: seg_start must increase within [0, period)");
  }
  LB_REQUIRE(nsteps >= 0 && dt > 0 && std::isfinite(dt), "lb_rk4_csr_td: bad step count or dt");
  LB_TRY_CUDA(lbi::rk4_csr_td(A0->m.M, A0->m.rowptr, A0->m.col, A0->m.val, Q1->m.rowptr, Q1->m.col, Q1->m.val,
                              A0->m.K, nseg, seg_start, seg_eps, period, t0, v, dt, nsteps, work, S(stream)),
              "lb_rk4_csr_td");
  return LB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ host API

namespace {

// Per-device stream and memory pool of the host-buffer interface.  The pool
// keeps what it has reserved (release threshold: unlimited) so that repeated
// calls of the same size reuse device memory without cudaMalloc / cudaFree
// (a cudaFree synchronizes the whole device); lb_host_release hands it back.
struct HostCtx {
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
};
std::mutex g_host_mu;
std::vector<HostCtx> g_host;

cudaError_t host_ctx(HostCtx* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_host_mu);
  if ((int)g_host.size() <= dev) g_host.resize(dev + 1);
  HostCtx& c = g_host[dev];
  if (!c.st) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if ((e = cudaMemPoolCreate(&c.pool, &props)) != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    if ((e = cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking)) != cudaSuccess) {
      c.st = nullptr;
      return e;
    }
  }
  *out = c;
  return cudaSuccess;
}

// Bytes the pool holds but no allocation uses: free for the next call.
size_t pool_spare(cudaMemPool_t pool) {
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess) return 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) return 0;
  return reserved > used ? (size_t)(reserved - used) : 0;
}

// Stream-ordered pool allocation on the library stream (freed with pool_free).
struct PoolBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  PoolBuf() = default;
  PoolBuf(const PoolBuf&) = delete;
  PoolBuf& operator=(const PoolBuf&) = delete;
  ~PoolBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  int alloc(const HostCtx& c, size_t n, const char* what) {
    st = c.st;
    const cudaError_t e = cudaMallocFromPoolAsync(&p, n ? n : 1, c.pool, c.st);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      p = nullptr;
      lbi::set_error("device allocation of %zu bytes for %s refused", n, what);
      return LB_ENOMEM;
    }
    if (e != cudaSuccess) {
      p = nullptr;
      return lbi::cuda_fail(e, what);
    }
    return LB_OK;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
  void free_now() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
  }
};

// Events around the phases of one call on the library stream.
struct PhaseClock {
  cudaEvent_t ev[LB_PHASES + 1] = {};
  bool ok = true;
  explicit PhaseClock(cudaStream_t st) : st_(st) {
    for (auto& e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  }
  ~PhaseClock() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
  void mark(int i) {
    if (ok) ok = cudaEventRecord(ev[i], st_) == cudaSuccess;
  }
  // ms[i] = time from mark i to mark i + 1 (marks not recorded count as 0)
  void read(double* ms, int from, int to) {
    for (int i = from; i < to; ++i) {
      float t = 0.f;
      ms[i] = (ok && cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) ? t : 0.0;
    }
    cudaGetLastError();
  }

 private:
  cudaStream_t st_;
};

// a_jk = sum_p gamma_p l_pj conj(l_pk) for one channel p, added onto a dense
// M x M complex matrix: one thread per pair of the channel's nonzeros, so
// each entry is touched once per channel.
__global__ void k_lowrank_add(int64_t M, int n, const int64_t* __restrict__ idx, const double2* __restrict__ val,
                              double gamma, double2* __restrict__ a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const double2 x = val[i], y = val[j];
  double2* o = a + idx[i] * M + idx[j];
  o->x += gamma * (x.x * y.x + x.y * y.y);
  o->y += gamma * (x.y * y.x - x.x * y.y);
}

// h_m = Re coef_m (stride-2 copy of the real parts), on st
cudaError_t real_part(const double2* coef, double* h, int64_t M, cudaStream_t st) {
  return cudaMemcpy2DAsync(h, sizeof(double), coef, 2 * sizeof(double), sizeof(double), (size_t)M,
                           cudaMemcpyDeviceToDevice, st);
}

void pool_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

}  // namespace

extern "C" {

int lb_host_release(void) {
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_host_release");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_host_release");
  LB_TRY_CUDA(cudaMemPoolTrimTo(c.pool, 0), "lb_host_release");
  return LB_OK;
}

int lb_expand_host(const lb_basis_t* b, const double* A, double* coef) {
  LB_REQUIRE(b && A && coef, "lb_expand_host: NULL argument");
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_expand_host");
  const size_t nn = (size_t)b->N * b->N;
  PoolBuf dA, dc;
  int rc;
  if ((rc = dA.alloc(c, 16 * nn, "A")) != LB_OK || (rc = dc.alloc(c, 16 * (size_t)b->M, "coef")) != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemcpyAsync(dA.p, A, 16 * nn, cudaMemcpyHostToDevice, c.st), "lb_expand_host: copy A");
  LB_TRY_CUDA(lbi::expand(b->view(), dA.as<double2>(), dc.as<double2>(), c.st), "lb_expand_host");
  LB_TRY_CUDA(cudaMemcpyAsync(coef, dc.p, 16 * (size_t)b->M, cudaMemcpyDeviceToHost, c.st), "lb_expand_host: copy");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_expand_host");
  return LB_OK;
}

int lb_rho_host(const lb_basis_t* b, const double* v, double* rho) {
  LB_REQUIRE(b && v && rho, "lb_rho_host: NULL argument");
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_rho_host");
  const size_t nn = (size_t)b->N * b->N;
  PoolBuf dv, dr;
  int rc;
  if ((rc = dv.alloc(c, 8 * (size_t)b->M, "v")) != LB_OK || (rc = dr.alloc(c, 16 * nn, "rho")) != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemcpyAsync(dv.p, v, 8 * (size_t)b->M, cudaMemcpyHostToDevice, c.st), "lb_rho_host: copy v");
  LB_TRY_CUDA(lbi::rho(b->view(), dv.as<double>(), dr.as<double2>(), c.st), "lb_rho_host");
  LB_TRY_CUDA(cudaMemcpyAsync(rho, dr.p, 16 * nn, cudaMemcpyDeviceToHost, c.st), "lb_rho_host: copy");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_rho_host");
  return LB_OK;
}

int lb_assemble(const lb_basis_t* b, const double* H, const lb_kossakowski* a, int format, int algorithm,
                int keep_parts, lb_system_t** out) {
  LB_REQUIRE(b && a && out, "lb_assemble: NULL argument");
  *out = nullptr;
  LB_REQUIRE(a->kind == LB_A_DENSE || a->kind == LB_A_LOWRANK, "lb_assemble: Kossakowski kind = %d", a->kind);
  LB_REQUIRE(format == LB_DENSE || format == LB_CSR, "lb_assemble: format = %d", format);
  LB_REQUIRE(algorithm == LB_ALG_JOIN || algorithm == LB_ALG_CLOSED, "lb_assemble: algorithm = %d", algorithm);
  if (a->kind == LB_A_DENSE) LB_REQUIRE(a->a != nullptr, "lb_assemble: dense Kossakowski matrix is NULL");
  if (a->kind == LB_A_LOWRANK) {
    LB_REQUIRE(a->nP >= 0 && a->nP <= 4096, "lb_assemble: nP = %d", a->nP);
    LB_REQUIRE(a->nP == 0 || (a->gamma && a->lp_ptr), "lb_assemble: NULL channel arrays");
    LB_REQUIRE(a->nP == 0 || a->lp_ptr[0] == 0, "lb_assemble: lp_ptr[0] must be 0");
    for (int p = 0; p < a->nP; ++p) {
      LB_REQUIRE(a->lp_ptr[p + 1] >= a->lp_ptr[p], "lb_assemble: lp_ptr not monotone");
      LB_REQUIRE(std::isfinite(a->gamma[p]), "lb_assemble: gamma[%d] not finite", p);
    }
    const int64_t nl = a->nP ? a->lp_ptr[a->nP] : 0;
    LB_REQUIRE(nl == 0 || (a->lp_idx && a->lp_val), "lb_assemble: NULL channel arrays");
    for (int64_t i = 0; i < nl; ++i)
      LB_REQUIRE(a->lp_idx[i] >= 0 && a->lp_idx[i] < b->M, "lb_assemble: lp_idx[%lld] out of range",
                 (long long)i);
  }
  if (format == LB_CSR) {
    if (a->kind == LB_A_DENSE) {
      lbi::set_error("lb_assemble: a CSR system needs a low-rank Kossakowski matrix (the sparse pattern keeps an "
                     "entry by the size of its terms, which the dense kernels do not form)");
      return LB_EUNSUPPORTED;
    }
    if (keep_parts) {
      lbi::set_error("lb_assemble: Q and R are not kept separately in a CSR system");
      return LB_EUNSUPPORTED;
    }
    LB_REQUIRE(b->M <= 0x7fffffffLL, "lb_assemble: M too large for int32 columns");
  } else {
    LB_REQUIRE(b->N <= lbi::kMaxDenseN, "lb_assemble: N = %d above %d for a dense system", b->N, lbi::kMaxDenseN);
  }
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_assemble: library stream");
  const int64_t M = b->M, N = b->N;
  const size_t mm = (size_t)M * (size_t)M;
  lb_system* sys = new lb_system;
  sys->basis = b;
  sys->M = M;
  sys->format = format;
  auto fail = [&](int rc) {
    lb_system_destroy(sys);
    return rc;
  };
  PhaseClock clk(c.st);
  const auto t0 = std::chrono::steady_clock::now();
  int rc;
  // device memory (admission against what is free plus what the pool holds spare)
  PoolBuf da, dH, dcoef, dh, dli, dlv;
  const int64_t nl = (a->kind == LB_A_LOWRANK && a->nP) ? a->lp_ptr[a->nP] : 0;
  if (format == LB_DENSE) {
    const size_t need = 16 * mm + 8 * mm * (keep_parts ? 3 : 1) + 64 * (size_t)M;
    size_t fr = 0, tot = 0;
    LB_TRY_CUDA(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    fr += pool_spare(c.pool);
    if (need > fr) {
      delete sys;
      lbi::set_error("lb_assemble: needs %zu bytes of device memory, %zu free", need, fr);
      return LB_ENOMEM;
    }
    PoolBuf dA, dQ, dR, dK;
    if ((rc = da.alloc(c, 16 * mm, "a")) != LB_OK || (rc = dA.alloc(c, 8 * mm, "A")) != LB_OK ||
        (rc = dK.alloc(c, 8 * (size_t)M, "K")) != LB_OK ||
        (keep_parts && ((rc = dQ.alloc(c, 8 * mm, "Q")) != LB_OK || (rc = dR.alloc(c, 8 * mm, "R")) != LB_OK)))
      return fail(rc);
    sys->A = dA.as<double>();
    sys->K = dK.as<double>();
    sys->Q = dQ.as<double>();
    sys->R = dR.as<double>();
    dA.release();
    dK.release();
    dQ.release();
    dR.release();
  }
  if (nl > 0) {
    if ((rc = dli.alloc(c, 8 * (size_t)nl, "channel indices")) != LB_OK ||
        (rc = dlv.alloc(c, 16 * (size_t)nl, "channel values")) != LB_OK)
      return fail(rc);
  }
  if (H) {
    if ((rc = dH.alloc(c, 16 * (size_t)N * N, "H")) != LB_OK || (rc = dcoef.alloc(c, 16 * (size_t)M, "coef")) != LB_OK ||
        (rc = dh.alloc(c, 8 * (size_t)M, "h")) != LB_OK)
      return fail(rc);
  }
  sys->ms[LB_PHASE_ALLOC] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  // inputs to the device
  clk.mark(LB_PHASE_H2D);
  cudaError_t e = cudaSuccess;
  if (H) e = cudaMemcpyAsync(dH.p, H, 16 * (size_t)N * N, cudaMemcpyHostToDevice, c.st);
  if (e == cudaSuccess && nl > 0) {
    e = cudaMemcpyAsync(dli.p, a->lp_idx, 8 * (size_t)nl, cudaMemcpyHostToDevice, c.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlv.p, a->lp_val, 16 * (size_t)nl, cudaMemcpyHostToDevice, c.st);
  }
  if (e == cudaSuccess && format == LB_DENSE && a->kind == LB_A_DENSE)
    e = lbi::upload_hermitian(reinterpret_cast<const double2*>(a->a), da.as<double2>(), M, c.st);
  if (e != cudaSuccess) return fail(lbi::cuda_fail(e, "lb_assemble: copy inputs"));
  // kernels
  clk.mark(LB_PHASE_KERNELS);
  if (H) {
    e = lbi::expand(b->view(), dH.as<double2>(), dcoef.as<double2>(), c.st);
    if (e == cudaSuccess) e = real_part(dcoef.as<double2>(), dh.as<double>(), M, c.st);
  }
  if (e == cudaSuccess && format == LB_DENSE && a->kind == LB_A_LOWRANK) {
    e = cudaMemsetAsync(da.p, 0, 16 * mm, c.st);
    for (int p = 0; p < a->nP && e == cudaSuccess; ++p) {
      const int64_t n = a->lp_ptr[p + 1] - a->lp_ptr[p];
      if (n == 0) continue;
      const int64_t pairs = n * n;
      k_lowrank_add<<<(unsigned)((pairs + 255) / 256), 256, 0, c.st>>>(
          M, (int)n, dli.as<int64_t>() + a->lp_ptr[p], dlv.as<double2>() + a->lp_ptr[p], a->gamma[p], da.as<double2>());
      lbi::note_launch(1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && format == LB_DENSE)
    e = lbi::assemble_dense(b->view(), H ? dh.as<double>() : nullptr, da.as<double2>(), sys->A, sys->Q, sys->R,
                            sys->K, algorithm, c.st);
  if (e == cudaSuccess && format == LB_CSR) {
    static const int64_t zero_ptr[1] = {0};
    e = lbi::assemble_lowrank_csr(b->view(), H ? dh.as<double>() : nullptr, a->nP, a->gamma,
                                  a->nP ? a->lp_ptr : zero_ptr, dli.as<int64_t>(), dlv.as<double2>(), &sys->csr, c.st);
    sys->K = sys->csr.K;
  }
  clk.mark(LB_PHASE_D2H);
  clk.mark(LB_PHASE_FREE);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      lbi::set_error("lb_assemble: device memory exhausted");
      return fail(LB_ENOMEM);
    }
    return fail(lbi::cuda_fail(e, "lb_assemble"));
  }
  // the staging buffers go back to the pool here (stream-ordered)
  const auto t1 = std::chrono::steady_clock::now();
  da.free_now();
  clk.mark(LB_PHASES);
  cudaStreamSynchronize(c.st);
  clk.read(sys->ms, LB_PHASE_H2D, LB_PHASES);
  sys->ms[LB_PHASE_FREE] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  *out = sys;
  return LB_OK;
}

int lb_system_timings(const lb_system_t* s, double* ms) {
  LB_REQUIRE(s && ms, "lb_system_timings: NULL argument");
  for (int i = 0; i < LB_PHASES; ++i) ms[i] = s->ms[i];
  return LB_OK;
}

int lb_system_info(const lb_system_t* s, int* format, int64_t* M, int64_t* nnz) {
  LB_REQUIRE(s != nullptr, "lb_system_info: NULL handle");
  if (format) *format = s->format;
  if (M) *M = s->M;
  if (nnz) *nnz = s->format == LB_CSR ? s->csr.nnz : s->M * s->M;
  return LB_OK;
}

int lb_system_get_csr(const lb_system_t* s, int64_t* rowptr, int32_t* col, double* val) {
  LB_REQUIRE(s != nullptr, "lb_system_get_csr: NULL handle");
  LB_REQUIRE(s->format == LB_CSR, "lb_system_get_csr: the system is dense");
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_system_get_csr");
  if (rowptr)
    LB_TRY_CUDA(cudaMemcpyAsync(rowptr, s->csr.rowptr, 8 * (size_t)(s->M + 1), cudaMemcpyDeviceToHost, c.st), "copy");
  if (col) LB_TRY_CUDA(cudaMemcpyAsync(col, s->csr.col, 4 * (size_t)s->csr.nnz, cudaMemcpyDeviceToHost, c.st), "copy");
  if (val) LB_TRY_CUDA(cudaMemcpyAsync(val, s->csr.val, 8 * (size_t)s->csr.nnz, cudaMemcpyDeviceToHost, c.st), "copy");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_system_get_csr");
  return LB_OK;
}

int lb_system_destroy(lb_system_t* s) {
  if (!s) return LB_OK;
  HostCtx c;
  const bool have = host_ctx(&c) == cudaSuccess;
  if (have) {  // pool memory, returned in the order of the library stream
    pool_free(s->A, c.st);
    pool_free(s->Q, c.st);
    pool_free(s->R, c.st);
    if (s->format == LB_DENSE) pool_free(s->K, c.st);
    pool_free(s->A32, c.st);
    pool_free(s->Abf, c.st);
    pool_free(s->scale, c.st);
  }
  cudaFree(s->csr.rowptr);
  cudaFree(s->csr.col);
  cudaFree(s->csr.val);
  cudaFree(s->csr.K);
  cudaFree(s->csr32);
  delete s;
  return LB_OK;
}

}  // extern "C"

namespace {

// File format of lb_system_save: a 64-byte header, then the parts.
struct SysFileHeader {
  char magic[8];     // "LBSYS001"
  int64_t N, M;
  int64_t parts;     // bit 0 A, 1 K, 2 Q, 3 R
  int64_t version;   // 1
  int64_t reserved[3];
};
static_assert(sizeof(SysFileHeader) == 64, "header is 64 bytes");

constexpr size_t kFileChunk = size_t(64) << 20;  // bytes per host bounce

bool write_device(FILE* f, const double* d, size_t count, std::string& err) {
  std::vector<char> buf(std::min(kFileChunk, 8 * count + 1));
  size_t done = 0;
  while (done < 8 * count) {
    const size_t n = std::min(buf.size(), 8 * count - done);
    const cudaError_t e = cudaMemcpy(buf.data(), reinterpret_cast<const char*>(d) + done, n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return false;
    }
    if (fwrite(buf.data(), 1, n, f) != n) {
      err = "short write";
      return false;
    }
    done += n;
  }
  return true;
}

bool read_device(FILE* f, double* d, size_t count, std::string& err) {
  std::vector<char> buf(std::min(kFileChunk, 8 * count + 1));
  size_t done = 0;
  while (done < 8 * count) {
    const size_t n = std::min(buf.size(), 8 * count - done);
    if (fread(buf.data(), 1, n, f) != n) {
      err = "file is truncated";
      return false;
    }
    const cudaError_t e = cudaMemcpy(reinterpret_cast<char*>(d) + done, buf.data(), n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return false;
    }
    done += n;
  }
  return true;
}

}  // namespace

extern "C" {

int lb_system_save(const lb_system_t* s, const char* path) {
  LB_REQUIRE(s && path, "lb_system_save: NULL argument");
  if (s->format != LB_DENSE) {
    lbi::set_error("lb_system_save: only dense systems are written to files");
    return LB_EUNSUPPORTED;
  }
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_system_save");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_system_save");
  FILE* f = fopen(path, "wb");
  LB_REQUIRE(f != nullptr, "lb_system_save: cannot open %s for writing", path);
  SysFileHeader h{};
  memcpy(h.magic, "LBSYS001", 8);
  h.N = s->basis->N;
  h.M = s->M;
  h.parts = (s->A ? 1 : 0) | (s->K ? 2 : 0) | (s->Q ? 4 : 0) | (s->R ? 8 : 0);
  h.version = 1;
  std::string err;
  const size_t mm = (size_t)s->M * (size_t)s->M;
  bool ok = fwrite(&h, sizeof h, 1, f) == 1;
  if (!ok) err = "short write";
  if (ok && s->A) ok = write_device(f, s->A, mm, err);
  if (ok && s->K) ok = write_device(f, s->K, (size_t)s->M, err);
  if (ok && s->Q) ok = write_device(f, s->Q, mm, err);
  if (ok && s->R) ok = write_device(f, s->R, mm, err);
  if (fclose(f) != 0 && ok) {
    ok = false;
    err = "close failed";
  }
  if (!ok) {
    cudaGetLastError();
    lbi::set_error("lb_system_save: %s: %s", path, err.c_str());
    return LB_EINVAL;
  }
  return LB_OK;
}

int lb_system_load(const lb_basis_t* b, const char* path, lb_system_t** out) {
  LB_REQUIRE(b && path && out, "lb_system_load: NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  LB_REQUIRE(f != nullptr, "lb_system_load: cannot open %s", path);
  SysFileHeader h{};
  const bool hdr = fread(&h, sizeof h, 1, f) == 1;
  if (!hdr || memcmp(h.magic, "LBSYS001", 8) != 0 || h.version != 1 || h.N != b->N || h.M != b->M ||
      !(h.parts & 1) || !(h.parts & 2)) {
    fclose(f);
    lbi::set_error("lb_system_load: %s is not a system file for N = %d", path, b->N);
    return LB_EINVAL;
  }
  const size_t mm = (size_t)b->M * (size_t)b->M;
  int rc;
  HostCtx c;
  const cudaError_t ec = host_ctx(&c);
  if (ec != cudaSuccess) {
    fclose(f);
    return lbi::cuda_fail(ec, "lb_system_load: library stream");
  }
  PoolBuf dA, dK, dQ, dR;
  if ((rc = dA.alloc(c, 8 * mm, "A")) != LB_OK || (rc = dK.alloc(c, 8 * (size_t)b->M, "K")) != LB_OK ||
      ((h.parts & 4) && (rc = dQ.alloc(c, 8 * mm, "Q")) != LB_OK) ||
      ((h.parts & 8) && (rc = dR.alloc(c, 8 * mm, "R")) != LB_OK)) {
    fclose(f);
    return rc;
  }
  const cudaError_t es = cudaStreamSynchronize(c.st);  // the copies below run on the legacy stream
  if (es != cudaSuccess) {
    fclose(f);
    return lbi::cuda_fail(es, "lb_system_load");
  }
  std::string err;
  bool ok = read_device(f, dA.as<double>(), mm, err) && read_device(f, dK.as<double>(), (size_t)b->M, err);
  if (ok && (h.parts & 4)) ok = read_device(f, dQ.as<double>(), mm, err);
  if (ok && (h.parts & 8)) ok = read_device(f, dR.as<double>(), mm, err);
  fclose(f);
  if (!ok) {
    cudaGetLastError();
    lbi::set_error("lb_system_load: %s: %s", path, err.c_str());
    return LB_EINVAL;
  }
  lb_system* s = new lb_system;
  s->basis = b;
  s->M = b->M;
  s->A = static_cast<double*>(dA.release());
  s->K = static_cast<double*>(dK.release());
  s->Q = static_cast<double*>(dQ.release());
  s->R = static_cast<double*>(dR.release());
  *out = s;
  return LB_OK;
}

int lb_system_get(const lb_system_t* s, int part, double* out) {
  LB_REQUIRE(s && out, "lb_system_get: NULL argument");
  const double* src = part == LB_SYS_A ? s->A : part == LB_SYS_Q ? s->Q : part == LB_SYS_R ? s->R
                      : part == LB_SYS_K ? s->K : nullptr;
  LB_REQUIRE(src != nullptr, "lb_system_get: part %d not available%s", part,
             s->format == LB_CSR && part != LB_SYS_K ? " (CSR system: use lb_system_get_csr)" : "");
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_system_get");
  const size_t n = part == LB_SYS_K ? (size_t)s->M : (size_t)s->M * (size_t)s->M;
  LB_TRY_CUDA(cudaMemcpyAsync(out, src, 8 * n, cudaMemcpyDeviceToHost, c.st), "lb_system_get");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_system_get");
  return LB_OK;
}

static int spectrum_status(int rc, cudaError_t ce, const char* what) {
  if (rc == 0) return LB_OK;
  if (rc == 1) {
    lbi::set_error("%s: the dense nonsymmetric eigensolver (libcusolver) could not be loaded", what);
    return LB_EUNSUPPORTED;
  }
  if (rc == 3) return lbi::cuda_fail(ce, what);
  lbi::set_error("%s: the eigensolver reported a failure", what);
  return LB_ECUDA;
}

int lb_spectrum(const double* A, int64_t M, double* eig, void* stream) {
  LB_REQUIRE(A && eig, "lb_spectrum: NULL argument");
  LB_REQUIRE(M >= 1, "lb_spectrum: M = %lld", (long long)M);
  cudaError_t ce = cudaSuccess;
  const int rc = lbi::spectrum_dense(A, M, reinterpret_cast<double2*>(eig), S(stream), &ce);
  return spectrum_status(rc, ce, "lb_spectrum");
}

int lb_spectrum_density(const double* eig, int64_t n, const double* box, int nre, int nim, double* density,
                        void* stream) {
  LB_REQUIRE(eig && box && density, "lb_spectrum_density: NULL argument");
  LB_REQUIRE(n >= 0 && nre >= 1 && nim >= 1, "lb_spectrum_density: bad sizes");
  LB_REQUIRE(std::isfinite(box[0]) && std::isfinite(box[1]) && std::isfinite(box[2]) && std::isfinite(box[3]) &&
                 box[1] > box[0] && box[3] > box[2],
             "lb_spectrum_density: empty or non-finite box");
  LB_TRY_CUDA(lbi::spectrum_density(reinterpret_cast<const double2*>(eig), n, box, nre, nim, density, S(stream)),
              "lb_spectrum_density");
  return LB_OK;
}

int lb_system_spectrum(const lb_system_t* s, double* eig) {
  LB_REQUIRE(s && eig, "lb_system_spectrum: NULL argument");
  LB_REQUIRE(s->format == LB_DENSE && s->A, "lb_system_spectrum: dense systems only");
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_system_spectrum");
  PoolBuf w;
  int rc;
  if ((rc = w.alloc(c, 16 * (size_t)s->M, "eigenvalues")) != LB_OK) return rc;
  cudaError_t ce = cudaSuccess;
  rc = spectrum_status(lbi::spectrum_dense(s->A, s->M, w.as<double2>(), c.st, &ce), ce, "lb_system_spectrum");
  if (rc != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemcpyAsync(eig, w.p, 16 * (size_t)s->M, cudaMemcpyDeviceToHost, c.st), "lb_system_spectrum");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_system_spectrum");
  return LB_OK;
}

static int integrate_steps(lb_system_t* s, int precision, int correct_every, const double* v0, double dt,
                           int64_t n, int64_t snap_every, double* v_out);

int lb_integrate(lb_system_t* s, int precision, int correct_every, const double* v0, double t, double dt,
                 int64_t snap_every, double* v_out) {
  LB_REQUIRE(s && v0 && v_out, "lb_integrate: NULL argument");
  LB_REQUIRE(dt > 0 && t >= 0 && std::isfinite(t) && std::isfinite(dt), "lb_integrate: bad t or dt");
  LB_REQUIRE(correct_every >= 0 && snap_every >= 0, "lb_integrate: negative correction or snapshot period");
  const double nr = std::nearbyint(t / dt);
  const int64_t n = (int64_t)nr;
  LB_REQUIRE(std::fabs(nr * dt - t) <= 1e-9 * t, "lb_integrate: t = %g is not a multiple of dt = %g", t, dt);
  LB_REQUIRE(snap_every == 0 || n % snap_every == 0, "lb_integrate: %lld steps are not a multiple of snap_every = %lld",
             (long long)n, (long long)snap_every);
  return integrate_steps(s, precision, correct_every, v0, dt, n, snap_every, v_out);
}

int lb_integrate_resume(lb_system_t* s, int precision, int correct_every, double* v, double dt, int64_t nsteps) {
  LB_REQUIRE(s && v, "lb_integrate_resume: NULL argument");
  LB_REQUIRE(dt > 0 && std::isfinite(dt) && nsteps >= 0 && correct_every >= 0,
             "lb_integrate_resume: bad dt, step count or correction period");
  return integrate_steps(s, precision, correct_every, v, dt, nsteps, 0, v);
}

static int integrate_steps(lb_system_t* s, int precision, int correct_every, const double* v0, double dt,
                           int64_t n, int64_t snap_every, double* v_out) {
  const int64_t M = s->M;
  const size_t mm = (size_t)M * (size_t)M;
  HostCtx c;
  LB_TRY_CUDA(host_ctx(&c), "lb_integrate: library stream");
  int rc;
  if (s->format == LB_CSR) {
    LB_REQUIRE(precision == LB_FP64 || precision == LB_FP32, "lb_integrate: CSR precision = %d", precision);
    LB_REQUIRE(snap_every == 0 || correct_every == 0 || precision == LB_FP64 || snap_every % correct_every == 0,
               "lb_integrate: on a CSR system snap_every must be a multiple of correct_every");
  } else {
    LB_REQUIRE(precision == LB_FP64 || precision == LB_FP32 || precision == LB_BF16, "lb_integrate: precision = %d",
               precision);
  }
  const void* Ap = s->format == LB_CSR ? (const void*)s->csr.val : (const void*)s->A;
  if (precision == LB_FP32 && s->format == LB_CSR) {
    if (!s->csr32) {
      DevBuf b32;
      if ((rc = alloc_or_enomem(b32, sizeof(float) * (size_t)(s->csr.nnz + 1), "FP32 values")) != LB_OK) return rc;
      LB_TRY_CUDA(lbi::to_f32(s->csr.nnz, s->csr.val, b32.as<float>(), c.st), "pack FP32 values");
      s->csr32 = static_cast<float*>(b32.release());
    }
    Ap = s->csr32;
  } else if (precision == LB_FP32) {
    if (!s->A32) {
      PoolBuf b32;
      if ((rc = b32.alloc(c, 4 * mm, "A32")) != LB_OK) return rc;
      LB_TRY_CUDA(lbi::pack_fp32(M, s->A, b32.as<float>(), c.st), "pack fp32");
      s->A32 = static_cast<float*>(b32.release());
    }
    Ap = s->A32;
  } else if (precision == LB_BF16) {
    if (!s->Abf) {
      PoolBuf bb, sc;
      if ((rc = bb.alloc(c, 2 * mm, "Abf16")) != LB_OK) return rc;
      if ((rc = sc.alloc(c, 4 * (size_t)M, "row scales")) != LB_OK) return rc;
      LB_TRY_CUDA(lbi::pack_bf16(M, s->A, bb.as<uint16_t>(), sc.as<float>(), c.st), "pack bf16");
      s->Abf = static_cast<uint16_t*>(bb.release());
      s->scale = static_cast<float*>(sc.release());
    }
    Ap = s->Abf;
  }
  const int64_t nsnap = snap_every ? n / snap_every : 0;
  PoolBuf dv, work, dsn;
  if ((rc = dv.alloc(c, 8 * (size_t)M, "v")) != LB_OK) return rc;
  if ((rc = work.alloc(c, lbi::rk4_workspace_bytes(M), "RK4 workspace")) != LB_OK) return rc;
  if (nsnap > 0 && (rc = dsn.alloc(c, 8 * (size_t)M * nsnap, "snapshots")) != LB_OK) return rc;
  LB_TRY_CUDA(cudaMemcpyAsync(dv.p, v0, 8 * (size_t)M, cudaMemcpyHostToDevice, c.st), "copy v0");
  if (s->format == LB_CSR) {
    const int64_t seg = nsnap > 0 ? snap_every : n;
    const int64_t nseg = nsnap > 0 ? nsnap : 1;
    for (int64_t i = 0; i < nseg; ++i) {
      LB_TRY_CUDA(lbi::rk4_csr(M, precision, s->csr.rowptr, s->csr.col, Ap, s->csr.val, correct_every, s->csr.K,
                               dv.as<double>(), dt, seg, work.p, c.st),
                  "RK4 (CSR)");
      if (nsnap > 0)
        LB_TRY_CUDA(cudaMemcpyAsync(dsn.as<double>() + (size_t)i * M, dv.p, 8 * (size_t)M, cudaMemcpyDeviceToDevice,
                                    c.st),
                    "snapshot");
    }
  } else {
    LB_TRY_CUDA(lbi::rk4_dense(M, precision, Ap, s->scale, s->A, correct_every, s->K, dv.as<double>(), dt, n,
                               nsnap > 0 ? dsn.as<double>() : nullptr, nsnap > 0 ? snap_every : 0, work.p, c.st),
                "RK4");
  }
  if (nsnap > 0)
    LB_TRY_CUDA(cudaMemcpyAsync(v_out, dsn.p, 8 * (size_t)M * nsnap, cudaMemcpyDeviceToHost, c.st), "copy snapshots");
  else
    LB_TRY_CUDA(cudaMemcpyAsync(v_out, dv.p, 8 * (size_t)M, cudaMemcpyDeviceToHost, c.st), "copy v");
  LB_TRY_CUDA(cudaStreamSynchronize(c.st), "lb_integrate");
  return LB_OK;
}

}  // extern "C"

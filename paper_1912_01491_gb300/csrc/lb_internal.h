// lb_internal.h -- declarations shared by the translation units of
// liblindblad.so (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lindblad.h"
#include "su_n.cuh"

// Device-resident basis: the lexicographic pair table and the per-level
// constants (layout of d_tab: c[N], lc[N], c2[N], inv[N+1]).
struct lb_basis {
  int N;
  int64_t P, M;
  int32_t* d_pair_ab = nullptr;  // P
  double* d_tab = nullptr;       // 4N + 1
  lb::BasisView view() const {
    lb::BasisView v;
    v.N = N; v.P = P; v.M = M;
    v.pair_ab = d_pair_ab;
    v.c = d_tab;
    v.lc = d_tab + N;
    v.c2 = d_tab + 2 * N;
    v.inv = d_tab + 3 * N;
    return v;
  }
};

namespace lbi {

// dense assembly keeps per-block tables of O(N) entries in shared memory
constexpr int kMaxDenseN = 512;

void set_error(const char* fmt, ...);
void note_launch(int n);
int cuda_fail(cudaError_t e, const char* what);

// kernel (a) and friends (lb_basis.cu)
cudaError_t build_tables(int N, int32_t* pair_ab, double* tab, cudaStream_t st);
cudaError_t structure_count(const lb::BasisView& B, int which, int64_t* per_m, cudaStream_t st);
cudaError_t structure_fill(const lb::BasisView& B, int which, const int64_t* offsets,
                           int32_t* idx3, double* val, cudaStream_t st);
cudaError_t expand(const lb::BasisView& B, const double2* A, double2* coef, cudaStream_t st);
cudaError_t rho(const lb::BasisView& B, const double* v, double2* out, cudaStream_t st);
// sum_i v_i F_i (rho without the 1/N identity part)
cudaError_t synth(const lb::BasisView& B, const double* v, double2* out, cudaStream_t st);

// dense assembly (lb_assemble.cu)
constexpr int kAssembleKernels = 7;
// Copy a Hermitian M x M a from host memory to the device: only the upper
// triangle crosses the link (one 2D copy per row block), the strict lower
// triangle is then written on the device as a_kj = conj(a_jk).
cudaError_t upload_hermitian(const double2* host, double2* dev, int64_t M, cudaStream_t st);
// ev (kAssembleKernels + 1 events, optional): the kernels run in sequence
// on st with an event between them.
cudaError_t assemble_dense(const lb::BasisView& B, const double* h, const double2* a,
                           double* A, double* Q, double* R, double* K, int algorithm, cudaStream_t st,
                           cudaEvent_t* ev = nullptr);
const char* assemble_kernel_name(int i);
cudaError_t join_terms(const lb::BasisView& B, unsigned long long* d_count, cudaStream_t st);

// sparse assembly (lb_csr.cu)
struct CsrOut {
  int64_t M = 0, nnz = 0, terms = 0;
  int64_t* rowptr = nullptr;  // M + 1
  int32_t* col = nullptr;     // nnz, sorted within rows
  double* val = nullptr;      // nnz
  double* K = nullptr;        // M
};
// Eigenvalues w[0..M) (complex) of the dense row-major M x M matrix A by the
// library's nonsymmetric eigensolver; 0 ok, 1 solver not found, 2 solver
// failure, 3 CUDA error (*ce).
int spectrum_dense(const double* A, int64_t M, double2* w, cudaStream_t st, cudaError_t* ce);
// Eigenvalues E (ascending) and eigenvectors (row j of Ub) of the Hermitian
// row-major N x N H; status as spectrum_dense.
int hermitian_eig(const double2* H, int N, double* E, double2* Ub, cudaStream_t st, cudaError_t* ce);
// Eigenvalue density on an nre x nim grid over box = {re_lo, re_hi, im_lo, im_hi}.
cudaError_t spectrum_density(const double2* w, int64_t n, const double* box, int nre, int nim, double* dens,
                             cudaStream_t st);
// off[0..n] = exclusive prefix sums of n int64 counts (off[n] = total);
// synchronous with respect to st.
cudaError_t exclusive_scan(const int64_t* counts, int64_t* off, int64_t n, cudaStream_t st);
cudaError_t assemble_lowrank_csr(const lb::BasisView& B, const double* h, int nP, const double* gamma_host,
                                 const int64_t* lp_ptr_host, const int64_t* lp_idx, const double2* lp_val,
                                 CsrOut* out, cudaStream_t st);
cudaError_t rk4_csr(int64_t M, int precision, const int64_t* rowptr, const int32_t* col, const void* val,
                    const double* val64, int correct_every, const double* K, double* v, double dt, int64_t nsteps,
                    void* work, cudaStream_t st);
cudaError_t to_f32(int64_t n, const double* x, float* y, cudaStream_t st);
cudaError_t rk4_csr_td(int64_t M, const int64_t* rowptr, const int32_t* col, const double* val,
                       const int64_t* rowptr1, const int32_t* col1, const double* val1, const double* K, int nseg,
                       const double* seg_start, const double* seg_eps, double T, double t0, double* v, double dt,
                       int64_t nsteps, void* work, cudaStream_t st);

// RK4 (lb_rk4.cu)
cudaError_t pack_fp32(int64_t M, const double* A, float* A32, cudaStream_t st);
cudaError_t pack_bf16(int64_t M, const double* A, uint16_t* Ab, float* scale, cudaStream_t st);
size_t rk4_workspace_bytes(int64_t M);
cudaError_t rk4_dense(int64_t M, int precision, const void* Ap, const float* scale,
                      const double* A64, int correct_every, const double* K, double* v,
                      double dt, int64_t nsteps, double* snaps, int64_t snap_every,
                      void* work, cudaStream_t st);

// batched form (lb_batch.cu): one realization of the cluster-persistent RK4
struct BatchItem {
  int64_t M;
  const float* A32;   // M x M
  const double* A64;  // M x M (for the correction) or null
  const double* K;    // M
  double* v;          // M, in/out
};
constexpr int kBatchMaxN = 64;

// propagator form (lb_prop.cu): batched Y = B + alpha A G over square
// M x M row-major matrices (B may be null), one launch over the 64 x 64
// tiles of every job; and batched FP64 y = K + alpha A x.
struct GemmTile {
  int job, ti, tj;
};
template <class T>
struct GemmJob {
  int64_t M;
  const T* A;
  const T* G;
  const T* B;
  T* Y;
  T alpha;
};
struct GemvJob {
  int64_t M;
  const double* A;
  const double* x;
  const double* K;
  double* y;
  double alpha;
};
// scratch: device memory for the job and tile lists (batch_gemm_scratch_bytes);
// both calls return after their kernel has finished on st.
template <class T>
cudaError_t batch_gemm(const std::vector<GemmJob<T>>& jobs, void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t batch_gemm_scratch_bytes(const std::vector<int64_t>& Ms);
cudaError_t batch_gemv64(const std::vector<GemvJob>& jobs, void* scratch, size_t scratch_bytes, cudaStream_t st);
cudaError_t add32(const float* A, const float* R, float* Y, int64_t n, cudaStream_t st);
cudaError_t add64(const double* A, const double* R, double* Y, int64_t n, cudaStream_t st);
// single system (lb_prop.cu): D' (FP64, or FP32 with R32 = D' - A) and c'
// for step h; then nsteps propagator steps of R states (V: R x M, FP64)
size_t propagator_form_workspace_bytes(int64_t M, int precision);
cudaError_t propagator_form(int64_t M, int precision, const double* A64, const float* A32, const double* K, double h,
                            void* Dp, float* R32, double* cp, void* work, size_t work_bytes, cudaStream_t st);
// FP64 checks (lb_steady.cu)
size_t steady_workspace_bytes(int64_t M, int restart);
// The Hamiltonian preconditioner of the steady-state GMRES (lb_steady.cu):
// basis, eigenvalues E and eigenvectors (rows of Ub) of H, shift sigma and
// scratch (X, T: N x N complex; coef: M complex; z: M).
struct PcView {
  lb::BasisView B;
  double* E;
  double2 *Ub, *X, *T, *coef;
  double* z;
  double sigma;
};
size_t steady_pc_workspace_bytes(int N, int64_t M, int restart);
int steady_pc_setup(const lb::BasisView& B, const double2* H, const double* A, double sigma, int restart,
                    void* work, PcView* pc, cudaStream_t st, cudaError_t* ce);
cudaError_t steady_state(int64_t M, const double* A, const double* K, double* v, double tol, int max_iter,
                         int restart, double* rel_res, int* iters, void* work, cudaStream_t st,
                         const PcView* pc = nullptr);
size_t rho_checks_workspace_bytes(int N);
cudaError_t rho_checks(const lb::BasisView& B, const double* V, int64_t nsnap, double delta, double* out_host,
                       void* work, cudaStream_t st);
size_t propagate_workspace_bytes(int64_t M, int R, int precision);
cudaError_t propagate(int64_t M, int R, int precision, const void* Dp, const float* R32, const double* A64,
                      const double* cp, int correct_every, double* V, double h, int64_t nsteps, double* snaps,
                      int64_t snap_every, void* work, cudaStream_t st);
// Cluster size the batched kernel uses for dimension M when none is chosen:
// the smallest of {1, 2, 4, 8, 16} whose slice of the FP32 matrix stays
// resident in shared memory, else 16.
int batch_default_cluster(int64_t M);
// Enqueue one launch over n items (host array) on st; the item list and work
// counter are allocated from pool (stream-ordered) and freed after the launch.
cudaError_t batch_launch_async(const BatchItem* items, int n, int C, int64_t nsteps, double dt, int correct_every,
                               cudaMemPool_t pool, cudaStream_t st);

}  // namespace lbi

/*
 * lindblad.h -- C ABI of liblindblad.so: the transformation of a GKSL
 * (Lindblad) generator into the real linear system dv/dt = (Q + R) v + K over
 * the generalized Gell-Mann basis, and its RK4 integration, on one sm_103a GPU.
 *
 * Method: Meyerov et al., "Transforming Lindblad Equations into Systems of
 * Real-Valued Linear Equations" -- Sec. 2 (basis, Eqs. (02)-(09)), Table 1
 * (Data Preparation steps 2.1-2.6, ODE Integration steps 3.1-3.2), Sec. 4.
 *
 * Conventions (all functions):
 *   - N is the Hilbert-space dimension, M = N*N - 1, P = N*(N-1)/2.
 *   - Basis order, 0-based: S_ab (pairs a<b, lexicographic) at 0..P-1,
 *     J_ab at P..2P-1, D_l (l = 1..N-1) at 2P..M-1.  D_l is the Hermitian,
 *     orthonormal matrix (sum_{k<l} E_kk - l E_ll)/sqrt(l(l+1)).
 *   - Complex arrays are interleaved (re, im) doubles; matrices are row-major.
 *   - The Kossakowski matrix `a` follows the index convention of Eqs. (08)
 *     and (09): L_D(rho) = sum_jk a_jk (F_j rho F_k - 1/2 {F_k F_j, rho}),
 *     i.e. a = K^T for the matrix K_mn of Eq. (1); a must be Hermitian and is
 *     passed as the full M x M matrix (both triangles; lb_assemble reads only
 *     the upper one for M > 2048).
 *   - Every function returns an int status (LB_OK = 0 on success).  On error
 *     nothing is half-written to caller buffers except where stated, no
 *     exception or abort crosses the ABI, and lb_last_error() returns a
 *     thread-local description of the last failure on the calling thread.
 *   - "device" pointers are CUDA device addresses on the current device;
 *     "host" pointers are ordinary (pageable or pinned) host memory.  Stream
 *     arguments are cudaStream_t values passed as void* (NULL = legacy
 *     default stream); device-pointer functions are asynchronous with
 *     respect to the host unless stated.
 *   - Caller-owned buffers are only read (inputs) or written (outputs) during
 *     the call and its stream work; the library keeps no reference to them.
 *   - Handles (lb_basis_t, lb_system_t) own device memory; they are not
 *     thread-safe: use one handle per host thread or serialise calls.
 */
#ifndef LINDBLAD_H
#define LINDBLAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LB_OK 0
#define LB_EINVAL 1         /* bad argument (size, pointer, range)           */
#define LB_ENOMEM 2         /* device memory refused (admission or cudaMalloc) */
#define LB_ECUDA 3          /* a CUDA runtime call or kernel failed           */
#define LB_ETIMEOUT 4       /* a bounded device-side wait ran out              */
#define LB_EUNSUPPORTED 5   /* valid request that this build does not handle   */
#define LB_EAGAIN 6         /* result not ready yet                            */

/* structure tensors (Eq. (05)) */
#define LB_F 0
#define LB_D 1

/* storage precision of the integration matrix A = Q + R */
#define LB_FP64 0
#define LB_FP32 1
#define LB_BF16 2

/* parts of an assembled system */
#define LB_SYS_A 0
#define LB_SYS_Q 1
#define LB_SYS_R 2
#define LB_SYS_K 3

/* storage format of an assembled system (lb_assemble) */
#define LB_DENSE 0
#define LB_CSR 1

/* kinds of Kossakowski matrix (lb_kossakowski) */
#define LB_A_DENSE 0
#define LB_A_LOWRANK 1

/* phases of a host-buffer call (lb_system_timings) */
#define LB_PHASE_ALLOC 0    /* host wall time of the device allocations (library pool) */
#define LB_PHASE_H2D 1      /* host -> device copies of the inputs */
#define LB_PHASE_KERNELS 2  /* expansion of H and assembly kernels */
#define LB_PHASE_D2H 3      /* device -> host copies (none in lb_assemble) */
#define LB_PHASE_FREE 4     /* return of the staging buffers to the pool */
#define LB_PHASES 5

typedef struct lb_basis lb_basis_t;
typedef struct lb_system lb_system_t;

/* Thread-local text of the last error on this thread ("" if none). */
const char *lb_last_error(void);

/* ABI version (major * 100 + minor). */
int lb_version(void);

/* ------------------------------------------------------------------------
 * a1 -- basis and structure constants.  Table 1 step 2.2, Sec. 4 item 2.2:
 * only the O(N^3) nonzero f_mns, d_mns (Eq. (05)) exist, each O(1) to
 * compute; they are enumerated by index arithmetic, never stored densely.
 * --------------------------------------------------------------------- */

/* Build the device index tables of the basis for dimension N (2 <= N <= 4096):
 * the lexicographic pair table and c_l = 1/sqrt(l(l+1)).  *out is owned by
 * the caller and released with lb_basis_destroy; it must outlive every
 * lb_system_t assembled from it.  Synchronous.  LB_EINVAL for bad N,
 * LB_ENOMEM / LB_ECUDA on device failure. */
int lb_basis_create(int N, void *stream, lb_basis_t **out);
int lb_basis_destroy(lb_basis_t *b);

/* N, M, P of a basis (any output pointer may be NULL). */
int lb_basis_dims(const lb_basis_t *b, int *N, int64_t *M, int64_t *P);

/* Label of basis index i: type 'S', 'J' (pair j<k) or 'D' (j = k = l). */
int lb_basis_label(const lb_basis_t *b, int64_t i, char *type, int *j, int *k);

/* Number of canonical nonzero triples (m <= n <= s) of f (which = LB_F) or
 * d (LB_D) of the basis, counted on the GPU by kernel (a) without storing
 * them.  Synchronous (default stream). */
int lb_structure_count(const lb_basis_t *b, int which, int64_t *nnz);

/* Kernel (a): enumerate the canonical nonzero triples, sorted
 * lexicographically by (m, n, s), into caller DEVICE buffers idx3 (3*nnz
 * int32) and val (nnz doubles) by a count pass, an exclusive scan and a fill
 * pass.  capacity is the buffer length in triples; *nnz always receives the
 * count, and LB_EINVAL is returned (buffers untouched) if capacity < nnz.
 * Synchronous with respect to `stream`. */
int lb_structure_export(const lb_basis_t *b, int which, int32_t *idx3, double *val,
                        int64_t capacity, int64_t *nnz, void *stream);

/* lb_structure_export without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory per
 * call -- processes whose framework's caching allocator has reserved the
 * device memory (a cudaMalloc there fails or fragments the pool, and a
 * cudaFree synchronizes the whole device), and real-time or embedded callers
 * that reserve all memory at start-up.  Arguments, outputs, ordering and
 * error behaviour are those of lb_structure_export; the caller passes the
 * basis and the output buffers.  The scratch (per-m counts and their scan)
 * is a file-scope device array of 2 x 65536 int64 (1 MiB) that every GPU
 * loading this library holds until the process exits; the entry point calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *   - Limit: M <= 65535 (N <= 256); a larger basis returns LB_EINVAL with a
 *     message naming the limit, and nothing is launched.
 *   - Set-up: every call looks up the array's device address on the current
 *     device with cudaGetSymbolAddress (nothing is cached, so the call stays
 *     valid after a cudaDeviceReset or a recreated context); the first call
 *     on a device loads the module there, so make it before any stream
 *     capture begins.
 *   - Sharing: all calls on a device use the same array, which keeps the last
 *     call's contents (every word a call reads is written earlier in the same
 *     call, so nothing needs clearing).  The call returns after its fill has
 *     finished on `stream`; calls whose GPU work overlaps (from several host
 *     threads at once, on any streams) race on the array and give wrong
 *     results. */
int lb_structure_export_noalloc(const lb_basis_t *b, int which, int32_t *idx3, double *val,
                                int64_t capacity, int64_t *nnz, void *stream);

/* Number of join terms W = #{(j,l,n,k,s): z_jln != 0, f_kls != 0} visited by
 * the dense R assembly (Eq. (09)); counted on the GPU.  Synchronous. */
int lb_join_terms(const lb_basis_t *b, int64_t *W);

/* ------------------------------------------------------------------------
 * a2 -- expansion and reconstruction.  Table 1 steps 2.1, 2.6, 3.2.
 * --------------------------------------------------------------------- */

/* Eq. (02): coef_j = Tr(F_j A), j = 0..M-1, for an N x N complex matrix A
 * (device, interleaved).  coef is M complex (device).  For Hermitian A the
 * coefficients are real; for a jump operator they are the complex l_j.  The
 * identity component Tr(A)/N is not part of coef. */
int lb_expand(const lb_basis_t *b, const double *A, double *coef, void *stream);

/* Eq. (rho): rho = 1/N + sum_i v_i F_i as an N x N complex matrix (device). */
int lb_rho(const lb_basis_t *b, const double *v, double *rho, void *stream);

/* lb_expand and lb_rho with host buffers (Table 1 steps 2.1, 2.6, 3.2):
 * A and rho are N x N complex (interleaved) in host memory, coef is M
 * complex, v is M doubles.  The device copies come from the library pool
 * and run on the library stream (see lb_assemble).  Synchronous. */
int lb_expand_host(const lb_basis_t *b, const double *A, double *coef);
int lb_rho_host(const lb_basis_t *b, const double *v, double *rho);

/* ------------------------------------------------------------------------
 * a3-a5 -- dense assembly.  Eqs. (07)-(09), Table 1 steps 2.3-2.5.
 * --------------------------------------------------------------------- */

/* Dense assembly from device buffers.
 *   h : M real Hamiltonian coefficients h_m = Tr(F_m H) (Eq. (07)), or NULL (H = 0)
 *   a : M x M complex Kossakowski matrix (convention above)
 * Outputs (each may be NULL, at least one of A, Q, R must not be):
 *   A = Q + R, Q, R : M x M doubles, row s = equation for dv_s/dt, column n
 *   K : M doubles (Eq. (08))
 * R follows Eq. (09) in the one-term form r_sn = -1/2 Re sum_jkl a_jk z_jln
 * f_kls (identical to the printed two-term form with prefactor -1/4 for
 * Hermitian a; Sec. 4 item 2.5), accumulated in FP64 by the thread or warp
 * that owns the entry (no atomics).  N <= 512 (LB_EINVAL otherwise).  Same as
 * lb_assemble_dense_ex with algorithm = LB_ALG_CLOSED, the fast form; pass
 * LB_ALG_JOIN there for the term-by-term join. */
int lb_assemble_dense(const lb_basis_t *b, const double *h, const double *a,
                      double *A, double *Q, double *R, double *K, void *stream);

/* algorithms of the dense R assembly */
#define LB_ALG_JOIN 0   /* every join term visited, as in Sec. 4 item 2.5 (O(N^5)) */
#define LB_ALG_CLOSED 1 /* the join terms summed in closed form, grouped by the
                           relation of the two edges of (s, n): completeness
                           of the D_l (sum_l delta_x(l) delta_y(l) = [x = y] - 1/N),
                           their Helmert prefix structure, the phase parity of
                           J edges, and vertex quadruples for disjoint edges
                           (signed sums of 8 entries of a, formed as integer
                           sums of aligned significands); O(N^4); same R up to
                           rounding */

/* lb_assemble_dense with a choice of algorithm (LB_ALG_JOIN or LB_ALG_CLOSED). */
int lb_assemble_dense_ex(const lb_basis_t *b, const double *h, const double *a,
                         double *A, double *Q, double *R, double *K, int algorithm,
                         void *stream);

/* The same assembly, with the device time of each of its kernels, measured
 * with CUDA events on `stream`, written to kernel_ms[0 .. count-1] (count =
 * lb_assemble_kernel_count(); lb_assemble_kernel_name(i) names kernel i; a
 * kernel that the requested outputs skip reports ~0).  Synchronous. */
int lb_assemble_dense_timed(const lb_basis_t *b, const double *h, const double *a,
                            double *A, double *Q, double *R, double *K, int algorithm,
                            void *stream, float *kernel_ms);
int lb_assemble_kernel_count(void);
const char *lb_assemble_kernel_name(int i);

/* ------------------------------------------------------------------------
 * a6-a8 -- RK4 integration (Table 1 step 3.1; Sec. 4 item 3), with the
 * matrix stored in FP64, FP32, or BF16 with per-row scales.
 * --------------------------------------------------------------------- */

/* A32 = fl32(A) (device, M x M). */
int lb_pack_fp32(int64_t M, const double *A, float *A32, void *stream);

/* Abf = bf16(A_sn / r_s), row_scale[s] = r_s = max_n |A_sn| (1 for a zero row). */
int lb_pack_bf16(int64_t M, const double *A, uint16_t *Abf, float *row_scale, void *stream);

/* Bytes of device workspace lb_rk4_dense needs for size M. */
size_t lb_rk4_workspace_bytes(int64_t M);

/* Classical RK4 with fixed step dt for dv/dt = A v + K, nsteps steps, all on
 * device.  precision selects the storage of Ap: LB_FP64 (double*), LB_FP32
 * (float*), LB_BF16 (uint16_t* bf16 with row_scale).  For FP32/BF16 the
 * stage products are FP32 multiply-adds of FP32-rounded stage vectors; the
 * state v and the stage combination stay FP64.  If correct_every > 0 and A64
 * is given, every correct_every steps the FP64 defect c = (A64 - A_lp) v at
 * the current v is formed in FP64 and added to K until the next correction.
 * v (M doubles) is the initial state on entry and the final state on exit.
 * snaps (may be NULL): after every snap_every steps a copy of v is stored in
 * row t/snap_every - 1 of snaps ((nsteps/snap_every) x M).
 * work: lb_rk4_workspace_bytes(M) bytes of device memory. */
int lb_rk4_dense(int64_t M, int precision, const void *Ap, const float *row_scale,
                 const double *A64, int correct_every, const double *K, double *v,
                 double dt, int64_t nsteps, double *snaps, int64_t snap_every,
                 void *work, void *stream);

/* Propagator form of classical RK4 for one system (Sec. 4 item 3): for
 * dv/dt = A v + K one RK4 step of size h is v <- v + h (D' v + c'), with
 *   D' = A + (h/2) A (A + (h/3) A (A + (h/4) A A)) = (P(hA) - 1)/h,
 *   P(x) = 1 + x + x^2/2 + x^3/6 + x^4/24,
 *   c' = K + (h/2) A (K + (h/3) A (K + (h/4) A K)),
 * which follows from writing the four stages as polynomials in hA applied to
 * A v + K.  A step then reads the matrix once (instead of four times), and
 * several initial states share that read.
 *
 * Bytes of device workspace for M, nrhs (1 <= nrhs <= 64) and precision
 * (LB_FP64 or LB_FP32); 0 for invalid arguments. */
size_t lb_propagator_workspace_bytes(int64_t M, int nrhs, int precision);

/* Form D' (Dp: M x M, double for LB_FP64, float for LB_FP32) and c' (cp: M
 * doubles) for step dt from the FP64 A64 and K (device).  LB_FP32 forms D'
 * from A32 = fl32(A64) with FP32 products and also returns R32 = D' - A32
 * (M x M floats) for the FP64 correction of lb_propagate; c' is always FP64.
 * Three matrix products by this library's tiled GEMM kernel.  Synchronous
 * with respect to stream. */
int lb_propagator_form(int64_t M, int precision, const double *A64, const float *A32, const double *K, double dt,
                       void *Dp, float *R32, double *cp, void *work, void *stream);

/* nsteps propagator steps of dt for nrhs states at once: V (device, nrhs x M
 * doubles, state r in row r) in/out.  Each step is one product of D' with
 * the block of states rounded to the precision of D' (FP64 or FP32), with
 * the state kept in FP64.  LB_FP32 with correct_every > 0 (and A64, R32
 * given): every correct_every steps the FP64 defect (A64 + R32 - D') v_r is
 * formed for every state and added to c' until the next one (A64 - A32 is
 * the storage error of A, A32 + R32 - D' the rounding of D').  snaps (may be
 * NULL): after every snap_every steps a copy of V goes to block
 * t/snap_every - 1 of snaps ((nsteps/snap_every) x nrhs x M).  dt must be the
 * step D' was formed for.  work: lb_propagator_workspace_bytes bytes. */
int lb_propagate(int64_t M, int nrhs, int precision, const void *Dp, const float *R32, const double *A64,
                 const double *cp, int correct_every, double *V, double dt, int64_t nsteps, double *snaps,
                 int64_t snap_every, void *work, void *stream);

/* ------------------------------------------------------------------------
 * FP64 checks on the device (Sec. 2: rho = 1/N + sum_i v_i F_i is a density
 * matrix, and the real system has the steady state of the Lindbladian).
 * --------------------------------------------------------------------- */

/* Bytes of device workspace of lb_steady_state for size M and restart
 * length `restart` (0: the default, min(M, 1024)); 0 for bad arguments. */
size_t lb_steady_workspace_bytes(int64_t M, int restart);

/* Steady state of dv/dt = A v + K: solve A v = -K (A = Q + R, M x M FP64
 * row-major, K: M, both device) by restarted GMRES(m) in FP64 with this
 * library's kernels (classical Gram-Schmidt with one reorthogonalisation
 * pass, Givens rotations on the host), m = restart (0: min(M, 1024); the
 * Krylov basis takes (m + 1) M doubles of workspace), from the initial guess
 * in v (device, M doubles; overwritten by the solution).  The Hamiltonian
 * part spreads the spectrum along the imaginary axis while the damping
 * keeps it near it, so long restarts converge where short ones stall.  Stops when the GMRES residual
 * estimate is <= tol ||K|| or after max_iter inner iterations;
 * *rel_residual receives the true relative residual ||K + A v|| / ||K|| of
 * the returned v (0 with v = 0 for K = 0) and *iterations the inner
 * iterations used.  Synchronous with respect to
 * stream.  work: lb_steady_workspace_bytes(M) bytes. */
int lb_steady_state(int64_t M, const double *A, const double *K, double *v, double tol, int max_iter, int restart,
                    double *rel_residual, int *iterations, void *work, void *stream);

/* Bytes of device workspace of lb_steady_state_pc for dimension N
 * (M = N^2 - 1) and restart length `restart`; 0 for bad arguments. */
size_t lb_steady_pc_workspace_bytes(int N, int64_t M, int restart);

/* lb_steady_state with a preconditioner from the Hamiltonian (Sec. 2: the
 * part Q of A acts on rho as -i[H, rho]).  In the eigenbasis of H (found on
 * the device by the CUDA toolkit's Hermitian eigensolver, loaded at run
 * time; LB_EUNSUPPORTED when it cannot be loaded), P = Q - sigma 1 is
 * diagonal with entries -i(E_j - E_k) - sigma, and GMRES runs on A P^-1
 * (right preconditioning: the residual is that of A v = -K).  sigma >= 0 is
 * the shift; sigma < 0 takes -Tr(A) / M, the mean damping rate (Tr Q = 0).
 * For a random Lindbladian, whose damping spreads little, GMRES then needs
 * a handful of iterations where the plain form needs hundreds.  H: device
 * N x N complex Hermitian (interleaved), the H of A; b: its basis.  work:
 * lb_steady_pc_workspace_bytes(N, M, restart) bytes, 256-byte aligned.
 * Other arguments and results as lb_steady_state. */
int lb_steady_state_pc(const lb_basis_t *b, const double *A, const double *K, const double *H, double sigma,
                       double *v, double tol, int max_iter, int restart, double *rel_residual, int *iterations,
                       void *work, void *stream);

/* Bytes of device workspace of lb_rho_checks for dimension N. */
size_t lb_rho_checks_workspace_bytes(int N);

/* For each of the nsnap states in V (device, nsnap x M doubles), rebuild
 * rho (Eq. (rho)) on the device and write to out (host, nsnap x 3):
 *   out[3k]     = Tr rho - 1,
 *   out[3k + 1] = max |rho_jk - conj(rho_kj)|,
 *   out[3k + 2] = the smallest pivot of the Cholesky factorisation of
 *                 rho + psd_shift 1 (complex, FP64; positive exactly when
 *                 the smallest eigenvalue of rho exceeds -psd_shift; the
 *                 first non-positive pivot ends the factorisation).
 * Synchronous with respect to stream.  work: lb_rho_checks_workspace_bytes(N). */
int lb_rho_checks(const lb_basis_t *b, const double *V, int64_t nsnap, double psd_shift, double *out, void *work,
                  void *stream);

/* ------------------------------------------------------------------------
 * Sparse models (Sec. 3: sparse H and a Kossakowski matrix of few channels,
 * P = 1 for the paper's sparse model): CSR assembly of A = Q + R and K, and
 * RK4 on CSR.
 * --------------------------------------------------------------------- */

typedef struct lb_csr lb_csr_t;

/* Assemble A = Q + R (CSR) and K for a_jk = sum_p gamma_p l_pj conj(l_pk).
 *   h      : M real Hamiltonian coefficients (device), or NULL (H = 0); its
 *            zero entries are skipped, so a sparse H costs O(nnz).
 *   nP     : number of channels p; gamma: nP rates (host)
 *   lp_ptr : nP + 1 offsets (host, lp_ptr[0] = 0) into lp_idx / lp_val
 *   lp_idx : basis indices of the nonzero l_pj (device int64)
 *   lp_val : the values l_pj (device, complex interleaved), e.g. from lb_expand
 * Eq. (09) is evaluated per channel as r_sn = -1/2 gamma_p Re sum_l W_ls U_ln,
 * U_ln = sum_j l_j z_jln, W_ls = sum_k conj(l_k) f_kls (a sparse product:
 * the terms are placed in buckets by row / column with count, scan and fill
 * passes, and each row of A is summed in a hash table keyed by column; the
 * diagonal components of l_p and of h enter through closed-form edge sums).
 * Pattern: an entry is stored iff |A_sn| exceeds 1e-12 times the sum of the
 * magnitudes of its terms (exact cancellations leave rounding residue only);
 * columns are sorted within rows.  Values are reproducible to rounding (the
 * order in which duplicate terms are summed is not fixed).  Indices within
 * one channel are expected to be distinct.  *out owns the device arrays (see
 * lb_csr_arrays); release with lb_csr_destroy.  Synchronous w.r.t. stream.
 * LB_ENOMEM when the intermediate lists do not fit; LB_EUNSUPPORTED when a
 * row of A has more than 8192 distinct columns. */
int lb_assemble_lowrank_csr(const lb_basis_t *b, const double *h, int nP, const double *gamma,
                            const int64_t *lp_ptr, const int64_t *lp_idx, const double *lp_val,
                            lb_csr_t **out, void *stream);

/* M, stored entries, and the number of summed terms (R products + Q terms). */
int lb_csr_info(const lb_csr_t *c, int64_t *M, int64_t *nnz, int64_t *terms);

/* Device arrays owned by the handle: rowptr (M+1 int64), col (nnz int32),
 * val (nnz doubles), K (M doubles).  Valid until lb_csr_destroy. */
int lb_csr_arrays(const lb_csr_t *c, const int64_t **rowptr, const int32_t **col,
                  const double **val, const double **K);
int lb_csr_destroy(lb_csr_t *c);

/* Copy the CSR arrays (and K) into caller buffers, host or device (any
 * pointer may be NULL to skip it).  Synchronous with respect to stream. */
int lb_csr_copy(const lb_csr_t *c, int64_t *rowptr, int32_t *col, double *val, double *K, void *stream);

/* RK4 on the CSR system (same stage structure as lb_rk4_dense): precision
 * LB_FP64, or LB_FP32 values (converted once and cached in the handle) with
 * FP32 products and, if correct_every > 0, the FP64 defect
 * (A64 - A32) v added to K every correct_every steps.  v (device, M doubles)
 * in/out; work: lb_rk4_workspace_bytes(M) bytes of device memory.  With
 * rows of fewer than 8 entries on average and a 16-byte aligned v, the
 * stages stream their rows through shared memory by bulk copies with
 * bounded waits; the call then returns after the steps have finished on
 * `stream`, and LB_ETIMEOUT if a wait ran out. */
int lb_rk4_csr(const lb_csr_t *c, int precision, int correct_every, double *v, double dt,
               int64_t nsteps, void *work, void *stream);

/* RK4 with a time-dependent Hamiltonian H(t) = H0 + eps(t) H1 (Sec. 3: the
 * periodically rocked dimer, Eq. (10), where eps(t) = E + A Theta(t)):
 * dv/dt = (A0 + eps(t) Q1) v + K with A0 = Q0 + R and K from the CSR system
 * A0 and Q1 the CSR matrix of Eq. (07) for H1 (e.g. lb_assemble_lowrank_csr
 * with h1 and no channels; its K is not used).  eps is periodic with period
 * `period` and piecewise constant: eps(t) = seg_eps[k] for (t mod period) in
 * [seg_start[k], seg_start[k + 1]) (seg_start[0] = 0, increasing; the last
 * segment ends at period).  Classical RK4 from time t0, each stage with eps
 * at its own time, the stages at the ends of a step taken 1e-6 dt inside it
 * (a step lying between two switches of eps sees one value in all four
 * stages); FP64.  v (device, M doubles) in/out; work:
 * lb_rk4_workspace_bytes(M).  Asynchronous on stream (seg arrays are host
 * memory, read during the call). */
int lb_rk4_csr_td(const lb_csr_t *A0, const lb_csr_t *Q1, int nseg, const double *seg_start, const double *seg_eps,
                  double period, double t0, double *v, double dt, int64_t nsteps, void *work, void *stream);

/* ------------------------------------------------------------------------
 * a9 -- batched form: many independent realizations of mixed N (the
 * ensemble sampling of Sec. 6, one sample per processor group), assembled
 * and integrated together.
 * --------------------------------------------------------------------- */

typedef struct lb_batch lb_batch_t;

/* A batch of `count` realizations with dimensions Ns[r] (2 <= N <= 64).  The
 * batch owns one basis per distinct N and, per realization, the assembled
 * A = Q + R (FP64 and FP32) and K.  Synchronous. */
int lb_batch_create(int count, const int *Ns, lb_batch_t **out);

/* Inputs and state of realization r: a (device M x M complex Kossakowski
 * matrix), h (device M real Hamiltonian coefficients, or NULL), v (device M
 * doubles: the initial state, overwritten by lb_batch_integrate).  The
 * pointers are kept (not copied) and must stay valid while the batch uses them. */
int lb_batch_set(lb_batch_t *b, int r, const double *a, const double *h, double *v);

/* Assemble every realization (dense, LB_ALG_JOIN or LB_ALG_CLOSED) and pack
 * its FP32 copy.  Synchronous. */
int lb_batch_assemble(lb_batch_t *b, int algorithm, void *stream);

/* Cluster size (1, 2, 4, 8, 16 blocks) used for realization r; default 1. */
int lb_batch_set_cluster(lb_batch_t *b, int r, int C);

/* Autotuner: bucket the realizations by N (bucket width `width`), time every
 * cluster size on each bucket for probe_steps RK4 steps, keep the fastest
 * (states restored afterwards).  choice (optional, count ints) receives it. */
int lb_batch_tune(lb_batch_t *b, int width, int probe_steps, double dt, void *stream, int *choice);

/* Storage and arithmetic of lb_batch_integrate and lb_batch_tune: LB_FP32
 * (default; FP32 matrix and products, FP64 state and optional correction) or
 * LB_FP64 (FP64 matrix and products; correct_every is ignored). */
int lb_batch_set_precision(lb_batch_t *b, int precision);

/* Integration form of lb_batch_integrate and lb_batch_tune. */
#define LB_FORM_RK4 0         /* the four RK4 stages per step (default) */
#define LB_FORM_PROPAGATOR 1  /* one product per step with D' = (P(hA) - 1)/h */

/* Select the integration form.  LB_FORM_PROPAGATOR: for the autonomous
 * system dv/dt = A v + K, one classical RK4 step of size h (Sec. 4 item 3)
 * equals v <- v + h (D' v + c') with
 *   D' = A + (h/2) A (A + (h/3) A (A + (h/4) A A)) = (P(hA) - 1)/h,
 *   P(x) = 1 + x + x^2/2 + x^3/6 + x^4/24,
 *   c' = K + (h/2) A (K + (h/3) A (K + (h/4) A K)),
 * so a step reads the matrix once and exchanges the state once.  D' and c'
 * are formed for the step h of the first integration (or by
 * lb_batch_form_propagator) and kept until h or the precision changes.
 * Precision LB_FP64: D' and c' in FP64, FP64 products.  LB_FP32: D' formed
 * from the FP32 A with FP32 products (its difference from A kept in FP32 as
 * well), c' in FP64, FP64 state; with correct_every > 0 the FP64 defect
 * (A64 + (D' - A)_FP32 - D'_FP32) v is added to c' every correct_every steps.
 * The trajectory equals classical RK4's up to rounding. */
int lb_batch_set_form(lb_batch_t *b, int form);

/* Form D' and c' of every realization for step dt in the batch's precision
 * now (three matrix products per realization, by this library's batched
 * tiled GEMM, and three FP64 matrix-vector products); ms (optional)
 * receives the device time.  Synchronous.  LB_ENOMEM if the device cannot
 * hold D' (and D' - A) beside the batch. */
int lb_batch_form_propagator(lb_batch_t *b, double dt, void *stream, float *ms);

/* RK4 for every realization, nsteps steps of dt, FP32 matrix with FP32
 * products, FP64 state, FP64 defect correction every correct_every steps (0:
 * none).  One persistent cluster launch per cluster-size group: a cluster
 * takes realizations from a queue (largest first), keeps its row slices of
 * the matrix in shared memory when they fit, and exchanges the stage
 * vector through distributed shared memory.  ms (optional) receives the
 * device time.  Synchronous. */
int lb_batch_integrate(lb_batch_t *b, int correct_every, double dt, int64_t nsteps, void *stream, float *ms);

/* Device pointers of realization r's assembled system (owned by the batch). */
int lb_batch_system(const lb_batch_t *b, int r, const double **A64, const float **A32, const double **K,
                    int64_t *M);

/* Copy realization r's FP64 A (M x M) and K (M) into caller buffers (host or
 * device; either may be NULL).  Synchronous with respect to stream. */
int lb_batch_copy_system(const lb_batch_t *b, int r, double *A64, double *K, void *stream);
int lb_batch_destroy(lb_batch_t *b);

/* ------------------------------------------------------------------------
 * Host-buffer interface (one call per paper step, inputs and outputs in
 * host memory, copies included; Table 1 steps 2.1-2.6 and 3.1-3.2).  The
 * assembled system stays on the device inside an lb_system_t.
 *
 * Device memory and ordering: every call runs on one non-blocking library
 * stream per device and takes its device memory from one library memory
 * pool per device, which keeps what it has reserved between calls (no
 * cudaMalloc / cudaFree, and no device-wide synchronization, once a size
 * has been seen); lb_host_release returns the spare memory.  Calls are
 * synchronous with respect to the host.  Concurrent calls from several
 * host threads are correct and run one after another on the library stream.
 * --------------------------------------------------------------------- */

/* The Kossakowski matrix of an assembly, in the convention of Eqs. (08) and
 * (09) (see above), either dense or as a sum over channels (Sec. 2: the
 * dissipator as a sum over jump operators, a_jk = sum_p gamma_p l_pj
 * conj(l_pk), with l_p the expansion of jump operator L_p, Eq. (02)).
 * All arrays are host memory, read during the call only. */
typedef struct lb_kossakowski {
  int kind;               /* LB_A_DENSE or LB_A_LOWRANK */
  const double *a;        /* LB_A_DENSE: M x M complex Hermitian (interleaved); only
                             its upper triangle j <= k is read when the array is
                             page-locked (then by the GPU over the host link) or
                             M > 2048; the whole array (pageable, M <= 2048) */
  int nP;                 /* LB_A_LOWRANK: number of channels (0 <= nP <= 4096) */
  const double *gamma;    /* nP rates */
  const int64_t *lp_ptr;  /* nP + 1 offsets into lp_idx / lp_val, lp_ptr[0] = 0 */
  const int64_t *lp_idx;  /* basis indices j (0 <= j < M) of the nonzero l_pj */
  const double *lp_val;   /* the values l_pj, complex interleaved */
} lb_kossakowski;

/* Expand H (host N x N complex Hermitian, may be NULL for H = 0; Eq. (02))
 * and assemble A = Q + R and K (Eqs. (07)-(09)) from the Kossakowski matrix
 * `a` into a new system *out (owned by the caller, released with
 * lb_system_destroy).
 *   format = LB_DENSE: A as M x M FP64 (N <= 512), by `algorithm`
 *     (LB_ALG_CLOSED or LB_ALG_JOIN); keep_parts != 0 also keeps Q and R.  A
 *     low-rank `a` is first formed as a dense matrix on the device.  The
 *     Hermitian upper triangle of a dense `a` crosses the host link and the
 *     lower one is mirrored on the device.  A page-locked (pinned, mapped)
 *     `a` is read by a kernel directly from host memory; a pageable one goes
 *     through the copy engine in row blocks.
 *   format = LB_CSR: A in CSR form from a low-rank `a` (the product form of
 *     lb_assemble_lowrank_csr, same pattern rule); `algorithm` is not used.
 *     A dense `a` or keep_parts != 0 give LB_EUNSUPPORTED.
 * LB_ENOMEM if the device cannot hold the dense buffers (checked against
 * free memory plus the pool's spare memory before any allocation) or an
 * allocation is refused.  The staging copy of `a` is returned to the pool
 * before the call returns.  Synchronous. */
int lb_assemble(const lb_basis_t *b, const double *H, const lb_kossakowski *a, int format, int algorithm,
                int keep_parts, lb_system_t **out);
int lb_system_destroy(lb_system_t *sys);

/* Format (LB_DENSE / LB_CSR), M and stored entries (M * M for dense) of a
 * system; any output pointer may be NULL. */
int lb_system_info(const lb_system_t *sys, int *format, int64_t *M, int64_t *nnz);

/* Times in ms of the phases of the lb_assemble call that built sys, indexed
 * by LB_PHASE_* (ms: LB_PHASES doubles).  Device phases are CUDA-event
 * times on the library stream; LB_PHASE_ALLOC and LB_PHASE_FREE are host
 * wall times.  Zero for systems from lb_system_load. */
int lb_system_timings(const lb_system_t *sys, double *ms);

/* Copy one part (LB_SYS_A, _Q, _R: M x M; LB_SYS_K: M) into host memory.
 * LB_EINVAL if the part was not kept (and for A, Q, R of a CSR system). */
int lb_system_get(const lb_system_t *sys, int part, double *out);

/* ------------------------------------------------------------------------
 * Spectrum of the generator (Sec. 6, Fig. 5: the complex eigenvalues
 * lambda_i, i = 2..N^2, of one random Lindbladian, counted on a grid of cells
 * and normalised by the cell area).  The eigenvalues of A = Q + R are those
 * of the N^2 x N^2 generator other than the steady state's.  They come from
 * the dense nonsymmetric eigensolver of the CUDA toolkit's solver library
 * (loaded at run time; LB_EUNSUPPORTED when it cannot be loaded), O(M^3) FP64
 * work: about 1e15 flops at N = 200, so practical up to N of about 70-100 on
 * one GPU.  The density grid is the library's own kernel.
 * --------------------------------------------------------------------- */

/* Eigenvalues of the dense row-major M x M FP64 matrix A (device) into eig
 * (device, 2 M doubles, complex interleaved, in the solver's order).  A is
 * not modified (the solver works on a copy, M^2 doubles of device memory).
 * Synchronous with respect to stream; LB_ECUDA if the solver fails. */
int lb_spectrum(const double *A, int64_t M, double *eig, void *stream);

/* The same for the A of a dense system, into host memory (eig: 2 M doubles,
 * complex interleaved).  LB_EINVAL for a CSR system. */
int lb_system_spectrum(const lb_system_t *sys, double *eig);

/* Density of n complex eigenvalues (device, interleaved) on an nre x nim
 * grid over the box {re_lo, re_hi, im_lo, im_hi} (host, 4 doubles): the
 * number in each cell [re_lo + a dre, re_lo + (a+1) dre) x [im_lo + b dim,
 * ...) divided by the cell area dre * dim, at density[a * nim + b] (device,
 * nre * nim doubles, overwritten).  Eigenvalues outside the box are not
 * counted.  Asynchronous on stream. */
int lb_spectrum_density(const double *eig, int64_t n, const double *box, int nre, int nim, double *density,
                        void *stream);

/* CSR arrays of a CSR system into host buffers (any may be NULL): rowptr
 * (M + 1 int64), col (nnz int32, sorted within rows), val (nnz doubles).
 * LB_EINVAL for a dense system. */
int lb_system_get_csr(const lb_system_t *sys, int64_t *rowptr, int32_t *col, double *val);

/* Classical RK4 (Sec. 4 item 3) from the host initial state v0 (M doubles)
 * for n = round(t/dt) steps (LB_EINVAL if |n dt - t| > 1e-9 t).
 *   snap_every = 0: v_out (host, M doubles) receives the final state.
 *   snap_every > 0: n must be a multiple of it (else LB_EINVAL); v_out
 *     (host, (n / snap_every) x M doubles) receives the state after every
 *     snap_every steps, row i after (i + 1) snap_every steps, so the last row
 *     is the final state.
 * Dense systems: precision LB_FP64, LB_FP32 or LB_BF16 with correct_every as
 * for lb_rk4_dense; the low-precision copy is made (and cached in the
 * system) on first use.  CSR systems: LB_FP64 or LB_FP32 as for lb_rk4_csr;
 * with LB_FP32 and correct_every > 0, snap_every must be a multiple of
 * correct_every (the correction restarts at every snapshot).  Synchronous. */
int lb_integrate(lb_system_t *sys, int precision, int correct_every, const double *v0, double t, double dt,
                 int64_t snap_every, double *v_out);

/* Return the spare device memory of the library pool of the current device
 * (after the library stream has finished).  The next host-buffer call
 * reserves again what it needs. */
int lb_host_release(void);

/* Checkpoint and resume.  There is no counterpart in the paper; it serves
 * long integrations that are stopped and continued.
 *
 * lb_system_save writes the system to the file `path`: a 64-byte header
 * ("LBSYS001", N, M, a mask of the parts present, format version), then A
 * (M x M FP64, row-major), K (M), and Q, R if they were kept, all little
 * endian.  It copies in bounded chunks through host memory and is
 * synchronous.  LB_EINVAL if the file cannot be written.
 *
 * lb_system_load reads such a file for basis b (whose N must match) into a
 * new system owned by the caller; the low-precision copies are made again on
 * first use.  LB_EINVAL for a missing, truncated or foreign file;
 * LB_ENOMEM / LB_ECUDA on device failure.
 *
 * lb_integrate_resume advances the host state v (M doubles, in place) by
 * nsteps RK4 steps of size dt.  When every earlier segment had a multiple of
 * correct_every steps (any length for LB_FP64, or for correct_every = 0),
 * the segments give the same bits as one lb_integrate over their total:
 * each segment starts from v exactly as a step boundary of one run does.
 * Synchronous. */
int lb_system_save(const lb_system_t *sys, const char *path);
int lb_system_load(const lb_basis_t *b, const char *path, lb_system_t **out);
int lb_integrate_resume(lb_system_t *sys, int precision, int correct_every, double *v, double dt,
                        int64_t nsteps);

/* ------------------------------------------------------------------------
 * Measurement helpers (no counterpart in the paper).
 * --------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched in the process so far. */
long long lb_launch_count(void);

/* FP64 fused multiply-add throughput of the current device in TFLOP/s
 * (2 flops per FMA), measured with eight independent FMA chains per thread
 * over 4 blocks of 256 threads per SM.  The roofline denominator of the
 * FP64-bound kernels.  Synchronous. */
int lb_probe_fp64(double *tflops);

/* ------------------------------------------------------------------------
 * a10 -- serving form.  Realizations of the random-Lindbladian model
 * (Sec. 6: independent samples of an ensemble) arrive one by one as
 * requests; each is assembled (Eqs. (07)-(09)) and integrated (RK4, Table 1
 * step 3) on the GPU while earlier ones are still running.  A server owns a
 * scheduler thread, a device-memory pool and per-request streams.
 *
 * Admission: a request holds lb_request_bytes(N, precision, H != NULL)
 * bytes of server memory from admission to completion (A64, the low-
 * precision copy, K, the state, the expansion of H and RK4 work vectors).
 * Requests are admitted in arrival order while fewer than `slots` are in
 * flight and their bytes fit in what `budget_bytes` has left; one that does
 * not fit is passed by later requests only until it has waited `bypass_ms`.
 * The caller's a, H and v0 stay caller-owned and are not counted: they are
 * read until the request's state reaches LB_REQ_ASSEMBLED, after which the
 * caller may free or reuse them.  v_out is written by the time the state is
 * LB_REQ_DONE.
 *
 * Engines: N <= 64 with LB_FP32 runs on the cluster-persistent batched
 * kernel (requests admitted together share one launch; cluster size from
 * lb_server_set_cluster, else the smallest size that keeps the matrix in
 * shared memory); every other request runs the fused RK4 stage kernels as a
 * CUDA graph of about 50 steps (a multiple of correct_every) replayed on its
 * own stream.  A request's result depends only on its own inputs, N and
 * precision, not on the other requests in flight.
 *
 * Thread safety: every lb_server_* / lb_submit / lb_poll / lb_wait call may
 * come from any host thread (one internal mutex).  All waits are bounded by
 * the caller's timeout; lb_server_destroy cancels queued requests and waits
 * for admitted ones to finish on the GPU.
 * --------------------------------------------------------------------- */

typedef struct lb_server lb_server_t;

typedef struct lb_request {
  int N;               /* 2 <= N <= 512 */
  int precision;       /* LB_FP64 | LB_FP32 | LB_BF16 */
  int correct_every;   /* FP64 defect-correction period for FP32/BF16 (0 = none) */
  double dt;
  int64_t nsteps;
  const double *H;     /* device N x N complex128 Hermitian (interleaved), or NULL */
  const double *a;     /* device M x M complex128 Hermitian Kossakowski matrix (Eq. (09) convention) */
  const double *v0;    /* device M: initial state */
  double *v_out;       /* device M: final state */
  void *stream;        /* caller's cudaStream_t: a, H, v0 are complete in its order at
                          submission (the server's work waits for it); NULL = legacy stream */
} lb_request;

#define LB_REQ_QUEUED 0
#define LB_REQ_RUNNING 1     /* admitted; a, H, v0 may still be read */
#define LB_REQ_ASSEMBLED 2   /* a, H, v0 no longer read */
#define LB_REQ_DONE 3
#define LB_REQ_FAILED 4
#define LB_REQ_CANCELLED 5

#define LB_ENGINE_CLUSTER 0
#define LB_ENGINE_STREAM 1

typedef struct lb_result {
  int state;           /* LB_REQ_* */
  int status;          /* LB_OK, or the error of a failed request */
  int engine;          /* LB_ENGINE_* */
  int cluster;         /* cluster size (cluster engine), else 0 */
  double queue_ms;     /* submission -> admission */
  double latency_ms;   /* submission -> completion seen by the host */
  double gpu_ms;       /* device time from the request's first enqueue to its result copy */
} lb_result;

/* Server memory one request holds (bytes), or -1 for invalid arguments. */
int64_t lb_request_bytes(int N, int precision, int with_H);

/* Create a server on the current device.  budget_bytes > 0, slots >= 1,
 * bypass_ms >= 0.  LB_ECUDA if the pool or streams cannot be created. */
int lb_server_create(int64_t budget_bytes, int slots, double bypass_ms, lb_server_t **out);

/* Cluster size C in {1, 2, 4, 8, 16} for requests of dimension N <= 64 on
 * the cluster engine (takes effect for requests admitted afterwards). */
int lb_server_set_cluster(lb_server_t *s, int N, int C);

/* Queue a request; *id identifies it.  LB_EINVAL for a malformed request,
 * LB_ENOMEM if it can never fit in the budget.  Returns at once. */
int lb_submit(lb_server_t *s, const lb_request *q, uint64_t *id);

/* State of a request.  LB_OK when done (out filled), LB_EAGAIN while queued
 * or running, the request's error code if it failed. */
int lb_poll(lb_server_t *s, uint64_t id, lb_result *out);

/* Wait at most timeout_ms for a request to finish.  LB_ETIMEOUT if it has
 * not (out holds its current state). */
int lb_wait(lb_server_t *s, uint64_t id, double timeout_ms, lb_result *out);

/* Nearest-rank p50 / p99 of the latency of completed requests, their
 * throughput (completed / (last completion - first submission), per s) and
 * count, since creation or the last lb_server_reset_stats. */
int lb_server_stats(lb_server_t *s, double *p50_ms, double *p99_ms, double *throughput, int64_t *completed);
int lb_server_reset_stats(lb_server_t *s);
int lb_server_destroy(lb_server_t *s);

/* Replay of the admission policy in virtual time (host only, no GPU):
 * request i arrives at arrival_ms[i] (non-decreasing), holds bytes[i] and
 * runs service_ms[i] once admitted.  start_ms / finish_ms receive its times
 * (-1 if it exceeds the budget).  For capacity planning and tests. */
int lb_sched_simulate(int n, const double *arrival_ms, const int64_t *bytes, const double *service_ms,
                      int64_t budget, int slots, double bypass_ms, double *start_ms, double *finish_ms);

#ifdef __cplusplus
}
#endif
#endif /* LINDBLAD_H */

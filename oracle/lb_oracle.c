/*
 * lb_oracle.c -- plain, slow CPU FP64 oracle for the transformation of a
 * GKSL (Lindblad) generator into the real linear system dv/dt = (Q+R)v + K
 * (Meyerov et al., "Transforming Lindblad Equations into Systems of
 * Real-Valued Linear Equations", Sec. 2, Eqs. (02)-(09)).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes, and how (deliberately naive):
 *   * the SU(N) basis {F_i} of Sec. 2 as explicit sparse N x N matrices
 *     (S^(j,k), J^(j,k), D^l; D^l is read as the Hermitian, orthonormal
 *     matrix (sum_{k<=l} e_k e_k^T - l e_{l+1} e_{l+1}^T)/sqrt(l(l+1)), the
 *     printed prefactor i/sqrt(l(l+1)) contradicts Tr(F_n F_m) = delta_nm);
 *     0-based order: S block (pairs j<k lexicographic), J block, D_1..D_{N-1};
 *   * f_mns = -i Tr(F_s [F_m,F_n]) and d_mns = Tr(F_s {F_m,F_n}) (Eq. (05))
 *     by multiplying the sparse basis matrices and projecting the commutator
 *     and anticommutator back onto the basis -- no closed-form rules;
 *   * expansion coefficients a_j = Tr(F_j A) (Eq. (02));
 *   * q_sn = sum_m h_m f_mns (Eq. (07));
 *   * k_s = (i/N) sum_jk a_jk f_jks (Eq. (08), with the sum over channels
 *     folded into the Kossakowski matrix a_jk = sum_p gamma_p l_pj conj(l_pk));
 *   * r_sn = -1/4 sum_jkl a_jk (z_jln f_kls + conj(z_kln) f_jls) (Eq. (09)
 *     with z = f + i d, Eq. (06)); the prefactor -1/4 (not the printed -1/2)
 *     is the one the brute-force definition Tr(F_s L_D(F_n)) fixes for this
 *     two-term form;
 *   * classical fourth-order Runge-Kutta for dv/dt = A v + K (Sec. 4, step 3).
 *
 * Values are "nonzero" when |x| > 1e-12 * (largest |x| of the tensor).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ basis */

typedef struct {
    int nnz;          /* number of stored entries            */
    int *row, *col;   /* positions                           */
    double *re, *im;  /* values                              */
} sp_mat;

typedef struct {
    int N;
    int64_t M, P;
    sp_mat *F;        /* F[0..M-1] */
    /* ordered nonzero triples of f and d: (m, n, s, value) */
    int64_t nf, nd;
    int32_t *f_idx;   /* 3 * nf */
    double *f_val;
    int32_t *d_idx;   /* 3 * nd */
    double *d_val;
} ora_ctx;

static void sp_alloc(sp_mat *A, int nnz) {
    A->nnz = nnz;
    A->row = (int *)malloc(sizeof(int) * (size_t)nnz);
    A->col = (int *)malloc(sizeof(int) * (size_t)nnz);
    A->re = (double *)calloc((size_t)nnz, sizeof(double));
    A->im = (double *)calloc((size_t)nnz, sizeof(double));
}

static void sp_free(sp_mat *A) {
    free(A->row); free(A->col); free(A->re); free(A->im);
}

/* Sec. 2, Eqs. for S^(j,k), J^(j,k), D^l (0-based indices). */
static void build_basis(ora_ctx *c) {
    int N = c->N;
    int64_t P = c->P, i = 0;
    double r2 = 1.0 / sqrt(2.0);
    c->F = (sp_mat *)calloc((size_t)c->M, sizeof(sp_mat));
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b, ++i) {
            sp_mat *S = &c->F[i];
            sp_alloc(S, 2);
            S->row[0] = a; S->col[0] = b; S->re[0] = r2;
            S->row[1] = b; S->col[1] = a; S->re[1] = r2;
            sp_mat *J = &c->F[P + i];
            sp_alloc(J, 2);
            J->row[0] = a; J->col[0] = b; J->im[0] = -r2;  /* -i/sqrt2 e_a e_b^T */
            J->row[1] = b; J->col[1] = a; J->im[1] = r2;   /* +i/sqrt2 e_b e_a^T */
        }
    for (int l = 1; l < N; ++l) {
        sp_mat *D = &c->F[2 * P + (l - 1)];
        double nrm = 1.0 / sqrt((double)l * (double)(l + 1));
        sp_alloc(D, l + 1);
        for (int k = 0; k < l; ++k) {
            D->row[k] = k; D->col[k] = k; D->re[k] = nrm;
        }
        D->row[l] = l; D->col[l] = l; D->re[l] = -(double)l * nrm;
    }
}

/* Dense N x N complex scratch with a list of touched positions. */
typedef struct {
    int N;
    double *re, *im;
    char *mark;
    int *touched;
    int nt;
} scratch;

static void scr_init(scratch *w, int N) {
    w->N = N;
    w->re = (double *)calloc((size_t)N * N, sizeof(double));
    w->im = (double *)calloc((size_t)N * N, sizeof(double));
    w->mark = (char *)calloc((size_t)N * N, 1);
    w->touched = (int *)malloc(sizeof(int) * (size_t)N * N);
    w->nt = 0;
}

static void scr_free(scratch *w) {
    free(w->re); free(w->im); free(w->mark); free(w->touched);
}

static void scr_add(scratch *w, int r, int c, double xr, double xi) {
    int p = r * w->N + c;
    if (!w->mark[p]) { w->mark[p] = 1; w->touched[w->nt++] = p; }
    w->re[p] += xr;
    w->im[p] += xi;
}

static void scr_clear(scratch *w) {
    for (int t = 0; t < w->nt; ++t) {
        int p = w->touched[t];
        w->re[p] = 0; w->im[p] = 0; w->mark[p] = 0;
    }
    w->nt = 0;
}

/* Tr(F_s X) = sum_pq (F_s)_pq X_qp for a dense X held in scratch. */
static void trace_with(const sp_mat *Fs, const double *Xr, const double *Xi,
                       int N, double *tr, double *ti) {
    double sr = 0, si = 0;
    for (int e = 0; e < Fs->nnz; ++e) {
        int q = Fs->col[e], p = Fs->row[e];
        double xr = Xr[q * N + p], xi = Xi[q * N + p];
        sr += Fs->re[e] * xr - Fs->im[e] * xi;
        si += Fs->re[e] * xi + Fs->im[e] * xr;
    }
    *tr = sr; *ti = si;
}

/* Same trace, summed over the touched positions of X instead (X sparse):
 * Tr(F_s X) = sum over touched (q,p) of (F_s)_pq X_qp.  Entries of F_s are
 * found by a scan of its (short) entry list. */
static void trace_touched(const sp_mat *Fs, const scratch *X, double *tr, double *ti) {
    int N = X->N;
    double sr = 0, si = 0;
    for (int t = 0; t < X->nt; ++t) {
        int pos = X->touched[t], q = pos / N, p = pos % N;
        for (int e = 0; e < Fs->nnz; ++e)
            if (Fs->row[e] == p && Fs->col[e] == q) {
                double xr = X->re[pos], xi = X->im[pos];
                sr += Fs->re[e] * xr - Fs->im[e] * xi;
                si += Fs->re[e] * xi + Fs->im[e] * xr;
            }
    }
    *tr = sr; *ti = si;
}

/* growable triple list */
typedef struct { int64_t n, cap; int32_t *idx; double *val; } tlist;

static void tl_push(tlist *t, int32_t m, int32_t n, int32_t s, double v) {
    if (t->n == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->idx = (int32_t *)realloc(t->idx, sizeof(int32_t) * 3 * (size_t)t->cap);
        t->val = (double *)realloc(t->val, sizeof(double) * (size_t)t->cap);
    }
    t->idx[3 * t->n] = m; t->idx[3 * t->n + 1] = n; t->idx[3 * t->n + 2] = s;
    t->val[t->n] = v;
    t->n++;
}

/* index of the pair (a,b), a<b, in lexicographic order */
static int64_t pair_index(int N, int a, int b) {
    return (int64_t)a * (2 * N - a - 1) / 2 + (b - a - 1);
}

/*
 * Eq. (05): enumerate all ordered (m,n,s) with f_mns or d_mns nonzero.
 * For every ordered pair (m,n) whose product F_m F_n can be nonzero, form
 * P = F_m F_n explicitly, then [F_m,F_n] = P - P^dagger and
 * {F_m,F_n} = P + P^dagger (the F are Hermitian), and take traces with every
 * basis element whose support meets the result.
 */
static void enumerate_fd(ora_ctx *c) {
    int N = c->N;
    int64_t M = c->M, P = c->P;
    /* elements touching each index v (support rows) */
    int **touch = (int **)malloc(sizeof(int *) * (size_t)N);
    int *ntouch = (int *)calloc((size_t)N, sizeof(int));
    for (int64_t i = 0; i < M; ++i)
        for (int e = 0; e < c->F[i].nnz; ++e) ntouch[c->F[i].row[e]]++;
    for (int v = 0; v < N; ++v) touch[v] = (int *)malloc(sizeof(int) * (size_t)(ntouch[v] + 1));
    int *fill = (int *)calloc((size_t)N, sizeof(int));
    for (int64_t i = 0; i < M; ++i)
        for (int e = 0; e < c->F[i].nnz; ++e) {
            int v = c->F[i].row[e];
            touch[v][fill[v]++] = (int)i;
        }

    tlist tf = {0, 0, NULL, NULL}, td = {0, 0, NULL, NULL};
    scratch Pm, Cm, Am;
    scr_init(&Pm, N); scr_init(&Cm, N); scr_init(&Am, N);
    char *cand_mark = (char *)calloc((size_t)M, 1);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);
    char *seen = (char *)calloc((size_t)M, 1);
    int64_t *nlist = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);
    double *fraw = NULL, *draw = NULL; /* values before thresholding */
    int64_t nraw = 0, capraw = 0;
    int32_t *rawidx = NULL;

    for (int64_t m = 0; m < M; ++m) {
        const sp_mat *Fm = &c->F[m];
        /* candidates n: elements whose rows meet the columns of F_m */
        int64_t nn = 0;
        for (int e = 0; e < Fm->nnz; ++e) {
            int v = Fm->col[e];
            for (int t = 0; t < ntouch[v]; ++t) {
                int n = touch[v][t];
                if (!seen[n]) { seen[n] = 1; nlist[nn++] = n; }
            }
        }
        for (int64_t q = 0; q < nn; ++q) {
            int64_t n = nlist[q];
            seen[n] = 0;
            const sp_mat *Fn = &c->F[n];
            /* P = F_m F_n */
            for (int e = 0; e < Fm->nnz; ++e)
                for (int g = 0; g < Fn->nnz; ++g)
                    if (Fm->col[e] == Fn->row[g]) {
                        double xr = Fm->re[e] * Fn->re[g] - Fm->im[e] * Fn->im[g];
                        double xi = Fm->re[e] * Fn->im[g] + Fm->im[e] * Fn->re[g];
                        scr_add(&Pm, Fm->row[e], Fn->col[g], xr, xi);
                    }
            if (Pm.nt == 0) continue;
            /* C = P - P^dag, A = P + P^dag */
            for (int t = 0; t < Pm.nt; ++t) {
                int p = Pm.touched[t], r = p / N, cc = p % N;
                double pr = Pm.re[p], pi = Pm.im[p];
                scr_add(&Cm, r, cc, pr, pi);
                scr_add(&Cm, cc, r, -pr, pi);     /* -(conj P)^T */
                scr_add(&Am, r, cc, pr, pi);
                scr_add(&Am, cc, r, pr, -pi);     /* +(conj P)^T */
            }
            /* candidate s: pairs on touched off-diagonal positions; every D
             * if a diagonal position was touched (a D has only diagonal
             * entries, so otherwise all its traces vanish) */
            int64_t ns = 0;
            int diag = 0;
            for (int t = 0; t < Cm.nt; ++t) {
                int p = Cm.touched[t], r = p / N, cc = p % N;
                if (r == cc) { diag = 1; continue; }
                int a = r < cc ? r : cc, b = r < cc ? cc : r;
                int64_t ps = pair_index(N, a, b);
                if (!cand_mark[ps]) { cand_mark[ps] = 1; cand[ns++] = ps; }
                if (!cand_mark[P + ps]) { cand_mark[P + ps] = 1; cand[ns++] = P + ps; }
            }
            for (int l = 1; diag && l < N; ++l) {
                int64_t s = 2 * P + (l - 1);
                if (!cand_mark[s]) { cand_mark[s] = 1; cand[ns++] = s; }
            }
            for (int64_t u = 0; u < ns; ++u) {
                int64_t s = cand[u];
                cand_mark[s] = 0;
                double cr, ci, ar, ai;
                if (c->F[s].nnz <= 2 || Cm.nt <= 2) {
                    /* short side: scan the touched positions */
                    trace_touched(&c->F[s], &Cm, &cr, &ci);
                    trace_touched(&c->F[s], &Am, &ar, &ai);
                } else {
                    trace_with(&c->F[s], Cm.re, Cm.im, N, &cr, &ci);
                    trace_with(&c->F[s], Am.re, Am.im, N, &ar, &ai);
                }
                /* f = -i Tr(F_s C) -> real part = Im Tr(F_s C); d = Tr(F_s A) */
                double fv = ci, dv = ar;
                if (fv != 0.0 || dv != 0.0) {
                    if (nraw == capraw) {
                        capraw = capraw ? 2 * capraw : 4096;
                        fraw = (double *)realloc(fraw, sizeof(double) * (size_t)capraw);
                        draw = (double *)realloc(draw, sizeof(double) * (size_t)capraw);
                        rawidx = (int32_t *)realloc(rawidx, sizeof(int32_t) * 3 * (size_t)capraw);
                    }
                    fraw[nraw] = fv; draw[nraw] = dv;
                    rawidx[3 * nraw] = (int32_t)m;
                    rawidx[3 * nraw + 1] = (int32_t)n;
                    rawidx[3 * nraw + 2] = (int32_t)s;
                    nraw++;
                }
            }
            scr_clear(&Pm); scr_clear(&Cm); scr_clear(&Am);
        }
    }
    /* threshold relative to the largest magnitude of each tensor */
    double fmax = 0, dmax = 0;
    for (int64_t r = 0; r < nraw; ++r) {
        if (fabs(fraw[r]) > fmax) fmax = fabs(fraw[r]);
        if (fabs(draw[r]) > dmax) dmax = fabs(draw[r]);
    }
    for (int64_t r = 0; r < nraw; ++r) {
        int32_t *x = &rawidx[3 * r];
        if (fabs(fraw[r]) > 1e-12 * fmax) tl_push(&tf, x[0], x[1], x[2], fraw[r]);
        if (fabs(draw[r]) > 1e-12 * dmax) tl_push(&td, x[0], x[1], x[2], draw[r]);
    }
    free(fraw); free(draw); free(rawidx);
    c->nf = tf.n; c->f_idx = tf.idx; c->f_val = tf.val;
    c->nd = td.n; c->d_idx = td.idx; c->d_val = td.val;

    scr_free(&Pm); scr_free(&Cm); scr_free(&Am);
    free(cand_mark); free(cand); free(seen); free(nlist);
    for (int v = 0; v < N; ++v) free(touch[v]);
    free(touch); free(ntouch); free(fill);
}

ora_ctx *ora_create(int N) {
    if (N < 2) return NULL;
    ora_ctx *c = (ora_ctx *)calloc(1, sizeof(ora_ctx));
    c->N = N;
    c->M = (int64_t)N * N - 1;
    c->P = (int64_t)N * (N - 1) / 2;
    build_basis(c);
    enumerate_fd(c);
    return c;
}

void ora_destroy(ora_ctx *c) {
    if (!c) return;
    for (int64_t i = 0; i < c->M; ++i) sp_free(&c->F[i]);
    free(c->F);
    free(c->f_idx); free(c->f_val); free(c->d_idx); free(c->d_val);
    free(c);
}

int64_t ora_M(const ora_ctx *c) { return c->M; }

/* Dense copy of basis element i (N x N complex, interleaved re,im). */
void ora_basis_dense(const ora_ctx *c, int64_t i, double *out) {
    int N = c->N;
    memset(out, 0, sizeof(double) * 2 * (size_t)N * N);
    const sp_mat *A = &c->F[i];
    for (int e = 0; e < A->nnz; ++e) {
        size_t p = (size_t)A->row[e] * N + A->col[e];
        out[2 * p] = A->re[e];
        out[2 * p + 1] = A->im[e];
    }
}

/* which: 0 = f, 1 = d.  ordered != 0 -> all ordered triples, else only m<=n<=s. */
int64_t ora_nnz(const ora_ctx *c, int which, int ordered) {
    int64_t n = which ? c->nd : c->nf;
    const int32_t *x = which ? c->d_idx : c->f_idx;
    if (ordered) return n;
    int64_t k = 0;
    for (int64_t r = 0; r < n; ++r)
        if (x[3 * r] <= x[3 * r + 1] && x[3 * r + 1] <= x[3 * r + 2]) k++;
    return k;
}

static const int32_t *g_sort_idx;
static int cmp_triple(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    const int32_t *x = &g_sort_idx[3 * a], *y = &g_sort_idx[3 * b];
    for (int q = 0; q < 3; ++q) {
        if (x[q] < y[q]) return -1;
        if (x[q] > y[q]) return 1;
    }
    return 0;
}

/* Canonical list (m<=n<=s), sorted lexicographically, with values. */
void ora_export(const ora_ctx *c, int which, int32_t *idx3, double *val) {
    int64_t n = which ? c->nd : c->nf;
    const int32_t *x = which ? c->d_idx : c->f_idx;
    const double *v = which ? c->d_val : c->f_val;
    int64_t k = 0;
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t r = 0; r < n; ++r)
        if (x[3 * r] <= x[3 * r + 1] && x[3 * r + 1] <= x[3 * r + 2]) ord[k++] = r;
    g_sort_idx = x;
    qsort(ord, (size_t)k, sizeof(int64_t), cmp_triple);
    for (int64_t q = 0; q < k; ++q) {
        int64_t r = ord[q];
        idx3[3 * q] = x[3 * r]; idx3[3 * q + 1] = x[3 * r + 1]; idx3[3 * q + 2] = x[3 * r + 2];
        val[q] = v[r];
    }
    free(ord);
}

/* All ordered triples (unsorted) -- for symmetry checks in the tests. */
void ora_export_ordered(const ora_ctx *c, int which, int32_t *idx3, double *val) {
    int64_t n = which ? c->nd : c->nf;
    memcpy(idx3, which ? c->d_idx : c->f_idx, sizeof(int32_t) * 3 * (size_t)n);
    memcpy(val, which ? c->d_val : c->f_val, sizeof(double) * (size_t)n);
}

/* Eq. (02): coef_j = Tr(F_j A) for j = 0..M-1 (complex, interleaved);
 * a0 = Tr(A)/N (complex).  A is N x N complex row-major, interleaved. */
void ora_expand(const ora_ctx *c, const double *A, double *coef, double *a0) {
    int N = c->N;
    for (int64_t j = 0; j < c->M; ++j) {
        const sp_mat *F = &c->F[j];
        double sr = 0, si = 0;
        for (int e = 0; e < F->nnz; ++e) {
            size_t q = (size_t)F->col[e] * N + F->row[e];
            double xr = A[2 * q], xi = A[2 * q + 1];
            sr += F->re[e] * xr - F->im[e] * xi;
            si += F->re[e] * xi + F->im[e] * xr;
        }
        coef[2 * j] = sr; coef[2 * j + 1] = si;
    }
    double tr = 0, ti = 0;
    for (int k = 0; k < N; ++k) { tr += A[2 * ((size_t)k * N + k)]; ti += A[2 * ((size_t)k * N + k) + 1]; }
    a0[0] = tr / N; a0[1] = ti / N;
}

/* Eq. (rho): rho = F_0 + sum_i v_i F_i, F_0 = 1/N.  Output N x N complex. */
void ora_rho(const ora_ctx *c, const double *v, double *rho) {
    int N = c->N;
    memset(rho, 0, sizeof(double) * 2 * (size_t)N * N);
    for (int k = 0; k < N; ++k) rho[2 * ((size_t)k * N + k)] = 1.0 / N;
    for (int64_t i = 0; i < c->M; ++i) {
        const sp_mat *F = &c->F[i];
        for (int e = 0; e < F->nnz; ++e) {
            size_t p = (size_t)F->row[e] * N + F->col[e];
            rho[2 * p] += v[i] * F->re[e];
            rho[2 * p + 1] += v[i] * F->im[e];
        }
    }
}

/* Eq. (07): Q[s*M+n] = sum_m h_m f_mns (dense M x M). */
void ora_Q(const ora_ctx *c, const double *h, double *Q) {
    int64_t M = c->M;
    memset(Q, 0, sizeof(double) * (size_t)M * M);
    for (int64_t r = 0; r < c->nf; ++r) {
        int32_t m = c->f_idx[3 * r], n = c->f_idx[3 * r + 1], s = c->f_idx[3 * r + 2];
        Q[(size_t)s * M + n] += h[m] * c->f_val[r];
    }
}

/* Eq. (08): k_s = (i/N) sum_jk a_jk f_jks; a is M x M complex (interleaved).
 * Kimag receives the imaginary part of the result (zero for Hermitian a). */
void ora_K(const ora_ctx *c, const double *a, double *K, double *Kimag) {
    int64_t M = c->M;
    double *sr = (double *)calloc((size_t)M, sizeof(double));
    double *si = (double *)calloc((size_t)M, sizeof(double));
    for (int64_t r = 0; r < c->nf; ++r) {
        int32_t j = c->f_idx[3 * r], k = c->f_idx[3 * r + 1], s = c->f_idx[3 * r + 2];
        size_t q = (size_t)j * M + k;
        sr[s] += a[2 * q] * c->f_val[r];
        si[s] += a[2 * q + 1] * c->f_val[r];
    }
    for (int64_t s = 0; s < M; ++s) {
        /* (i/N)(sr + i si) = (-si + i sr)/N */
        K[s] = -si[s] / c->N;
        if (Kimag) Kimag[s] = sr[s] / c->N;
    }
    free(sr); free(si);
}

/* Eq. (08) with a given only where the sum reads it: ima[r] = Im a_jk for the
 * r-th ordered nonzero f_jks, in the order of ora_export_ordered.  For
 * Hermitian a, K_s = -(1/N) sum_jk Im(a_jk) f_jks (the real part of the
 * sum drops out, as in ora_K). */
void ora_K_on_f(const ora_ctx *c, const double *ima, double *K) {
    int64_t M = c->M;
    for (int64_t s = 0; s < M; ++s) K[s] = 0.0;
    for (int64_t r = 0; r < c->nf; ++r) {
        int32_t s = c->f_idx[3 * r + 2];
        K[s] += ima[r] * c->f_val[r];
    }
    for (int64_t s = 0; s < M; ++s) K[s] = -K[s] / c->N;
}

/* Lists grouped by the middle index l: F-section (k,s,f_kls) and
 * Z-section (j,n,z_jln); f and d never share a position, so z items are
 * either (f,0) or (0,d). */
typedef struct {
    int64_t *fptr, *zptr;
    int32_t *fk, *fs; double *fv;
    int32_t *zj, *zn; double *zr, *zi;
} sections;

static void build_sections(const ora_ctx *c, sections *S) {
    int64_t M = c->M;
    S->fptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    S->zptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    for (int64_t r = 0; r < c->nf; ++r) { S->fptr[c->f_idx[3 * r + 1] + 1]++; S->zptr[c->f_idx[3 * r + 1] + 1]++; }
    for (int64_t r = 0; r < c->nd; ++r) S->zptr[c->d_idx[3 * r + 1] + 1]++;
    for (int64_t l = 0; l < M; ++l) { S->fptr[l + 1] += S->fptr[l]; S->zptr[l + 1] += S->zptr[l]; }
    int64_t nf = S->fptr[M], nz = S->zptr[M];
    S->fk = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf); S->fs = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf);
    S->fv = (double *)malloc(sizeof(double) * (size_t)nf);
    S->zj = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz); S->zn = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz);
    S->zr = (double *)malloc(sizeof(double) * (size_t)nz); S->zi = (double *)malloc(sizeof(double) * (size_t)nz);
    int64_t *pf = (int64_t *)malloc(sizeof(int64_t) * (size_t)M), *pz = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);
    memcpy(pf, S->fptr, sizeof(int64_t) * (size_t)M); memcpy(pz, S->zptr, sizeof(int64_t) * (size_t)M);
    for (int64_t r = 0; r < c->nf; ++r) {
        int32_t a = c->f_idx[3 * r], l = c->f_idx[3 * r + 1], b = c->f_idx[3 * r + 2];
        int64_t q = pf[l]++;
        S->fk[q] = a; S->fs[q] = b; S->fv[q] = c->f_val[r];
        q = pz[l]++;
        S->zj[q] = a; S->zn[q] = b; S->zr[q] = c->f_val[r]; S->zi[q] = 0.0;
    }
    for (int64_t r = 0; r < c->nd; ++r) {
        int32_t a = c->d_idx[3 * r], l = c->d_idx[3 * r + 1], b = c->d_idx[3 * r + 2];
        int64_t q = pz[l]++;
        S->zj[q] = a; S->zn[q] = b; S->zr[q] = 0.0; S->zi[q] = c->d_val[r];
    }
    free(pf); free(pz);
}

static void free_sections(sections *S) {
    free(S->fptr); free(S->zptr); free(S->fk); free(S->fs); free(S->fv);
    free(S->zj); free(S->zn); free(S->zr); free(S->zi);
}

/* Number of join terms W = sum_l |Z-section(l)| * |F-section(l)|. */
int64_t ora_join_terms(const ora_ctx *c) {
    sections S;
    build_sections(c, &S);
    int64_t W = 0;
    for (int64_t l = 0; l < c->M; ++l)
        W += (S.zptr[l + 1] - S.zptr[l]) * (S.fptr[l + 1] - S.fptr[l]);
    free_sections(&S);
    return W;
}

/*
 * Eq. (09), both printed terms, prefactor -1/4:
 *   r_sn = -1/4 sum_l sum_jk a_jk ( z_jln f_kls + conj(z_kln) f_jls ).
 * R receives the real part (M x M, R[s*M+n]); Rimag (optional) the imaginary
 * part, which must vanish; Sc (optional) the scale 1/4 sum |term|.
 */
void ora_R(const ora_ctx *c, const double *a, double *R, double *Rimag, double *Sc) {
    int64_t M = c->M;
    sections S;
    build_sections(c, &S);
    double *acc_i = (double *)calloc((size_t)M * M, sizeof(double));
    double *acc_s = (double *)calloc((size_t)M * M, sizeof(double));
    memset(R, 0, sizeof(double) * (size_t)M * M);
    for (int64_t l = 0; l < M; ++l) {
        for (int64_t zq = S.zptr[l]; zq < S.zptr[l + 1]; ++zq) {
            int32_t x = S.zj[zq], n = S.zn[zq];
            double zr = S.zr[zq], zi = S.zi[zq];
            for (int64_t fq = S.fptr[l]; fq < S.fptr[l + 1]; ++fq) {
                int32_t y = S.fk[fq], s = S.fs[fq];
                double fv = S.fv[fq];
                size_t o = (size_t)s * M + n;
                /* first term: j = x, k = y: a_jk z_jln f_kls */
                size_t q1 = (size_t)x * M + y;
                double ar = a[2 * q1], ai = a[2 * q1 + 1];
                double t1r = (ar * zr - ai * zi) * fv, t1i = (ar * zi + ai * zr) * fv;
                /* second term: k = x, j = y: a_jk conj(z_kln) f_jls */
                size_t q2 = (size_t)y * M + x;
                double br = a[2 * q2], bi = a[2 * q2 + 1];
                double t2r = (br * zr + bi * zi) * fv, t2i = (bi * zr - br * zi) * fv;
                R[o] += t1r + t2r;
                acc_i[o] += t1i + t2i;
                acc_s[o] += sqrt(t1r * t1r + t1i * t1i) + sqrt(t2r * t2r + t2i * t2i);
            }
        }
    }
    for (size_t o = 0; o < (size_t)M * M; ++o) {
        R[o] *= -0.25;
        if (Rimag) Rimag[o] = -0.25 * acc_i[o];
        if (Sc) Sc[o] = 0.25 * acc_s[o];
    }
    free(acc_i); free(acc_s);
    free_sections(&S);
}

/* Lists grouped by the LAST index, sorted by the middle one, for evaluating
 * single entries r_sn: Fc(s) = {(k,l,f_kls)}, Zc(n) = {(j,l,z_jln)}. */
typedef struct {
    int64_t *fptr, *zptr;
    int32_t *fk, *fl; double *fv;
    int32_t *zj, *zl; double *zr, *zi;
} columns;

static int64_t *g_key;
static int cmp_key(const void *pa, const void *pb) {
    int64_t a = g_key[*(const int64_t *)pa], b = g_key[*(const int64_t *)pb];
    return a < b ? -1 : (a > b ? 1 : 0);
}

static void build_columns(const ora_ctx *c, columns *C) {
    int64_t M = c->M, nf = c->nf, nz = c->nf + c->nd;
    C->fptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    C->zptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    /* sort f items by (last, middle) and z items likewise */
    int64_t *kf = (int64_t *)malloc(sizeof(int64_t) * (size_t)nf), *of = (int64_t *)malloc(sizeof(int64_t) * (size_t)nf);
    for (int64_t r = 0; r < nf; ++r) { kf[r] = (int64_t)c->f_idx[3 * r + 2] * M + c->f_idx[3 * r + 1]; of[r] = r; }
    g_key = kf; qsort(of, (size_t)nf, sizeof(int64_t), cmp_key);
    int64_t *kz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nz), *oz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nz);
    for (int64_t r = 0; r < nz; ++r) {
        const int32_t *x = r < nf ? &c->f_idx[3 * r] : &c->d_idx[3 * (r - nf)];
        kz[r] = (int64_t)x[2] * M + x[1]; oz[r] = r;
    }
    g_key = kz; qsort(oz, (size_t)nz, sizeof(int64_t), cmp_key);
    C->fk = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf); C->fl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf);
    C->fv = (double *)malloc(sizeof(double) * (size_t)nf);
    C->zj = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz); C->zl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz);
    C->zr = (double *)malloc(sizeof(double) * (size_t)nz); C->zi = (double *)malloc(sizeof(double) * (size_t)nz);
    for (int64_t q = 0; q < nf; ++q) {
        int64_t r = of[q];
        C->fk[q] = c->f_idx[3 * r]; C->fl[q] = c->f_idx[3 * r + 1]; C->fv[q] = c->f_val[r];
        C->fptr[c->f_idx[3 * r + 2] + 1]++;
    }
    for (int64_t q = 0; q < nz; ++q) {
        int64_t r = oz[q];
        if (r < nf) {
            C->zj[q] = c->f_idx[3 * r]; C->zl[q] = c->f_idx[3 * r + 1];
            C->zr[q] = c->f_val[r]; C->zi[q] = 0.0;
            C->zptr[c->f_idx[3 * r + 2] + 1]++;
        } else {
            r -= nf;
            C->zj[q] = c->d_idx[3 * r]; C->zl[q] = c->d_idx[3 * r + 1];
            C->zr[q] = 0.0; C->zi[q] = c->d_val[r];
            C->zptr[c->d_idx[3 * r + 2] + 1]++;
        }
    }
    for (int64_t s = 0; s < M; ++s) { C->fptr[s + 1] += C->fptr[s]; C->zptr[s + 1] += C->zptr[s]; }
    free(kf); free(of); free(kz); free(oz);
}

static void free_columns(columns *C) {
    free(C->fptr); free(C->zptr); free(C->fk); free(C->fl); free(C->fv);
    free(C->zj); free(C->zl); free(C->zr); free(C->zi);
}

/*
 * Eq. (09) for selected entries (s_i, n_i) only; same two-term form and
 * prefactor as ora_R.  a_at(j,k) reads the dense M x M complex matrix.
 * Entries are independent, so they may be spread over OpenMP threads.
 */
void ora_R_entries(const ora_ctx *c, const double *a, int64_t cnt,
                   const int64_t *si, const int64_t *ni, double *out,
                   double *out_imag, double *out_scale) {
    int64_t M = c->M;
    columns C;
    build_columns(c, &C);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < cnt; ++e) {
        int64_t s = si[e], n = ni[e];
        double accr = 0, acci = 0, accs = 0;
        int64_t pf = C.fptr[s], ef = C.fptr[s + 1];
        int64_t pz = C.zptr[n], ez = C.zptr[n + 1];
        /* merge-join on the middle index l (both lists sorted by l) */
        while (pf < ef && pz < ez) {
            int32_t lf = C.fl[pf], lz = C.zl[pz];
            if (lf < lz) { pf++; continue; }
            if (lz < lf) { pz++; continue; }
            int64_t f0 = pf, z0 = pz;
            while (pf < ef && C.fl[pf] == lf) pf++;
            while (pz < ez && C.zl[pz] == lf) pz++;
            for (int64_t zq = z0; zq < pz; ++zq)
                for (int64_t fq = f0; fq < pf; ++fq) {
                    int32_t x = C.zj[zq], y = C.fk[fq];
                    double zr = C.zr[zq], zi = C.zi[zq], fv = C.fv[fq];
                    size_t q1 = (size_t)x * M + y, q2 = (size_t)y * M + x;
                    double ar = a[2 * q1], ai = a[2 * q1 + 1];
                    double br = a[2 * q2], bi = a[2 * q2 + 1];
                    double t1r = (ar * zr - ai * zi) * fv, t1i = (ar * zi + ai * zr) * fv;
                    double t2r = (br * zr + bi * zi) * fv, t2i = (bi * zr - br * zi) * fv;
                    accr += t1r + t2r; acci += t1i + t2i;
                    accs += sqrt(t1r * t1r + t1i * t1i) + sqrt(t2r * t2r + t2i * t2i);
                }
        }
        out[e] = -0.25 * accr;
        if (out_imag) out_imag[e] = -0.25 * acci;
        if (out_scale) out_scale[e] = 0.25 * accs;
    }
    free_columns(&C);
}

/*
 * The rows of a that ora_R_entries_rows needs for entries with row indices
 * si: the first indices k of every f_kls with s in si (both terms of
 * Eq. (09) read a only at (j,k) and (k,j) with such a k).  Returns the count;
 * fills out (sorted, unique) when out != NULL and cap suffices.
 */
int64_t ora_R_rows_needed(const ora_ctx *c, int64_t cnt, const int64_t *si, int64_t *out, int64_t cap) {
    int64_t M = c->M;
    columns C;
    build_columns(c, &C);
    char *mark = (char *)calloc((size_t)M, 1);
    for (int64_t e = 0; e < cnt; ++e)
        for (int64_t q = C.fptr[si[e]]; q < C.fptr[si[e] + 1]; ++q) mark[C.fk[q]] = 1;
    int64_t n = 0;
    for (int64_t k = 0; k < M; ++k)
        if (mark[k]) {
            if (out && n < cap) out[n] = k;
            n++;
        }
    free(mark);
    free_columns(&C);
    return n;
}

/*
 * Eq. (09) at selected entries, with a given only by some of its rows:
 * rows[r*M + j] = a_{row_ids[r], j} (row_ids sorted).  Same two-term form and
 * prefactor as ora_R; an a_jk whose row is not supplied is read as
 * conj(a_kj) (a is Hermitian).  Returns -1 if a needed value is missing.
 */
static int find_row(const int64_t *ids, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ids[mid] == k) return (int)mid;
        if (ids[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int ora_R_entries_rows(const ora_ctx *c, int64_t nrows, const int64_t *row_ids, const double *rows,
                       int64_t cnt, const int64_t *si, const int64_t *ni, double *out, double *out_scale) {
    int64_t M = c->M;
    columns C;
    build_columns(c, &C);
    int missing = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : missing)
    for (int64_t e = 0; e < cnt; ++e) {
        int64_t s = si[e], n = ni[e];
        double accr = 0, accs = 0;
        int64_t pf = C.fptr[s], ef = C.fptr[s + 1];
        int64_t pz = C.zptr[n], ez = C.zptr[n + 1];
        while (pf < ef && pz < ez) {
            int32_t lf = C.fl[pf], lz = C.zl[pz];
            if (lf < lz) { pf++; continue; }
            if (lz < lf) { pz++; continue; }
            int64_t f0 = pf, z0 = pz;
            while (pf < ef && C.fl[pf] == lf) pf++;
            while (pz < ez && C.zl[pz] == lf) pz++;
            for (int64_t fq = f0; fq < pf; ++fq) {
                int32_t y = C.fk[fq];
                int r = find_row(row_ids, nrows, y);
                if (r < 0) { missing = 1; continue; }
                const double *row = rows + 2 * (size_t)r * M;
                for (int64_t zq = z0; zq < pz; ++zq) {
                    int32_t x = C.zj[zq];
                    double zr = C.zr[zq], zi = C.zi[zq], fv = C.fv[fq];
                    /* a_xy = conj(a_yx), a_yx from row y */
                    double br = row[2 * (size_t)x], bi = row[2 * (size_t)x + 1];
                    double ar = br, ai = -bi;
                    double t1r = (ar * zr - ai * zi) * fv, t1i = (ar * zi + ai * zr) * fv;
                    double t2r = (br * zr + bi * zi) * fv, t2i = (bi * zr - br * zi) * fv;
                    accr += t1r + t2r;
                    accs += sqrt(t1r * t1r + t1i * t1i) + sqrt(t2r * t2r + t2i * t2i);
                }
            }
        }
        out[e] = -0.25 * accr;
        if (out_scale) out_scale[e] = 0.25 * accs;
    }
    free_columns(&C);
    return missing ? -1 : 0;
}

/* Eq. (07) for selected entries. */
void ora_Q_entries(const ora_ctx *c, const double *h, int64_t cnt,
                   const int64_t *si, const int64_t *ni, double *out) {
    columns C;
    build_columns(c, &C);
    for (int64_t e = 0; e < cnt; ++e) {
        int64_t s = si[e], n = ni[e];
        double acc = 0;
        /* f_mns with last index s and middle index n: Fc(s) items with l == n */
        for (int64_t q = C.fptr[s]; q < C.fptr[s + 1]; ++q)
            if (C.fl[q] == n) acc += h[C.fk[q]] * C.fv[q];
        out[e] = acc;
    }
    free_columns(&C);
}

/*
 * Eq. (09) for a Kossakowski matrix given in spectral (low-rank) form,
 * a_jk = sum_p gamma_p l_pj conj(l_pk), with sparse l_p.  Only the nonzero
 * a_jk are visited.  Output dense M x M (small N) plus the symbolic mask:
 * mask[s*M+n] = 1 iff some (p, j, k, l) with l_pj != 0, l_pk != 0,
 * z_jln != 0 and f_kls != 0 reaches (s, n).
 * lp_ptr: P+1 offsets into (lp_idx, lp_re, lp_im).
 */
void ora_R_lowrank(const ora_ctx *c, int nP, const double *gamma,
                   const int64_t *lp_ptr, const int64_t *lp_idx,
                   const double *lp_re, const double *lp_im,
                   double *R, unsigned char *mask) {
    int64_t M = c->M;
    sections S;
    build_sections(c, &S);
    memset(R, 0, sizeof(double) * (size_t)M * M);
    if (mask) memset(mask, 0, (size_t)M * M);
    /* per-element sorted lists of (l, n) for z and (l, s) for f keyed by
     * the FIRST index, derived from the sections */
    /* simple approach: for every nonzero a_jk, loop over all l and test */
    for (int p = 0; p < nP; ++p) {
        for (int64_t u = lp_ptr[p]; u < lp_ptr[p + 1]; ++u)
            for (int64_t w = lp_ptr[p]; w < lp_ptr[p + 1]; ++w) {
                int64_t j = lp_idx[u], k = lp_idx[w];
                /* a_jk = gamma l_j conj(l_k) */
                double ar = gamma[p] * (lp_re[u] * lp_re[w] + lp_im[u] * lp_im[w]);
                double ai = gamma[p] * (lp_im[u] * lp_re[w] - lp_re[u] * lp_im[w]);
                for (int64_t l = 0; l < M; ++l) {
                    for (int64_t zq = S.zptr[l]; zq < S.zptr[l + 1]; ++zq) {
                        int32_t x = S.zj[zq], n = S.zn[zq];
                        if (x != j && x != k) continue;
                        for (int64_t fq = S.fptr[l]; fq < S.fptr[l + 1]; ++fq) {
                            int32_t y = S.fk[fq], s = S.fs[fq];
                            double zr = S.zr[zq], zi = S.zi[zq], fv = S.fv[fq];
                            size_t o = (size_t)s * M + n;
                            if (x == j && y == k) {  /* a_jk z_jln f_kls */
                                R[o] += (ar * zr - ai * zi) * fv;
                                if (mask) mask[o] = 1;
                            }
                            if (x == k && y == j) {  /* a_jk conj(z_kln) f_jls */
                                R[o] += (ar * zr + ai * zi) * fv;
                                if (mask) mask[o] = 1;
                            }
                        }
                    }
                }
            }
    }
    for (size_t o = 0; o < (size_t)M * M; ++o) R[o] *= -0.25;
    free_sections(&S);
}

/* ---------------------------------------------- sparse (CSR) assembly */

/* open-addressing map (s*M + n) -> value, for the sparse generator */
typedef struct { int64_t cap, n; int64_t *key; double *val, *abs; } hmap;

static void hm_init(hmap *h, int64_t cap) {
    int64_t c = 1024;
    while (c < 2 * cap) c <<= 1;
    h->cap = c; h->n = 0;
    h->key = (int64_t *)malloc(sizeof(int64_t) * (size_t)c);
    h->val = (double *)calloc((size_t)c, sizeof(double));
    h->abs = (double *)calloc((size_t)c, sizeof(double));
    for (int64_t i = 0; i < c; ++i) h->key[i] = -1;
}

static void hm_add(hmap *h, int64_t key, double v, double a);

static void hm_grow(hmap *h) {
    hmap g;
    hm_init(&g, h->cap);
    for (int64_t i = 0; i < h->cap; ++i)
        if (h->key[i] >= 0) hm_add(&g, h->key[i], h->val[i], h->abs[i]);
    free(h->key); free(h->val); free(h->abs);
    *h = g;
}

/* value v with its absolute size a (for the entry's scale) */
static void hm_add(hmap *h, int64_t key, double v, double a) {
    if (2 * (h->n + 1) > h->cap) hm_grow(h);
    uint64_t x = (uint64_t)key * 0x9E3779B97F4A7C15ULL;
    int64_t i = (int64_t)(x >> 11) & (h->cap - 1);
    while (h->key[i] >= 0 && h->key[i] != key) i = (i + 1) & (h->cap - 1);
    if (h->key[i] < 0) { h->key[i] = key; h->n++; }
    h->val[i] += v;
    h->abs[i] += a;
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Lists keyed by the FIRST index: Ff(k) = {(l, s, f_kls)}, Zf(j) = {(l, n, z_jln)}. */
typedef struct {
    int64_t *fptr, *zptr;
    int32_t *fl, *fs; double *fv;
    int32_t *zl, *zn; double *zr, *zi;
} firsts;

static void build_firsts(const ora_ctx *c, firsts *F) {
    int64_t M = c->M, nf = c->nf, nz = c->nf + c->nd;
    F->fptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    F->zptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    /* order the items by (first, middle) */
    int64_t *kf = (int64_t *)malloc(sizeof(int64_t) * (size_t)nf), *of = (int64_t *)malloc(sizeof(int64_t) * (size_t)nf);
    for (int64_t r = 0; r < nf; ++r) { kf[r] = (int64_t)c->f_idx[3 * r] * M + c->f_idx[3 * r + 1]; of[r] = r; }
    g_key = kf; qsort(of, (size_t)nf, sizeof(int64_t), cmp_key);
    int64_t *kz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nz), *oz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nz);
    for (int64_t r = 0; r < nz; ++r) {
        const int32_t *x = r < nf ? &c->f_idx[3 * r] : &c->d_idx[3 * (r - nf)];
        kz[r] = (int64_t)x[0] * M + x[1]; oz[r] = r;
    }
    g_key = kz; qsort(oz, (size_t)nz, sizeof(int64_t), cmp_key);
    F->fl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf); F->fs = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf);
    F->fv = (double *)malloc(sizeof(double) * (size_t)nf);
    F->zl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz); F->zn = (int32_t *)malloc(sizeof(int32_t) * (size_t)nz);
    F->zr = (double *)malloc(sizeof(double) * (size_t)nz); F->zi = (double *)malloc(sizeof(double) * (size_t)nz);
    for (int64_t q = 0; q < nf; ++q) {
        const int32_t *x = &c->f_idx[3 * of[q]];
        F->fl[q] = x[1]; F->fs[q] = x[2]; F->fv[q] = c->f_val[of[q]];
        F->fptr[x[0] + 1]++;
    }
    for (int64_t q = 0; q < nz; ++q) {
        int64_t r = oz[q];
        const int32_t *x = r < nf ? &c->f_idx[3 * r] : &c->d_idx[3 * (r - nf)];
        F->zl[q] = x[1]; F->zn[q] = x[2];
        F->zr[q] = r < nf ? c->f_val[r] : 0.0;
        F->zi[q] = r < nf ? 0.0 : c->d_val[r - nf];
        F->zptr[x[0] + 1]++;
    }
    for (int64_t i = 0; i < M; ++i) { F->fptr[i + 1] += F->fptr[i]; F->zptr[i + 1] += F->zptr[i]; }
    free(kf); free(of); free(kz); free(oz);
}

static void free_firsts(firsts *F) {
    free(F->fptr); free(F->zptr); free(F->fl); free(F->fs); free(F->fv);
    free(F->zl); free(F->zn); free(F->zr); free(F->zi);
}

/*
 * The generator for a Kossakowski matrix in spectral form,
 * a_jk = sum_p gamma_p l_pj conj(l_pk) (sparse l_p), and sparse real h, as a
 * CSR matrix A = Q + R.  Terms: h_m f_mns with h_m != 0 (Eq. (07)) and
 * a_jk z_jln f_kls, a_jk conj(z_kln) f_jls with (j, k) in the support of some
 * l_p (Eq. (09), two-term form, prefactor -1/4).  Pattern: the (s, n) whose
 * summed value exceeds 1e-12 times the sum of its terms' magnitudes --
 * entries whose terms cancel exactly (most of the ones the terms reach, for
 * ladder-type models) are dropped, genuine nonzeros kept.
 * Also K (Eq. (08)), dense.  The Eq. (09) sums run over the nonzero a_jk,
 * joining the first-index lists of j and k on the middle index l.
 * Arrays are malloc'ed; release with ora_free.
 */
int64_t ora_lowrank_csr(const ora_ctx *c, const double *h, int nP, const double *gamma,
                        const int64_t *lp_ptr, const int64_t *lp_idx, const double *lp_re,
                        const double *lp_im, int64_t **rowptr_out, int32_t **col_out,
                        double **val_out, double **mag_out, double *K) {
    int64_t M = c->M;
    firsts F;
    build_firsts(c, &F);
    hmap hm;
    hm_init(&hm, 16 * M);
    /* Q */
    if (h)
        for (int64_t m = 0; m < M; ++m) {
            if (h[m] == 0.0) continue;
            for (int64_t q = F.fptr[m]; q < F.fptr[m + 1]; ++q)
                hm_add(&hm, (int64_t)F.fs[q] * M + F.fl[q], h[m] * F.fv[q], fabs(h[m] * F.fv[q]));  /* f_{m n s}: n = l, s */
        }
    /* the union of the channel supports, and a_jk on it */
    memset(K, 0, sizeof(double) * (size_t)M);
    double *Ki = (double *)calloc((size_t)M, sizeof(double));
    for (int p = 0; p < nP; ++p)
        for (int64_t u = lp_ptr[p]; u < lp_ptr[p + 1]; ++u)
            for (int64_t w = lp_ptr[p]; w < lp_ptr[p + 1]; ++w) {
                int64_t j = lp_idx[u], k = lp_idx[w];
                double ar = gamma[p] * (lp_re[u] * lp_re[w] + lp_im[u] * lp_im[w]);
                double ai = gamma[p] * (lp_im[u] * lp_re[w] - lp_re[u] * lp_im[w]);
                /* term 1: a_jk z_jln f_kls; term 2 of the pair (k, j) is added when
                 * the loop reaches (k, j): a_kj conj(z_jln) f_kls, i.e. the printed
                 * a_jk conj(z_kln) f_jls with the names exchanged */
                int64_t zq = F.zptr[j], ze = F.zptr[j + 1], fq = F.fptr[k], fe = F.fptr[k + 1];
                /* merge-join on l (both lists sorted by l) */
                while (zq < ze && fq < fe) {
                    int32_t lz = F.zl[zq], lf = F.fl[fq];
                    if (lz < lf) { zq++; continue; }
                    if (lf < lz) { fq++; continue; }
                    int64_t z0 = zq, f0 = fq;
                    while (zq < ze && F.zl[zq] == lz) zq++;
                    while (fq < fe && F.fl[fq] == lz) fq++;
                    for (int64_t a = z0; a < zq; ++a)
                        for (int64_t b = f0; b < fq; ++b) {
                            double zr = F.zr[a], zi = F.zi[a], fv = F.fv[b];
                            int64_t key = (int64_t)F.fs[b] * M + F.zn[a];
                            /* a_jk z f */
                            double t1 = (ar * zr - ai * zi) * fv;
                            /* the second printed term, written for the pair (j', k') = (k, j):
                             * a_{k j} conj(z_{j l n}) f_{k l s} -- a_kj = conj(a_jk) */
                            double t2 = (ar * zr - ai * zi) * fv;
                            double mag = sqrt(ar * ar + ai * ai) * sqrt(zr * zr + zi * zi) * fabs(fv);
                            hm_add(&hm, key, -0.25 * (t1 + t2), 0.5 * mag);
                        }
                }
                /* Eq. (08): (i/N) a_jk f_jks */
                for (int64_t b = F.fptr[j]; b < F.fptr[j + 1]; ++b)
                    if (F.fl[b] == k) {
                        K[F.fs[b]] += -ai * F.fv[b] / c->N;
                        Ki[F.fs[b]] += ar * F.fv[b] / c->N;
                    }
            }
    free(Ki);
    /* to CSR, columns sorted; an entry is kept iff its value is not below
     * 1e-12 of the sum of the magnitudes of its terms (terms that cancel
     * exactly leave rounding residue only) */
    int64_t nnz = 0, t = 0;
    for (int64_t i = 0; i < hm.cap; ++i)
        if (hm.key[i] >= 0 && fabs(hm.val[i]) > 1e-12 * hm.abs[i]) nnz++;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz + 1));
    for (int64_t i = 0; i < hm.cap; ++i)
        if (hm.key[i] >= 0 && fabs(hm.val[i]) > 1e-12 * hm.abs[i]) keys[t++] = hm.key[i];
    qsort(keys, (size_t)nnz, sizeof(int64_t), cmp_i64);
    int64_t *rowptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    double *val = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *mag = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t key = keys[e];
        uint64_t x = (uint64_t)key * 0x9E3779B97F4A7C15ULL;
        int64_t i = (int64_t)(x >> 11) & (hm.cap - 1);
        while (hm.key[i] != key) i = (i + 1) & (hm.cap - 1);
        rowptr[key / M + 1]++;
        col[e] = (int32_t)(key % M);
        val[e] = hm.val[i];
        mag[e] = hm.abs[i];
    }
    for (int64_t s = 0; s < M; ++s) rowptr[s + 1] += rowptr[s];
    free(keys); free(hm.key); free(hm.val); free(hm.abs);
    free_firsts(&F);
    *rowptr_out = rowptr; *col_out = col; *val_out = val; *mag_out = mag;
    return nnz;
}

void ora_free(void *p) { free(p); }

/* -------------------------------------------------------------- RK4 */

/* y = A x + K (dense, row-major M x M) */
static void dense_rhs(int64_t M, const double *A, const double *K, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < M; ++s) {
        const double *row = A + (size_t)s * M;
        double acc = 0;
        for (int64_t n = 0; n < M; ++n) acc += row[n] * x[n];
        y[s] = acc + K[s];
    }
}

/*
 * Classical RK4 with fixed step dt for dv/dt = A v + K (Eq. (04) with
 * time-independent Q and R), nsteps steps.  Snapshots of v after every
 * snap_every steps go to out ((nsteps/snap_every) x M); the final v to vout.
 */
void ora_rk4_dense(int64_t M, const double *A, const double *K, const double *v0,
                   double dt, int64_t nsteps, int64_t snap_every, double *out, double *vout) {
    double *v = (double *)malloc(sizeof(double) * (size_t)M);
    double *x = (double *)malloc(sizeof(double) * (size_t)M);
    double *k1 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k2 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k3 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k4 = (double *)malloc(sizeof(double) * (size_t)M);
    memcpy(v, v0, sizeof(double) * (size_t)M);
    int64_t snap = 0;
    for (int64_t t = 0; t < nsteps; ++t) {
        dense_rhs(M, A, K, v, k1);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k1[i];
        dense_rhs(M, A, K, x, k2);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k2[i];
        dense_rhs(M, A, K, x, k3);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + dt * k3[i];
        dense_rhs(M, A, K, x, k4);
        for (int64_t i = 0; i < M; ++i)
            v[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        if (out && snap_every > 0 && (t + 1) % snap_every == 0) {
            memcpy(out + (size_t)snap * M, v, sizeof(double) * (size_t)M);
            snap++;
        }
    }
    if (vout) memcpy(vout, v, sizeof(double) * (size_t)M);
    free(v); free(x); free(k1); free(k2); free(k3); free(k4);
}

/* y = A x + K for CSR A (int64 row pointers, int32 columns). */
static void csr_rhs(int64_t M, const int64_t *rp, const int32_t *ci, const double *val,
                    const double *K, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < M; ++s) {
        double acc = 0;
        for (int64_t q = rp[s]; q < rp[s + 1]; ++q) acc += val[q] * x[ci[q]];
        y[s] = acc + (K ? K[s] : 0.0);
    }
}

void ora_rk4_csr(int64_t M, const int64_t *rp, const int32_t *ci, const double *val,
                 const double *K, const double *v0, double dt, int64_t nsteps, double *vout) {
    double *v = (double *)malloc(sizeof(double) * (size_t)M);
    double *x = (double *)malloc(sizeof(double) * (size_t)M);
    double *k1 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k2 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k3 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k4 = (double *)malloc(sizeof(double) * (size_t)M);
    memcpy(v, v0, sizeof(double) * (size_t)M);
    for (int64_t t = 0; t < nsteps; ++t) {
        csr_rhs(M, rp, ci, val, K, v, k1);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k1[i];
        csr_rhs(M, rp, ci, val, K, x, k2);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k2[i];
        csr_rhs(M, rp, ci, val, K, x, k3);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + dt * k3[i];
        csr_rhs(M, rp, ci, val, K, x, k4);
        for (int64_t i = 0; i < M; ++i)
            v[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    memcpy(vout, v, sizeof(double) * (size_t)M);
    free(v); free(x); free(k1); free(k2); free(k3); free(k4);
}

/*
 * Classical RK4 for the time-dependent system dv/dt = (A0 + eps(t) Q1) v + K
 * (Eq. (04) with Q(t) = Q0 + eps(t) Q1, Sec. 3: the rocked dimer): every
 * stage uses eps at its own time, the stages at the ends of the step taken
 * just inside it (t + 1e-6 dt, t + dt/2, t + dt/2, t + dt - 1e-6 dt), so
 * that a step lying between two switches of eps sees one value in all four
 * stages whatever the rounding of its end times.  eps is periodic with
 * period T: eps(t) = seg_eps[k] for (t mod T) in [seg_start[k],
 * seg_start[k + 1]) (seg_start[0] = 0, the last segment ends at T).  A0, Q1
 * dense M x M; nsteps steps from time t0.
 */
static double eps_at(double t, int nseg, const double *seg_start, const double *seg_eps, double T) {
    double u = fmod(t, T);
    if (u < 0) u += T;
    int k = 0;
    while (k + 1 < nseg && u >= seg_start[k + 1]) ++k;
    return seg_eps[k];
}

static void td_rhs(int64_t M, const double *A0, const double *Q1, double eps, const double *K,
                   const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < M; ++s) {
        const double *a = A0 + (size_t)s * M, *q = Q1 + (size_t)s * M;
        double acc = 0;
        for (int64_t n = 0; n < M; ++n) acc += (a[n] + eps * q[n]) * x[n];
        y[s] = acc + K[s];
    }
}

void ora_rk4_dense_td(int64_t M, const double *A0, const double *Q1, const double *K, int nseg,
                      const double *seg_start, const double *seg_eps, double T, double t0,
                      const double *v0, double dt, int64_t nsteps, double *vout) {
    double *v = (double *)malloc(sizeof(double) * (size_t)M);
    double *x = (double *)malloc(sizeof(double) * (size_t)M);
    double *k1 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k2 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k3 = (double *)malloc(sizeof(double) * (size_t)M);
    double *k4 = (double *)malloc(sizeof(double) * (size_t)M);
    memcpy(v, v0, sizeof(double) * (size_t)M);
    for (int64_t n = 0; n < nsteps; ++n) {
        const double t = t0 + (double)n * dt;
        td_rhs(M, A0, Q1, eps_at(t + 1e-6 * dt, nseg, seg_start, seg_eps, T), K, v, k1);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k1[i];
        td_rhs(M, A0, Q1, eps_at(t + 0.5 * dt, nseg, seg_start, seg_eps, T), K, x, k2);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + 0.5 * dt * k2[i];
        td_rhs(M, A0, Q1, eps_at(t + 0.5 * dt, nseg, seg_start, seg_eps, T), K, x, k3);
        for (int64_t i = 0; i < M; ++i) x[i] = v[i] + dt * k3[i];
        td_rhs(M, A0, Q1, eps_at(t + dt - 1e-6 * dt, nseg, seg_start, seg_eps, T), K, x, k4);
        for (int64_t i = 0; i < M; ++i)
            v[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    memcpy(vout, v, sizeof(double) * (size_t)M);
    free(v); free(x); free(k1); free(k2); free(k3); free(k4);
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

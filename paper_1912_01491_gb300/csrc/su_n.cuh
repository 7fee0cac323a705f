// su_n.cuh -- index arithmetic of the generalized Gell-Mann (SU(N)) basis and
// closed-form structure constants, shared by all kernels of the library.
//
// Basis (Sec. 2, Eqs. for S^(j,k), J^(j,k), D^l), 0-based:
//   index i <  P       : S_ab = (E_ab + E_ba)/sqrt2,          pair p = i
//   P <= i < 2P        : J_ab = -i (E_ab - E_ba)/sqrt2,       pair p = i - P
//   2P <= i < M        : D_l  = (sum_{k<l} E_kk - l E_ll)/sqrt(l(l+1)), l = i - 2P + 1
// with P = N(N-1)/2, M = N^2 - 1, pairs (a<b) in lexicographic order.  D_l is
// the Hermitian, orthonormal reading of the printed D^l (Tr(F_n F_m) = delta).
//
// Structure constants (Eq. (05)) from one trace:  with T = Tr(F_s F_m F_n),
//   f_mns = -i Tr(F_s [F_m, F_n]) = 2 Im T,   d_mns = Tr(F_s {F_m, F_n}) = 2 Re T,
// because Tr(F_s F_n F_m) = conj(T) for Hermitian F.  And z = f + i d (Eq. (06))
// gives z_jln = 2 i Tr(F_n F_l F_j).
//
// T is nonzero in exactly three situations, each with a closed form:
//   * three pair elements whose edges form a triangle p-q-r:
//       T = c_x(p->q) c_y(q->r) c_w(r->p),  c = coefficient of E_uv in F,
//     c_S(u->v) = 1/sqrt2, c_J(u->v) = -i/sqrt2 (u<v) or +i/sqrt2 (u>v);
//   * two pair elements on the same edge (a,b) and one D_l (rotated first):
//       Tr(D_l F_u F_v) = delta_a(l) c_u(a->b) c_v(b->a) + delta_b(l) c_u(b->a) c_v(a->b);
//   * three diagonal elements: Tr(D_l D_m D_n) = sum_k delta_k(l) delta_k(m) delta_k(n)
//       = c_r if the two smallest of {l,m,n} are equal (p = q < r),
//         (1 - p) c_p if l = m = n = p, else 0,
//   with delta_k(l) = (D_l)_kk = c_l (k<l), -l c_l (k=l), 0 (k>l), c_l = 1/sqrt(l(l+1)).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define LB_HD __host__ __device__ __forceinline__
#else
#define LB_HD inline
#endif

namespace lb {

constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr double kInv2Sqrt2 = 0.35355339059327376220;

enum ElemKind : int { kS = 0, kJ = 1, kD = 2 };

// Read-only tables of one basis, resident in device memory.
struct BasisView {
  int N;
  int64_t P, M;
  const int32_t* pair_ab;  // P entries, (a << 16) | b
  const double* c;         // c[l] = 1/sqrt(l(l+1)),   l = 1..N-1 (c[0] unused)
  const double* lc;        // lc[l] = -l * c[l]
  const double* c2;        // c2[l] = c[l]^2 = 1/(l(l+1))
  const double* inv;       // inv[l] = 1/l, l = 1..N  (sum_{l=x}^{y} c2[l] = inv[x] - inv[y+1])
};

struct Elem {
  int kind;  // kS, kJ, kD
  int a, b;  // pair: a < b;  D: a = b = l
};

LB_HD int64_t pair_index(int N, int a, int b) {  // a < b
  return (int64_t)a * (2 * N - a - 1) / 2 + (b - a - 1);
}

LB_HD int64_t pair_index_any(int N, int u, int v) {
  return u < v ? pair_index(N, u, v) : pair_index(N, v, u);
}

LB_HD int64_t elem_index(const BasisView& B, int kind, int a, int b) {
  if (kind == kD) return 2 * B.P + (a - 1);
  return (int64_t)kind * B.P + pair_index_any(B.N, a, b);
}

LB_HD int64_t d_index(const BasisView& B, int l) { return 2 * B.P + (l - 1); }

LB_HD Elem decode(const BasisView& B, int64_t i) {
  Elem e;
  if (i < 2 * B.P) {
    int64_t p = i < B.P ? i : i - B.P;
#if defined(__CUDA_ARCH__)
    int32_t ab = __ldg(B.pair_ab + p);
#else
    int32_t ab = B.pair_ab[p];
#endif
    e.kind = i < B.P ? kS : kJ;
    e.a = ab >> 16;
    e.b = ab & 0xffff;
  } else {
    e.kind = kD;
    e.a = e.b = (int)(i - 2 * B.P + 1);
  }
  return e;
}

LB_HD int64_t partner(const BasisView& B, int64_t i) {  // S_ab <-> J_ab
  return i < B.P ? i + B.P : i - B.P;
}

LB_HD double ld_c(const BasisView& B, int l) {
#if defined(__CUDA_ARCH__)
  return __ldg(B.c + l);
#else
  return B.c[l];
#endif
}

LB_HD double ld_lc(const BasisView& B, int l) {
#if defined(__CUDA_ARCH__)
  return __ldg(B.lc + l);
#else
  return B.lc[l];
#endif
}

// delta_k(l) = (D_l)_kk
LB_HD double delta(const BasisView& B, int k, int l) {
  return k < l ? ld_c(B, l) : (k == l ? ld_lc(B, l) : 0.0);
}

// Phase (power of i, mod 4) of the coefficient of E_uv in a pair element
// of kind `kind` on edge {u, v}:  S -> 1 (i^0),  J -> -i (i^3) if u < v, +i (i^1) if u > v.
LB_HD int coef_phase(int kind, int u, int v) { return kind == kS ? 0 : (u < v ? 3 : 1); }

// i^k as (re, im)
LB_HD void ipow(int k, double& re, double& im) {
  k &= 3;
  re = (k == 0) ? 1.0 : (k == 2 ? -1.0 : 0.0);
  im = (k == 1) ? 1.0 : (k == 3 ? -1.0 : 0.0);
}

// The common vertex of two edges sharing exactly one vertex, or -1.
LB_HD int common_vertex(const Elem& x, const Elem& y) {
  int c = -1, n = 0;
  if (x.a == y.a || x.a == y.b) { c = x.a; ++n; }
  if (x.b == y.a || x.b == y.b) { c = x.b; ++n; }
  return n == 1 ? c : -1;
}

// Tr(D_l F_u F_v) for pair elements u, v (zero unless on the same edge).
LB_HD void trace_dpp(const BasisView& B, int l, const Elem& u, const Elem& v, double& re, double& im) {
  re = im = 0.0;
  if (u.a != v.a || u.b != v.b) return;
  int a = u.a, b = u.b;
  double r1, i1, r2, i2;
  ipow(coef_phase(u.kind, a, b) + coef_phase(v.kind, b, a), r1, i1);
  ipow(coef_phase(u.kind, b, a) + coef_phase(v.kind, a, b), r2, i2);
  double da = delta(B, a, l), db = delta(B, b, l);
  re = 0.5 * (da * r1 + db * r2);
  im = 0.5 * (da * i1 + db * i2);
}

// Tr(D_l D_m D_n)
LB_HD double trace_ddd(const BasisView& B, int l, int m, int n) {
  int p = l, q = m, r = n, t;
  if (p > q) { t = p; p = q; q = t; }
  if (q > r) { t = q; q = r; r = t; }
  if (p > q) { t = p; p = q; q = t; }
  if (p != q) return 0.0;
  if (q < r) return ld_c(B, r);
  return (double)(1 - p) * ld_c(B, p);
}

// T = Tr(F_x F_y F_w) for any three basis elements.
LB_HD void trace3(const BasisView& B, const Elem& x, const Elem& y, const Elem& w, double& re, double& im) {
  re = im = 0.0;
  int nd = (x.kind == kD) + (y.kind == kD) + (w.kind == kD);
  if (nd == 0) {
    int q = common_vertex(x, y), r = common_vertex(y, w), p = common_vertex(w, x);
    if (p < 0 || q < 0 || r < 0 || p == q || q == r || p == r) return;
    int ph = coef_phase(x.kind, p, q) + coef_phase(y.kind, q, r) + coef_phase(w.kind, r, p);
    ipow(ph, re, im);
    re *= kInv2Sqrt2;
    im *= kInv2Sqrt2;
  } else if (nd == 1) {
    // rotate cyclically so that the diagonal element comes first
    if (x.kind == kD) trace_dpp(B, x.a, y, w, re, im);
    else if (y.kind == kD) trace_dpp(B, y.a, w, x, re, im);
    else trace_dpp(B, w.a, x, y, re, im);
  } else if (nd == 3) {
    re = trace_ddd(B, x.a, y.a, w.a);
  }
  // nd == 2: diagonal x diagonal x off-diagonal has zero trace
}

// f_mns and d_mns (Eq. (05)) through T = Tr(F_s F_m F_n).
LB_HD void fd_value(const BasisView& B, const Elem& m, const Elem& n, const Elem& s, double& f, double& d) {
  double re, im;
  trace3(B, s, m, n, re, im);
  f = 2.0 * im;
  d = 2.0 * re;
}

LB_HD double f_value(const BasisView& B, const Elem& m, const Elem& n, const Elem& s) {
  double f, d;
  fd_value(B, m, n, s, f, d);
  return f;
}

// The edge of the two non-shared vertices of two edges sharing exactly one vertex.
LB_HD void third_edge(const Elem& x, const Elem& y, int v, int& lo, int& hi) {
  int u = (x.a == v) ? x.b : x.a;
  int w = (y.a == v) ? y.b : y.a;
  lo = u < w ? u : w;
  hi = u < w ? w : u;
}

LB_HD Elem make_pair(int kind, int u, int v) {
  Elem e;
  e.kind = kind;
  e.a = u < v ? u : v;
  e.b = u < v ? v : u;
  return e;
}

LB_HD Elem make_d(int l) {
  Elem e;
  e.kind = kD;
  e.a = e.b = l;
  return e;
}

LB_HD int imax(int a, int b) { return a > b ? a : b; }
LB_HD int imin(int a, int b) { return a < b ? a : b; }

}  // namespace lb

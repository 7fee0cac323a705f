// lb_assemble.cu -- kernel (b): dense assembly of Q (Eq. (07)), R (Eq. (09))
// and K (Eq. (08)); Table 1 steps 2.3-2.5.
//
// R is computed owner-computes: the thread that owns entry (s, n) evaluates
//     r_sn = -1/2 sum_l sum_k sum_j f_kls Re(a_jk z_jln),   z = f + i d,
// visiting exactly the join terms with f_kls != 0 and z_jln != 0 -- the join
// of the F-section (k, s) and Z-section (j, n) of every shared l that the
// paper's Sec. 4 item 2.5 describes -- enumerated by index arithmetic
// instead of searched.  (The printed two-term form with prefactor -1/4 is
// the same sum, since its second term is the complex conjugate of the first
// for Hermitian a.)  With e(x) the edge of a pair element x:
//   * l = D_lambda: f_{k D s} != 0 only for pair s, k = partner(s) and
//     lambda in [max(a_s,1), b_s]; the Z-section of D_lambda couples n to
//     j = n (d) and j = partner(n) (f) for pair n, to j = D_min for n = D;
//     this part carries the O(N^5) work of dense R.
//   * l a pair element: f_{k l s} != 0 if e(l) shares exactly one vertex
//     with e(s) (k = the third edge of the triangle) or l = partner(s)
//     (k = D_mu); z_{j l n} != 0 if e(l) shares one vertex with e(n)
//     (j = the third edge, both types) or e(l) = e(n) (j = D_mu).
// That is the JOIN algorithm (LB_ALG_JOIN).  The CLOSED algorithm (the
// default) groups the entries by the relation of their two edges -- disjoint
// (vertex quadruples), meeting at one vertex, the same edge, pair x diagonal,
// diagonal x diagonal -- and sums each group's join terms in closed form;
// an entry is written by one kernel and, for edges that meet, completed by
// one later kernel on the same stream.  No atomics on either path.
#include <algorithm>

#include "lb_internal.h"

namespace {

using namespace lb;

struct AView {
  const double2* a;
  int64_t M;
};

LB_HD double2 ldA(const AView& A, int64_t j, int64_t k) {
#if defined(__CUDA_ARCH__)
  return __ldg(A.a + j * A.M + k);
#else
  return A.a[j * A.M + k];
#endif
}

// a_jk read from row k (a is Hermitian: a_jk = conj(a_kj)); lanes that vary
// j at fixed k then read one contiguous row.
LB_HD double2 ldA_row(const AView& A, int64_t j, int64_t k) {
  double2 t = ldA(A, k, j);
  t.y = -t.y;
  return t;
}

template <bool COUNT>
struct EntryAcc {
  double acc = 0.0;  // sum f_kls Re(a_jk z_jln)
  unsigned long long terms = 0;
};

// One join term (j, l, k) of entry (s, n): f_kls Re(a_jk z_jln),
// Re(a z) = Re(a) f_jln - Im(a) d_jln.
template <bool COUNT>
LB_HD void add_term(const BasisView& B, const AView& A, const Elem& en,
                                         const Elem& ej, int64_t j, const Elem& el, int64_t k,
                                         double fk, EntryAcc<COUNT>& E) {
  double fj, dj;
  fd_value(B, ej, el, en, fj, dj);
  if (fj == 0.0 && dj == 0.0) return;
  if (COUNT) {
    ++E.terms;
  } else {
    const double2 av = ldA(A, j, k);
    E.acc += fk * (av.x * fj - av.y * dj);
  }
}

// l is a pair element with a single k (pair element); j runs over both types
// of one edge (ju, jv).
template <bool COUNT>
LB_HD void pair_l_two_j(const BasisView& B, const AView& A, const Elem& es,
                                             const Elem& en, const Elem& el, const Elem& ek,
                                             int ju, int jv, EntryAcc<COUNT>& E) {
  const double fk = f_value(B, ek, el, es);
  if (fk == 0.0) return;
  const int64_t k = elem_index(B, ek.kind, ek.a, ek.b);
  for (int tj = kS; tj <= kJ; ++tj) {
    const Elem ej = make_pair(tj, ju, jv);
    add_term<COUNT>(B, A, en, ej, elem_index(B, tj, ju, jv), el, k, fk, E);
  }
}

// l is a pair element on the edge of n; j runs over D_mu for mu in [lo, hi].
template <bool COUNT>
LB_HD void pair_l_d_j(const BasisView& B, const AView& A, const Elem& en,
                                           const Elem& el, int64_t k, double fk, int lo, int hi,
                                           EntryAcc<COUNT>& E) {
  for (int mu = lo; mu <= hi; ++mu) {
    add_term<COUNT>(B, A, en, make_d(mu), d_index(B, mu), el, k, fk, E);
  }
}

template <bool COUNT>
__host__ __device__ void entry(const BasisView& B, const AView& A, const double* h, int64_t s, int64_t n,
                      EntryAcc<COUNT>& E, double& q) {
  const int N = B.N;
  const Elem es = decode(B, s), en = decode(B, n);
  q = 0.0;
  if (es.kind != kD) {
    const int as = es.a, bs = es.b, ts = es.kind;
    const int64_t sb = partner(B, s);
    const Elem esb = make_pair(1 - ts, as, bs);
    const int lo_s = imax(as, 1);  // f(partner(s), D_l, s) != 0 for l in [lo_s, bs]
    const double sgs = ts == kS ? 1.0 : -1.0;
    if (en.kind != kD) {
      // ------------------------------------------------ s pair, n pair
      const int an = en.a, bn = en.b, tn = en.kind;
      const int64_t nb = partner(B, n);
      const double sgn = tn == kS ? 1.0 : -1.0;
      // Part D: l = D_lambda, k = partner(s), j in {n (d), partner(n) (f)}.
      //   f(partner(s), D, s) = sgs * (delta_as - delta_bs)
      //   f(partner(n), D, n) = sgn * (delta_an - delta_bn),  d(n, D, n) = delta_an + delta_bn
      {
        const int lo = imax(lo_s, imax(an, 1));
        double accf = 0.0, accd = 0.0;
        for (int lam = lo; lam <= bs; ++lam) {
          const double cl = ld_c(B, lam), lcl = ld_lc(B, lam);
          const double das = as < lam ? cl : (as == lam ? lcl : 0.0);
          const double dbs = bs < lam ? cl : (bs == lam ? lcl : 0.0);
          const double dan = an < lam ? cl : (an == lam ? lcl : 0.0);
          const double dbn = bn < lam ? cl : (bn == lam ? lcl : 0.0);
          const double gs = das - dbs;
          const double gn = dan - dbn, hn = dan + dbn;
          if (COUNT) {
            E.terms += (gn != 0.0) + (hn != 0.0);
          } else {
            accf = fma(gs, gn, accf);
            accd = fma(gs, hn, accd);
          }
        }
        if (!COUNT && lo <= bs) {
          const double2 a1 = ldA_row(A, nb, sb);  // a_{partner(n), partner(s)}
          const double2 a2 = ldA_row(A, n, sb);   // a_{n, partner(s)}
          E.acc += sgs * (sgn * a1.x * accf - a2.y * accd);
        }
      }
      // Part P: l a pair element.
      int shared = 0, cv = -1;
      if (as == an || as == bn) { ++shared; cv = as; }
      if (bs == an || bs == bn) { ++shared; cv = bs; }
      if (shared == 0) {
        // e(l) = (v, w), v in e(s), w in e(n); k on (v', w), j on (v, w').
        for (int vi = 0; vi < 2; ++vi) {
          const int v = vi ? bs : as, vp = vi ? as : bs;
          for (int wi = 0; wi < 2; ++wi) {
            const int w = wi ? bn : an, wp = wi ? an : bn;
            for (int tl = kS; tl <= kJ; ++tl) {
              const Elem el = make_pair(tl, v, w);
              const Elem ek = make_pair(1 ^ tl ^ ts, vp, w);
              pair_l_two_j<COUNT>(B, A, es, en, el, ek, v, wp, E);
            }
          }
        }
      } else if (shared == 1) {
        const int v = cv;
        const int p = (as == v) ? bs : as;  // e(s) = (v, p)
        const int qv = (an == v) ? bn : an; // e(n) = (v, q)
        // (A1) e(l) = (v, w), w not in {v, p, q}: k on (p, w), j on (q, w)
        for (int w = 0; w < N; ++w) {
          if (w == v || w == p || w == qv) continue;
          for (int tl = kS; tl <= kJ; ++tl) {
            const Elem el = make_pair(tl, v, w);
            const Elem ek = make_pair(1 ^ tl ^ ts, p, w);
            pair_l_two_j<COUNT>(B, A, es, en, el, ek, qv, w, E);
          }
        }
        // (A2) e(l) = (p, q): k on (v, q), j on (v, p)
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, p, qv);
          const Elem ek = make_pair(1 ^ tl ^ ts, v, qv);
          pair_l_two_j<COUNT>(B, A, es, en, el, ek, v, p, E);
        }
        // (A3) e(l) = e(n): k on (p, q); j = D_mu
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, an, bn);
          const Elem ek = make_pair(1 ^ tl ^ ts, p, qv);
          const double fk = f_value(B, ek, el, es);
          if (fk == 0.0) continue;
          const int64_t k = elem_index(B, ek.kind, ek.a, ek.b);
          if (tl == tn) pair_l_d_j<COUNT>(B, A, en, el, k, fk, imax(an, 1), N - 1, E);
          else pair_l_d_j<COUNT>(B, A, en, el, k, fk, imax(an, 1), bn, E);
        }
        // (B) l = partner(s): k = D_mu, j on (p, q)
        for (int mu = lo_s; mu <= bs; ++mu) {
          const Elem ek = make_d(mu);
          const double fk = f_value(B, ek, esb, es);
          if (fk == 0.0) continue;
          const int64_t k = d_index(B, mu);
          for (int tj = kS; tj <= kJ; ++tj) {
            const Elem ej = make_pair(tj, p, qv);
            add_term<COUNT>(B, A, en, ej, elem_index(B, tj, p, qv), esb, k, fk, E);
          }
        }
      } else {
        // same edge (a, b): (A) e(l) = (v, w), v in e(s), w outside; k and j on (v', w)
        for (int w = 0; w < N; ++w) {
          if (w == as || w == bs) continue;
          for (int vi = 0; vi < 2; ++vi) {
            const int v = vi ? bs : as, vp = vi ? as : bs;
            for (int tl = kS; tl <= kJ; ++tl) {
              const Elem el = make_pair(tl, v, w);
              const Elem ek = make_pair(1 ^ tl ^ ts, vp, w);
              pair_l_two_j<COUNT>(B, A, es, en, el, ek, vp, w, E);
            }
          }
        }
        // (B) l = partner(s): k = D_mu; j = D_nu from the fiber of (partner(s), n)
        for (int mu = lo_s; mu <= bs; ++mu) {
          const Elem ek = make_d(mu);
          const double fk = f_value(B, ek, esb, es);
          if (fk == 0.0) continue;
          const int64_t k = d_index(B, mu);
          if (sb == n) pair_l_d_j<COUNT>(B, A, en, esb, k, fk, lo_s, N - 1, E);
          else pair_l_d_j<COUNT>(B, A, en, esb, k, fk, lo_s, bs, E);
        }
      }
      // Q (Eq. (07)): q_sn = sum_m h_m f_mns
      if (h != nullptr && !COUNT) {
        if (shared == 1) {
          const int p = (as == cv) ? bs : as, qv = (an == cv) ? bn : an;
          const Elem em = make_pair(1 ^ tn ^ ts, p, qv);
          q += h[elem_index(B, em.kind, em.a, em.b)] * f_value(B, em, en, es);
        } else if (shared == 2 && tn != ts) {
          for (int lam = lo_s; lam <= bs; ++lam) q += h[d_index(B, lam)] * f_value(B, make_d(lam), en, es);
        }
      }
    } else {
      // ------------------------------------------------ s pair, n = D_nu
      const int nu = en.a;
      // Part D: l = D_lambda, k = partner(s), j = D from the d-fiber of (D_lambda, D_nu)
      for (int lam = lo_s; lam <= bs; ++lam) {
        const Elem el = make_d(lam);
        const double fk = f_value(B, esb, el, es);
        if (fk == 0.0) continue;
        if (lam != nu) {
          const int j = imin(lam, nu);
          add_term<COUNT>(B, A, en, make_d(j), d_index(B, j), el, sb, fk, E);
        } else {
          for (int mu = lam; mu < N; ++mu) {
            if (mu == 1 && lam == 1) continue;
            add_term<COUNT>(B, A, en, make_d(mu), d_index(B, mu), el, sb, fk, E);
          }
        }
      }
      // Part P (A): e(l) = (v, w) sharing one vertex with e(s); k on (v', w);
      // j in {l (d), partner(l) (f)}
      for (int w = 0; w < N; ++w) {
        if (w == as || w == bs) continue;
        for (int vi = 0; vi < 2; ++vi) {
          const int v = vi ? bs : as, vp = vi ? as : bs;
          for (int tl = kS; tl <= kJ; ++tl) {
            const Elem el = make_pair(tl, v, w);
            const Elem ek = make_pair(1 ^ tl ^ ts, vp, w);
            const double fk = f_value(B, ek, el, es);
            if (fk == 0.0) continue;
            const int64_t k = elem_index(B, ek.kind, ek.a, ek.b);
            const int64_t li = elem_index(B, tl, v, w);
            add_term<COUNT>(B, A, en, el, li, el, k, fk, E);
            const Elem elb = make_pair(1 - tl, v, w);
            add_term<COUNT>(B, A, en, elb, partner(B, li), el, k, fk, E);
          }
        }
      }
      // Part P (B): l = partner(s), k = D_mu, j in {partner(s) (d), s (f)}
      for (int mu = lo_s; mu <= bs; ++mu) {
        const Elem ek = make_d(mu);
        const double fk = f_value(B, ek, esb, es);
        if (fk == 0.0) continue;
        const int64_t k = d_index(B, mu);
        add_term<COUNT>(B, A, en, esb, sb, esb, k, fk, E);
        add_term<COUNT>(B, A, en, es, s, esb, k, fk, E);
      }
      if (h != nullptr && !COUNT && nu >= lo_s && nu <= bs) q += h[sb] * f_value(B, esb, en, es);
    }
  } else {
    const int nu = es.a;
    if (en.kind != kD) {
      // ------------------------------------------------ s = D_nu, n pair
      // l pair with nu in [max(a_l,1), b_l], k = partner(l).
      const int an = en.a, bn = en.b, tn = en.kind;
      for (int vi = 0; vi < 2; ++vi) {
        const int v = vi ? bn : an, vp = vi ? an : bn;
        for (int w = 0; w < N; ++w) {
          if (w == an || w == bn) continue;
          const int lo = imin(v, w), hi = imax(v, w);
          if (nu < imax(lo, 1) || nu > hi) continue;
          for (int tl = kS; tl <= kJ; ++tl) {
            const Elem el = make_pair(tl, v, w);
            const Elem ek = make_pair(1 - tl, v, w);
            pair_l_two_j<COUNT>(B, A, es, en, el, ek, vp, w, E);
          }
        }
      }
      if (nu >= imax(an, 1) && nu <= bn) {
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, an, bn);
          const Elem ek = make_pair(1 - tl, an, bn);
          const double fk = f_value(B, ek, el, es);
          if (fk == 0.0) continue;
          const int64_t k = elem_index(B, ek.kind, an, bn);
          if (tl == tn) pair_l_d_j<COUNT>(B, A, en, el, k, fk, imax(an, 1), N - 1, E);
          else pair_l_d_j<COUNT>(B, A, en, el, k, fk, imax(an, 1), bn, E);
        }
        if (h != nullptr && !COUNT) {
          const int64_t nb = partner(B, n);
          q += h[nb] * f_value(B, make_pair(1 - tn, an, bn), en, es);
        }
      }
    } else {
      // ------------------------------------------------ s = D_nu, n = D_mu
      // l on an edge (x, y) with x <= nu <= y, k = partner(l), j in {l (d), partner(l) (f)}
      for (int x = 0; x <= nu; ++x) {
        for (int y = imax(nu, x + 1); y < N; ++y) {
          for (int tl = kS; tl <= kJ; ++tl) {
            const Elem el = make_pair(tl, x, y);
            const Elem ek = make_pair(1 - tl, x, y);
            const double fk = f_value(B, ek, el, es);
            if (fk == 0.0) continue;
            const int64_t li = elem_index(B, tl, x, y);
            const int64_t k = partner(B, li);
            add_term<COUNT>(B, A, en, el, li, el, k, fk, E);
            add_term<COUNT>(B, A, en, ek, k, el, k, fk, E);
          }
        }
      }
    }
  }
}

// One thread per entry; a block covers 256 consecutive columns n of one row s.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_assemble(BasisView B, AView A, const double* __restrict__ h,
                                                  double* __restrict__ Aout, double* __restrict__ Qout,
                                                  double* __restrict__ Rout,
                                                  unsigned long long* __restrict__ count) {
  const int64_t M = B.M;
  const int64_t chunks = (M + 255) / 256;
  const int64_t s = blockIdx.x / chunks;
  const int64_t n = (blockIdx.x % chunks) * 256 + threadIdx.x;
  EntryAcc<COUNT> E;
  double q = 0.0;
  if (n < M) entry<COUNT>(B, A, h, s, n, E, q);
  if (COUNT) {
    unsigned long long t = E.terms;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(count, t);
    return;
  }
  if (n >= M) return;
  const double r = -0.5 * E.acc;
  const int64_t o = s * M + n;
  if (Rout) Rout[o] = r;
  if (Qout) Qout[o] = q;
  if (Aout) Aout[o] = q + r;
}

// Eq. (08): k_s = (i/N) sum_jk a_jk f_jks = -(1/N) sum_jk Im(a_jk) f_jks.
// One warp per s; lanes stride over the j candidates.
// CLOSED: the diagonal rows are left to k_kvec_diag_* below.
template <bool CLOSED>
__global__ void k_kvec(BasisView B, AView A, double* __restrict__ K) {
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= (CLOSED ? 2 * B.P : B.M)) return;
  const int N = B.N;
  const Elem es = decode(B, s);
  double acc = 0.0;
  if (es.kind != kD) {
    const int as = es.a, bs = es.b, ts = es.kind;
    const int64_t sb = partner(B, s);
    const Elem esb = make_pair(1 - ts, as, bs);
    // j pair sharing one vertex with e(s): j = (v, w), k on (v', w)
    const int nw = 2 * N;
    for (int t = lane; t < nw; t += 32) {
      const int vi = t / N, w = t % N;
      if (w == as || w == bs) continue;
      const int v = vi ? bs : as, vp = vi ? as : bs;
      for (int tj = kS; tj <= kJ; ++tj) {
        const Elem ej = make_pair(tj, v, w);
        const Elem ek = make_pair(1 ^ tj ^ ts, vp, w);
        const double f = f_value(B, ej, ek, es);
        if (f != 0.0) acc += ldA(A, elem_index(B, tj, v, w), elem_index(B, ek.kind, vp, w)).y * f;
      }
    }
    // j = partner(s), k = D_l  and  j = D_l, k = partner(s)
    for (int l = imax(as, 1) + lane; l <= bs; l += 32) {
      const Elem ed = make_d(l);
      const int64_t di = d_index(B, l);
      acc += ldA(A, sb, di).y * f_value(B, esb, ed, es);
      acc += ldA(A, di, sb).y * f_value(B, ed, esb, es);
    }
  } else {
    const int nu = es.a;
    // j on an edge (x, y) with x <= nu <= y, k = partner(j)
    const int64_t cnt = (int64_t)(nu + 1) * N;
    for (int64_t t = lane; t < cnt; t += 32) {
      const int x = (int)(t / N), y = (int)(t % N);
      if (y <= x || y < nu) continue;
      for (int tj = kS; tj <= kJ; ++tj) {
        const Elem ej = make_pair(tj, x, y);
        const Elem ek = make_pair(1 - tj, x, y);
        const double f = f_value(B, ej, ek, es);
        if (f != 0.0) {
          const int64_t j = elem_index(B, tj, x, y);
          acc += ldA(A, j, partner(B, j)).y * f;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) K[s] = -acc / (double)N;
}

// K on the diagonal rows in closed form.  The only nonzero f_{j k D_nu} with
// pair j, k are f(S_xy, J_xy, D_nu) = delta_x(nu) - delta_y(nu) = -f(J_xy,
// S_xy, D_nu), and a is Hermitian, so with g_xy = 2 Im a_{S_xy, J_xy}
//   K_{D_nu} = -(1/N) sum_{x<y} (delta_x(nu) - delta_y(nu)) g_xy
//            = -(1/N) sum_k delta_k(nu) G_k,  G_k = sum_{y>k} g_ky - sum_{x<k} g_xk,
// and sum_k delta_k(nu) G_k = c_nu sum_{k<nu} G_k - nu c_nu G_nu (the prefix
// form of the Helmert vectors).  k_kvec_diag_g: one block per vertex k, a
// fixed-order reduction; k_kvec_diag: the prefix over k (one warp) and the
// rows.
__global__ void __launch_bounds__(128) k_kvec_diag_g(BasisView B, AView A, double* __restrict__ G) {
  const int N = B.N, k = blockIdx.x;
  double acc = 0.0;
  for (int u = threadIdx.x; u < N; u += blockDim.x) {
    if (u == k) continue;
    const int64_t p = pair_index_any(N, k, u);
    const double g = 2.0 * ldA(A, p, B.P + p).y;
    acc += u > k ? g : -g;
  }
  __shared__ double red[4];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) G[k] = (red[0] + red[1]) + (red[2] + red[3]);
}

__device__ __forceinline__ void warp_prefix(double* arr, int n);  // below
__device__ __forceinline__ void warp_suffix(const double* x, double* y, int n);  // below

__global__ void __launch_bounds__(256) k_kvec_diag(BasisView B, const double* __restrict__ G,
                                                    double* __restrict__ K) {
  __shared__ double pre[lbi::kMaxDenseN + 1];  // pre[nu] = sum_{k < nu} G_k
  const int N = B.N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) pre[k + 1] = G[k];
  if (threadIdx.x == 0) pre[0] = 0.0;
  __syncthreads();
  if (threadIdx.x < 32) warp_prefix(pre, N);
  __syncthreads();
  for (int nu = 1 + threadIdx.x; nu < N; nu += blockDim.x)
    K[d_index(B, nu)] = -(ld_c(B, nu) * pre[nu] + ld_lc(B, nu) * G[nu]) / (double)N;
}

// ---------------------------------------------------------------------------
// Production path.  The same join terms as entry<>, split by the relation of
// the edges of s and n so that no warp carries another case's O(N) loops:
//   k_entries : every entry -- the l = D_lambda part of pair-pair entries,
//               the l-pair part of pair-pair entries on disjoint edges (16
//               terms), entries with a diagonal s or n (via entry<>), and Q;
//   k_shared  : the l-pair part of pair-pair entries whose edges share one
//               vertex; one block per ordered vertex pair (p, q), entries
//               s on (v, p), n on (v, q) for all v, with the entries of a
//               common to every v staged in shared memory;
//   k_same    : the l-pair part of pair-pair entries on the same edge; one
//               block per edge.
// A triangle value is +-1/sqrt2, so a triangle-triangle term is +-1/2 Re(a)
// or +-1/2 Im(a): its sign comes from integer phase arithmetic and the term
// costs one FP64 add.

// +-1 of a triangle constant: f = Im(i^ph)/sqrt2 (odd ph), d = Re(i^ph)/sqrt2 (even ph)
LB_HD int sgn_f(int ph) { return ((ph & 3) == 1) ? 1 : -1; }
LB_HD int sgn_d(int ph) { return ((ph & 3) == 0) ? 1 : -1; }

// s * x for s = +-1, by flipping the sign bit (no FP64 instruction)
__device__ __forceinline__ double sgn_mul(int s, double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((unsigned long long)(s < 0) << 63));
}

// -x/2, exactly, by exponent and sign-bit arithmetic for normal x (no FP64
// instruction); zero, subnormal, inf and nan take the FP64 multiply.
__device__ __forceinline__ double neg_half(double x) {
  const long long b = __double_as_longlong(x);
  const long long ex = (b >> 52) & 0x7ff;
  if (ex > 1 && ex < 0x7ff) return __longlong_as_double((b - (1LL << 52)) ^ (long long)(1ULL << 63));
  return -0.5 * x;
}

// 2x, exactly, by exponent arithmetic for normal x below the top binade (no
// FP64 instruction); zero, subnormal, inf and nan take the FP64 add.
__device__ __forceinline__ double twice(double x) {
  const long long b = __double_as_longlong(x);
  const long long ex = (b >> 52) & 0x7ff;
  if (ex >= 1 && ex < 0x7fe) return __longlong_as_double(b + (1LL << 52));
  return x + x;
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// delta_x(lam) = (D_lam)_xx
__device__ __forceinline__ double dlt(const BasisView& B, int x, int lam) {
  return x < lam ? ld_c(B, lam) : (x == lam ? ld_lc(B, lam) : 0.0);
}

// sum_{lam=x}^{y} c_lam^2: term by term (the join) or as 1/x - 1/(y+1)
template <int ALG>
__device__ __forceinline__ double seg_c2(const BasisView& B, int x, int y) {
  if (x > y) return 0.0;
  if (ALG == LB_ALG_CLOSED) return __ldg(B.inv + x) - __ldg(B.inv + y + 1);
  double s = 0.0;
  for (int l = x; l <= y; ++l) s += __ldg(B.c2 + l);
  return s;
}

// Pair s = (as, bs), pair n = (an, bn): the l = D_lambda part,
//   sum_lam f(partner(s), D, s) [Re a_{partner(n), partner(s)} f(partner(n), D, n)
//                                 - Im a_{n, partner(s)} d(n, D, n)].
// Inside (lo, hi) away from the four edge end points every factor is c_lam
// (or 0, 2 c_lam past b_n), so the sum runs over c_lam^2 between the sorted
// end points, which are evaluated from the delta's in full.
template <int ALG>
__device__ __forceinline__ double part_d_pp(const BasisView& B, const AView& A, int as, int bs, int ts,
                                            int an, int bn, int tn, int64_t sb, int64_t n, int64_t nb) {
  const int lo = imax(imax(as, an), 1), hi = bs;
  if (lo > hi) return 0.0;
  int sp0 = as, sp1 = an, sp2 = bn, sp3 = bs, t;
  if (sp0 > sp1) { t = sp0; sp0 = sp1; sp1 = t; }
  if (sp2 > sp3) { t = sp2; sp2 = sp3; sp3 = t; }
  if (sp0 > sp2) { t = sp0; sp0 = sp2; sp2 = t; }
  if (sp1 > sp3) { t = sp1; sp1 = sp3; sp3 = t; }
  if (sp1 > sp2) { t = sp1; sp1 = sp2; sp2 = t; }
  const int sp[4] = {sp0, sp1, sp2, sp3};
  double accf = 0.0, accd = 0.0;
  int prev = lo;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int x = sp[i];
    if (x < prev || x > hi) continue;
    if (prev <= x - 1) {
      const double S = seg_c2<ALG>(B, prev, x - 1);
      if (x - 1 < bn) { accf += S; accd += S; } else { accd += 2.0 * S; }
    }
    const double das = dlt(B, as, x), dbs = dlt(B, bs, x), dan = dlt(B, an, x), dbn = dlt(B, bn, x);
    const double gs = das - dbs;
    accf = fma(gs, dan - dbn, accf);
    accd = fma(gs, dan + dbn, accd);
    prev = x + 1;
  }
  if (prev <= hi) {
    const double S = seg_c2<ALG>(B, prev, hi);
    if (hi < bn) { accf += S; accd += S; } else { accd += 2.0 * S; }
  }
  const double2 a1 = ldA_row(A, nb, sb);  // a_{partner(n), partner(s)}
  const double2 a2 = ldA_row(A, n, sb);   // a_{n, partner(s)}
  const double sgs = ts == kS ? 1.0 : -1.0, sgn = tn == kS ? 1.0 : -1.0;
  return sgs * (sgn * a1.x * accf - a2.y * accd);
}

// Pair s, pair n on disjoint edges: e(l) = (v, w), v in e(s), w in e(n);
// k on (v', w), j on (v, w') with both types.  Lanes of a warp run over
// consecutive n, so a_jk is read from the row (j or k) that is common to
// the warp.
__device__ __forceinline__ double part_p_disjoint(const BasisView& B, const AView& A, int as, int bs, int ts,
                                                  int an, int bn, int tn) {
  const int N = B.N;
  const int64_t P = B.P;
  double acc2 = 0.0;
#pragma unroll
  for (int vi = 0; vi < 2; ++vi) {
    const int v = vi ? bs : as, vp = vi ? as : bs;
    const int phs = coef_phase(ts, v, vp);
#pragma unroll
    for (int wi = 0; wi < 2; ++wi) {
      const int w = wi ? bn : an, wp = wi ? an : bn;
      const int phn = coef_phase(tn, w, wp);
      const int64_t pk = pair_index_any(N, vp, w), pj = pair_index_any(N, v, wp);
#pragma unroll
      for (int tl = 0; tl < 2; ++tl) {
        const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int phl_wv = coef_phase(tl, w, v), phl_vw = coef_phase(tl, v, w);
        const int sk = sgn_f(phs + coef_phase(tk, vp, w) + phl_wv);
        const int sf = sgn_f(phn + coef_phase(tjf, wp, v) + phl_vw);
        const int sd = sgn_d(phn + coef_phase(tjd, wp, v) + phl_vw);
        const int64_t k = tk * P + pk, jf = tjf * P + pj, jd = tjd * P + pj;
        double2 a1, a2;
        if (wi == 0) {
          a1 = ldA_row(A, jf, k);
          a2 = ldA_row(A, jd, k);
        } else {
          a1 = ldA(A, jf, k);
          a2 = ldA(A, jd, k);
        }
        acc2 += sgn_mul(sk * sf, a1.x);
        acc2 -= sgn_mul(sk * sd, a2.y);
      }
    }
  }
  return 0.5 * acc2;
}

// Pair-pair block (s, n < 2P); one thread per entry, 256 consecutive n per block.
template <int ALG>
__global__ void __launch_bounds__(256) k_entries(BasisView B, AView A, const double* __restrict__ h,
                                                 double* __restrict__ Aout, double* __restrict__ Qout,
                                                 double* __restrict__ Rout) {
  const int64_t M = B.M, P2 = 2 * B.P;
  const int64_t chunks = (P2 + 255) / 256;
  const int64_t s = blockIdx.x / chunks;
  const int64_t n = (blockIdx.x % chunks) * 256 + threadIdx.x;
  if (n >= P2) return;
  const Elem es = decode(B, s), en = decode(B, n);
  double q = 0.0;
  const int as = es.a, bs = es.b, ts = es.kind, an = en.a, bn = en.b, tn = en.kind;
  double acc = part_d_pp<ALG>(B, A, as, bs, ts, an, bn, tn, partner(B, s), n, partner(B, n));
  int shared = 0, cv = -1;
  if (as == an || as == bn) { ++shared; cv = as; }
  if (bs == an || bs == bn) { ++shared; cv = bs; }
  if (shared == 0)
    acc += part_p_disjoint(B, A, as, bs, ts, an, bn, tn);
  if (h != nullptr) {
    if (shared == 1) {
      const int p = (as == cv) ? bs : as, qv = (an == cv) ? bn : an;
      const Elem em = make_pair(1 ^ tn ^ ts, p, qv);
      q = __ldg(h + elem_index(B, em.kind, em.a, em.b)) * f_value(B, em, en, es);
    } else if (shared == 2 && tn != ts) {
      for (int lam = imax(as, 1); lam <= bs; ++lam)
        q += __ldg(h + d_index(B, lam)) * f_value(B, make_d(lam), en, es);
    }
  }
  const double r = -0.5 * acc;
  const int64_t o = s * M + n;
  if (Rout) Rout[o] = r;
  if (Qout) Qout[o] = q;
  if (Aout) Aout[o] = q + r;
}

// Sign tables of the disjoint-edge closed form.  For disjoint edges e(s),
// e(n) the l-pair part of Eq. (09) runs over l = (v, w) with v on e(s) and
// w on e(n); the term of (v, w, l) and that of (v', w', l') (the other ends,
// the matching type of l') read the same entry of a, once as a_jk and once
// as a_kj = conj(a_jk), with equal contributions, so the eight terms with
// v = a_s, doubled, give the sum.  For v = a_s < v' = b_s and
// (w, w') = (a_n, b_n) (wi = 0) or (b_n, a_n) (wi = 1),
// every coefficient phase in the eight terms of the (S, S) and (S, J) sums
// depends only on three vertex orders: b0 = [w < v], b1 = [v' < w],
// b2 = [w' < v].  Bit (8 idx + 4 tn + 2 tl + {0: f term, 1: d term}) of
// table wi is set when that term enters with a minus sign (idx = b0 + 2 b1 +
// 4 b2; the minus of the d term and the conjugation of the wi = 0 reads are
// included).
constexpr int cp_(int t, bool x_lt_y) { return t == kS ? 0 : (x_lt_y ? 3 : 1); }
constexpr int sf_(int ph) { return (ph & 3) == 1 ? 1 : -1; }
constexpr int sd_(int ph) { return (ph & 3) == 0 ? 1 : -1; }
constexpr unsigned long long disjoint_sign_table(int wi) {
  unsigned long long T = 0;
  for (int idx = 0; idx < 8; ++idx) {
    const bool b0 = idx & 1, b1 = (idx >> 1) & 1, b2 = (idx >> 2) & 1;
    const int isg = wi ? 1 : -1;
    for (int tn = 0; tn < 2; ++tn) {
      const int phn = cp_(tn, wi == 0);  // coef_phase(tn, w, w'): w < w' iff wi = 0
      for (int tl = 0; tl < 2; ++tl) {
        const int tk = 1 ^ tl, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int sk = sf_(cp_(tk, b1) + cp_(tl, b0));
        const int sf = sf_(phn + cp_(tjf, b2) + cp_(tl, !b0));
        const int sd = sd_(phn + cp_(tjd, b2) + cp_(tl, !b0));
        const unsigned long long nf = (sk * sf) < 0, nd = (-(sk * sd * isg)) < 0;
        T |= nf << (idx * 8 + tn * 4 + tl * 2);
        T |= nd << (idx * 8 + tn * 4 + tl * 2 + 1);
      }
    }
  }
  return T;
}
constexpr unsigned long long kDisjointSign0 = disjoint_sign_table(0);
constexpr unsigned long long kDisjointSign1 = disjoint_sign_table(1);

// Fixed-point summation of the disjoint-edge terms.  GB300's FP64 unit is
// narrow (2 lanes per clock per SM) while the integer pipes are 64 lanes
// wide, so the signed terms of an entry are added exactly as 64-bit integers
// instead of with FP64 adds: each value's 53-bit significand is placed at bit
// 57 of an int64 for the largest exponent E among the values that are summed
// together, and shifted right by E - e_i (truncation error < 2^-57 of the
// largest value per term).  The signed sums of 8 terms are formed in int64
// (|sum| < 2^61), and each result is rounded once to the nearest double, with
// the -1/2 of Eq. (09) applied to the exponent and sign.  Values that are not
// finite, or too small for the exponent arithmetic, take the FP64 path.
struct FxTerm {
  unsigned long long mant;  // significand with the implicit bit set
  int e;                    // biased exponent field (0 for zero and subnormals)
  unsigned neg;             // sign bit
};

// The implicit bit is set unconditionally: a zero or subnormal value has
// e = 0, and the callers only align to E >= 64, so its shift E - e >= 63
// drops it entirely (its magnitude is below 2^-1022, under the 2^-57
// truncation of the largest term).
__device__ __forceinline__ FxTerm fx_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  FxTerm t;
  t.mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  t.e = (int)((b >> 52) & 0x7ff);
  t.neg = (unsigned)(b >> 63);
  return t;
}

// biased exponent of x (zero and subnormals: 1)
__device__ __forceinline__ int fx_exponent(double x) {
  return max((__double2hiint(x) >> 20) & 0x7ff, 1);
}

// term aligned to exponent E (E >= 64), negated when its sign bit is set
__device__ __forceinline__ long long fx_align(const FxTerm& t, int E) {
  const int sh = E - t.e;
  const unsigned long long m = sh < 63 ? ((t.mant << 5) >> sh) : 0ull;
  return t.neg ? -(long long)m : (long long)m;
}



// ---------------------------------------------------------------------------
// Disjoint pair x pair entries by vertex quadruple.  For four vertices
// p < q < r < t the three perfect matchings
//   m = 0: (p,q) | (r,t),   m = 1: (p,r) | (q,t),   m = 2: (p,t) | (q,r)
// each give two ordered edge pairs (s, n), four type pairs each: 24 entries.
// The closed form of an entry on matching m reads the a-block between the
// two edges of each other matching (the k/j edge pairs of Eq. (09)), so the
// 24 entries of the quadruple read the same 12 entries of a (one orientation
// per matching; the other follows from a = a^dagger), and with the vertex
// order fixed every sign is a compile-time constant.  Labels 0..3 stand for
// p, q, r, t.
constexpr int kQuadEdge[3][2][2] = {{{0, 1}, {2, 3}}, {{0, 2}, {1, 3}}, {{0, 3}, {1, 2}}};

struct QuadTerm {
  int y, i, j, c, neg;  // value D[y][i][j][c] (c: 0 re, 1 im), negated if neg
};

constexpr int quad_edge_of(int x, int y) {  // 2 m + e for the edge (x < y)
  for (int m = 0; m < 3; ++m)
    for (int e = 0; e < 2; ++e)
      if (kQuadEdge[m][e][0] == x && kQuadEdge[m][e][1] == y) return 2 * m + e;
  return -1;
}

// Term `slot` (0..3: the (S,S) sum, 4..7: the (S,J) sum) of edge pair wi for
// the output of matching m with s = edge ori, n = edge 1 - ori.  The loaded
// values D[y][i][j] are a[e1 i][e2 j] for y = 0, 1 and a[e2 i][e1 j] for
// y = 2 (e1 = the edge holding p); the sums take X[tj][tk] = a_jk for wi = 1
// and its conjugate for wi = 0, as the sign tables assume.
constexpr QuadTerm quad_term(int m, int ori, int wi, int slot) {
  const int as = kQuadEdge[m][ori][0], bs = kQuadEdge[m][ori][1];
  const int an = kQuadEdge[m][1 - ori][0], bn = kQuadEdge[m][1 - ori][1];
  const int w = wi ? bn : an, wp = wi ? an : bn;
  const int j0 = as < wp ? as : wp, j1 = as < wp ? wp : as;
  const int me = quad_edge_of(j0, j1);
  const int y = me / 2;
  const bool jfirst = (me % 2) == 0;
  const int idx = (w < as ? 1 : 0) | ((bs < w ? 1 : 0) << 1) | ((wp < as ? 1 : 0) << 2);
  const unsigned mb = (unsigned)(((wi ? kDisjointSign1 : kDisjointSign0) >> (8 * idx)) & 0xffu);
  // slots: (tj, tk, comp) = (1,1,re) (0,1,im) (0,0,re) (1,0,im) | (0,1,re) (1,1,im) (1,0,re) (0,0,im)
  constexpr int stj[8] = {1, 0, 0, 1, 0, 1, 1, 0};
  constexpr int stk[8] = {1, 1, 0, 0, 1, 1, 0, 0};
  constexpr int sc[8] = {0, 1, 0, 1, 0, 1, 0, 1};
  const int tj = stj[slot], tk = stk[slot], c = sc[slot];
  int neg = (int)((mb >> slot) & 1u);
  // a_jk = L_y[tj][tk] when j is e1 of matching y, else conj(L_y[tk][tj])
  const int t1 = jfirst ? tj : tk, t2 = jfirst ? tk : tj;
  const int conj = (wi == 0 ? 1 : 0) + (jfirst ? 0 : 1);
  if (c == 1 && (conj & 1)) neg ^= 1;
  QuadTerm r{y, t1, t2, c, neg};
  if (y == 2) {  // loaded as a[e2][e1] = conj(L_2) transposed
    r.i = t2;
    r.j = t1;
    if (c == 1) r.neg ^= 1;
  }
  return r;
}

template <class T, int MM, int ORI, int WI, int SLOT>
__device__ __forceinline__ T quad_val(const T (&D)[3][2][2][2]) {
  constexpr QuadTerm q = quad_term(MM, ORI, WI, SLOT);
  return q.neg ? -D[q.y][q.i][q.j][q.c] : D[q.y][q.i][q.j][q.c];
}

template <class T, int MM, int ORI, int WI>
__device__ __forceinline__ T quad_sum(const T (&D)[3][2][2][2], int half) {
  return half == 0 ? (quad_val<T, MM, ORI, WI, 0>(D) + quad_val<T, MM, ORI, WI, 1>(D)) +
                         (quad_val<T, MM, ORI, WI, 2>(D) + quad_val<T, MM, ORI, WI, 3>(D))
                   : (quad_val<T, MM, ORI, WI, 4>(D) + quad_val<T, MM, ORI, WI, 5>(D)) +
                         (quad_val<T, MM, ORI, WI, 6>(D) + quad_val<T, MM, ORI, WI, 7>(D));
}

// -s/2 * 2^(E - 1080) (s in units of 2^(E - 1080)), rounded to the nearest
// double (ties to even), with integer operations only: GB300's FP64 pipe
// issues about two lanes per clock per SM, so an int64 -> double conversion
// there costs a warp ~64 cycles of that pipe, while these shifts, a count of
// leading zeros and the rounding increment run on the integer pipes and
// leave the FP64 pipe free (4% faster at N = 200, same bits).  |s| < 2^61;
// the caller has checked that the exponent stays normal.  The biased
// exponent of |s| 2^(E - 1081) is E + 5 - lz; the significand with its
// leading bit is added onto (exponent - 1) << 52, so a rounding carry into
// bit 53 moves into the exponent.
__device__ __forceinline__ double quad_out(long long s, int E) {
  if (s == 0) return 0.0;
  const unsigned long long neg = (unsigned long long)(s >> 63);
  unsigned long long m = ((unsigned long long)s ^ neg) - neg;
  const int lz = __clzll((long long)m);
  m <<= lz;
  unsigned long long mant = m >> 11;
  const unsigned rem = (unsigned)m & 0x7ffu;
  mant += (unsigned long long)((rem > 0x400u) | ((rem == 0x400u) & ((unsigned)mant & 1u)));
  const unsigned long long bits = ((unsigned long long)(E + 4 - lz) << 52) + mant;
  return __longlong_as_double((long long)(bits ^ (~neg & 0x8000000000000000ull)));  // the sign of -s
}

struct QuadIdx {
  int64_t e[6];  // pair index of the edges (0,1) (2,3) (0,2) (1,3) (0,3) (1,2)
};

constexpr int quad_slot(int x, int y) { return quad_edge_of(x, y); }  // 2 m + e -> e[] slot

template <int MM, int ORI>
__device__ __forceinline__ void quad_store(const QuadIdx& I, int64_t P, int64_t M, const double (&o)[4],
                                           double* __restrict__ Aout, double* __restrict__ Qout,
                                           double* __restrict__ Rout) {
  constexpr int es = quad_slot(kQuadEdge[MM][ORI][0], kQuadEdge[MM][ORI][1]);
  constexpr int en = quad_slot(kQuadEdge[MM][1 - ORI][0], kQuadEdge[MM][1 - ORI][1]);
  const int64_t s = I.e[es], n = I.e[en];
#pragma unroll
  for (int ts = 0; ts < 2; ++ts)
#pragma unroll
    for (int tn = 0; tn < 2; ++tn) {
      const int64_t off = ((int64_t)ts * P + s) * M + (int64_t)tn * P + n;
      const double v = o[ts * 2 + tn];
      if (Aout) Aout[off] = v;
      if (Rout) Rout[off] = v;
      if (Qout) Qout[off] = 0.0;  // Q vanishes on disjoint edges
    }
}


// Fixed-point form of one output group (always computed; a group that is not
// exact is stored again by the FP64 path afterwards).
template <int MM, int ORI>
__device__ __forceinline__ void quad_group(const long long (&D)[3][2][2][2], int E, int64_t P, int64_t M,
                                           const QuadIdx& I, double* __restrict__ Aout, double* __restrict__ Qout,
                                           double* __restrict__ Rout) {
  const long long xs0 = quad_sum<long long, MM, ORI, 0>(D, 0), xs1 = quad_sum<long long, MM, ORI, 1>(D, 0);
  const long long xj0 = quad_sum<long long, MM, ORI, 0>(D, 1), xj1 = quad_sum<long long, MM, ORI, 1>(D, 1);
  const double o[4] = {quad_out(xs0 + xs1, E),   // (S, S)
                       quad_out(xj0 + xj1, E),   // (S, J)
                       quad_out(xj0 - xj1, E),   // (J, S)
                       quad_out(xs1 - xs0, E)};  // (J, J)
  quad_store<MM, ORI>(I, P, M, o, Aout, Qout, Rout);
}

// FP64 form of one output group (values not finite, or too small for the
// fixed-point form).
template <int MM, int ORI>
__device__ __forceinline__ void quad_group_fp64_t(const double (&V)[3][2][2][2], double (&o)[4]) {
  const double xs0 = quad_sum<double, MM, ORI, 0>(V, 0), xs1 = quad_sum<double, MM, ORI, 1>(V, 0);
  const double xj0 = quad_sum<double, MM, ORI, 0>(V, 1), xj1 = quad_sum<double, MM, ORI, 1>(V, 1);
  o[0] = -0.5 * (xs0 + xs1);
  o[1] = -0.5 * (xj0 + xj1);
  o[2] = -0.5 * (xj0 - xj1);
  o[3] = -0.5 * (xs1 - xs0);
}

// FP64 form of the eight entries of matching MM from the loaded values.
template <int MM>
__device__ __forceinline__ void quad_fp64_matching(const double2 (&L)[3][2][2], int64_t P, int64_t M,
                                                   const QuadIdx& I, double* __restrict__ Aout,
                                                   double* __restrict__ Qout, double* __restrict__ Rout) {
  double V[3][2][2][2];
#pragma unroll
  for (int y = 0; y < 3; ++y)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        V[y][i][j][0] = L[y][i][j].x;
        V[y][i][j][1] = L[y][i][j].y;
      }
  double o[4];
  quad_group_fp64_t<MM, 0>(V, o);
  quad_store<MM, 0>(I, P, M, o, Aout, Qout, Rout);
  quad_group_fp64_t<MM, 1>(V, o);
  quad_store<MM, 1>(I, P, M, o, Aout, Qout, Rout);
}

// The 12 a values of quadruple (p, q, r, t), where u = (r, t): matching 0
// from rows (p,q), matching 1 from rows (p,r), matching 2 from rows (q,r)
// (one orientation each).
struct QuadLoad {
  double2 L[3][2][2];
};

__device__ __forceinline__ void quad_index(int64_t pq, int64_t u, int r, int t, int64_t base_p, int64_t base_q,
                                           QuadIdx& I) {
  I.e[0] = pq;
  I.e[1] = u;
  I.e[2] = base_p + r;
  I.e[3] = base_q + t;
  I.e[4] = base_p + t;
  I.e[5] = base_q + r;
}

__device__ __forceinline__ void quad_load(const AView& A, int64_t P, int64_t M, const QuadIdx& I, QuadLoad& q) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      q.L[0][i][j] = __ldg(A.a + (i * P + I.e[0]) * M + j * P + I.e[1]);
      q.L[1][i][j] = __ldg(A.a + (i * P + I.e[2]) * M + j * P + I.e[3]);
      q.L[2][i][j] = __ldg(A.a + (i * P + I.e[5]) * M + j * P + I.e[4]);
    }
}

// All 12 values are aligned to one exponent E (the quadruple's largest); an
// output matching whose own values lie more than 10 binades below E is
// formed in FP64 instead.
__device__ __forceinline__ void quad_emit(const double2 (&L)[3][2][2], int64_t P, int64_t M, const QuadIdx& I,
                                          double* __restrict__ Aout, double* __restrict__ Qout,
                                          double* __restrict__ Rout) {
  int Ey[3];
#pragma unroll
  for (int y = 0; y < 3; ++y) {
    Ey[y] = 1;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        Ey[y] = max(Ey[y], max(fx_exponent(L[y][i][j].x), fx_exponent(L[y][i][j].y)));
  }
  const int E = max(Ey[0], max(Ey[1], Ey[2]));
  const bool ok = E >= 64 && E <= 2040;
  const bool ex0 = ok && E - max(Ey[1], Ey[2]) <= 10;  // matching 0 reads matchings 1 and 2
  const bool ex1 = ok && E - max(Ey[0], Ey[2]) <= 10;
  const bool ex2 = ok && E - max(Ey[0], Ey[1]) <= 10;
  if (ex0 && ex1 && ex2) {
    long long D[3][2][2][2];
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          D[y][i][j][0] = fx_align(fx_split(L[y][i][j].x), E);
          D[y][i][j][1] = fx_align(fx_split(L[y][i][j].y), E);
        }
    quad_group<0, 0>(D, E, P, M, I, Aout, Qout, Rout);
    quad_group<0, 1>(D, E, P, M, I, Aout, Qout, Rout);
    quad_group<1, 0>(D, E, P, M, I, Aout, Qout, Rout);
    quad_group<1, 1>(D, E, P, M, I, Aout, Qout, Rout);
    quad_group<2, 0>(D, E, P, M, I, Aout, Qout, Rout);
    quad_group<2, 1>(D, E, P, M, I, Aout, Qout, Rout);
  } else {  // rare: values not finite, tiny, or of widely different magnitude
    quad_fp64_matching<0>(L, P, M, I, Aout, Qout, Rout);
    quad_fp64_matching<1>(L, P, M, I, Aout, Qout, Rout);
    quad_fp64_matching<2>(L, P, M, I, Aout, Qout, Rout);
  }
}

// One block per edge (p, q); its warps run over tiles of the edges (r, t)
// with q < r < t.  A tile is kTileR consecutive r by kTileT consecutive t,
// lane = kTileT (r - rbase) + (t - t0).  The r-groups are laid on one grid
// from the top, rbase = N - 1 - kTileR (g + 1) for g = 0, 1, ..., the same
// for every q (lanes with r <= q are idle), so the blocks of (p, q) and
// (p, q + 1), which start close together, visit the rows (r, t) in the same
// order and at about the same time.  In a tile the stores whose column is
// (p, r) or (q, r) cover kTileR adjacent columns and those whose column is
// (p, t), (q, t) or (r, t) kTileT, so these output sectors are written
// nearly whole by one warp instruction; the stores into column (p, q) are
// 8 bytes per row, and their sector neighbours come from the blocks of the
// neighbouring q at about the same time.  A warp issues the loads of its
// next tile before it forms and stores the current one, so the loads stay in
// flight across the arithmetic.
constexpr int kTileR = 8, kTileT = 4;
static_assert(kTileR * kTileT == 32, "a tile is one warp");

struct QuadTile {
  int64_t k;    // tile index within the block
  int64_t cum;  // tiles of the r-groups before this one
  int rbase;    // r = rbase + lane / kTileT
  int t0, cg;   // first t of the group and its number of t-tiles
};

// Start the r-group whose lowest r is rbase, for the block of q.
__device__ __forceinline__ void quad_group_start(int N, int q, int rbase, QuadTile& T) {
  T.rbase = rbase;
  T.t0 = max(rbase, q + 1) + 1;
  T.cg = (N - T.t0 + kTileT - 1) / kTileT;
}

// Move to tile k (>= the current one); false past the last r-group.
__device__ __forceinline__ bool quad_tile_seek(int N, int q, QuadTile& T, int64_t k) {
  T.k = k;
  while (k >= T.cum + T.cg) {
    if (T.rbase <= q + 1) return false;  // that group held r = q + 1
    T.cum += T.cg;
    quad_group_start(N, q, T.rbase - kTileR, T);
  }
  return true;
}

constexpr int kQuadThreads = 256;
// at most 168 registers: no spills, and a little faster than the 182 the
// compiler takes without a cap
__global__ void __maxnreg__(168) k_disjoint4(BasisView B, AView A, double* __restrict__ Aout,
                                                               double* __restrict__ Qout, double* __restrict__ Rout) {
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t pq = blockIdx.x;
  const int32_t abq = __ldg(B.pair_ab + pq);
  const int p = abq >> 16, q = abq & 0xffff;
  if (q + 2 >= N) return;
  const int64_t base_p = (int64_t)p * (2 * N - p - 1) / 2 - p - 1;  // pair_index(p, y) = base_p + y
  const int64_t base_q = (int64_t)q * (2 * N - q - 1) / 2 - q - 1;
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  QuadTile T;
  T.cum = 0;
  quad_group_start(N, q, N - 1 - kTileR, T);
  if (!quad_tile_seek(N, q, T, threadIdx.x >> 5)) return;
  auto coords = [&](const QuadTile& X, int& r, int& t) {
    r = X.rbase + lane / kTileT;
    t = X.t0 + kTileT * (int)(X.k - X.cum) + lane % kTileT;
    return r > q && r <= N - 2 && t <= N - 1 && t > r;
  };
  auto index = [&](int r, int t, QuadIdx& I) {
    const int64_t base_r = (int64_t)r * (2 * N - r - 1) / 2 - r - 1;
    quad_index(pq, base_r + t, r, t, base_p, base_q, I);
  };
  int r, t;
  bool ok = coords(T, r, t);
  QuadIdx I;
  QuadLoad cur;
  if (ok) {
    index(r, t, I);
    quad_load(A, P, M, I, cur);
  }
  while (true) {
    QuadTile Tn = T;
    const bool more = quad_tile_seek(N, q, Tn, T.k + nw);
    int rn = 0, tn = 0;
    const bool okn = more && coords(Tn, rn, tn);
    QuadIdx In;
    QuadLoad nxt;
    if (okn) {
      index(rn, tn, In);
      quad_load(A, P, M, In, nxt);
    }
    if (ok) quad_emit(cur.L, P, M, I, Aout, Qout, Rout);
    if (!more) break;
    T = Tn;
    ok = okn;
    I = In;
    cur = nxt;
  }
}

// Pair row s = (as, bs) type ts, diagonal columns n = D_nu.  One block per
// row; the a entries every nu of the row needs are staged in shared memory:
//   Y[x] = a[partner(s)][D_x],  Z[x] = a[s][D_x],
//   W[(vi, w, tl)] = (a(l, k), a(partner(l), k)),  l = (v, w) tl, k = (v', w) (1^tl^ts).
// With g_s = delta_as - delta_bs, h_s = delta_as + delta_bs:
//   l = D_lam (lam in [lo_s, bs]), k = partner(s), f = sgs g_s(lam); j = D_min(lam,nu)
//     with d = 2 c_max(lam,nu), or for lam = nu every D_mu, mu >= nu;
//   l = (v, w) sharing one vertex with e(s): k on (v', w) (triangle), j = l
//     (d = h_l(nu)) and j = partner(l) (f = -+ g_l(nu));
//   l = partner(s): k = D_mu, f = -sgs g_s(mu); j = partner(s) (d = h_s(nu)),
//     j = s (f = sgs g_s(nu)).
constexpr int kRowThreads = 128;

__global__ void __launch_bounds__(kRowThreads) k_pd(BasisView B, AView A, const double* __restrict__ h,
                                                    double* __restrict__ Aout, double* __restrict__ Qout,
                                                    double* __restrict__ Rout) {
  extern __shared__ double2 sp[];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t s = blockIdx.x;
  const Elem es = decode(B, s);
  const int as = es.a, bs = es.b, ts = es.kind;
  const int64_t sb = partner(B, s);
  const int lo_s = imax(as, 1);
  const double sgs = ts == kS ? 1.0 : -1.0;
  double2* Y = sp;          // [N]
  double2* Z = sp + N;      // [N]
  double2* Wt = sp + 2 * N; // [2][N][2] pairs of values -> 8N double2
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    Y[x] = x >= 1 ? ldA(A, sb, d_index(B, x)) : make_double2(0.0, 0.0);
    Z[x] = x >= 1 ? ldA(A, s, d_index(B, x)) : make_double2(0.0, 0.0);
  }
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) {
    const int vi = t / (2 * N), w = (t / 2) % N, tl = t & 1;
    double2 v0 = make_double2(0.0, 0.0), v1 = v0;
    if (w != as && w != bs) {
      const int v = vi ? bs : as, vp = vi ? as : bs;
      const int64_t pl = pair_index_any(N, v, w), pk = pair_index_any(N, vp, w);
      const int64_t k = (int64_t)(1 ^ tl ^ ts) * P + pk;
      v0 = ldA(A, (int64_t)tl * P + pl, k);
      v1 = ldA(A, (int64_t)(1 - tl) * P + pl, k);
    }
    Wt[2 * t] = v0;
    Wt[2 * t + 1] = v1;
  }
  __syncthreads();
  for (int nu = 1 + threadIdx.x; nu < N; nu += blockDim.x) {
    // l = D_lam
    double accD = 0.0;
    for (int lam = lo_s; lam <= bs; ++lam) {
      const double gs = dlt(B, as, lam) - dlt(B, bs, lam);
      if (lam != nu) {
        const int jm = imin(lam, nu), mx = imax(lam, nu);
        accD = fma(gs, Y[jm].y * 2.0 * ld_c(B, mx), accD);  // -Im a(D_j, partner(s)) = Im Y
      } else {
        double t2 = 0.0;
        for (int mu = nu; mu < N; ++mu) {
          if (mu == 1 && nu == 1) continue;
          const double d = mu > nu ? 2.0 * ld_c(B, mu) : 2.0 * (double)(1 - nu) * ld_c(B, nu);
          t2 = fma(Y[mu].y, d, t2);
        }
        accD = fma(gs, t2, accD);
      }
    }
    double acc = sgs * accD;
    // l = (v, w) on an edge sharing one vertex with e(s)
    double accA = 0.0;
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi ? bs : as, vp = vi ? as : bs;
      const int phs = coef_phase(ts, v, vp);
      for (int w = 0; w < N; ++w) {
        if (w == as || w == bs) continue;
        const int x = imin(v, w), y = imax(v, w);
        if (nu < imax(x, 1)) continue;  // both the d- and the f-fiber vanish
        const double dx = dlt(B, x, nu), dy = dlt(B, y, nu);
        const double hl = (x == 0 && y == 1 && nu == 1) ? 0.0 : dx + dy, gl = dx - dy;
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) {
          const int tk = 1 ^ tl ^ ts;
          const int sk = sgn_f(phs + coef_phase(tk, vp, w) + coef_phase(tl, w, v));
          const double2 al = Wt[2 * ((vi * N + w) * 2 + tl)], alb = Wt[2 * ((vi * N + w) * 2 + tl) + 1];
          const double fl = tl == kS ? -gl : gl;  // f(partner(l), l, D_nu)
          accA += sgn_mul(sk, alb.x * fl - al.y * hl);
        }
      }
    }
    acc += accA * kInvSqrt2;
    // l = partner(s), k = D_mu
    {
      const double gnu = (nu >= lo_s && nu <= bs) ? dlt(B, as, nu) - dlt(B, bs, nu) : 0.0;
      const double hnu = (nu >= lo_s && !(as == 0 && bs == 1 && nu == 1)) ? dlt(B, as, nu) + dlt(B, bs, nu) : 0.0;
      double c1 = 0.0, c2 = 0.0;
      for (int mu = lo_s; mu <= bs; ++mu) {
        const double g = dlt(B, as, mu) - dlt(B, bs, mu);
        c1 = fma(g, Z[mu].x, c1);
        c2 = fma(g, Y[mu].y, c2);
      }
      acc += -gnu * c1 + sgs * hnu * c2;
    }
    double q = 0.0;
    if (h != nullptr && nu >= lo_s && nu <= bs) q = __ldg(h + sb) * sgs * (dlt(B, as, nu) - dlt(B, bs, nu));
    const double r = -0.5 * acc;
    const int64_t o = s * M + d_index(B, nu);
    if (Rout) Rout[o] = r;
    if (Qout) Qout[o] = q;
    if (Aout) Aout[o] = q + r;
  }
}

// Diagonal row s = D_nu, pair columns n = (an, bn) type tn; one thread per entry.
//   l = (v, w) sharing one vertex with e(n), nu in [max(x,1), y] for {x,y} = {v,w}:
//     k = partner(l), f = -+ g_l(nu); j on (v', w), both types (triangle);
//   l on e(n) itself when nu in [max(an,1), bn]: k = partner(l); j = D_mu
//     (d = h_n(mu) if l = n, f = -+ g_n(mu) if l = partner(n)).
__global__ void __launch_bounds__(256) k_dp(BasisView B, AView A, const double* __restrict__ h,
                                            double* __restrict__ Aout, double* __restrict__ Qout,
                                            double* __restrict__ Rout) {
  const int N = B.N;
  const int64_t P = B.P, M = B.M, P2 = 2 * P;
  const int64_t chunks = (P2 + 255) / 256;
  const int nu = 1 + (int)(blockIdx.x / chunks);
  const int64_t n = (blockIdx.x % chunks) * 256 + threadIdx.x;
  if (n >= P2) return;
  const Elem en = decode(B, n);
  const int an = en.a, bn = en.b, tn = en.kind;
  double acc2 = 0.0;
  for (int vi = 0; vi < 2; ++vi) {
    const int v = vi ? bn : an, vp = vi ? an : bn;
    const int phn = coef_phase(tn, v, vp);
    for (int w = 0; w < N; ++w) {
      if (w == an || w == bn) continue;
      const int x = imin(v, w), y = imax(v, w);
      if (nu < imax(x, 1) || nu > y) continue;
      const double gl = dlt(B, x, nu) - dlt(B, y, nu);
      const int64_t pl = pair_index_any(N, v, w), pj = pair_index_any(N, vp, w);
#pragma unroll
      for (int tl = 0; tl < 2; ++tl) {
        const int tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int phl = coef_phase(tl, w, v);
        const int sf = sgn_f(phn + coef_phase(tjf, vp, w) + phl);
        const int sd = sgn_d(phn + coef_phase(tjd, vp, w) + phl);
        const int64_t kb = (int64_t)(1 - tl) * P + pl;  // partner(l)
        // read from the row that is common to the lanes of a warp (v = an: k; v = bn: j)
        const double2 a1 = vi ? ldA(A, (int64_t)tjf * P + pj, kb) : ldA_row(A, (int64_t)tjf * P + pj, kb);
        const double2 a2 = vi ? ldA(A, (int64_t)tjd * P + pj, kb) : ldA_row(A, (int64_t)tjd * P + pj, kb);
        const double t = sgn_mul(sf, a1.x) - sgn_mul(sd, a2.y);
        acc2 += tl == kS ? -gl * t : gl * t;
      }
    }
  }
  double acc = acc2 * kInvSqrt2;
  double q = 0.0;
  const int lo_n = imax(an, 1);
  if (nu >= lo_n && nu <= bn) {
    const double gn = dlt(B, an, nu) - dlt(B, bn, nu);
    const int64_t nb = partner(B, n);
    for (int tl = 0; tl < 2; ++tl) {
      const double fk = tl == kS ? -gn : gn;  // f(partner(l), l, D_nu), l on e(n)
      const int64_t kb = (int64_t)(1 - tl) * P + (n % P);
      double t = 0.0;
      if (tl == tn) {
        for (int mu = lo_n; mu < N; ++mu) {
          if (an == 0 && bn == 1 && mu == 1) continue;
          t -= ldA(A, d_index(B, mu), kb).y * (dlt(B, an, mu) + dlt(B, bn, mu));
        }
      } else {
        for (int mu = lo_n; mu <= bn; ++mu) t += ldA(A, d_index(B, mu), kb).x * (dlt(B, an, mu) - dlt(B, bn, mu));
        if (tn == kS) t = -t;
      }
      acc = fma(fk, t, acc);
    }
    if (h != nullptr) q = __ldg(h + nb) * (tn == kS ? -gn : gn);
  }
  const double r = -0.5 * acc;
  const int64_t o = d_index(B, nu) * M + n;
  if (Rout) Rout[o] = r;
  if (Qout) Qout[o] = q;
  if (Aout) Aout[o] = q + r;
}

// Diagonal row s = D_nu, diagonal column n = D_mu; one warp per entry.  Only
// l = (x, y) with x <= min(nu, mu), y >= nu contribute, k = partner(l); the
// two types of l combine to
//   g_xy(nu) g_xy(mu) (Re a_{S S} + Re a_{J J}) + 2 g_xy(nu) h_xy(mu) Im a_{S J}.
__global__ void __launch_bounds__(256) k_dd(BasisView B, AView A, double* __restrict__ Aout,
                                            double* __restrict__ Qout, double* __restrict__ Rout) {
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= (int64_t)(N - 1) * (N - 1)) return;
  const int nu = 1 + (int)(e / (N - 1)), mu = 1 + (int)(e % (N - 1));
  const int xm = imin(nu, mu);
  double acc = 0.0;
  const int64_t cnt = (int64_t)(xm + 1) * N;
  for (int64_t t = lane; t < cnt; t += 32) {
    const int x = (int)(t / N), y = (int)(t % N);
    if (y <= x || y < nu) continue;
    const double gn = dlt(B, x, nu) - dlt(B, y, nu);
    const double gm = dlt(B, x, mu) - dlt(B, y, mu);
    const double hm = (x == 0 && y == 1 && mu == 1) ? 0.0 : dlt(B, x, mu) + dlt(B, y, mu);
    const int64_t p = pair_index(N, x, y);
    const double ass = ldA(A, p, p).x, ajj = ldA(A, P + p, P + p).x, asj = ldA(A, p, P + p).y;
    acc = fma(gn, fma(gm, ass + ajj, 2.0 * hm * asj), acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const double r = -0.5 * acc;
    const int64_t o = d_index(B, nu) * M + d_index(B, mu);
    if (Rout) Rout[o] = r;
    if (Qout) Qout[o] = 0.0;
    if (Aout) Aout[o] = r;
  }
}

// ---------------------------------------------------------------------------
// Diagonal blocks through the Helmert structure of the D_l.  With d_l the
// vector of the diagonal of D_l (d_l[k] = delta_k(l)), g_xy(l) = d_l[x] -
// d_l[y] and h_xy(l) = d_l[x] + d_l[y], sums over pairs x < y of the form
// sum g_xy(nu) (g_xy(mu) W_xy + 2 h_xy(mu) V_xy) are d_nu^T G d_mu with the
// N x N matrix
//   G = sum_{x<y} W_xy (e_x - e_y)(e_x - e_y)^T + 2 V_xy (e_x - e_y)(e_x + e_y)^T,
// and every d_l^T x is c_l sum_{k<l} x_k - l c_l x_l: a prefix sum.  So the
// diagonal x diagonal block costs O(N^2) instead of O(N^4).

// W_xy = Re a(S_xy, S_xy) + Re a(J_xy, J_xy), V_xy = Im a(S_xy, J_xy), x < y
__device__ __forceinline__ void dd_wv(const BasisView& B, const AView& A, int x, int y, double& W, double& V) {
  const int64_t p = pair_index(B.N, x, y);
  W = ldA(A, p, p).x + ldA(A, B.P + p, B.P + p).x;
  V = ldA(A, p, B.P + p).y;
}

// The diagonal x diagonal block, R[D_nu][D_mu] = -1/2 sum_{x<y} g_xy(nu)
// (g_xy(mu) W_xy + 2 h_xy(mu) V_xy), by cells of constant coefficient.  The
// vertices split at lo = min(nu, mu) and hi = max(nu, mu) into the classes
// [0, lo), {lo}, (lo, hi), {hi}, (hi, N); g_xy(l) and h_xy(l) depend only on
// the classes of x and y (delta_x(l) is c_l below l, -l c_l at l, 0 above),
// and g_xy(nu) != 0 needs x <= nu <= y, so every pair whose coefficient is
// not zero lies in a cell (class of x) x (class of y) with x's class before
// y's.  A cell's sum of W (or V) comes from tables of sums of terms that
// all enter the entry: a point, a column prefix sum_{x<a} X_xy, a row range
// from row suffixes RS[x][b] = sum_{y>=b, y>x} X_xy, or a corner range from
// C[a][b] = sum_{x<a, y>=b, x<y} X_xy.  No cell sums pairs whose coefficient
// is zero, so no such terms are added and cancelled (the prefix form
// d_nu^T G d_mu over all pairs would cancel them only up to rounding,
// relative to their own size).  O(N^2) tables, O(1) per entry.
struct DDTables {
  double *W, *V;      // [N][N], x < y
  double *RSW, *RSV;  // [N][N + 1]
  double *CPW, *CPV;  // [N][N + 1]: CP[y][a] = sum_{x<a, x<y} X_xy
  double *CW, *CV;    // [N + 1][N + 1]
  static size_t doubles(int N) { return 2 * (size_t)N * N + 4 * (size_t)N * (N + 1) + 2 * (size_t)(N + 1) * (N + 1); }
  static DDTables carve(double* base, int N) {
    DDTables t;
    const size_t nn = (size_t)N * N, nr = (size_t)N * (N + 1), cc = (size_t)(N + 1) * (N + 1);
    t.W = base;
    t.V = t.W + nn;
    t.RSW = t.V + nn;
    t.RSV = t.RSW + nr;
    t.CPW = t.RSV + nr;
    t.CPV = t.CPW + nr;
    t.CW = t.CPV + nr;
    t.CV = t.CW + cc;
    return t;
  }
};

// Row x of W and V, and their row suffixes.  One block per x.
__global__ void __launch_bounds__(128) k_dd_rows(BasisView B, AView A, DDTables T) {
  const int N = B.N, x = blockIdx.x;
  for (int y = threadIdx.x; y < N; y += blockDim.x) {
    double W = 0.0, V = 0.0;
    if (y > x) dd_wv(B, A, x, y, W, V);
    T.W[(int64_t)x * N + y] = W;
    T.V[(int64_t)x * N + y] = V;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const double* X = (threadIdx.x ? T.V : T.W) + (int64_t)x * N;
    double* RS = (threadIdx.x ? T.RSV : T.RSW) + (int64_t)x * (N + 1);
    double acc = 0.0;
    RS[N] = 0.0;
    for (int b = N - 1; b >= 0; --b) {
      if (b > x) acc += X[b];
      RS[b] = acc;
    }
  }
}

// Column prefixes CP[y][a] and corner sums C[a][b] = sum_{x<a} RS[x][b]:
// thread t < 2N takes column y = t / 2 (W or V), thread t in [2N, 4N + 2)
// takes corner column b.
__global__ void __launch_bounds__(128) k_dd_cols(BasisView B, DDTables T) {
  const int N = B.N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 2 * N) {
    const int y = t >> 1, wv = t & 1;
    const double* X = wv ? T.V : T.W;
    double* CP = (wv ? T.CPV : T.CPW) + (int64_t)y * (N + 1);
    double acc = 0.0;
    CP[0] = 0.0;
    for (int a = 0; a < N; ++a) {
      if (a < y) acc += X[(int64_t)a * N + y];
      CP[a + 1] = acc;
    }
  } else if (t < 2 * N + 2 * (N + 1)) {
    const int u = t - 2 * N, b = u >> 1, wv = u & 1;
    const double* RS = wv ? T.RSV : T.RSW;
    double* C = wv ? T.CV : T.CW;
    double acc = 0.0;
    C[b] = 0.0;  // a = 0
    for (int a = 1; a <= N; ++a) {
      acc += RS[(int64_t)(a - 1) * (N + 1) + b];
      C[(int64_t)a * (N + 1) + b] = acc;
    }
  }
}

// Sum of X over the cell [x0, x1) x [y0, y1) (x1 <= y0) from the tables.
__device__ __forceinline__ double dd_cell(const double* X, const double* RS, const double* CP, const double* C,
                                          int N, int x0, int x1, int y0, int y1) {
  if (x1 - x0 == 1 && y1 - y0 == 1) return X[(int64_t)x0 * N + y0];
  if (y1 - y0 == 1) return CP[(int64_t)y0 * (N + 1) + x1];  // x0 = 0
  if (x1 - x0 == 1) return RS[(int64_t)x0 * (N + 1) + y0] - RS[(int64_t)x0 * (N + 1) + y1];
  return C[(int64_t)x1 * (N + 1) + y0] - C[(int64_t)x1 * (N + 1) + y1];  // x0 = 0
}

// One thread per entry (nu, mu), nu, mu in 1..N-1.
__global__ void __launch_bounds__(256) k_dd_cells(BasisView B, DDTables T, double* __restrict__ Aout,
                                                  double* __restrict__ Qout, double* __restrict__ Rout) {
  const int N = B.N;
  const int64_t M = B.M;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)(N - 1) * (N - 1)) return;
  const int nu = 1 + (int)(e / (N - 1)), mu = 1 + (int)(e % (N - 1));
  const int lo = imin(nu, mu), hi = imax(nu, mu);
  int c0[5], c1[5], nc = 0;
  auto add = [&](int a, int b) {
    if (b > a) {
      c0[nc] = a;
      c1[nc] = b;
      ++nc;
    }
  };
  add(0, lo);
  add(lo, lo + 1);
  if (hi > lo) {
    add(lo + 1, hi);
    add(hi, hi + 1);
  }
  add(hi + 1, N);
  double acc = 0.0;
  for (int i = 0; i < nc; ++i) {
    const int x = c0[i];
    const double dxn = dlt(B, x, nu), dxm = dlt(B, x, mu);
    for (int j = i + 1; j < nc; ++j) {
      const int y = c0[j];
      const double g = dxn - dlt(B, y, nu);
      if (g == 0.0) continue;
      const double dym = dlt(B, y, mu);
      const double cw = g * (dxm - dym), cv = 2.0 * g * (dxm + dym);
      if (cw != 0.0) acc = fma(cw, dd_cell(T.W, T.RSW, T.CPW, T.CW, N, c0[i], c1[i], c0[j], c1[j]), acc);
      if (cv != 0.0) acc = fma(cv, dd_cell(T.V, T.RSV, T.CPV, T.CV, N, c0[i], c1[i], c0[j], c1[j]), acc);
    }
  }
  const double r = -0.5 * acc;
  const int64_t o = d_index(B, nu) * M + d_index(B, mu);
  if (Rout) Rout[o] = r;
  if (Qout) Qout[o] = 0.0;
  if (Aout) Aout[o] = r;
}

// Tables of the D x D block X[lam][mu] = a[D_lam][D_mu] for the same-edge
// entries' D-section sums: CXr[lam][mu] = c_lam Re X[lam][mu] and the
// suffix sums SXi[k][mu] = sum_{lam >= k} c_lam Im X[lam][mu] (k = 0..N,
// SXi[N][mu] = 0).  One block per column mu >= 1; row-major N-wide tables.
__global__ void __launch_bounds__(128) k_dtab(BasisView B, AView A, double* __restrict__ CXr,
                                              double* __restrict__ SXi) {
  __shared__ double xi[lbi::kMaxDenseN];
  __shared__ double sx[lbi::kMaxDenseN + 1];
  const int N = B.N, mu = 1 + blockIdx.x;
  for (int lam = threadIdx.x; lam < N; lam += blockDim.x) {
    double cr = 0.0, ci = 0.0;
    if (lam >= 1) {
      const double c = ld_c(B, lam);
      const double2 x = ldA(A, d_index(B, lam), d_index(B, mu));
      cr = c * x.x;
      ci = c * x.y;
    }
    CXr[(int64_t)lam * N + mu] = cr;
    xi[lam] = ci;
  }
  __syncthreads();
  if (threadIdx.x < 32) warp_suffix(xi, sx, N);
  __syncthreads();
  for (int k = threadIdx.x; k <= N; k += blockDim.x) SXi[(int64_t)k * N + mu] = sx[k];
}

// Pair-pair entries whose edges share one vertex v: s on (v, p), n on (v, q).
// Shared memory: T1[w][tj][tk] = a[(q,w) tj][(p,w) tk],  T2[mu][t] = a[D_mu][(p,q) t].
__global__ void __launch_bounds__(256) k_shared(BasisView B, AView A, double* __restrict__ Aout,
                                                double* __restrict__ Rout) {
  extern __shared__ double2 sm[];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int p = blockIdx.x / (N - 1);
  int q = blockIdx.x % (N - 1);
  if (q >= p) ++q;
  double2* T1 = sm;
  double2* T2 = sm + 4 * N;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) {
    const int w = t >> 2, tj = (t >> 1) & 1, tk = t & 1;
    double2 val = make_double2(0.0, 0.0);
    if (w != p && w != q) val = ldA(A, tj * P + pair_index_any(N, q, w), tk * P + pair_index_any(N, p, w));
    T1[t] = val;
  }
  const int64_t ppq = pair_index_any(N, p, q);
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int mu = t >> 1, tt = t & 1;
    T2[t] = mu >= 1 ? ldA(A, d_index(B, mu), tt * P + ppq) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < N; v += nw) {
    if (v == p || v == q) continue;
    const int64_t pvp = pair_index_any(N, v, p), pvq = pair_index_any(N, v, q);
    for (int combo = 0; combo < 4; ++combo) {
      const int ts = combo >> 1, tn = combo & 1;
      double acc2 = 0.0, accD = 0.0;
      // (A1) e(l) = (v, w), w not in {v, p, q}: k on (p, w), j on (q, w)
      for (int w = lane; w < N; w += 32) {
        if (w == v || w == p || w == q) continue;
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) {
          const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
          const int phl = coef_phase(tl, w, v);
          const int sk = sgn_f(coef_phase(ts, v, p) + coef_phase(tk, p, w) + phl);
          const int base = coef_phase(tn, v, q) + phl;
          const int sf = sgn_f(base + coef_phase(tjf, q, w));
          const int sd = sgn_d(base + coef_phase(tjd, q, w));
          acc2 += sgn_mul(sk * sf, T1[4 * w + 2 * tjf + tk].x);
          acc2 -= sgn_mul(sk * sd, T1[4 * w + 2 * tjd + tk].y);
        }
      }
      // (A3) e(l) = e(n) = (v, q): k on (p, q), j = D_mu
      {
        const int lo = imin(v, q), hi = imax(v, q);
        for (int tl = 0; tl < 2; ++tl) {
          const int tk = 1 ^ tl ^ ts;
          const int sk = sgn_f(coef_phase(ts, v, p) + coef_phase(tk, p, q) + coef_phase(tl, q, v));
          double part = 0.0;
          if (tl == tn) {  // d(D_mu, n, n) = delta_lo + delta_hi, mu >= max(lo,1), not (0,1,1)
            for (int mu = imax(lo, 1) + lane; mu < N; mu += 32) {
              if (lo == 0 && hi == 1 && mu == 1) continue;
              part -= T2[2 * mu + tk].y * (dlt(B, lo, mu) + dlt(B, hi, mu));
            }
          } else {  // f(D_mu, partner(n), n) = -+(delta_lo - delta_hi), mu in [max(lo,1), hi]
            for (int mu = imax(lo, 1) + lane; mu <= hi; mu += 32)
              part += T2[2 * mu + tk].x * (dlt(B, lo, mu) - dlt(B, hi, mu));
            if (tn == kS) part = -part;
          }
          accD += sgn_mul(sk, part) * kInvSqrt2;
        }
      }
      // (B) l = partner(s) on (v, p): k = D_mu, j on (p, q)
      {
        const int lo = imin(v, p), hi = imax(v, p), tl = 1 - ts;
        const int tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int base = coef_phase(tn, v, q) + coef_phase(tl, p, v);
        const int sf = sgn_f(base + coef_phase(tjf, q, p));
        const int sd = sgn_d(base + coef_phase(tjd, q, p));
        double part = 0.0;
        for (int mu = imax(lo, 1) + lane; mu <= hi; mu += 32) {
          const double g = dlt(B, lo, mu) - dlt(B, hi, mu);
          part = fma(g, sgn_mul(sf, T2[2 * mu + tjf].x) + sgn_mul(sd, T2[2 * mu + tjd].y), part);
        }
        if (ts == kS) part = -part;  // f(D_mu, partner(s), s) = -+ g_s(mu)
        accD += part * kInvSqrt2;
      }
      // (A2) e(l) = (p, q): k on (v, q), j on (v, p)
      if (lane == 0) {
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) {
          const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
          const int sk = sgn_f(coef_phase(ts, p, v) + coef_phase(tk, v, q) + coef_phase(tl, q, p));
          const int base = coef_phase(tn, q, v) + coef_phase(tl, p, q);
          const int sf = sgn_f(base + coef_phase(tjf, v, p));
          const int sd = sgn_d(base + coef_phase(tjd, v, p));
          const int64_t k = tk * P + pvq;
          const double2 a1 = ldA(A, tjf * P + pvp, k), a2 = ldA(A, tjd * P + pvp, k);
          acc2 += sgn_mul(sk * sf, a1.x);
          acc2 -= sgn_mul(sk * sd, a2.y);
        }
      }
      const double tot = warp_sum(0.5 * acc2 + accD);
      if (lane == 0) {
        const double r = -0.5 * tot;
        const int64_t o = (ts * P + pvp) * M + (tn * P + pvq);
        if (Rout) Rout[o] += r;
        if (Aout) Aout[o] += r;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Closed-form variants (LB_ALG_CLOSED) of k_shared and k_pd.  Inside the sum
// over the free vertex w of an l = (v, w) family (and over the levels mu of a
// D-fiber) every coefficient -- triangle signs, delta_w(nu), the order of w
// and v -- only changes where w crosses one of a few fixed vertices, so the
// sum is a handful of interval sums of the staged a values, taken from
// prefix sums: O(1) per entry after O(N) staging per block.

// sum_{w=lo}^{hi} x_w from a prefix array pre[w+1] = sum_{w' <= w} x_w'
__device__ __forceinline__ double isum(const double* pre, int lo, int hi) {
  return lo <= hi ? pre[hi + 1] - pre[lo] : 0.0;
}

// In-place prefix sums arr[1..n] of one array (arr[0] = 0 on entry) by one
// whole warp: every lane sums a contiguous segment of about n/32 values, an
// exclusive shuffle scan of the segment sums gives each lane its offset, and
// the lane writes its running sums.  GB300's FP64 pipe takes a warp
// instruction at the same cost whether 1 or 32 lanes are active, so a scan
// by one lane per array costs n warp instructions; this one costs about
// 2 n/32 + 5.
__device__ __forceinline__ void warp_prefix(double* arr, int n) {
  const int lane = threadIdx.x & 31;
  const int seg = (n + 31) >> 5;
  const int lo = 1 + lane * seg, hi = min(n, lo + seg - 1);
  double t = 0.0;
  for (int i = lo; i <= hi; ++i) t += arr[i];
  double inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  double run = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) run = 0.0;
  for (int i = lo; i <= hi; ++i) {
    run += arr[i];
    arr[i] = run;
  }
}

// Suffix sums y[k] = sum_{w >= k} x[w], k = 0..n-1, and y[n] = 0, by one
// whole warp (segments from the top, as in warp_prefix).
__device__ __forceinline__ void warp_suffix(const double* x, double* y, int n) {
  const int lane = threadIdx.x & 31;
  const int seg = (n + 31) >> 5;
  const int hi = n - 1 - lane * seg, lo = max(0, hi - seg + 1);
  double t = 0.0;
  for (int i = hi; i >= lo; --i) t += x[i];
  double inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  double run = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) run = 0.0;
  for (int i = hi; i >= lo; --i) {
    run += x[i];
    y[i] = run;
  }
  if (lane == 0) y[n] = 0.0;
}


constexpr double kNegHalfInvSqrt2 = -0.5 * kInvSqrt2;  // exact: a power-of-two scaling

// Staged data of one unordered vertex pair {p < q}, and accessors for the
// orientation (P_, Q_) = (p, q) (tr = 0) or (q, p) (tr = 1).  For (q, p) the
// staged a[(q,w) tj][(p,w) tk] becomes a[(p,w) tj][(q,w) tk] = conj(a[(q,w) tk][(p,w) tj]).
struct PairStage {
  const double* PX;  // [4][L] Re a[(q,w) tj][(p,w) tk] at w, index tj*2+tk
  const double* PY;  // [4][L] Im
  const double* TX;  // [2][L] Re a[D_mu][(p,q) t] (raw, index mu)
  const double* TY;  // [2][L] Im
  const double* CX;  // [2][L] c_mu Re a[D_mu][(p,q) t]
  const double* CY;  // [2][L] c_mu Im
  const double* DX;  // [2][L] (D x)_k = sum_mu delta_k(mu) Re a[D_mu][(p,q) t], k = 0..N-1
  const double* DY;  // [2][L] the same for Im
  const double* TOT; // [32] signed totals of the (A1) sums, see k_shared_closed
  int L;
  // sum_mu (delta_lo(mu) + sg delta_hi(mu)) x_mu for lo < hi (the d-vector form of dsum)
  __device__ __forceinline__ double dx(int t, int lo, int hi, double sg) const { return DX[t * L + lo] + sg * DX[t * L + hi]; }
  __device__ __forceinline__ double dy(int t, int lo, int hi, double sg) const { return DY[t * L + lo] + sg * DY[t * L + hi]; }
  // Re / Im of a[(Q_,w) tj][(P_,w) tk] for orientation tr (P_, Q_ = p, q or q, p)
  __device__ __forceinline__ double sre(int tr, int tj, int tk, int w) const {
    return PX[(tr ? tk * 2 + tj : tj * 2 + tk) * L + w];
  }
  __device__ __forceinline__ double sim(int tr, int tj, int tk, int w) const {
    const double x = PY[(tr ? tk * 2 + tj : tj * 2 + tk) * L + w];
    return tr ? -x : x;
  }
};

// l-pair part of the pair x pair entry s on (v, P_), n on (v, Q_) (edges
// sharing the vertex v), in closed form, split into the terms that do not
// depend on v (block constants: the block totals of (A1) and the D-vector
// values at P_ and Q_ of (A3) and (B)), formed once per block for each
// orientation, type pair and position of v against P_ and Q_, and the terms
// at v, formed per entry.  The entry is -1/4 acc2 - 1/(2 sqrt2) accD.
//
// (A1): all w outside {v, P_, Q_}.  Every J edge's phase moves by 2 when its
// vertex order flips, which flips the sign of f (odd phase sums) and of d
// (even sums); the order of w and v enters sk and sf (sd) once each and
// cancels, so with sigma(w) = (-1)^([P_ < w] tk + [Q_ < w] tj) the sum is
// kappa (TOT - sigma(v) X(v)), TOT the block's signed total over all w.
// (A3): e(l) = (v, Q_), k on (P_, Q_), j = D_mu.  (B): l = partner(s) on
// (v, P_), k = D_mu, j on (P_, Q_).  (A2): e(l) = (P_, Q_), k on (v, Q_), j
// on (v, P_), from the four values X[tj][tk] = a[(tj, (v, P_))][(tk, (v, Q_))].
struct SharedSigns {  // the integer signs of one (ts, tn, tl) at one position of v
  int kf, kd, sfv, sdv;
};

__device__ __forceinline__ SharedSigns shared_signs_a1(int ts, int tn, int tl, int a_, int b_, int pv, int qv) {
  const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
  const int sk = sgn_f(a_ + tk + tl);  // phases at [P_ < w] = [w < v] = 0
  SharedSigns g;
  g.kf = sk * sgn_f(b_ + tl + tjf);
  g.kd = sk * sgn_d(b_ + tl + tjd);
  g.sfv = ((pv & tk) ^ (qv & tjf)) ? -1 : 1;
  g.sdv = ((pv & tk) ^ (qv & tjd)) ? -1 : 1;
  return g;
}

// Block constant of orientation tr, type pair (ts, tn), and v with
// [P_ < v] = pv, [Q_ < v] = qv (v stands for any vertex in that position).
__device__ __forceinline__ double shared_entry_const(const PairStage& S, int tr, int P_, int Q_, int pv, int qv,
                                                     int ts, int tn) {
  // a vertex v with the given position: only its comparisons with P_, Q_ enter
  const int vlo_p = pv ? 0 : 1, vlo_q = qv ? 0 : 1;  // [v < P_], [v < Q_]
  const int a_ = ts == kS ? 0 : (vlo_p ? 3 : 1), b_ = tn == kS ? 0 : (vlo_q ? 3 : 1);
  double acc2 = 0.0, accD = 0.0;
#pragma unroll
  for (int tl = 0; tl < 2; ++tl) {
    const SharedSigns g = shared_signs_a1(ts, tn, tl, a_, b_, pv, qv);
    const double* T = S.TOT + ((tr * 2 + ts) * 2 + tn) * 4 + tl * 2;
    acc2 += sgn_mul(g.kf, T[0]);
    acc2 -= sgn_mul(g.kd, T[1]);
  }
  // (A3): the value at Q_ of DX / DY
#pragma unroll
  for (int tl = 0; tl < 2; ++tl) {
    const int tk = 1 ^ tl ^ ts;
    const int ph_v_p = ts == kS ? 0 : (vlo_p ? 3 : 1);            // coef_phase(ts, v, P_)
    const int ph_q_v = tl == kS ? 0 : (vlo_q ? 1 : 3);            // coef_phase(tl, Q_, v)
    const int sk = sgn_f(ph_v_p + coef_phase(tk, P_, Q_) + ph_q_v);
    double part;
    if (tl == tn) part = -S.DY[tk * S.L + Q_];
    else {
      const double x = S.DX[tk * S.L + Q_];  // dx(lo, hi, -1) = X[lo] - X[hi], negated for tn = S
      part = tn == kS ? (vlo_q ? x : -x) : (vlo_q ? -x : x);
    }
    accD += sgn_mul(sk, part);
  }
  // (B): the values at P_
  {
    const int tl = 1 - ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
    const int ph_v_q = tn == kS ? 0 : (vlo_q ? 3 : 1);  // coef_phase(tn, v, Q_)
    const int ph_p_v = tl == kS ? 0 : (vlo_p ? 1 : 3);  // coef_phase(tl, P_, v)
    const int base = ph_v_q + ph_p_v;
    const int sf = sgn_f(base + coef_phase(tjf, Q_, P_));
    const int sd = sgn_d(base + coef_phase(tjd, Q_, P_));
    // dx(lo, hi, -1) = X[lo] - X[hi]: the P_ value enters with - when P_ is the upper end
    const double part = sgn_mul(sf, S.DX[tjf * S.L + P_]) + sgn_mul(sd, S.DY[tjd * S.L + P_]);
    const double pp = vlo_p ? -part : part;
    accD += ts == kS ? -pp : pp;
  }
  return fma(-0.25, acc2, kNegHalfInvSqrt2 * accD);
}

// The terms at v of the same entry, to be scaled as in shared_entry_const:
// t[0..7] the signed terms of acc2 ((A1) at v, then (A2)), and accD (t[8],
// t[9] are left to the caller).
__device__ __forceinline__ void shared_entry_var(const double2 (&X)[2][2], const PairStage& S, int tr, int P_,
                                                 int Q_, int v, int ts, int tn, double (&t)[10], double& accD) {
  const int pv = P_ < v ? 1 : 0, qv = Q_ < v ? 1 : 0;
  const int a_ = coef_phase(ts, v, P_), b_ = coef_phase(tn, v, Q_);
#pragma unroll
  for (int tl = 0; tl < 2; ++tl) {  // (A1) at v
    const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
    const SharedSigns g = shared_signs_a1(ts, tn, tl, a_, b_, pv, qv);
    t[2 * tl] = sgn_mul(-g.kf * g.sfv, S.sre(tr, tjf, tk, v));
    t[2 * tl + 1] = sgn_mul(g.kd * g.sdv, S.sim(tr, tjd, tk, v));
  }
#pragma unroll
  for (int tl = 0; tl < 2; ++tl) {  // (A2)
    const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
    const int sk = sgn_f(coef_phase(ts, P_, v) + coef_phase(tk, v, Q_) + coef_phase(tl, Q_, P_));
    const int base = coef_phase(tn, Q_, v) + coef_phase(tl, P_, Q_);
    const int sf = sgn_f(base + coef_phase(tjf, v, P_));
    const int sd = sgn_d(base + coef_phase(tjd, v, P_));
    t[4 + 2 * tl] = sgn_mul(sk * sf, X[tjf][tk].x);
    t[5 + 2 * tl] = sgn_mul(-sk * sd, X[tjd][tk].y);
  }
  // accD starts from its first term (an add to 0.0 is an FP64 instruction of its own)
  const int vlo_q = v < Q_, vlo_p = v < P_;
#pragma unroll
  for (int tl = 0; tl < 2; ++tl) {  // (A3) at v
    const int tk = 1 ^ tl ^ ts;
    const int sk = sgn_f(coef_phase(ts, v, P_) + coef_phase(tk, P_, Q_) + coef_phase(tl, Q_, v));
    double part;
    if (tl == tn) part = -S.DY[tk * S.L + v];
    else {
      const double x = S.DX[tk * S.L + v];  // dx(lo, hi, -1) = X[lo] - X[hi], negated for tn = S
      part = tn == kS ? (vlo_q ? -x : x) : (vlo_q ? x : -x);
    }
    accD = tl == 0 ? sgn_mul(sk, part) : accD + sgn_mul(sk, part);
  }
  {  // (B) at v
    const int tl = 1 - ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
    const int base = coef_phase(tn, v, Q_) + coef_phase(tl, P_, v);
    const int sf = sgn_f(base + coef_phase(tjf, Q_, P_));
    const int sd = sgn_d(base + coef_phase(tjd, Q_, P_));
    const double part = sgn_mul(sf, S.DX[tjf * S.L + v]) + sgn_mul(sd, S.DY[tjd * S.L + v]);
    const double pv_ = vlo_p ? part : -part;
    accD += ts == kS ? -pv_ : pv_;
  }
}

// -(t[0] + ... + t[7] + 2 t[8] + 2 t[9]) / 4, exactly rounded: the ten terms
// in int64 fixed point at their largest exponent (see fx_split / fx_align;
// truncation below 2^-57 of the largest term), one rounding at the end.
// GB300's FP64 pipe takes a warp instruction in about 64 cycles of an SM
// sub-partition against 2 for an integer one, so the ten-term sum costs the
// FP64 pipe nothing.  false (and *out untouched) for values that are not
// finite or too small for the exponent arithmetic.
__device__ __forceinline__ bool fx_quarter_sum10(const double (&t)[10], double* out) {
  int E = 1;
#pragma unroll
  for (int i = 0; i < 10; ++i) E = max(E, fx_exponent(t[i]) + (i >= 8 ? 1 : 0));
  if (E < 65 || E > 2040) return false;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    FxTerm f = fx_split(t[i]);
    if (i >= 8) f.e += 1;  // 2 t[i]: the same significand one binade up
    s += fx_align(f, E);
  }
  *out = quad_out(s, E - 1);  // -s/2 2^(E - 1 - 1080) = -(sum)/4
  return true;
}

// Diagonal row D_nu, pair column n on {p, q} of type tn, in closed form: the
// l = (v, w) families for v = p and v = q (k = partner(l), j on (v', w)), the
// l on e(n) itself (j = D_mu), and Q.  Returns (R entry, Q entry).  A family
// is sum_w (delta_w(nu) - delta_v(nu)) U_w with U_w = sigma_v(w) sum_tl
// tau_l (sf Re a - sd Im a), built by k_shared_closed (see there) as raw
// values RU, prefix sums PU (PU[k] = sum_{w<k}) and suffix sums SU (SU[k] =
// sum_{w>=k}).  The coefficient delta_w(nu) - delta_v(nu) is c_nu times an
// integer that is constant on w < nu, w = nu and w > nu and vanishes on one
// of these ranges, so the family is formed from the two ranges whose terms
// enter Eq. (09), never as a total minus terms that do not (those would
// cancel only up to rounding, relative to their own size):
//   v < nu:  -c_nu ((nu + 1) U_nu + SU[nu + 1])
//   v = nu:   c_nu ((nu + 1) PU[nu] + nu SU[nu + 1])      (U_v = 0)
//   v > nu:   c_nu (PU[nu] - nu U_nu)
__device__ __forceinline__ void dp_entry_closed(const BasisView& B, const PairStage& S, const double* PU,
                                                const double* RU, const double* SU, const double* h, int p,
                                                int q, int nu, int tn, double& r, double& qout) {
  const int N = B.N;
  const int64_t P = B.P;
  const int L = S.L;
  const double cnu = ld_c(B, nu), fnu = (double)nu;
  double acc2 = 0.0;
#pragma unroll
  for (int tr = 0; tr < 2; ++tr) {
    const int o = (tr * 2 + tn) * L;
    const int v = tr ? q : p;
    double fam;
    if (v < nu) fam = -((fnu + 1.0) * RU[o + nu] + SU[o + nu + 1]);
    else if (v == nu) fam = (fnu + 1.0) * PU[o + nu] + fnu * SU[o + nu + 1];
    else fam = PU[o + nu] - fnu * RU[o + nu];
    acc2 = fma(cnu, fam, acc2);
  }
  double acc = acc2 * kInvSqrt2;
  qout = 0.0;
  const int lo_n = imax(p, 1);
  if (nu >= lo_n && nu <= q) {
    const double gn = dlt(B, p, nu) - dlt(B, q, nu);
    for (int tl = 0; tl < 2; ++tl) {
      const double fk = tl == kS ? -gn : gn;  // f(partner(l), l, D_nu), l on e(n)
      const int tkb = 1 - tl;
      double t;
      if (tl == tn) t = -S.dy(tkb, p, q, 1.0);
      else t = (tn == kS ? -1.0 : 1.0) * S.dx(tkb, p, q, -1.0);
      acc = fma(fk, t, acc);
    }
    if (h != nullptr) qout = __ldg(h + (int64_t)(1 - tn) * P + pair_index(N, p, q)) * (tn == kS ? -gn : gn);
  }
  r = -0.5 * acc;
}

// One block per unordered vertex pair {p < q}: the l-pair part of every
// pair x pair entry on edges (v, p), (v, q) in both orientations, and the
// diagonal x pair entries of the edge (p, q).
__global__ void __launch_bounds__(256, 3) k_shared_closed(BasisView B, AView A, const double* __restrict__ h,
                                                       double* __restrict__ Aout, double* __restrict__ Qout,
                                                       double* __restrict__ Rout) {
  extern __shared__ double sc[];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int32_t ab = __ldg(B.pair_ab + blockIdx.x);
  const int p = ab >> 16, q = ab & 0xffff;
  const int L = N + 1;
  double* PX = sc;
  double* PY = sc + 4 * L;
  double* TX = sc + 8 * L;
  double* TY = sc + 10 * L;
  double* CX = sc + 12 * L;
  double* CY = sc + 14 * L;
  double* PU = sc + 16 * L;  // [4][L]: prefix over w of U for (tr, tn)
  double* DXs = sc + 20 * L;  // [2][L]
  double* DYs = sc + 22 * L;  // [2][L]
  double* RU = sc + 24 * L;   // [4][L]: U at w (raw)
  double* SU = sc + 28 * L;   // [4][L]: suffix over w of U
  __shared__ double TOTs[32];
  const int64_t ppq = blockIdx.x;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) {
    const int w = t >> 2, jk = t & 3, tj = jk >> 1, tk = jk & 1;
    double2 val = make_double2(0.0, 0.0);
    if (w != p && w != q) val = ldA(A, tj * P + pair_index_any(N, q, w), tk * P + pair_index_any(N, p, w));
    PX[jk * L + w] = val.x;
    PY[jk * L + w] = val.y;
  }
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int mu = t >> 1, tt = t & 1;
    const double2 val = mu >= 1 ? ldA(A, d_index(B, mu), tt * P + ppq) : make_double2(0.0, 0.0);
    TX[tt * L + mu] = val.x;
    TY[tt * L + mu] = val.y;
    CX[tt * L + mu] = mu >= 1 ? ld_c(B, mu) * val.x : 0.0;
    CY[tt * L + mu] = mu >= 1 ? ld_c(B, mu) * val.y : 0.0;
  }
  __syncthreads();
  {
    // warps 0..3: suffix sums of CX[0], CX[1], CY[0], CY[1] into the (not
    // yet used) SU arrays: sums of the terms mu > k only, never a total
    // minus the terms below k
    const int wi = threadIdx.x >> 5;
    if (wi < 4) warp_suffix(wi < 2 ? CX + wi * L : CY + (wi - 2) * L, SU + wi * L, N);
  }
  __syncthreads();
  // (D x)_k for the four staged D-column vectors: sum_{mu > k} c_mu x_mu + delta_k(k) x_k
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) {
    const int arr = t / N, k = t % N, tt = arr & 1;
    const double* X = (arr < 2 ? TX : TY) + tt * L;
    double d = SU[arr * L + k + 1];  // mu from k + 1 to N - 1
    if (k >= 1) d += dlt(B, k, k) * X[k];
    (arr < 2 ? DXs : DYs)[tt * L + k] = d;
  }
  // (A1) totals: for (tr, ts, tn, tl), sum over w of sigma(w) X with
  // sigma(w) = (-1)^([P_ < w] tk + [Q_ < w] tj), f (Re, tj = tjf) and d (Im,
  // tj = tjd).  sigma is constant on the three vertex ranges w < p,
  // p < w < q and w > q (the staged values at p and q are zero), so each
  // total is a signed sum of three range sums of one staged array: 8 arrays
  // (PX and PY of the four (tj, tk)) x 3 ranges, 8 threads per range sum.
  __shared__ double RS[8][3];
  if (threadIdx.x < 24 * 8) {
    const int c = threadIdx.x >> 3, sub = threadIdx.x & 7;
    const int arr = c / 3, rg = c % 3;
    const double* X = (arr < 4 ? PX : PY) + (arr & 3) * L;
    const int lo = rg == 0 ? 0 : (rg == 1 ? p + 1 : q + 1), hi = rg == 0 ? p : (rg == 1 ? q : N);
    double acc = 0.0;
    for (int w = lo + sub; w < hi; w += 8) acc += X[w];
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, 8);
    if (sub == 0) RS[arr][rg] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int c = threadIdx.x;
    const int tr = c >> 4, ts = (c >> 3) & 1, tn = (c >> 2) & 1, tl = (c >> 1) & 1, fd = c & 1;
    const int tk = 1 ^ tl ^ ts, tj = fd ? (tl ^ tn) : (1 ^ tl ^ tn);
    // the staged array of sre / sim(tr, tj, tk, .), and sim's sign for tr = 1
    const int arr = (fd ? 4 : 0) + (tr ? tk * 2 + tj : tj * 2 + tk);
    // sigma on p < w < q: [P_ < w] = [P_ == p]; on w > q both flags are set
    const int s1 = (tr ? tj : tk) ? -1 : 1, s2 = (tk ^ tj) ? -1 : 1;
    const double t = RS[arr][0] + sgn_mul(s1, RS[arr][1]) + sgn_mul(s2, RS[arr][2]);
    TOTs[c] = (fd && tr) ? -t : t;
  }
  __syncthreads();
  const PairStage S{PX, PY, TX, TY, CX, CY, DXs, DYs, TOTs, L};
  // block constants of the shared-vertex entries: (tr, ts, tn, [P_ < v], [Q_ < v])
  __shared__ double CST[32];
  if (threadIdx.x < 32) {
    const int c = threadIdx.x, tr = c >> 4, ts = (c >> 3) & 1, tn = (c >> 2) & 1, pv = (c >> 1) & 1, qv = c & 1;
    CST[c] = shared_entry_const(S, tr, tr ? q : p, tr ? p : q, pv, qv, ts, tn);
  }
  // diagonal x pair families: for orientation tr (v = p or q, v' the other)
  // and column type tn, U_w = sigma_v(w) sum_tl tau_l (sf X_re - sd X_im) at
  // the single w, with X the staged a[(v',w) tj][(v,w) tk] (k = partner(l)),
  // tau_l = -1 for l of type S and sigma_v(w) = [w < v] - [w > v]; the entry's
  // sum over w is d_nu^T U - delta_v(nu) sum_w U_w.
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) {
    const int tr = t / (2 * N), tn = (t / N) & 1, w = t % N;
    double u = 0.0;
    if (w != p && w != q) {
      const int v = tr ? q : p, vp = tr ? p : q;
#pragma unroll
      for (int tl = 0; tl < 2; ++tl) {
        const int tjf = 1 ^ tl ^ tn, tjd = tl ^ tn, tkb = 1 - tl;
        const int phl = coef_phase(tl, w, v);
        const int phn = coef_phase(tn, v, vp);
        const int sf = sgn_f(phn + coef_phase(tjf, vp, w) + phl);
        const int sd = sgn_d(phn + coef_phase(tjd, vp, w) + phl);
        const double tv = sgn_mul(sf, S.sre(tr, tjf, tkb, w)) - sgn_mul(sd, S.sim(tr, tjd, tkb, w));
        u += tl == kS ? -tv : tv;
      }
      if (w > v) u = -u;
    }
    PU[(tr * 2 + tn) * L + w + 1] = u;
    RU[(tr * 2 + tn) * L + w] = u;
  }
  if (threadIdx.x < 4) PU[threadIdx.x * L] = 0.0;
  __syncthreads();
  {
    const int wi = threadIdx.x >> 5;  // warps 0..3: prefix of U, 4..7: suffix
    if (wi < 4)
      warp_prefix(PU + wi * L, N);
    else if (wi < 8)
      warp_suffix(RU + (wi - 4) * L, SU + (wi - 4) * L, N);
  }
  __syncthreads();
  // pair x pair, edges sharing a vertex: 2 orientations x N vertices v, the
  // four type pairs of one (orientation, v) from the four a values
  // X[tj][tk] = a[(tj, (v, P_))][(tk, (v, Q_))], written whole: the l-pair
  // part above, the D-section part (completeness form, -1/2 sgs (sgn cf
  // Re a_{partner(n) partner(s)} - cd Im a_{n partner(s)}) with cf, cd = +-1
  // from the position of v) and Q = h_m f_{m n s} on the triangle (P_, Q_, v)
  // with m the edge (P_, Q_) of type 1 ^ ts ^ tn.
  {
    const double hq[2] = {h ? __ldg(h + ppq) * kInvSqrt2 : 0.0, h ? __ldg(h + P + ppq) * kInvSqrt2 : 0.0};
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int tr = t / N, v = t % N;
      if (v == p || v == q) continue;
      const int P_ = tr ? q : p, Q_ = tr ? p : q;
      const int64_t pvp = pair_index_any(N, v, P_), pvq = pair_index_any(N, v, Q_);
      double2 X[2][2];
#pragma unroll
      for (int tj = 0; tj < 2; ++tj)
#pragma unroll
        for (int tk = 0; tk < 2; ++tk) X[tj][tk] = ldA(A, tj * P + pvp, tk * P + pvq);
      const int cf = ((v < P_) == (v < Q_)) ? 1 : -1, cd = v < P_ ? 1 : -1;
#pragma unroll
      for (int combo = 0; combo < 4; ++combo) {
        const int ts = combo >> 1, tn = combo & 1;
        const int sgs = ts == kS ? 1 : -1, sgn = tn == kS ? 1 : -1;
        // a_{partner(n) partner(s)} = conj(X[1-ts][1-tn]), a_{n partner(s)} = conj(X[1-ts][tn])
        double tt[10], accD;
        shared_entry_var(X, S, tr, P_, Q_, v, ts, tn, tt, accD);
        tt[8] = sgn_mul(sgs * sgn * cf, X[1 - ts][1 - tn].x);
        tt[9] = sgn_mul(sgs * cd, X[1 - ts][tn].y);
        const int ci = (((tr * 2 + ts) * 2 + tn) * 2 + (P_ < v ? 1 : 0)) * 2 + (Q_ < v ? 1 : 0);
        // -acc2/4 - am/2 = -(acc2 + 2 am)/4 in fixed point; FP64 for the rare
        // values outside its range
        double q1;
        if (!fx_quarter_sum10(tt, &q1)) {
          double acc2 = tt[0];
#pragma unroll
          for (int i = 1; i < 8; ++i) acc2 += tt[i];
          q1 = fma(-0.25, acc2, neg_half(tt[8] + tt[9]));
        }
        const double r = fma(kNegHalfInvSqrt2, accD, CST[ci] + q1);
        const int tm = 1 ^ tn ^ ts;
        const int ph = coef_phase(ts, v, P_) + coef_phase(tm, P_, Q_) + coef_phase(tn, Q_, v);
        const double qv = (ph & 1) ? sgn_mul(sgn_f(ph), hq[tm]) : 0.0;
        const int64_t o = (ts * P + pvp) * M + (tn * P + pvq);
        if (Rout) Rout[o] = r;
        if (Qout) Qout[o] = qv;
        if (Aout) Aout[o] = qv + r;
      }
    }
  }
  // diagonal x pair
  for (int t = threadIdx.x; t < 2 * (N - 1); t += blockDim.x) {
    const int nu = 1 + (t >> 1), tn = t & 1;
    double r, qv;
    dp_entry_closed(B, S, PU, RU, SU, h, p, q, nu, tn, r, qv);
    const int64_t o = d_index(B, nu) * M + (tn * P + ppq);
    if (Rout) Rout[o] = r;
    if (Qout) Qout[o] = qv;
    if (Aout) Aout[o] = qv + r;
  }
}

// Closed-form k_pd (pair row s, diagonal columns D_nu) and, when K is
// given, K_s.  Per row, with gs(x) = delta_as(x) - delta_bs(x), which is c_x
// for as < x < bs, lc_as at x = as >= 1 and (1 + bs) c_bs at x = bs:
//   YY[x] = Im a[partner(s)][D_x]; PCA, the prefix of c_x YY[x] over
//     x > as (zero up to as), and SCY, the suffix of c_x YY[x]: the sums of
//     gs(x) YY[x] over x are PCA values plus the two ends, and every sum
//     takes only the entry's own terms (a difference of two prefixes would
//     cancel other terms, with their rounding);
//   the sum of 2 gs(x) c_x over x from max(lo_s, nu + 1) to bs is 2/(nu + 1)
//     for as <= nu < bs and 0 otherwise (sum_{x=l}^{m} c_x^2 = 1/l - 1/(m + 1),
//     lc_as c_as = -1/(as + 1), (1 + bs) c_bs^2 = 1/bs);
//   U1S[w] = the sum over the two vertices v of e(s) of U1(v)_w, raw and as
//     a prefix over w; the totals U2(v) = sum_w U2(v)_w (see below);
//   c1 = sum gs(mu) Re a[s][D_mu];  LY = sum of sk Im a(l, k) over the
//     triangle terms (K's triangle part).
// K_s = -(1/N) sum_jk Im(a_jk) f_jks: the triangle terms have
// f(l, k, s) = -sk/sqrt2, and j = partner(s), k = D_l together with
// j = D_l, k = partner(s) give 2 sgs sum_l gs(l) YY[l].
constexpr int kPdRed = 4;  // block totals: U2(as), U2(bs), c1, LY

__global__ void __launch_bounds__(kRowThreads) k_pd_closed(BasisView B, AView A, const double* __restrict__ h,
                                                           double* __restrict__ Aout, double* __restrict__ Qout,
                                                           double* __restrict__ Rout, double* __restrict__ K) {
  extern __shared__ double sq[];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t s = blockIdx.x;
  const Elem es = decode(B, s);
  const int as = es.a, bs = es.b, ts = es.kind;
  const int64_t sb = partner(B, s);
  const int lo_s = imax(as, 1);
  const int L = N + 1;
  double* YY = sq;            // Im a[partner(s)][D_x]   (raw, index x)
  double* PCA = sq + L;       // prefix of c_x YY[x] over x > as
  double* PU1 = sq + 2 * L;   // prefix over w of U1S
  double* RU1 = sq + 3 * L;   // U1S at w (raw)
  double* CY = sq + 4 * L;    // c_x YY[x] (raw)
  double* SCY = sq + 5 * L;   // suffix of c_x YY[x]: SCY[k] = sum_{x >= k}
  __shared__ double red[kPdRed][kRowThreads];
  __shared__ double cst[kPdRed + 1];  // totals, then sum_{x in [lo_s, bs]} gs(x) YY[x]
  // l = (v, w) sharing the vertex v with e(s): with bx = Re a(partner(l), k),
  // ly = Im a(l, k), sk the sign of f(k, l, s), sigma = [w < v] - [w > v] and
  // tau = -1 for l of type S, the family contributes
  //   sum_w sk (tau sigma (delta_w(nu) - delta_v(nu)) bx - (delta_v(nu) + delta_w(nu)) ly)
  //   = d_nu^T U1 + delta_v(nu) U2,  U1_w = sk (tau sigma bx - ly),  U2 = sum_w sk (-tau sigma bx - ly),
  // and d_nu^T U1 = c_nu sum_{w<nu} U1_w + delta_nu(nu) U1_nu (a prefix over w).
  // The two tl of one (v, w) enter every entry with the same coefficients,
  // and so do the two v for U1, so they are summed here.
  double t_u2a = 0.0, t_u2b = 0.0, t_c1 = 0.0, t_ly = 0.0;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const double y = x >= 1 ? ldA(A, sb, d_index(B, x)).y : 0.0;
    YY[x] = y;
    const double cy = x >= 1 ? ld_c(B, x) * y : 0.0;
    CY[x] = cy;
    PCA[x + 1] = x > as ? cy : 0.0;
    if (x >= lo_s && x <= bs) t_c1 = fma(dlt(B, as, x) - dlt(B, bs, x), ldA(A, s, d_index(B, x)).x, t_c1);
    double u1s = 0.0, u1v[2];
    if (x != as && x != bs) {
      const int w = x;
#pragma unroll
      for (int vi = 0; vi < 2; ++vi) {
        const int v = vi ? bs : as, vp = vi ? as : bs;
        const int64_t pl = pair_index_any(N, v, w), pk = pair_index_any(N, vp, w);
        double lyv[2], bxv[2];
#pragma unroll
        for (int tl = 0; tl < 2; ++tl) {
          const int64_t k = (int64_t)(1 ^ tl ^ ts) * P + pk;
          const int tk = 1 ^ tl ^ ts;
          const int sk = sgn_f(coef_phase(ts, v, vp) + coef_phase(tk, vp, w) + coef_phase(tl, w, v));
          const int st = ((tl == kS) != (w < v)) ? sk : -sk;  // sk tau sigma
          lyv[tl] = sgn_mul(sk, ldA(A, (int64_t)tl * P + pl, k).y);
          bxv[tl] = sgn_mul(st, ldA(A, (int64_t)(1 - tl) * P + pl, k).x);
        }
        // u1 = Pb - Ly, u2 = -Pb - Ly
        const double pb = bxv[0] + bxv[1], ly = lyv[0] + lyv[1];
        u1v[vi] = pb - ly;
        if (vi) t_u2b -= pb + ly;
        else t_u2a -= pb + ly;
        t_ly += ly;
      }
      u1s = u1v[0] + u1v[1];
    }
    PU1[x + 1] = u1s;
    RU1[x] = u1s;
  }
  red[0][threadIdx.x] = t_u2a;
  red[1][threadIdx.x] = t_u2b;
  red[2][threadIdx.x] = t_c1;
  red[3][threadIdx.x] = t_ly;
  if (threadIdx.x == 0) PCA[0] = PU1[0] = 0.0;
  __syncthreads();
  // warps 0, 1, 2: the prefix sums PCA and PU1 and the suffix SCY; warp 3:
  // the four block totals
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  static_assert(kRowThreads == 128 && kPdRed == 4, "four warps: three scans, four totals");
  if (wid < 2) {
    warp_prefix(wid == 0 ? PCA : PU1, N);
    if (wid == 0) {
      __syncwarp();
      if (lane == 0) {  // sum_{x in [lo_s, bs]} gs(x) YY[x]: the two ends and the own terms between
        const double tas = as >= 1 ? ld_lc(B, as) * YY[as] : 0.0;
        const double tbs = (ld_c(B, bs) - ld_lc(B, bs)) * YY[bs];
        cst[kPdRed] = (tas + tbs) + PCA[bs];
      }
    }
  } else if (wid == 2) {
    warp_suffix(CY, SCY, N);
  } else {
#pragma unroll
    for (int r = 0; r < kPdRed; ++r) {
      double t = (red[r][lane] + red[r][lane + 32]) + (red[r][lane + 64] + red[r][lane + 96]);
      t = warp_sum(t);
      if (lane == 0) cst[r] = t;
    }
  }
  __syncthreads();
  const double u2a = cst[0], u2b = cst[1], c1 = cst[2], gy = cst[kPdRed];
  const int sgs = ts == kS ? 1 : -1;
  if (K != nullptr && threadIdx.x == 0)
    K[s] = -(fma(cst[3], -kInvSqrt2, twice(sgn_mul(sgs, gy)))) / (double)N;
  // the ends of sum_{x = lo_s}^{min(bs, nu - 1)} gs(x) YY[x]
  const double tas = as >= 1 ? ld_lc(B, as) * YY[as] : 0.0;
  const double tab = tas + (ld_c(B, bs) - ld_lc(B, bs)) * YY[bs];
  // per entry about 18 FP64 instructions: signs and the exact factors 2 and
  // -1/2 are applied to the bits with integer operations
  const double hsb = h != nullptr ? __ldg(h + sb) : 0.0;
  for (int nu = 1 + threadIdx.x; nu < N; nu += blockDim.x) {
    const double cnu = ld_c(B, nu);
    const bool inr = nu >= lo_s && nu <= bs;
    const double gs = inr ? dlt(B, as, nu) - dlt(B, bs, nu) : 0.0;
    // l = D_lam: sum_{lam < nu} gs(lam) YY[lam] and sum_{lam > nu} 2 gs(lam) c_lam
    const int hi = imin(bs - 1, nu - 1);
    double g1 = hi >= as + 1 ? PCA[hi + 1] : 0.0;
    g1 += nu > bs ? tab : (nu > as ? tas : 0.0);
    double accD = twice(cnu) * g1;
    if (nu >= as && nu < bs) accD = fma(YY[nu], twice(__ldg(B.inv + nu + 1)), accD);
    if (inr) {
      double t2 = twice(SCY[nu + 1]);
      if (nu != 1) t2 = fma(twice(cnu + ld_lc(B, nu)), YY[nu], t2);  // 2 (1 - nu) c_nu
      accD = fma(gs, t2, accD);
    }
    double acc = sgn_mul(sgs, accD);
    // l = (v, w) sharing a vertex with e(s): d_nu^T U1 + delta_v(nu) U2 per v
    double accA = cnu * PU1[nu];
    accA = fma(dlt(B, nu, nu), RU1[nu], accA);
    accA = fma(dlt(B, as, nu), u2a, accA);
    accA = fma(dlt(B, bs, nu), u2b, accA);
    acc = fma(accA, kInvSqrt2, acc);
    // l = partner(s), k = D_mu
    {
      const double hnu = (nu >= lo_s && !(as == 0 && bs == 1 && nu == 1)) ? dlt(B, as, nu) + dlt(B, bs, nu) : 0.0;
      acc = fma(-gs, c1, acc);
      acc = fma(hnu, sgn_mul(sgs, gy), acc);
    }
    const double q = inr ? sgn_mul(sgs, hsb * gs) : 0.0;
    const double r = neg_half(acc);
    const int64_t o = s * M + d_index(B, nu);
    if (Rout) Rout[o] = r;
    if (Qout) Qout[o] = q;
    if (Aout) Aout[o] = q + r;
  }
}

// Pair-pair entries on the same edge (a, b): s, n in {S_ab, J_ab}.  One block
// per edge; shared memory: G[mu] = f(D_mu, partner(s), s), Z[nu] = the
// z-fiber of (partner(s), n) at D_nu.
constexpr int kSameThreads = 128;

__global__ void __launch_bounds__(kSameThreads) k_same(BasisView B, AView A, double* __restrict__ Aout,
                                                       double* __restrict__ Rout) {
  extern __shared__ double shd[];  // G[N], Z[N]
  __shared__ double red[kSameThreads / 32];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t e = blockIdx.x;
  const int32_t ab = __ldg(B.pair_ab + e);
  const int a = ab >> 16, b = ab & 0xffff;
  for (int combo = 0; combo < 4; ++combo) {
    const int ts = combo >> 1, tn = combo & 1;
    const bool dfib = ts != tn;  // n = partner(s) = l: d-fiber; n = s: f-fiber of partner(n)
    __syncthreads();  // red[] (and G, Z) of the previous combination have been read
    double* G = shd;
    double* Z = shd + N;
    {
      const int lo = imax(a, 1);
      for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const double g = (t >= lo && t <= b) ? dlt(B, a, t) - dlt(B, b, t) : 0.0;
        G[t] = ts == kS ? -g : g;
        double z = 0.0;
        if (dfib) {
          if (t >= lo && !(a == 0 && b == 1 && t == 1)) z = dlt(B, a, t) + dlt(B, b, t);
        } else if (t >= lo && t <= b) {
          z = dlt(B, a, t) - dlt(B, b, t);
          if (tn == kS) z = -z;
        }
        Z[t] = z;
      }
      __syncthreads();
    }
    double acc2 = 0.0, accD = 0.0;
    // (A) e(l) = (v, w), v in {a, b}, w outside: k and j on (v', w)
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int vi = t / N, w = t % N;
      if (w == a || w == b) continue;
      const int v = vi ? b : a, vp = vi ? a : b;
      const int64_t pw = pair_index_any(N, vp, w);
#pragma unroll
      for (int tl = 0; tl < 2; ++tl) {
        const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int phl = coef_phase(tl, w, v);
        const int sk = sgn_f(coef_phase(ts, v, vp) + coef_phase(tk, vp, w) + phl);
        const int base = coef_phase(tn, v, vp) + phl;
        const int sf = sgn_f(base + coef_phase(tjf, vp, w));
        const int sd = sgn_d(base + coef_phase(tjd, vp, w));
        const double2 a1 = ldA(A, tjf * P + pw, tk * P + pw), a2 = ldA(A, tjd * P + pw, tk * P + pw);
        acc2 += sgn_mul(sk * sf, a1.x);
        acc2 -= sgn_mul(sk * sd, a2.y);
      }
    }
    // (B) l = partner(s): k = D_mu, j = D_nu, i.e. sum_{mu,nu} G_mu Z_nu X[nu][mu] with
    //     G = -+ D^T (e_a - e_b), Z = D^T (e_a + e_b) (d-fibre) or -+ D^T (e_a - e_b),
    //     X = -Im or Re of the D x D block of a: entries of H = D X D^T
    {  // every join term of the D x D block
      const int lo = imax(a, 1), nhi = dfib ? N - 1 : b;
      for (int mu = lo + threadIdx.x; mu <= b; mu += blockDim.x) {
        const int64_t kmu = d_index(B, mu);
        double inner = 0.0;
        for (int nu = lo; nu <= nhi; ++nu) {
          const double2 av = ldA(A, d_index(B, nu), kmu);
          inner = fma(Z[nu], dfib ? -av.y : av.x, inner);
        }
        accD = fma(G[mu], inner, accD);
      }
    }
    double tot = warp_sum(0.5 * acc2 + accD);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int i = 0; i < kSameThreads / 32; ++i) sum += red[i];
      const double r = -0.5 * sum;
      const int64_t o = (ts * P + e) * M + (tn * P + e);
      if (Rout) Rout[o] += r;
      if (Aout) Aout[o] += r;
    }
  }
}

// Same edge (a, b), closed form: the four type pairs (ts, tn) of the block's
// edge at once.  For each (v, w) with w outside the edge the four values
// a[(tj, (v', w))][(tk, (v', w))], tj, tk in {S, J}, are loaded once and
// enter every (ts, tn, tl) term (the per-pair sums keep the order of one pair
// at a time); the l = partner(s) part sums the D x D block over the edge's
// window from the tables of k_dtab.  The block also forms the entries'
// D-section part (by completeness, -+Re a of the partner pair) and Q, and
// writes the four entries whole.
__global__ void __launch_bounds__(kSameThreads) k_same_closed(BasisView B, AView A, const double* __restrict__ h,
                                                              const double* __restrict__ CXr,
                                                              const double* __restrict__ SXi,
                                                              double* __restrict__ Aout, double* __restrict__ Qout,
                                                              double* __restrict__ Rout) {
  __shared__ double red[5][kSameThreads];  // per thread: the four entries' sums, the Q sum
  __shared__ double tot[5];
  const int N = B.N;
  const int64_t P = B.P, M = B.M;
  const int64_t e = blockIdx.x;
  const int32_t ab = __ldg(B.pair_ab + e);
  const int a = ab >> 16, b = ab & 0xffff;
  double acc2[4] = {0.0, 0.0, 0.0, 0.0};  // index ts * 2 + tn
  // (A) e(l) = (v, w), v in {a, b}, w outside: k and j on (v', w)
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int vi = t / N, w = t % N;
    if (w == a || w == b) continue;
    const int v = vi ? b : a, vp = vi ? a : b;
    const int64_t pw = pair_index_any(N, vp, w);
    double2 X[2][2];  // X[tj][tk] = a[(tj, (v', w))][(tk, (v', w))]
#pragma unroll
    for (int tj = 0; tj < 2; ++tj)
#pragma unroll
      for (int tk = 0; tk < 2; ++tk) X[tj][tk] = ldA(A, tj * P + pw, tk * P + pw);
#pragma unroll
    for (int combo = 0; combo < 4; ++combo) {
      const int ts = combo >> 1, tn = combo & 1;
#pragma unroll
      for (int tl = 0; tl < 2; ++tl) {
        const int tk = 1 ^ tl ^ ts, tjf = 1 ^ tl ^ tn, tjd = tl ^ tn;
        const int phl = coef_phase(tl, w, v);
        const int sk = sgn_f(coef_phase(ts, v, vp) + coef_phase(tk, vp, w) + phl);
        const int base = coef_phase(tn, v, vp) + phl;
        const int sf = sgn_f(base + coef_phase(tjf, vp, w));
        const int sd = sgn_d(base + coef_phase(tjd, vp, w));
        acc2[combo] += sgn_mul(sk * sf, X[tjf][tk].x);
        acc2[combo] -= sgn_mul(sk * sd, X[tjd][tk].y);
      }
    }
  }
  // (B) l = partner(s): k = D_mu, j = D_lam, summed over the entry's own
  // terms only.  With g = D^T (e_a - e_b) (support W = [max(a, 1), b]:
  // lc_a at a, c_mu between, c_b - lc_b at b) and h = D^T (e_a + e_b):
  //   f-fibre (ts = tn): sum_{mu in W} g_mu sum_{lam in W} g_lam Re X[lam][mu],
  //   d-fibre (ts != tn): sum_{mu in W} g_mu sum_lam h_lam Im X[lam][mu],
  // the inner d sum from suffix sums over lam > a and lam > b (every term of
  // them enters; h vanishes only at lam = 1 for the edge (0, 1)), the inner
  // f sum term by term over the window (a difference of two longer sums
  // would cancel terms outside it, with their rounding).
  double tf = 0.0, td = 0.0;
  {
    const int lo = imax(a, 1);
    for (int mu = lo + threadIdx.x; mu <= b; mu += blockDim.x) {
      const double gmu = dlt(B, a, mu) - dlt(B, b, mu);
      const double2 xb = ldA(A, d_index(B, b), d_index(B, mu));
      const double2 xa = a >= 1 ? ldA(A, d_index(B, a), d_index(B, mu)) : make_double2(0.0, 0.0);
      double inner = (ld_c(B, b) - ld_lc(B, b)) * xb.x;
      for (int lam = a + 1; lam < b; ++lam) inner += CXr[(int64_t)lam * N + mu];
      if (a >= 1) inner = fma(ld_lc(B, a), xa.x, inner);
      tf = fma(gmu, inner, tf);
      double j;
      if (a == 0 && b == 1) {
        j = twice(SXi[(int64_t)2 * N + mu]);
      } else {
        j = SXi[(int64_t)(a + 1) * N + mu] + SXi[(int64_t)(b + 1) * N + mu];
        j = fma(ld_lc(B, b), xb.y, j);
        if (a >= 1) j = fma(ld_lc(B, a), xa.y, j);
      }
      td = fma(gmu, j, td);
    }
  }
  double accD[4];
#pragma unroll
  for (int combo = 0; combo < 4; ++combo) {
    const int ts = combo >> 1, tn = combo & 1;
    const double sgs = ts == kS ? -1.0 : 1.0;
    accD[combo] = ts != tn ? -sgs * td : sgs * (tn == kS ? -1.0 : 1.0) * tf;
  }
  // Q of the type-changing pairs: sum_lam h_{D_lam} f(D_lam, J_ab, S_ab) over
  // lam in [max(a, 1), b], f = delta_b(lam) - delta_a(lam); the lam < b terms
  // take -h c_lam from delta_a, lam = b takes h_b (lc_b - c_b) and lam = a
  // (a >= 1) -h_a lc_a.  The c_lam sum is split over the block.
  double hc = 0.0;
  if (h != nullptr)
    for (int lam = a + 1 + threadIdx.x; lam <= b; lam += blockDim.x) hc += __ldg(h + d_index(B, lam)) * ld_c(B, lam);
  // block sums: the partial sums go to shared memory and one warp reduces
  // each of the five (fewer FP64 warp instructions than a shuffle
  // reduction per warp and value)
#pragma unroll
  for (int combo = 0; combo < 4; ++combo) red[combo][threadIdx.x] = fma(0.5, acc2[combo], accD[combo]);
  red[4][threadIdx.x] = hc;
  __syncthreads();
  static_assert(kSameThreads == 128, "four warps reduce five sums of 128 values");
  {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = wid; i < 5; i += 4) {
      const double t = warp_sum((red[i][lane] + red[i][lane + 32]) + (red[i][lane + 64] + red[i][lane + 96]));
      if (lane == 0) tot[i] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int combo = threadIdx.x, ts = combo >> 1, tn = combo & 1;
    const double sum = tot[combo], hsum = tot[4];
    // the D-section part (completeness form): -1/2 sgs sgn 2 Re a_{partner(n) partner(s)}
    const double2 a1 = ldA_row(A, (int64_t)(1 - tn) * P + e, (int64_t)(1 - ts) * P + e);
    const double r = sgn_mul((ts == tn) ? -1 : 1, a1.x) + -0.5 * sum;
    double q = 0.0;
    if (h != nullptr && ts != tn) {
      double qsj = __ldg(h + d_index(B, b)) * ld_lc(B, b) - hsum;
      if (a >= 1) qsj -= __ldg(h + d_index(B, a)) * ld_lc(B, a);
      q = ts == kS ? qsj : -qsj;
    }
    const int64_t o = (ts * P + e) * M + (tn * P + e);
    if (Rout) Rout[o] = r;
    if (Qout) Qout[o] = q;
    if (Aout) Aout[o] = q + r;
  }
}

// ---------------------------------------------------------------------------
// Lower triangle of a Hermitian a from its upper triangle: a_kj = conj(a_jk)
// for k > j, through a 32 x 32 tile in shared memory so that both the read of
// the upper tile and the write of the lower tile are row-contiguous.  Block
// (x, y) writes tile row y, tile column x (x <= y) and reads tile (x, y) of
// the upper side, which no block writes.
__global__ void __launch_bounds__(256) k_mirror_lower(double2* __restrict__ a, int64_t M) {
  const int64_t tc = blockIdx.x, tr = blockIdx.y;
  if (tc > tr) return;
  __shared__ double2 t[32][33];
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = tc * 32 + y, c = tr * 32 + threadIdx.x;
    if (r < M && c < M) t[y][threadIdx.x] = a[r * M + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = tr * 32 + y, c = tc * 32 + threadIdx.x;
    if (r < M && c < M && r > c) {
      double2 v = t[threadIdx.x][y];
      v.y = -v.y;
      a[r * M + c] = v;
    }
  }
}

// Upper triangle (columns c >= r of every row r) of a from page-locked host
// memory that is mapped into the device address space, read by the SMs over
// the host link: each block walks whole rows with eight 16-byte loads in
// flight per thread, so that the link, not the latency of one load, sets the
// rate.  Reads stay within the M x M host array.
__global__ void __launch_bounds__(256) k_upload_upper(const double2* __restrict__ host, double2* __restrict__ dev,
                                                      int64_t M) {
  constexpr int kU = 8;
  for (int64_t r = blockIdx.x; r < M; r += gridDim.x) {
    const double2* __restrict__ src = host + r * M;
    double2* __restrict__ dst = dev + r * M;
    for (int64_t c0 = r + threadIdx.x; c0 < M; c0 += 256 * kU) {
      double2 v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t c = c0 + 256 * u;
        if (c < M) v[u] = src[c];
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t c = c0 + 256 * u;
        if (c < M) dst[c] = v[u];
      }
    }
  }
}

}  // namespace

namespace lbi {

cudaError_t upload_hermitian(const double2* host, double2* dev, int64_t M, cudaStream_t st) {
  // Page-locked host memory mapped into the device address space: the SMs
  // read the upper triangle directly (no staging copy), then the mirror.
  cudaPointerAttributes pa;
  const cudaError_t qa = cudaPointerGetAttributes(&pa, host);
  if (qa == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr) {
    int dev_id = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev_id);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>(M, (int64_t)sms * 8);
    k_upload_upper<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const double2*>(pa.devicePointer), dev, M);
    const unsigned nt = (unsigned)((M + 31) / 32);
    k_mirror_lower<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(dev, M);
    note_launch(2);
    return cudaGetLastError();
  }
  if (qa != cudaSuccess) cudaGetLastError();  // the failed query's error is not the caller's
  if (M <= 2048) return cudaMemcpyAsync(dev, host, sizeof(double2) * M * M, cudaMemcpyHostToDevice, st);
  // row block [j0, j1) brings columns [j0, M): the upper triangle and the
  // lower half of the diagonal block
  const int64_t h = std::max<int64_t>(256, (M + 63) / 64);
  cudaError_t e = cudaSuccess;
  for (int64_t j0 = 0; j0 < M && e == cudaSuccess; j0 += h) {
    const int64_t j1 = std::min(M, j0 + h);
    e = cudaMemcpy2DAsync(dev + j0 * M + j0, sizeof(double2) * M, host + j0 * M + j0, sizeof(double2) * M,
                          sizeof(double2) * (M - j0), j1 - j0, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return e;
  const unsigned nt = (unsigned)((M + 31) / 32);
  k_mirror_lower<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(dev, M);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t assemble_dense(const lb::BasisView& B, const double* h, const double2* a, double* A,
                           double* Q, double* R, double* K, int algorithm, cudaStream_t st,
                           cudaEvent_t* ev) {
  AView av{a, B.M};
  const int N = B.N;
  const int64_t P2 = 2 * B.P;
  const int64_t chunks = (P2 + 255) / 256;
  if (P2 * chunks > 0x7fffffffLL || N > kMaxDenseN) return cudaErrorInvalidConfiguration;
  const bool closed = algorithm == LB_ALG_CLOSED;
  cudaError_t e = cudaSuccess;
  // ev (optional, kAssembleKernels + 1 events): recorded before the first and
  // after every kernel of the sequence below, launched or not.
  auto mark = [&](int i) {
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[i], st);
  };
  mark(0);
  const bool dense_out = A || Q || R;
  // 0: pair x pair (closed: disjoint edges, one lane per vertex quadruple in warp tiles)
  if (dense_out) {
    if (closed) {
      if (N >= 4) {
        k_disjoint4<<<(unsigned)B.P, kQuadThreads, 0, st>>>(B, av, A, Q, R);
        note_launch(1);
      }
    } else {
      k_entries<LB_ALG_JOIN><<<(unsigned)(P2 * chunks), 256, 0, st>>>(B, av, h, A, Q, R);
      note_launch(1);
    }
  }
  mark(1);
  // 1: pair x diagonal
  if (dense_out && e == cudaSuccess) {
    if (closed) {
      const size_t smem = sizeof(double) * 6 * (size_t)(N + 1);
      e = cudaFuncSetAttribute(k_pd_closed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_pd_closed<<<(unsigned)P2, kRowThreads, smem, st>>>(B, av, h, A, Q, R, K);
    } else {
      const size_t smem = sizeof(double2) * 10 * (size_t)N;
      e = cudaFuncSetAttribute(k_pd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_pd<<<(unsigned)P2, kRowThreads, smem, st>>>(B, av, h, A, Q, R);
    }
    note_launch(1);
  }
  mark(2);
  // 2: diagonal x pair (closed: produced by k_shared_closed below)
  if (dense_out && !closed && e == cudaSuccess) {
    k_dp<<<(unsigned)((N - 1) * chunks), 256, 0, st>>>(B, av, h, A, Q, R);
    note_launch(1);
  }
  mark(3);
  // closed: stream-ordered scratch for the D x D tables (same edge), the vertex sums of K's
  // diagonal rows and the diagonal x diagonal tables
  double* scratch = nullptr;
  const size_t dd_at = 3 * (size_t)N * N + N;
  if (closed && e == cudaSuccess && (dense_out || K))
    e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(double) * (dd_at + DDTables::doubles(N)), st);
  // 3: diagonal x diagonal (closed: cells of constant coefficient from row,
  //    column and corner sums)
  if (dense_out && e == cudaSuccess && N >= 2) {
    if (closed) {
      const DDTables T = DDTables::carve(scratch + dd_at, N);
      const int cols = 2 * N + 2 * (N + 1);
      const int64_t ents = (int64_t)(N - 1) * (N - 1);
      k_dd_rows<<<(unsigned)N, 128, 0, st>>>(B, av, T);
      k_dd_cols<<<(unsigned)((cols + 127) / 128), 128, 0, st>>>(B, T);
      k_dd_cells<<<(unsigned)((ents + 255) / 256), 256, 0, st>>>(B, T, A, Q, R);
      note_launch(3);
    } else {
      const int64_t dd_warps = (int64_t)(N - 1) * (N - 1);
      k_dd<<<(unsigned)((dd_warps * 32 + 255) / 256), 256, 0, st>>>(B, av, A, Q, R);
      note_launch(1);
    }
  }
  mark(4);
  // 4: pair x pair on edges sharing one vertex (join: adds to R / A);
  //    closed: one block per vertex pair writes these entries whole (the
  //    D-section and Q parts too) and the diagonal x pair entries
  if (dense_out && closed && e == cudaSuccess) {
    const size_t smem = sizeof(double) * 32 * (size_t)(N + 1);
    e = cudaFuncSetAttribute(k_shared_closed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_shared_closed<<<(unsigned)B.P, 256, smem, st>>>(B, av, h, A, Q, R);
    note_launch(1);
  } else if ((A || R) && N >= 3 && e == cudaSuccess) {
    const size_t smem = sizeof(double2) * 6 * (size_t)N;
    e = cudaFuncSetAttribute(k_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_shared<<<(unsigned)(N * (N - 1)), 256, smem, st>>>(B, av, A, R);
    note_launch(1);
  }
  mark(5);
  // 5: pair x pair on the same edge (closed: written whole, Q included; join:
  //    adds to R / A); its D-section sums come from H = D X D^T of the D x D
  //    block of a (stream-ordered scratch)
  if ((closed ? dense_out : (A || R)) && e == cudaSuccess) {
    if (closed) {
      double* CXr = scratch;                     // N x N
      double* SXi = scratch + (size_t)N * N;     // (N + 1) x N
      if (N >= 2) {
        k_dtab<<<(unsigned)(N - 1), 128, 0, st>>>(B, av, CXr, SXi);
        note_launch(1);
      }
      k_same_closed<<<(unsigned)B.P, kSameThreads, 0, st>>>(B, av, h, CXr, SXi, A, Q, R);
      note_launch(1);
    } else {
      k_same<<<(unsigned)B.P, kSameThreads, sizeof(double) * 2 * N, st>>>(B, av, A, R);
      note_launch(1);
    }
  }
  mark(6);
  // 6: K (closed: the diagonal rows from the vertex sums G in the scratch)
  if (K && e == cudaSuccess) {
    if (closed) {
      // the pair rows of K come from k_pd_closed when it runs
      const int64_t warps = 2 * B.P;
      if (warps > 0 && !dense_out) {
        k_kvec<true><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(B, av, K);
        note_launch(1);
      }
      double* G = scratch + 3 * (size_t)N * N;
      k_kvec_diag_g<<<(unsigned)N, 128, 0, st>>>(B, av, G);
      k_kvec_diag<<<1, 256, 0, st>>>(B, G, K);
      note_launch(2);
    } else {
      const int64_t warps = B.M;
      k_kvec<false><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(B, av, K);
      note_launch(1);
    }
  }
  mark(7);
  if (scratch) {
    const cudaError_t ef = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = ef;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

const char* assemble_kernel_name(int i) {
  static const char* names[kAssembleKernels] = {
      "k_entries (pair x pair; closed: disjoint edges by vertex quadruple)", "k_pd (pair x diagonal)",
      "k_dp (diagonal x pair)", "k_dd (diagonal x diagonal)",
      "k_shared (edges sharing a vertex; closed: whole entries, + diagonal x pair)",
      "k_same (same edge; closed: whole entries)", "k_kvec (K)"};
  return (i >= 0 && i < kAssembleKernels) ? names[i] : nullptr;
}

cudaError_t join_terms(const lb::BasisView& B, unsigned long long* d_count, cudaStream_t st) {
  AView av{nullptr, B.M};
  const int64_t chunks = (B.M + 255) / 256;
  const int64_t blocks = chunks * B.M;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_assemble<true><<<(unsigned)blocks, 256, 0, st>>>(B, av, nullptr, nullptr, nullptr, nullptr, d_count);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace lbi

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
// No atomics: every entry is written once, rows of R contiguous per warp.
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
__global__ void k_kvec(BasisView B, AView A, double* __restrict__ K) {
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= B.M) return;
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

}  // namespace

namespace lbi {

cudaError_t assemble_dense(const lb::BasisView& B, const double* h, const double2* a, double* A,
                           double* Q, double* R, double* K, cudaStream_t st) {
  AView av{a, B.M};
  const int64_t chunks = (B.M + 255) / 256;
  const int64_t blocks = chunks * B.M;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (A || Q || R) {
    k_assemble<false><<<(unsigned)blocks, 256, 0, st>>>(B, av, h, A, Q, R, nullptr);
    note_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (K) {
    const int64_t warps = B.M;
    k_kvec<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(B, av, K);
    note_launch(1);
  }
  return cudaGetLastError();
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

// lb_csr.cu -- sparse (CSR) assembly of A = Q + R and K for a Kossakowski
// matrix in spectral form a_jk = sum_p gamma_p l_pj conj(l_pk) with sparse
// l_p and a sparse Hamiltonian (Eqs. (07)-(09); Sec. 3's sparse model class,
// P = 1 jump operator), and the fused RK4 step on CSR (Sec. 4 item 3).
//
// Eq. (09) factorises per channel:
//   r_sn = -1/2 gamma_p Re sum_l W_ls U_ln,
//   U_ln = sum_j l_j z_jln,   W_ls = sum_k conj(l_k) f_kls,
// so R is a sparse product.  Every step is a count / scan / fill pass of this
// file's own kernels (no library sort):
//   1. the fibres of the nonzero l_j and l_k emit the U terms into buckets by
//      row l and the W terms into buckets by column s, each term tagged with
//      its channel; the Q terms h_m f_mns go into buckets by row s.  A bucket
//      is filled through a per-bucket cursor after an exclusive scan of the
//      counts (terms of one bucket keep no particular order);
//   2. one warp per row s (one block for long rows) accumulates the row in a
//      hash table keyed by column n: every W term (p, l) of column s times
//      every U term of row l with the same channel, and the row's Q terms;
//      the value and the sum of the magnitudes of its terms are summed per
//      column.  An entry is kept when its value exceeds 1e-12 times that
//      magnitude (entries whose terms cancel exactly -- most of those the
//      terms reach -- carry only rounding residue).  A first pass counts the
//      kept entries of each row, a scan gives the row pointers, a second pass
//      writes the columns in ascending order with their values.
// Duplicate terms (the same (l, n) from several j) are summed in the order
// the fill placed them, so values are reproducible to rounding only.
#include "lb_internal.h"

namespace {

using namespace lb;

// The fibres of a pair element, cut into 2N - 1 slices so that one thread
// takes one slice: slice t < N holds the entries whose third vertex is
// w = t (none for w on the element's edge), slice t >= N the entries with
// D_lam, lam = t - N + 1: fiber_slices(N) slices per element.
__host__ __device__ inline int fiber_slices(int N) { return 2 * N - 1; }

// Slice t of the f-fibre of the pair element k: every (l, s) with
// f_{k l s} != 0, with the value.
template <class Emit>
__device__ void f_fiber_slice(const BasisView& B, int64_t k, int t, Emit& emit) {
  const int N = B.N;
  const Elem ek = decode(B, k);
  const int a = ek.a, b = ek.b, tk = ek.kind;
  if (t < N) {
    const int w = t;
    if (w == a || w == b) return;
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi ? b : a, vp = vi ? a : b;
      for (int tl = kS; tl <= kJ; ++tl) {
        const Elem el = make_pair(tl, v, w), es = make_pair(1 ^ tk ^ tl, vp, w);
        emit(elem_index(B, tl, v, w), elem_index(B, es.kind, vp, w), f_value(B, ek, el, es));
      }
    }
  } else {
    const int lam = t - N + 1;
    if (lam < imax(a, 1) || lam > b) return;
    const Elem ekb = make_pair(1 - tk, a, b);
    const int64_t kb = partner(B, k);
    emit(kb, d_index(B, lam), f_value(B, ek, ekb, make_d(lam)));
    emit(d_index(B, lam), kb, f_value(B, ek, make_d(lam), ekb));
  }
}

// Slice t of the z-fibre of the pair element j: every (l, n) with
// z_{j l n} != 0, with z = f + i d.
template <class Emit>
__device__ void z_fiber_slice(const BasisView& B, int64_t j, int t, Emit& emit) {
  const int N = B.N;
  const Elem ej = decode(B, j);
  const int a = ej.a, b = ej.b, tj = ej.kind;
  double f, d;
  if (t < N) {
    const int w = t;
    if (w == a || w == b) return;
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi ? b : a, vp = vi ? a : b;
      for (int tl = kS; tl <= kJ; ++tl) {
        const Elem el = make_pair(tl, v, w);
        const int64_t l = elem_index(B, tl, v, w);
        const Elem enf = make_pair(1 ^ tj ^ tl, vp, w), end = make_pair(tj ^ tl, vp, w);
        fd_value(B, ej, el, enf, f, d);
        emit(l, elem_index(B, enf.kind, vp, w), f, 0.0);
        fd_value(B, ej, el, end, f, d);
        emit(l, elem_index(B, end.kind, vp, w), 0.0, d);
      }
    }
  } else {
    const int lam = t - N + 1;
    if (lam < imax(a, 1)) return;
    const Elem ejb = make_pair(1 - tj, a, b), ed = make_d(lam);
    const int64_t jb = partner(B, j);
    if (lam <= b) {  // f-fibres: (partner(j), D) and (D, partner(j))
      fd_value(B, ej, ejb, ed, f, d);
      emit(jb, d_index(B, lam), f, 0.0);
      fd_value(B, ej, ed, ejb, f, d);
      emit(d_index(B, lam), jb, f, 0.0);
    }
    if (!(a == 0 && b == 1 && lam == 1)) {  // d-fibres: (j, D) and (D, j)
      fd_value(B, ej, ej, ed, f, d);
      emit(j, d_index(B, lam), 0.0, d);
      fd_value(B, ej, ed, ej, f, d);
      emit(d_index(B, lam), j, 0.0, d);
    }
  }
}

// Channel of a flattened nonzero index u (lp_ptr has nP + 1 entries).
__device__ __forceinline__ int channel_of(const int64_t* lp_ptr, int nP, int64_t u) {
  int p = 0;
  while (p + 1 < nP && lp_ptr[p + 1] <= u) ++p;
  return p;
}

// A bucketed term: channel p (-1 for Q), index x (l of a W term, n of a U or
// Q term), value (re, im) and the magnitude of its terms.
struct BTerm {
  int32_t p, x;
  double re, im, mag;
};

// Count mode (out == nullptr): one more term in bucket b.  Fill mode: the
// term goes to off[b] + (the bucket's cursor, advanced atomically).
struct Bucketer {
  unsigned long long* cnt;  // count, then cursor (reset to 0 between the passes)
  const int64_t* off;
  BTerm* out;
  __device__ __forceinline__ void put(int64_t b, int p, int64_t x, double re, double im, double mag) const {
    const unsigned long long k = atomicAdd(cnt + b, 1ull);
    if (out) out[off[b] + (int64_t)k] = BTerm{p, (int32_t)x, re, im, mag};
  }
};

// W terms into buckets by column s: (p, l, conj(l_k) f_kls, |l_k f|); one
// thread per (nonzero u of a pair element, fibre slice).
__global__ void k_w_bucket(BasisView B, int nP, const int64_t* lp_ptr, const int64_t* lp_idx, const double2* lp_val,
                           int64_t nu, Bucketer bk) {
  const int S = fiber_slices(B.N);
  const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= nu * S) return;
  const int64_t u = it / S;
  const int64_t k = lp_idx[u];
  if (k >= 2 * B.P) return;  // diagonal components: k_dpart_bucket
  const int p = channel_of(lp_ptr, nP, u);
  const double2 lk = lp_val[u];
  const double am = sqrt(lk.x * lk.x + lk.y * lk.y);
  auto emit = [&](int64_t l, int64_t s, double f) { bk.put(s, p, l, lk.x * f, -lk.y * f, am * fabs(f)); };
  f_fiber_slice(B, k, (int)(it % S), emit);
}

// U terms into buckets by row l: (p, n, l_j z_jln, |l_j z|); one thread per
// (nonzero u of a pair element, fibre slice).
__global__ void k_u_bucket(BasisView B, int nP, const int64_t* lp_ptr, const int64_t* lp_idx, const double2* lp_val,
                           int64_t nu, Bucketer bk) {
  const int S = fiber_slices(B.N);
  const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= nu * S) return;
  const int64_t u = it / S;
  const int64_t j = lp_idx[u];
  if (j >= 2 * B.P) return;  // diagonal components: k_dpart_bucket, k_udd_bucket
  const int p = channel_of(lp_ptr, nP, u);
  const double2 lj = lp_val[u];
  const double am = sqrt(lj.x * lj.x + lj.y * lj.y);
  auto emit = [&](int64_t l, int64_t n, double zr, double zi) {
    bk.put(l, p, n, lj.x * zr - lj.y * zi, lj.x * zi + lj.y * zr, am * sqrt(zr * zr + zi * zi));
  };
  z_fiber_slice(B, j, (int)(it % S), emit);
}

// The pair indices m < 2P with h_m != 0, in any order: list, *count.
__global__ void k_h_nonzero(int64_t P2, const double* h, int64_t* list, unsigned long long* count) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m < P2 && h[m] != 0.0) list[atomicAdd(count, 1ull)] = m;
}

// Q terms of the nonzero pair coefficients h_m into buckets by row s:
// f_{m n s} for (n, s) on the fibre of m; one thread per (m, fibre slice).
__global__ void k_q_pair_bucket(BasisView B, const double* h, const int64_t* hlist, int64_t nh, Bucketer bk) {
  const int S = fiber_slices(B.N);
  const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= nh * S) return;
  const int64_t m = hlist[it / S];
  const double hm = h[m];
  auto emit = [&](int64_t n, int64_t s, double f) { bk.put(s, -1, n, hm * f, 0.0, fabs(hm * f)); };
  f_fiber_slice(B, m, (int)(it % S), emit);
}

// ------------------------------------------------ diagonal components
// The diagonal part of a vector x over the D_nu (nu = 1..N-1) enters the
// products only through edge sums of delta_x(nu) = (D_nu)_xx (c_nu for
// x < nu, -nu c_nu at x = nu, 0 above): with f(D_nu, S_xy, J_xy) =
// delta_x(nu) - delta_y(nu) and d(D_nu, l, l) = delta_x(nu) + delta_y(nu)
// (l on (x, y)), over nu in [max(x, 1), y] resp. nu >= max(x, 1),
//   G_xy = [x >= 1] x_x lc_x + sum_{x < nu < y} x_nu c_nu + x_y (c_y - lc_y),
//   H_xy = [x >= 1] x_x lc_x + sum_{x < nu < y} x_nu c_nu + x_y (c_y + lc_y)
//          + 2 sum_{nu > y} x_nu c_nu,
// and d(D_nu, D_lam, D_mu) = 2 sum_k delta_k(nu) delta_k(lam) delta_k(mu).
// One thread per (source, x) walks y upward keeping the running sum over
// x < nu < y, so every sum holds exactly the terms of its edge; each term
// carries the sum of the magnitudes of its parts.

// Diagonal components of every channel: dl[p N + nu] (complex), hasD[p].
__global__ void k_dscatter(const BasisView B, int nP, const int64_t* lp_ptr, const int64_t* lp_idx,
                           const double2* lp_val, int64_t nu_tot, double2* dl, int* hasD) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nu_tot) return;
  const int64_t k = lp_idx[u];
  if (k < 2 * B.P) return;
  const int p = channel_of(lp_ptr, nP, u);
  const int64_t i = (int64_t)p * B.N + (k - 2 * B.P + 1);
  atomicAdd(&dl[i].x, lp_val[u].x);
  atomicAdd(&dl[i].y, lp_val[u].y);
  hasD[p] = 1;
}

// suf[p N + y] = sum_{nu > y} x_nu c_nu and sufm the same over |x_nu| c_nu.
__global__ void k_dsuffix(const BasisView B, int nP, const double2* dl, const int* hasD, double2* suf, double* sufm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nP || !hasD[p]) return;
  const int N = B.N;
  const double2* x = dl + (int64_t)p * N;
  double2 r = make_double2(0.0, 0.0);
  double rm = 0.0;
  for (int y = N - 1; y >= 0; --y) {
    suf[(int64_t)p * N + y] = r;
    sufm[(int64_t)p * N + y] = rm;
    if (y >= 1) {
      const double c = ld_c(B, y);
      r.x += x[y].x * c;
      r.y += x[y].y * c;
      rm += sqrt(x[y].x * x[y].x + x[y].y * x[y].y) * c;
    }
  }
}

// W and U terms of the diagonal components of channel p on edge (x, y):
//   W(l = S, s = J) = conj(G),  W(l = J, s = S) = -conj(G),
//   U(S, J) = G,  U(J, S) = -G,  U(S, S) = U(J, J) = i H.
// mode 0: W terms, mode 1: U terms.
__global__ void k_dpart_bucket(const BasisView B, int nP, const double2* dl, const int* hasD, const double2* suf,
                               const double* sufm, int mode, Bucketer bk) {
  const int N = B.N;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nP * N) return;
  const int p = (int)(t / N), x = (int)(t % N);
  if (!hasD[p]) return;
  const double2* dx = dl + (int64_t)p * N;
  const double2 head = x >= 1 ? make_double2(dx[x].x * ld_lc(B, x), dx[x].y * ld_lc(B, x)) : make_double2(0.0, 0.0);
  const double headm = x >= 1 ? sqrt(dx[x].x * dx[x].x + dx[x].y * dx[x].y) * fabs(ld_lc(B, x)) : 0.0;
  double2 run = make_double2(0.0, 0.0);
  double runm = 0.0;
  const int64_t P = B.P;
  for (int y = x + 1; y < N; ++y) {
    const double cy = ld_c(B, y), lcy = ld_lc(B, y);
    const double2 xy = dx[y];
    const double ay = sqrt(xy.x * xy.x + xy.y * xy.y);
    const double2 G = make_double2(head.x + run.x + xy.x * (cy - lcy), head.y + run.y + xy.y * (cy - lcy));
    const double Gm = headm + runm + ay * (cy - lcy);
    const int64_t e = pair_index(N, x, y), eS = e, eJ = P + e;
    if (mode == 0) {
      if (Gm > 0.0) {
        bk.put(eJ, p, eS, G.x, -G.y, Gm);
        bk.put(eS, p, eJ, -G.x, G.y, Gm);
      }
    } else {
      const double2 sy = suf[(int64_t)p * N + y];
      const double H_re = head.x + run.x + xy.x * (cy + lcy) + 2.0 * sy.x;
      const double H_im = head.y + run.y + xy.y * (cy + lcy) + 2.0 * sy.y;
      const double Hm = headm + runm + ay * fabs(cy + lcy) + 2.0 * sufm[(int64_t)p * N + y];
      if (Gm > 0.0) {
        bk.put(eS, p, eJ, G.x, G.y, Gm);
        bk.put(eJ, p, eS, -G.x, -G.y, Gm);
      }
      if (Hm > 0.0) {
        bk.put(eS, p, eS, -H_im, H_re, Hm);
        bk.put(eJ, p, eJ, -H_im, H_re, Hm);
      }
    }
    if (y < N - 1) {  // x < nu < y' for the next y' = y + 1
      run.x += xy.x * cy;
      run.y += xy.y * cy;
      runm += ay * cy;
    }
  }
}

// U terms of the diagonal components on the D x D block, row D_lam, column
// D_mu (one thread each): i 2 c_lam x_mu (mu < lam), i 2 c_mu x_lam
// (mu > lam), i (2 sum_{nu > lam} x_nu c_nu + 2 (1 - lam) c_lam x_lam) (mu = lam).
__global__ void k_udd_bucket(const BasisView B, int nP, const double2* dl, const int* hasD, const double2* suf,
                             const double* sufm, Bucketer bk) {
  const int N = B.N, D = N - 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nP * D * D) return;
  const int p = (int)(t / ((int64_t)D * D));
  if (!hasD[p]) return;
  const int lam = 1 + (int)((t / D) % D), mu = 1 + (int)(t % D);
  const double2* x = dl + (int64_t)p * N;
  double re, im, mag;
  if (mu != lam) {
    const double c2 = 2.0 * ld_c(B, mu < lam ? lam : mu);
    const double2 v = x[mu < lam ? mu : lam];
    re = -c2 * v.y;
    im = c2 * v.x;
    mag = c2 * sqrt(v.x * v.x + v.y * v.y);
  } else {
    const double cc = 2.0 * (ld_c(B, lam) + ld_lc(B, lam));  // 2 (1 - lam) c_lam
    const double2 sy = suf[(int64_t)p * N + lam];
    const double sr = 2.0 * sy.x + cc * x[lam].x, si = 2.0 * sy.y + cc * x[lam].y;
    re = -si;
    im = sr;
    mag = 2.0 * sufm[(int64_t)p * N + lam] + fabs(cc) * sqrt(x[lam].x * x[lam].x + x[lam].y * x[lam].y);
  }
  if (mag > 0.0) bk.put(d_index(B, lam), p, d_index(B, mu), re, im, mag);
}

// Q terms of the diagonal coefficients h_{D_lam}: only (S_xy, J_xy) and
// (J_xy, S_xy), q_{S J} = sum_lam h_{D_lam} f(D_lam, J_xy, S_xy) = -G_xy[h]
// and q_{J S} = -q_{S J}.  One warp per x: the lanes take 32 consecutive y
// at a time, and the sums over x < lam < y are a warp prefix scan of
// h_lam c_lam (and of |h_lam| c_lam) over that window plus the window's
// carry, so each holds exactly the terms of its edge.
__global__ void k_q_diag_bucket(BasisView B, const double* h, Bucketer bk) {
  const int N = B.N;
  const int x = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (x >= N) return;
  const double* hd = h + 2 * B.P - 1;  // hd[nu] = h_{D_nu}
  const double head = x >= 1 ? hd[x] * ld_lc(B, x) : 0.0;
  const double headm = x >= 1 ? fabs(hd[x] * ld_lc(B, x)) : 0.0;
  double carry = 0.0, carrym = 0.0;  // sums over x < lam < (the window's first y)
  for (int y0 = x + 1; y0 < N; y0 += 32) {
    const int y = y0 + lane;
    const bool in = y < N;
    const double cy = in ? ld_c(B, y) : 0.0, lcy = in ? ld_lc(B, y) : 0.0, hy = in ? hd[y] : 0.0;
    double t = hy * cy, tm = fabs(hy) * cy;  // the term lam = y, for the larger y
    double it = t, itm = tm;                  // inclusive prefix over the window
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, it, o), um = __shfl_up_sync(0xffffffffu, itm, o);
      if (lane >= o) {
        it += u;
        itm += um;
      }
    }
    double ex = __shfl_up_sync(0xffffffffu, it, 1), exm = __shfl_up_sync(0xffffffffu, itm, 1);
    if (lane == 0) {
      ex = 0.0;
      exm = 0.0;
    }
    const double run = carry + ex, runm = carrym + exm;  // x < lam < y
    if (in) {
      const double G = head + run + hy * (cy - lcy);
      const double Gm = headm + runm + fabs(hy) * (cy - lcy);
      if (Gm > 0.0) {
        const int64_t e = pair_index(N, x, y);
        bk.put(e, -1, B.P + e, -G, 0.0, Gm);
        bk.put(B.P + e, -1, e, G, 0.0, Gm);
      }
    }
    carry += __shfl_sync(0xffffffffu, it, 31);
    carrym += __shfl_sync(0xffffffffu, itm, 31);
  }
}

// K (Eq. (08)): k_s = -(1/N) sum_jk Im(a_jk) f_jks over pairs (j, k) of one
// channel's support, a_jk = gamma l_j conj(l_k).
__global__ void k_k_lowrank(BasisView B, int nP, const int64_t* lp_ptr, const double* gamma,
                            const int64_t* lp_idx, const double2* lp_val, double* K) {
  const int p = blockIdx.y;
  const int64_t base = lp_ptr[p], n = lp_ptr[p + 1] - base;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t u = base + t / n, w = base + t % n;
  const int64_t j = lp_idx[u], k = lp_idx[w];
  const double2 lj = lp_val[u], lk = lp_val[w];
  const double aim = gamma[p] * (lj.y * lk.x - lj.x * lk.y);  // Im(l_j conj(l_k))
  if (aim == 0.0) return;
  const Elem ej = decode(B, j), ek = decode(B, k);
  const double inv = -1.0 / (double)B.N;
  auto add = [&](const Elem& es, int64_t s) {
    const double f = f_value(B, ej, ek, es);
    if (f != 0.0) atomicAdd(K + s, inv * aim * f);
  };
  if (ej.kind != kD && ek.kind != kD) {
    if (ej.a == ek.a && ej.b == ek.b) {
      if (ej.kind != ek.kind)
        for (int lam = imax(ej.a, 1); lam <= ej.b; ++lam) add(make_d(lam), d_index(B, lam));
    } else {
      const int cv = common_vertex(ej, ek);
      if (cv >= 0) {
        int lo, hi;
        third_edge(ej, ek, cv, lo, hi);
        const int t3 = 1 ^ ej.kind ^ ek.kind;
        add(make_pair(t3, lo, hi), elem_index(B, t3, lo, hi));
      }
    }
  } else if (ej.kind != kD) {
    add(make_pair(1 - ej.kind, ej.a, ej.b), partner(B, j));
  } else if (ek.kind != kD) {
    add(make_pair(1 - ek.kind, ek.a, ek.b), partner(B, k));
  }
}

// ---------------------------------------------------------------- scan
// Exclusive prefix sums of n int64 counts into off[0..n] (off[n] = total),
// in three passes: tile sums, a scan of the tile sums by one block, and the
// tile scans with their offsets.  A tile is 256 threads x 8 counts.
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t* warp_tot, int64_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  total = warp_tot[kScanThreads / 32 - 1];
  const int64_t before = wid > 0 ? warp_tot[wid - 1] : 0;
  const int64_t r = before + inc - x;
  __syncthreads();
  return r;
}

template <class C>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const C* cnt, int64_t n, int64_t* off,
                                                             int64_t* tile_sum, int add) {
  __shared__ int64_t wt[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems], s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? (int64_t)cnt[base + i] : 0;
    s += v[i];
  }
  int64_t total;
  int64_t run = block_excl_scan(s, wt, total);
  if (!add) {
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
    return;
  }
  run += tile_sum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) off[base + i] = run;
    run += v[i];
  }
}

// Exclusive scan of the tile sums in place (one block, chunks of 256); the
// grand total goes to *total.
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int64_t* tile_sum, int64_t nt, int64_t* total) {
  __shared__ int64_t wt[kScanThreads / 32];
  int64_t carry = 0;
  for (int64_t b = 0; b < nt; b += kScanThreads) {
    const int64_t i = b + threadIdx.x;
    const int64_t x = i < nt ? tile_sum[i] : 0;
    int64_t tot;
    const int64_t e = block_excl_scan(x, wt, tot);
    if (i < nt) tile_sum[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

// ---------------------------------------------------------------- rows
constexpr int kRowCap = 512;          // hash slots of one warp (rows up to 256 terms)
constexpr int kRowBound = 256;        // terms above which a row takes the block path
constexpr int kRowWarps = 4;
constexpr int kLongCap = 8192;        // hash slots of one block (long rows), per column partition
constexpr int kLongThreads = 256;
constexpr int32_t kEmpty = -1;

struct RowInputs {
  int64_t M;
  const double* gamma;
  const int64_t *woff, *uoff, *qoff;  // bucket offsets (M + 1 each; qoff may be null)
  const BTerm *w, *u, *q;
};

__device__ __forceinline__ uint32_t col_hash(int32_t n) { return (uint32_t)n * 2654435761u; }

// Add (v, m) to column n; false if the table is full.  Slots come from the
// low bits of the column's hash (partitions, in the long path, from the high
// bits).
__device__ __forceinline__ bool hash_add(int32_t* keys, double* val, double* mag, uint32_t mask, int32_t n, double v,
                                         double m) {
  uint32_t h = col_hash(n) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t k = atomicCAS(keys + h, kEmpty, n);
    if (k == kEmpty || k == n) {
      atomicAdd(val + h, v);
      atomicAdd(mag + h, m);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

// Number of product and Q terms of row s (an upper bound of its columns).
__device__ __forceinline__ int64_t row_terms(const RowInputs& I, int64_t s, int lane, int width) {
  int64_t t = 0;
  for (int64_t i = I.woff[s] + lane; i < I.woff[s + 1]; i += width) {
    const int64_t l = I.w[i].x;
    t += I.uoff[l + 1] - I.uoff[l];
  }
  if (lane == 0 && I.qoff) t += I.qoff[s + 1] - I.qoff[s];
  return t;
}

// One warp adds (v, m) of every lane to the lane's column key (kEmpty: no
// term) without atomic additions: lanes with the same key are grouped by
// __match_any_sync, the group's lowest lane sums the group's terms in lane
// order (shuffles) and alone updates the column's slot, which it finds or
// claims by compare-and-swap on the key.  Leaders of different groups hold
// different keys, hence different slots.  False if the table is full.
__device__ __forceinline__ bool warp_add(int32_t* keys, double* val, double* mag, uint32_t mask, int32_t key,
                                         double v, double m, int lane) {
  const unsigned active = __ballot_sync(0xffffffffu, key != kEmpty);
  const unsigned grp = __match_any_sync(0xffffffffu, key) & active;
  unsigned rem = key != kEmpty ? grp & ~(1u << lane) : 0u;
  double sv = v, sm = m;
  while (__any_sync(0xffffffffu, rem != 0u)) {
    const int src = rem ? __ffs(rem) - 1 : lane;
    const double ov = __shfl_sync(0xffffffffu, v, src), om = __shfl_sync(0xffffffffu, m, src);
    if (rem) {
      sv += ov;
      sm += om;
      rem &= rem - 1u;
    }
  }
  bool ok = true;
  if (key != kEmpty && lane == __ffs(grp) - 1) {
    ok = false;
    uint32_t h = col_hash(key) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const int32_t k = atomicCAS(keys + h, kEmpty, key);
      if (k == kEmpty || k == key) {
        val[h] += sv;
        mag[h] += sm;
        ok = true;
        break;
      }
      h = (h + 1) & mask;
    }
  }
  __syncwarp();
  return ok;
}

// One W term of a chunk, scaled for its products (a product with the U term
// u is (a Re u + b Im u, m |u|) = (-1/2 g Re(w u), 1/2 g |w| |u|)), with the
// start of its U row and the chunk-local offset of its first product.
struct WStage {
  double a, b, m;
  int64_t ubeg;
  int32_t p, pre;
};

// Exclusive prefix of x over the WIDTH threads (WIDTH = 32: one warp;
// WIDTH = kLongThreads: the block, with a barrier); *total = the sum.
template <int WIDTH>
__device__ __forceinline__ int excl_prefix(int x, int* tot_s, int* total) {
  if (WIDTH == 32) {
    const int lane = threadIdx.x & 31;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - x;
  } else {
    int64_t t64;
    const int64_t r = block_excl_scan((int64_t)x, reinterpret_cast<int64_t*>(tot_s), t64);
    *total = (int)t64;
    return (int)r;
  }
}

template <int WIDTH>
__device__ __forceinline__ void width_sync() {
  if (WIDTH == 32) __syncwarp();
  else __syncthreads();
}

// Accumulate row s into the table, the columns of partition `part` of
// `nparts` only (hash high bits): the products of the W terms of column s
// with the U rows they name, taken WIDTH W terms at a time and spread over
// the threads one product each (a thread finds its W term by binary search
// of the chunk's prefix offsets), then the row's Q terms.
template <int WIDTH>
__device__ bool row_accumulate(const RowInputs& I, int64_t s, int t, WStage* ws, int* tot_s, int32_t* keys,
                               double* val, double* mag, uint32_t mask, int part, int nparts) {
  bool ok = true;
  const uint32_t pshift = 32 - (nparts > 1 ? __ffs(nparts) - 1 : 0);
  auto mine = [&](int32_t n) { return nparts == 1 || (int)(col_hash(n) >> pshift) == part; };
  const int64_t w0 = I.woff[s], w1 = I.woff[s + 1];
  for (int64_t c = w0; c < w1; c += WIDTH) {
    const int cnt = (int)(w1 - c < WIDTH ? w1 - c : WIDTH);
    int len = 0;
    WStage st{};
    if (t < cnt) {
      const BTerm wt = I.w[c + t];
      const double hg = 0.5 * I.gamma[wt.p];
      st.a = -hg * wt.re;
      st.b = hg * wt.im;
      st.m = hg * wt.mag;
      st.p = wt.p;
      st.ubeg = I.uoff[wt.x];
      len = (int)(I.uoff[wt.x + 1] - st.ubeg);
    }
    int total;
    st.pre = excl_prefix<WIDTH>(len, tot_s, &total);
    if (t < cnt) ws[t] = st;
    width_sync<WIDTH>();
    // rounds of WIDTH products (warp-uniform, for the warp path's collective add)
    for (int f0 = 0; f0 < total; f0 += WIDTH) {
      const int f = f0 + t;
      int32_t key = kEmpty;
      double v = 0.0, m = 0.0;
      if (f < total) {
        int lo = 0, hi = cnt - 1;  // the last i with ws[i].pre <= f
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ws[mid].pre <= f) lo = mid; else hi = mid - 1;
        }
        const WStage& w = ws[lo];
        const BTerm ut = I.u[w.ubeg + (f - w.pre)];
        if (ut.p == w.p && mine(ut.x)) {
          key = ut.x;
          v = fma(w.a, ut.re, w.b * ut.im);
          m = w.m * ut.mag;
        }
      }
      if (WIDTH == 32) ok &= warp_add(keys, val, mag, mask, key, v, m, t);
      else if (key != kEmpty) ok &= hash_add(keys, val, mag, mask, key, v, m);
    }
    width_sync<WIDTH>();
  }
  if (I.qoff) {
    const int64_t q0 = I.qoff[s], q1 = I.qoff[s + 1];
    for (int64_t i0 = q0; i0 < q1; i0 += WIDTH) {
      const int64_t i = i0 + t;
      int32_t key = kEmpty;
      double v = 0.0, m = 0.0;
      if (i < q1) {
        const BTerm qt = I.q[i];
        if (mine(qt.x)) {
          key = qt.x;
          v = qt.re;
          m = qt.mag;
        }
      }
      if (WIDTH == 32) ok &= warp_add(keys, val, mag, mask, key, v, m, t);
      else if (key != kEmpty) ok &= hash_add(keys, val, mag, mask, key, v, m);
    }
  }
  return ok;
}

__device__ __forceinline__ bool kept(int32_t k, double v, double m) { return k != kEmpty && fabs(v) > 1e-12 * m; }

// Move the kept entries of a table of `cap` slots (a multiple of 32) to its
// front and return their number.  Called by one whole warp.  First the
// occupied slots move to the front with integer tests only, then the kept
// test (|value| > 1e-12 x magnitude, FP64) runs over the occupied ones: the
// FP64 pipe takes a warp instruction at the same cost whatever its active
// lanes, and most slots are empty.  Each pass goes 32 slots at a time by
// ballot; a slot is read before any lane writes at or below it.
__device__ __forceinline__ int warp_compact(int32_t* keys, double* val, double* mag, int cap, int lane) {
  int occ = 0;
  for (int base = 0; base < cap; base += 32) {
    const int a = base + lane;
    const int32_t k = keys[a];
    const double v = val[a], m = mag[a];
    const bool used = k != kEmpty;
    const unsigned bal = __ballot_sync(0xffffffffu, used);
    __syncwarp();
    if (used) {
      const int pos = occ + __popc(bal & ((1u << lane) - 1u));
      keys[pos] = k;
      val[pos] = v;
      mag[pos] = m;
    }
    occ += __popc(bal);
    __syncwarp();
  }
  int run = 0;
  for (int base = 0; base < occ; base += 32) {
    const int a = base + lane;
    int32_t k = kEmpty;
    double v = 0.0, m = 0.0;
    if (a < occ) {
      k = keys[a];
      v = val[a];
      m = mag[a];
    }
    const bool kp = kept(k, v, m);
    const unsigned bal = __ballot_sync(0xffffffffu, kp);
    __syncwarp();
    if (kp) {
      const int pos = run + __popc(bal & ((1u << lane) - 1u));
      keys[pos] = k;
      val[pos] = v;
    }
    run += __popc(bal);
    __syncwarp();
  }
  return run;
}

// Terms of every row (one warp per row): bound[s]; rows of more than
// kRowBound terms go to the long list.
__global__ void __launch_bounds__(kRowWarps * 32) k_row_terms(RowInputs I, unsigned long long* bound,
                                                             int64_t* longlist, unsigned long long* nlong) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kRowWarps + wid;
  if (s >= I.M) return;
  int64_t t = row_terms(I, s, lane, 32);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) {
    bound[s] = (unsigned long long)t;
    if (t > kRowBound) longlist[atomicAdd(nlong, 1ull)] = s;
  }
}

// One warp per row of at most kRowBound terms, in a table of the smallest
// power of two >= 2 x terms slots (at least 64): accumulate the row once and
// write its kept entries (unordered) to the row's scratch range (tmpoff[s],
// room for bound[s] >= kept entries) and their number to rowcount[s].
__global__ void __launch_bounds__(kRowWarps * 32) k_rows_warp(RowInputs I, const unsigned long long* bound,
                                                             const int64_t* tmpoff, int32_t* tcol, double* tval,
                                                             unsigned long long* rowcount, int* status) {
  __shared__ int32_t keys_s[kRowWarps][kRowCap];
  __shared__ double val_s[kRowWarps][kRowCap], mag_s[kRowWarps][kRowCap];
  __shared__ WStage ws_s[kRowWarps][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kRowWarps + wid;
  if (s >= I.M) return;
  const unsigned long long tb = bound[s];
  if (tb > (unsigned long long)kRowBound) return;
  int cap = 64;
  while (cap < 2 * (int)tb) cap <<= 1;
  int32_t* keys = keys_s[wid];
  double* val = val_s[wid];
  double* mag = mag_s[wid];
  for (int a = lane; a < cap; a += 32) {
    keys[a] = kEmpty;
    val[a] = 0.0;
    mag[a] = 0.0;
  }
  __syncwarp();
  const bool ok = row_accumulate<32>(I, s, lane, ws_s[wid], nullptr, keys, val, mag, cap - 1, 0, 1);
  if (!ok) atomicExch(status, 1);  // not reached: at most cap / 2 columns
  __syncwarp();
  const int k = warp_compact(keys, val, mag, cap, lane);
  for (int e = lane; e < k; e += 32) {
    tcol[tmpoff[s] + e] = keys[e];
    tval[tmpoff[s] + e] = val[e];
  }
  if (lane == 0) rowcount[s] = (unsigned long long)k;
}

// One block per long row.  The row's columns are split by the high bits of
// their hash into the smallest power-of-two number of partitions with at
// most kLongCap / 2 terms each on average; each partition is accumulated in
// a table of kLongCap slots in shared memory and its kept entries appended
// to the row's scratch range.  A partition with more distinct columns than
// slots sets *status = 2.
__global__ void __launch_bounds__(kLongThreads) k_rows_long(RowInputs I, const int64_t* longlist,
                                                           const unsigned long long* bound, const int64_t* tmpoff,
                                                           int32_t* tcol, double* tval, unsigned long long* rowcount,
                                                           int* status) {
  extern __shared__ __align__(16) unsigned char lsm[];
  double* val = reinterpret_cast<double*>(lsm);
  double* mag = val + kLongCap;
  int32_t* keys = reinterpret_cast<int32_t*>(mag + kLongCap);
  __shared__ WStage ws[kLongThreads];
  __shared__ int64_t tot_s[kLongThreads / 32];
  __shared__ int kk;
  const int64_t s = longlist[blockIdx.x];
  int nparts = 1;
  while ((unsigned long long)nparts * (kLongCap / 2) < bound[s] && nparts < (1 << 20)) nparts <<= 1;
  int total = 0;
  for (int part = 0; part < nparts; ++part) {
    for (int a = threadIdx.x; a < kLongCap; a += kLongThreads) {
      keys[a] = kEmpty;
      val[a] = 0.0;
      mag[a] = 0.0;
    }
    __syncthreads();
    const bool ok = row_accumulate<kLongThreads>(I, s, threadIdx.x, ws, reinterpret_cast<int*>(tot_s), keys, val, mag,
                                                 kLongCap - 1, part, nparts);
    if (!ok) atomicExch(status, 2);
    __syncthreads();
    if (threadIdx.x < 32) {  // compaction by warp 0
      const int k = warp_compact(keys, val, mag, kLongCap, threadIdx.x);
      if (threadIdx.x == 0) kk = k;
    }
    __syncthreads();
    const int k = kk;
    for (int e = threadIdx.x; e < k; e += kLongThreads) {
      tcol[tmpoff[s] + total + e] = keys[e];
      tval[tmpoff[s] + total + e] = val[e];
    }
    total += k;
    __syncthreads();
  }
  if (threadIdx.x == 0) rowcount[s] = (unsigned long long)total;
}

// Rows from the scratch ranges to their CSR place in ascending column order
// (one warp per row; an entry's rank is the number of the row's entries with
// a smaller column).
__global__ void __launch_bounds__(256) k_rows_copy(int64_t M, const int64_t* tmpoff, const int32_t* tcol,
                                                  const double* tval, const int64_t* rowptr, int32_t* col,
                                                  double* val) {
  const int64_t s = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const int64_t src = tmpoff[s], dst = rowptr[s], k = rowptr[s + 1] - rowptr[s];
  for (int64_t i = lane; i < k; i += 32) {
    const int32_t ki = tcol[src + i];
    int64_t rank = 0;
    for (int64_t j = 0; j < k; ++j) rank += tcol[src + j] < ki ? 1 : 0;
    col[dst + rank] = ki;
    val[dst + rank] = tval[src + i];
  }
}

inline unsigned nb(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

namespace lbi {

// Owning device allocation helper for this file (freed on scope exit).
struct Buf {
  void* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, n ? n : 16); }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

#define CK(x)                             \
  do {                                    \
    cudaError_t _e = (x);                 \
    if (_e != cudaSuccess) return _e;     \
  } while (0)

// off[0..n] = exclusive prefix sums of the n counts (off[n] = the total).
template <class C>
static cudaError_t scan_device(const C* cnt, int64_t* off, int64_t n, cudaStream_t st) {
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  Buf ts;
  CK(ts.alloc(sizeof(int64_t) * (size_t)(nt + 1)));
  if (nt > 0) {
    k_scan_tiles<C><<<(unsigned)nt, kScanThreads, 0, st>>>(cnt, n, off, ts.as<int64_t>(), 0);
    k_scan_top<<<1, kScanThreads, 0, st>>>(ts.as<int64_t>(), nt, off + n);
    k_scan_tiles<C><<<(unsigned)nt, kScanThreads, 0, st>>>(cnt, n, off, ts.as<int64_t>(), 1);
    note_launch(3);
  } else {
    CK(cudaMemsetAsync(off, 0, sizeof(int64_t), st));
  }
  // the tile sums are freed when this returns: the scan must be complete
  return cudaStreamSynchronize(st);
}

// The same, and *total (host) = off[n].
static cudaError_t scan_counts(const unsigned long long* cnt, int64_t* off, int64_t n, int64_t* total,
                               cudaStream_t st) {
  CK(scan_device(cnt, off, n, st));
  CK(cudaMemcpyAsync(total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  return cudaStreamSynchronize(st);
}

cudaError_t exclusive_scan(const int64_t* counts, int64_t* off, int64_t n, cudaStream_t st) {
  return scan_device(counts, off, n, st);
}

// Buckets of terms: counts (M + 1), offsets (M + 1), the terms.
struct Buckets {
  Buf cnt, off, terms;
  int64_t total = 0;
};

// Count with `emit(bucketer)`, scan, reset the cursors, fill with `emit`.
template <class Emit>
static cudaError_t build_buckets(int64_t M, Buckets& b, Emit emit, cudaStream_t st) {
  CK(b.cnt.alloc(sizeof(unsigned long long) * (size_t)(M + 1)));
  CK(b.off.alloc(sizeof(int64_t) * (size_t)(M + 1)));
  CK(cudaMemsetAsync(b.cnt.p, 0, sizeof(unsigned long long) * (size_t)(M + 1), st));
  CK(emit(Bucketer{b.cnt.as<unsigned long long>(), nullptr, nullptr}));
  CK(scan_counts(b.cnt.as<unsigned long long>(), b.off.as<int64_t>(), M, &b.total, st));
  CK(b.terms.alloc(sizeof(BTerm) * (size_t)b.total));
  CK(cudaMemsetAsync(b.cnt.p, 0, sizeof(unsigned long long) * (size_t)(M + 1), st));
  if (b.total > 0) CK(emit(Bucketer{b.cnt.as<unsigned long long>(), b.off.as<int64_t>(), b.terms.as<BTerm>()}));
  return cudaSuccess;
}

cudaError_t assemble_lowrank_csr(const lb::BasisView& B, const double* h, int nP, const double* gamma_host,
                                 const int64_t* lp_ptr_host, const int64_t* lp_idx, const double2* lp_val,
                                 CsrOut* out, cudaStream_t st) {
  const int64_t M = B.M;
  const int64_t nu = lp_ptr_host[nP];
  Buf dptr, dgamma;
  CK(dptr.alloc(sizeof(int64_t) * (nP + 1)));
  CK(dgamma.alloc(sizeof(double) * (nP > 0 ? nP : 1)));
  CK(cudaMemcpyAsync(dptr.p, lp_ptr_host, sizeof(int64_t) * (nP + 1), cudaMemcpyHostToDevice, st));
  if (nP > 0) CK(cudaMemcpyAsync(dgamma.p, gamma_host, sizeof(double) * nP, cudaMemcpyHostToDevice, st));
  const int64_t* dp = dptr.as<int64_t>();
  // ---- diagonal components of the channels: dense per channel, suffix sums
  const int N = B.N;
  Buf dl, hasD, suf, sufm;
  CK(dl.alloc(sizeof(double2) * (size_t)nP * N));
  CK(hasD.alloc(sizeof(int) * (size_t)(nP > 0 ? nP : 1)));
  CK(suf.alloc(sizeof(double2) * (size_t)nP * N));
  CK(sufm.alloc(sizeof(double) * (size_t)nP * N));
  CK(cudaMemsetAsync(dl.p, 0, sizeof(double2) * (size_t)nP * N, st));
  CK(cudaMemsetAsync(hasD.p, 0, sizeof(int) * (size_t)(nP > 0 ? nP : 1), st));
  if (nu > 0) {
    k_dscatter<<<nb(nu, 256), 256, 0, st>>>(B, nP, dp, lp_idx, lp_val, nu, dl.as<double2>(), hasD.as<int>());
    k_dsuffix<<<nb(nP, 128), 128, 0, st>>>(B, nP, dl.as<double2>(), hasD.as<int>(), suf.as<double2>(),
                                           sufm.as<double>());
    note_launch(2);
  }
  const int64_t ndp = (int64_t)nP * N, ndd = (int64_t)nP * (N - 1) * (N - 1);
  const int S = fiber_slices(N);
  // ---- W (by column s), U (by row l), Q (by row s)
  Buckets W, U, Q;
  CK(build_buckets(M, W, [&](Bucketer bk) {
    if (nu > 0) {
      k_w_bucket<<<nb(nu * S, 256), 256, 0, st>>>(B, nP, dp, lp_idx, lp_val, nu, bk);
      k_dpart_bucket<<<nb(ndp, 128), 128, 0, st>>>(B, nP, dl.as<double2>(), hasD.as<int>(), suf.as<double2>(),
                                                   sufm.as<double>(), 0, bk);
      note_launch(2);
    }
    return cudaGetLastError();
  }, st));
  CK(build_buckets(M, U, [&](Bucketer bk) {
    if (nu > 0) {
      k_u_bucket<<<nb(nu * S, 256), 256, 0, st>>>(B, nP, dp, lp_idx, lp_val, nu, bk);
      k_dpart_bucket<<<nb(ndp, 128), 128, 0, st>>>(B, nP, dl.as<double2>(), hasD.as<int>(), suf.as<double2>(),
                                                   sufm.as<double>(), 1, bk);
      note_launch(2);
      if (ndd > 0) {
        k_udd_bucket<<<nb(ndd, 256), 256, 0, st>>>(B, nP, dl.as<double2>(), hasD.as<int>(), suf.as<double2>(),
                                                   sufm.as<double>(), bk);
        note_launch(1);
      }
    }
    return cudaGetLastError();
  }, st));
  if (h) {
    Buf hlist, hcount;
    CK(hlist.alloc(sizeof(int64_t) * (size_t)(2 * B.P)));
    CK(hcount.alloc(sizeof(unsigned long long)));
    CK(cudaMemsetAsync(hcount.p, 0, sizeof(unsigned long long), st));
    k_h_nonzero<<<nb(2 * B.P, 256), 256, 0, st>>>(2 * B.P, h, hlist.as<int64_t>(), hcount.as<unsigned long long>());
    note_launch(1);
    unsigned long long nh = 0;
    CK(cudaMemcpyAsync(&nh, hcount.p, sizeof(nh), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(build_buckets(M, Q, [&](Bucketer bk) {
      if (nh > 0) {
        k_q_pair_bucket<<<nb((int64_t)nh * S, 256), 256, 0, st>>>(B, h, hlist.as<int64_t>(), (int64_t)nh, bk);
        note_launch(1);
      }
      k_q_diag_bucket<<<nb((int64_t)N * 32, 256), 256, 0, st>>>(B, h, bk);
      note_launch(1);
      return cudaGetLastError();
    }, st));
  }
  // ---- rows: term bounds, one accumulation into scratch ranges, CSR
  RowInputs I{M, dgamma.as<double>(), W.off.as<int64_t>(), U.off.as<int64_t>(), h ? Q.off.as<int64_t>() : nullptr,
              W.terms.as<BTerm>(), U.terms.as<BTerm>(), h ? Q.terms.as<BTerm>() : nullptr};
  Buf bound, tmpoff, longlist, ctr;  // ctr: [0] long rows, [1] status
  CK(bound.alloc(sizeof(unsigned long long) * (size_t)(M + 1)));
  CK(tmpoff.alloc(sizeof(int64_t) * (size_t)(M + 1)));
  CK(longlist.alloc(sizeof(int64_t) * (size_t)M));
  CK(ctr.alloc(sizeof(unsigned long long) * 2));
  CK(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long) * 2, st));
  unsigned long long* c = ctr.as<unsigned long long>();
  int* status = reinterpret_cast<int*>(c + 1);
  const unsigned rgrid = nb(M, kRowWarps);
  k_row_terms<<<rgrid, kRowWarps * 32, 0, st>>>(I, bound.as<unsigned long long>(), longlist.as<int64_t>(), c);
  note_launch(1);
  int64_t nterms = 0;
  CK(scan_counts(bound.as<unsigned long long>(), tmpoff.as<int64_t>(), M, &nterms, st));
  unsigned long long hc[2];
  CK(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int64_t nlong = (int64_t)hc[0];
  Buf tcol, tval, rowc;
  CK(tcol.alloc(sizeof(int32_t) * (size_t)(nterms + 1)));
  CK(tval.alloc(sizeof(double) * (size_t)(nterms + 1)));
  CK(rowc.alloc(sizeof(unsigned long long) * (size_t)(M + 1)));
  k_rows_warp<<<rgrid, kRowWarps * 32, 0, st>>>(I, bound.as<unsigned long long>(), tmpoff.as<int64_t>(),
                                                tcol.as<int32_t>(), tval.as<double>(), rowc.as<unsigned long long>(),
                                                status);
  note_launch(1);
  if (nlong > 0) {
    const size_t lsmem = (sizeof(double) * 2 + sizeof(int32_t)) * (size_t)kLongCap;
    CK(cudaFuncSetAttribute(k_rows_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    k_rows_long<<<(unsigned)nlong, kLongThreads, lsmem, st>>>(I, longlist.as<int64_t>(),
                                                             bound.as<unsigned long long>(), tmpoff.as<int64_t>(),
                                                             tcol.as<int32_t>(), tval.as<double>(),
                                                             rowc.as<unsigned long long>(), status);
    note_launch(1);
  }
  Buf rowptr;
  CK(rowptr.alloc(sizeof(int64_t) * (size_t)(M + 1)));
  int64_t nnz = 0;
  CK(scan_counts(rowc.as<unsigned long long>(), rowptr.as<int64_t>(), M, &nnz, st));
  CK(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hc[1] != 0) return cudaErrorNotSupported;  // a row has more than kLongCap distinct columns
  Buf col, val, K;
  CK(col.alloc(sizeof(int32_t) * (size_t)(nnz + 1)));
  CK(val.alloc(sizeof(double) * (size_t)(nnz + 1)));
  CK(K.alloc(sizeof(double) * (size_t)M));
  k_rows_copy<<<nb(M, 8), 256, 0, st>>>(M, tmpoff.as<int64_t>(), tcol.as<int32_t>(), tval.as<double>(),
                                        rowptr.as<int64_t>(), col.as<int32_t>(), val.as<double>());
  note_launch(1);
  // ---- K
  CK(cudaMemsetAsync(K.p, 0, sizeof(double) * M, st));
  int64_t maxn = 0;
  for (int p = 0; p < nP; ++p) maxn = lp_ptr_host[p + 1] - lp_ptr_host[p] > maxn ? lp_ptr_host[p + 1] - lp_ptr_host[p] : maxn;
  if (maxn > 0) {
    dim3 grid(nb(maxn * maxn, 256), nP);
    k_k_lowrank<<<grid, 256, 0, st>>>(B, nP, dp, dgamma.as<double>(), lp_idx, lp_val, K.as<double>());
    note_launch(1);
  }
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  out->M = M;
  out->nnz = nnz;
  out->rowptr = rowptr.as<int64_t>();
  rowptr.p = nullptr;
  out->col = col.as<int32_t>();
  col.p = nullptr;
  out->val = val.as<double>();
  val.p = nullptr;
  out->K = K.as<double>();
  K.p = nullptr;
  out->terms = nterms;
  return cudaSuccess;
}

}  // namespace lbi

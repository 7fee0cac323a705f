// lb_csr.cu -- sparse (CSR) assembly of A = Q + R and K for a Kossakowski
// matrix in spectral form a_jk = sum_p gamma_p l_pj conj(l_pk) with sparse
// l_p and a sparse Hamiltonian (Eqs. (07)-(09); Sec. 3's sparse model class,
// P = 1 jump operator), and the fused RK4 step on CSR (Sec. 4 item 3).
//
// Eq. (09) factorises per channel:
//   r_sn = -1/2 gamma_p Re sum_l W_ls U_ln,
//   U_ln = sum_j l_j z_jln,   W_ls = sum_k conj(l_k) f_kls,
// so R is a sparse product: the fibres of the nonzero l_j give U and W as
// coordinate lists (count pass, scan, fill pass), a radix sort by (p, l, .)
// and a reduction by key merge duplicates, and every W entry is multiplied
// with the U row of its l.  The products and the Q terms h_m f_mns are
// sorted by (s, n) and reduced; an entry is kept when its value exceeds
// 1e-12 times the sum of the magnitudes of its terms (entries whose terms
// cancel exactly -- most of those the terms reach -- carry only rounding
// residue).  Magnitudes are carried through U and W as sum |l_j z_jln| etc.
#include <cub/cub.cuh>

#include "lb_internal.h"

namespace {

using namespace lb;

struct CTerm {  // a complex coordinate entry with the magnitude of its terms
  double re, im, mag;
};

struct RTerm {  // a real coordinate entry with the magnitude of its terms
  double val, mag;
};

struct CTermSum {
  __host__ __device__ CTerm operator()(const CTerm& a, const CTerm& b) const {
    return CTerm{a.re + b.re, a.im + b.im, a.mag + b.mag};
  }
};

struct RTermSum {
  __host__ __device__ RTerm operator()(const RTerm& a, const RTerm& b) const {
    return RTerm{a.val + b.val, a.mag + b.mag};
  }
};

// Every (l, s) with f_{k l s} != 0, with the value.
template <class Emit>
__device__ void for_each_f_fiber(const BasisView& B, int64_t k, Emit& emit) {
  const int N = B.N;
  const Elem ek = decode(B, k);
  if (ek.kind != kD) {
    const int a = ek.a, b = ek.b, tk = ek.kind;
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi ? b : a, vp = vi ? a : b;
      for (int w = 0; w < N; ++w) {
        if (w == a || w == b) continue;
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, v, w), es = make_pair(1 ^ tk ^ tl, vp, w);
          emit(elem_index(B, tl, v, w), elem_index(B, es.kind, vp, w), f_value(B, ek, el, es));
        }
      }
    }
    const Elem ekb = make_pair(1 - tk, a, b);
    const int64_t kb = partner(B, k);
    for (int lam = imax(a, 1); lam <= b; ++lam) {
      emit(kb, d_index(B, lam), f_value(B, ek, ekb, make_d(lam)));
      emit(d_index(B, lam), kb, f_value(B, ek, make_d(lam), ekb));
    }
  } else {
    const int nu = ek.a;
    for (int x = 0; x <= nu; ++x)
      for (int y = imax(nu, x + 1); y < N; ++y)
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, x, y), es = make_pair(1 - tl, x, y);
          emit(elem_index(B, tl, x, y), elem_index(B, 1 - tl, x, y), f_value(B, ek, el, es));
        }
  }
}

// Every (l, n) with z_{j l n} != 0, with z = f + i d.
template <class Emit>
__device__ void for_each_z_fiber(const BasisView& B, int64_t j, Emit& emit) {
  const int N = B.N;
  const Elem ej = decode(B, j);
  double f, d;
  if (ej.kind != kD) {
    const int a = ej.a, b = ej.b, tj = ej.kind;
    for (int vi = 0; vi < 2; ++vi) {
      const int v = vi ? b : a, vp = vi ? a : b;
      for (int w = 0; w < N; ++w) {
        if (w == a || w == b) continue;
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
    }
    const Elem ejb = make_pair(1 - tj, a, b);
    const int64_t jb = partner(B, j);
    for (int lam = imax(a, 1); lam < N; ++lam) {
      const Elem ed = make_d(lam);
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
  } else {
    const int nu = ej.a;
    for (int x = 0; x < N; ++x)
      for (int y = x + 1; y < N; ++y) {
        if (nu < imax(x, 1)) continue;
        for (int tl = kS; tl <= kJ; ++tl) {
          const Elem el = make_pair(tl, x, y), elb = make_pair(1 - tl, x, y);
          const int64_t l = elem_index(B, tl, x, y);
          if (nu <= y) {
            fd_value(B, ej, el, elb, f, d);
            emit(l, partner(B, l), f, 0.0);
          }
          if (!(x == 0 && y == 1 && nu == 1)) {
            fd_value(B, ej, el, el, f, d);
            emit(l, l, 0.0, d);
          }
        }
      }
    for (int lam = 1; lam < N; ++lam) {
      if (lam != nu) {
        const int m = imin(lam, nu);
        emit(d_index(B, lam), d_index(B, m), 0.0, 2.0 * trace_ddd(B, m, lam, nu));
      } else {
        for (int mu = nu; mu < N; ++mu) {
          if (mu == 1 && nu == 1) continue;
          emit(d_index(B, lam), d_index(B, mu), 0.0, 2.0 * trace_ddd(B, mu, lam, nu));
        }
      }
    }
  }
}

struct Counter {
  int64_t n = 0;
  __device__ void operator()(int64_t, int64_t, double) { ++n; }
  __device__ void operator()(int64_t, int64_t, double, double) { ++n; }
};

// Channel of a flattened nonzero index u (lp_ptr has nP + 1 entries).
__device__ __forceinline__ int channel_of(const int64_t* lp_ptr, int nP, int64_t u) {
  int p = 0;
  while (p + 1 < nP && lp_ptr[p + 1] <= u) ++p;
  return p;
}

// W terms: key = (p M + l) M + s, value conj(l_k) f_kls, magnitude |l_k f|.
__global__ void k_w_terms(BasisView B, int nP, const int64_t* lp_ptr, const int64_t* lp_idx,
                          const double2* lp_val, int64_t nu, const int64_t* off, int64_t* key, CTerm* val,
                          int64_t* count) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nu) return;
  const int p = channel_of(lp_ptr, nP, u);
  const int64_t k = lp_idx[u], M = B.M;
  const double2 lk = lp_val[u];
  if (count) {
    Counter c;
    for_each_f_fiber(B, k, c);
    count[u] = c.n;
    return;
  }
  int64_t o = off[u];
  auto emit = [&](int64_t l, int64_t s, double f) {
    key[o] = ((int64_t)p * M + l) * M + s;
    val[o] = CTerm{lk.x * f, -lk.y * f, sqrt(lk.x * lk.x + lk.y * lk.y) * fabs(f)};
    ++o;
  };
  for_each_f_fiber(B, k, emit);
}

// U terms: key = (p M + l) M + n, value l_j z_jln, magnitude |l_j z|.
__global__ void k_u_terms(BasisView B, int nP, const int64_t* lp_ptr, const int64_t* lp_idx,
                          const double2* lp_val, int64_t nu, const int64_t* off, int64_t* key, CTerm* val,
                          int64_t* count) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nu) return;
  const int p = channel_of(lp_ptr, nP, u);
  const int64_t j = lp_idx[u], M = B.M;
  const double2 lj = lp_val[u];
  if (count) {
    Counter c;
    for_each_z_fiber(B, j, c);
    count[u] = c.n;
    return;
  }
  int64_t o = off[u];
  auto emit = [&](int64_t l, int64_t n, double zr, double zi) {
    key[o] = ((int64_t)p * M + l) * M + n;
    val[o] = CTerm{lj.x * zr - lj.y * zi, lj.x * zi + lj.y * zr,
                   sqrt(lj.x * lj.x + lj.y * lj.y) * sqrt(zr * zr + zi * zi)};
    ++o;
  };
  for_each_z_fiber(B, j, emit);
}

__device__ __forceinline__ int64_t lower_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Products of each W entry with the U row of its (p, l): count or fill terms
// key2 = s M + n, value -1/2 gamma_p Re(W U), magnitude 1/2 gamma_p |W| |U|.
__global__ void k_products(int64_t M, int nP, const double* gamma, const int64_t* wkey, const CTerm* wval,
                           int64_t nw, const int64_t* ukey, const CTerm* uval, int64_t nuq, const int64_t* off,
                           int64_t* key2, RTerm* val2, int64_t* count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int64_t pl = wkey[i] / M, s = wkey[i] % M;
  const int64_t lo = lower_bound_i64(ukey, nuq, pl * M), hi = lower_bound_i64(ukey, nuq, (pl + 1) * M);
  if (count) {
    count[i] = hi - lo;
    return;
  }
  const int p = (int)(pl / M);
  const double g = gamma[p];
  const CTerm w = wval[i];
  int64_t o = off[i];
  for (int64_t q = lo; q < hi; ++q) {
    const CTerm u = uval[q];
    key2[o] = s * M + ukey[q] % M;
    val2[o] = RTerm{-0.5 * g * (w.re * u.re - w.im * u.im), 0.5 * g * w.mag * u.mag};
    ++o;
  }
}

// Q terms of the pair coefficients h_m (m < 2P, h_m != 0): f_{m n s}, (n, s) from the fibre.
__global__ void k_q_pair_terms(BasisView B, const double* h, const int64_t* off, int64_t* key2, RTerm* val2,
                               int64_t* count) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= 2 * B.P) return;
  const double hm = h[m];
  if (hm == 0.0) {
    if (count) count[m] = 0;
    return;
  }
  if (count) {
    Counter c;
    for_each_f_fiber(B, m, c);
    count[m] = c.n;
    return;
  }
  int64_t o = off[m];
  const int64_t M = B.M;
  auto emit = [&](int64_t n, int64_t s, double f) {
    key2[o] = s * M + n;
    val2[o] = RTerm{hm * f, fabs(hm * f)};
    ++o;
  };
  for_each_f_fiber(B, m, emit);
}

// Q terms of the diagonal coefficients h_{D_lam}: they reach only (S_xy, J_xy)
// and (J_xy, S_xy), with f(D_lam, J, S) etc.; one thread per edge, two terms.
__global__ void k_q_diag_terms(BasisView B, const double* h, int64_t* key2, RTerm* val2) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B.P) return;
  const int32_t ab = __ldg(B.pair_ab + e);
  const int x = ab >> 16, y = ab & 0xffff;
  double v = 0.0, mag = 0.0;  // sum_lam h_{D_lam} f(D_lam, J_xy, S_xy)
  for (int lam = imax(x, 1); lam <= y; ++lam) {
    const double t = h[d_index(B, lam)] * f_value(B, make_d(lam), make_pair(kJ, x, y), make_pair(kS, x, y));
    v += t;
    mag += fabs(t);
  }
  const int64_t M = B.M, sS = e, sJ = B.P + e;
  key2[2 * e] = sS * M + sJ;  // q_{S J} = sum h f_{m J S}
  val2[2 * e] = RTerm{v, mag};
  key2[2 * e + 1] = sJ * M + sS;  // q_{J S} = -q_{S J}
  val2[2 * e + 1] = RTerm{-v, mag};
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

// Keep entries with |value| > 1e-12 * magnitude: flags and row counts.
__global__ void k_keep(int64_t n, const int64_t* key, const RTerm* val, int64_t M, int* keep) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  keep[i] = fabs(val[i].val) > 1e-12 * val[i].mag ? 1 : 0;
}

__global__ void k_compact(int64_t n, const int64_t* key, const RTerm* val, const int* keep, const int64_t* pos,
                          int64_t M, int64_t* rowcount, int32_t* col, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  const int64_t o = pos[i];
  col[o] = (int32_t)(key[i] % M);
  out[o] = val[i].val;
  atomicAdd(reinterpret_cast<unsigned long long*>(rowcount + key[i] / M), 1ULL);
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

// exclusive scan of n int64 counts into off (n + 1 entries); returns the total
static cudaError_t scan_counts(const int64_t* count, int64_t* off, int64_t n, int64_t* total, cudaStream_t st) {
  size_t tmp = 0;
  CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp, count, off, (int)(n + 1), st));
  Buf t;
  CK(t.alloc(tmp));
  CK(cub::DeviceScan::ExclusiveSum(t.p, tmp, count, off, (int)(n + 1), st));
  CK(cudaMemcpyAsync(total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  return cudaStreamSynchronize(st);
}

// sort (key, value) pairs and merge equal keys with op; returns unique count
template <class V, class Op>
static cudaError_t sort_reduce(int64_t n, Buf& key, Buf& val, Buf& okey, Buf& oval, int64_t* nuniq, Op op,
                               int end_bit, cudaStream_t st) {
  Buf k2, v2, tmp, nout;
  CK(k2.alloc(sizeof(int64_t) * n));
  CK(v2.alloc(sizeof(V) * n));
  size_t tb = 0;
  CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, key.as<int64_t>(), k2.as<int64_t>(), val.as<V>(), v2.as<V>(),
                                     (int)n, 0, end_bit, st));
  CK(tmp.alloc(tb));
  CK(cub::DeviceRadixSort::SortPairs(tmp.p, tb, key.as<int64_t>(), k2.as<int64_t>(), val.as<V>(), v2.as<V>(),
                                     (int)n, 0, end_bit, st));
  CK(okey.alloc(sizeof(int64_t) * n));
  CK(oval.alloc(sizeof(V) * n));
  CK(nout.alloc(sizeof(int64_t)));
  size_t tr = 0;
  CK(cub::DeviceReduce::ReduceByKey(nullptr, tr, k2.as<int64_t>(), okey.as<int64_t>(), v2.as<V>(), oval.as<V>(),
                                    nout.as<int64_t>(), op, (int)n, st));
  Buf tmp2;
  CK(tmp2.alloc(tr));
  CK(cub::DeviceReduce::ReduceByKey(tmp2.p, tr, k2.as<int64_t>(), okey.as<int64_t>(), v2.as<V>(), oval.as<V>(),
                                    nout.as<int64_t>(), op, (int)n, st));
  CK(cudaMemcpyAsync(nuniq, nout.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  return cudaStreamSynchronize(st);
}

static int bits_for(int64_t x) {
  int b = 1;
  while (b < 63 && (int64_t(1) << b) <= x) ++b;
  return b;
}

cudaError_t assemble_lowrank_csr(const lb::BasisView& B, const double* h, int nP, const double* gamma_host,
                                 const int64_t* lp_ptr_host, const int64_t* lp_idx, const double2* lp_val,
                                 CsrOut* out, cudaStream_t st) {
  const int64_t M = B.M;
  const int64_t nu = lp_ptr_host[nP];
  Buf dptr, dgamma;
  CK(dptr.alloc(sizeof(int64_t) * (nP + 1)));
  CK(dgamma.alloc(sizeof(double) * nP));
  CK(cudaMemcpyAsync(dptr.p, lp_ptr_host, sizeof(int64_t) * (nP + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dgamma.p, gamma_host, sizeof(double) * nP, cudaMemcpyHostToDevice, st));
  const int kb = bits_for((int64_t)nP * M * M);
  // ---- W and U coordinate lists
  int64_t nwt = 0, nut = 0;
  Buf cnt, off, wkey, wval, ukey, uval;
  CK(cnt.alloc(sizeof(int64_t) * (nu + 1)));
  CK(off.alloc(sizeof(int64_t) * (nu + 1)));
  CK(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (nu + 1), st));
  if (nu > 0) {
    k_w_terms<<<nb(nu, 128), 128, 0, st>>>(B, nP, dptr.as<int64_t>(), lp_idx, lp_val, nu, nullptr, nullptr,
                                           nullptr, cnt.as<int64_t>());
    note_launch(1);
  }
  CK(scan_counts(cnt.as<int64_t>(), off.as<int64_t>(), nu, &nwt, st));
  CK(wkey.alloc(sizeof(int64_t) * nwt));
  CK(wval.alloc(sizeof(CTerm) * nwt));
  if (nu > 0) {
    k_w_terms<<<nb(nu, 128), 128, 0, st>>>(B, nP, dptr.as<int64_t>(), lp_idx, lp_val, nu, off.as<int64_t>(),
                                           wkey.as<int64_t>(), wval.as<CTerm>(), nullptr);
    k_u_terms<<<nb(nu, 128), 128, 0, st>>>(B, nP, dptr.as<int64_t>(), lp_idx, lp_val, nu, nullptr, nullptr,
                                           nullptr, cnt.as<int64_t>());
    note_launch(2);
  }
  CK(scan_counts(cnt.as<int64_t>(), off.as<int64_t>(), nu, &nut, st));
  CK(ukey.alloc(sizeof(int64_t) * nut));
  CK(uval.alloc(sizeof(CTerm) * nut));
  if (nu > 0) {
    k_u_terms<<<nb(nu, 128), 128, 0, st>>>(B, nP, dptr.as<int64_t>(), lp_idx, lp_val, nu, off.as<int64_t>(),
                                           ukey.as<int64_t>(), uval.as<CTerm>(), nullptr);
    note_launch(1);
  }
  Buf wk, wv, uk, uv;
  int64_t nw = 0, nuq = 0;
  if (nwt > 0) CK(sort_reduce<CTerm>(nwt, wkey, wval, wk, wv, &nw, CTermSum(), kb, st));
  if (nut > 0) CK(sort_reduce<CTerm>(nut, ukey, uval, uk, uv, &nuq, CTermSum(), kb, st));
  // ---- R products and Q terms into one (s, n) coordinate list
  Buf pcnt, poff;
  int64_t np = 0;
  CK(pcnt.alloc(sizeof(int64_t) * (nw + 1)));
  CK(poff.alloc(sizeof(int64_t) * (nw + 1)));
  CK(cudaMemsetAsync(pcnt.p, 0, sizeof(int64_t) * (nw + 1), st));
  if (nw > 0 && nuq > 0) {
    k_products<<<nb(nw, 256), 256, 0, st>>>(M, nP, dgamma.as<double>(), wk.as<int64_t>(), wv.as<CTerm>(), nw,
                                            uk.as<int64_t>(), uv.as<CTerm>(), nuq, nullptr, nullptr, nullptr,
                                            pcnt.as<int64_t>());
    note_launch(1);
  }
  CK(scan_counts(pcnt.as<int64_t>(), poff.as<int64_t>(), nw, &np, st));
  int64_t nqp = 0;
  Buf qcnt, qoff;
  const int64_t P2 = 2 * B.P;
  if (h) {
    CK(qcnt.alloc(sizeof(int64_t) * (P2 + 1)));
    CK(qoff.alloc(sizeof(int64_t) * (P2 + 1)));
    CK(cudaMemsetAsync(qcnt.p, 0, sizeof(int64_t) * (P2 + 1), st));
    k_q_pair_terms<<<nb(P2, 128), 128, 0, st>>>(B, h, nullptr, nullptr, nullptr, qcnt.as<int64_t>());
    note_launch(1);
    CK(scan_counts(qcnt.as<int64_t>(), qoff.as<int64_t>(), P2, &nqp, st));
  }
  const int64_t nqd = h ? 2 * B.P : 0;
  const int64_t nt = np + nqp + nqd;
  Buf tkey, tval;
  CK(tkey.alloc(sizeof(int64_t) * nt));
  CK(tval.alloc(sizeof(RTerm) * nt));
  if (np > 0) {
    k_products<<<nb(nw, 256), 256, 0, st>>>(M, nP, dgamma.as<double>(), wk.as<int64_t>(), wv.as<CTerm>(), nw,
                                            uk.as<int64_t>(), uv.as<CTerm>(), nuq, poff.as<int64_t>(),
                                            tkey.as<int64_t>(), tval.as<RTerm>(), nullptr);
    note_launch(1);
  }
  if (nqp > 0) {
    k_q_pair_terms<<<nb(P2, 128), 128, 0, st>>>(B, h, qoff.as<int64_t>(), tkey.as<int64_t>() + np,
                                               tval.as<RTerm>() + np, nullptr);
    note_launch(1);
  }
  if (nqd > 0) {
    k_q_diag_terms<<<nb(B.P, 128), 128, 0, st>>>(B, h, tkey.as<int64_t>() + np + nqp,
                                                tval.as<RTerm>() + np + nqp);
    note_launch(1);
  }
  // ---- reduce by (s, n), keep, CSR
  Buf fk, fv;
  int64_t nf = 0;
  if (nt > 0) CK(sort_reduce<RTerm>(nt, tkey, tval, fk, fv, &nf, RTermSum(), bits_for(M * M), st));
  Buf keep, pos, rowc;
  CK(keep.alloc(sizeof(int) * (nf + 1)));
  CK(pos.alloc(sizeof(int64_t) * (nf + 1)));
  CK(rowc.alloc(sizeof(int64_t) * (M + 1)));
  CK(cudaMemsetAsync(rowc.p, 0, sizeof(int64_t) * (M + 1), st));
  int64_t nnz = 0;
  if (nf > 0) {
    k_keep<<<nb(nf, 256), 256, 0, st>>>(nf, fk.as<int64_t>(), fv.as<RTerm>(), M, keep.as<int>());
    note_launch(1);
    size_t tmp = 0;
    CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp, keep.as<int>(), pos.as<int64_t>(), (int)nf, st));
    Buf t;
    CK(t.alloc(tmp));
    CK(cub::DeviceScan::ExclusiveSum(t.p, tmp, keep.as<int>(), pos.as<int64_t>(), (int)nf, st));
    int64_t lastpos = 0;
    int lastkeep = 0;
    CK(cudaMemcpyAsync(&lastpos, pos.as<int64_t>() + nf - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&lastkeep, keep.as<int>() + nf - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nnz = lastpos + lastkeep;
  }
  Buf rowptr, col, val, K;
  CK(rowptr.alloc(sizeof(int64_t) * (M + 1)));
  CK(col.alloc(sizeof(int32_t) * (nnz + 1)));
  CK(val.alloc(sizeof(double) * (nnz + 1)));
  CK(K.alloc(sizeof(double) * M));
  if (nf > 0) {
    k_compact<<<nb(nf, 256), 256, 0, st>>>(nf, fk.as<int64_t>(), fv.as<RTerm>(), keep.as<int>(),
                                          pos.as<int64_t>(), M, rowc.as<int64_t>(), col.as<int32_t>(),
                                          val.as<double>());
    note_launch(1);
  }
  int64_t total = 0;
  CK(scan_counts(rowc.as<int64_t>(), rowptr.as<int64_t>(), M, &total, st));
  // ---- K
  CK(cudaMemsetAsync(K.p, 0, sizeof(double) * M, st));
  int64_t maxn = 0;
  for (int p = 0; p < nP; ++p) maxn = lp_ptr_host[p + 1] - lp_ptr_host[p] > maxn ? lp_ptr_host[p + 1] - lp_ptr_host[p] : maxn;
  if (maxn > 0) {
    dim3 grid(nb(maxn * maxn, 256), nP);
    k_k_lowrank<<<grid, 256, 0, st>>>(B, nP, dptr.as<int64_t>(), dgamma.as<double>(), lp_idx, lp_val, K.as<double>());
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
  out->terms = np + nqp + nqd;
  return cudaSuccess;
}

}  // namespace lbi

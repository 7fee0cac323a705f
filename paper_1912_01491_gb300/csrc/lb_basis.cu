// lb_basis.cu -- kernel (a): index-arithmetic enumeration of the nonzero
// structure constants f_mns, d_mns (Eq. (05); Table 1 step 2.2), plus the
// basis index tables, the expansion of Eq. (02) and the reconstruction of
// Eq. (rho).
//
// Canonical lists hold each unordered triple once as m <= n <= s, sorted by
// (m, n, s).  Thread m walks its partners n in increasing index order and
// for each the third indices s >= n in increasing order, so a count pass,
// an exclusive scan over m and a fill pass give the sorted list without any
// sort.  The nonzero triples fall into three classes:
//   * three pair elements whose edges form a triangle a-b-c: for given
//     types of two of them the type of the third is fixed by parity (f: odd
//     number of J's, d: even);
//   * two pair elements on one edge (a,b) and D_l: f(S_ab, J_ab, D_l) != 0
//     for max(a,1) <= l <= b; d(S_ab, S_ab, D_l) = d(J_ab, J_ab, D_l) != 0
//     for l >= max(a,1) except (a,b,l) = (0,1,1);
//   * d(D_l, D_l, D_r) for r >= l except l = r = 1 (canonical form of the
//     "two smallest equal" rule).
#include <cub/cub.cuh>

#include "lb_internal.h"

namespace {

using namespace lb;

__global__ void k_tables(int N, int32_t* pair_ab, double* tab) {
  int64_t P = (int64_t)N * (N - 1) / 2;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < P) {
    // invert the lexicographic pair index
    int a = 0;
    int64_t p = t;
    // rows have N-1-a entries; a linear walk is O(N) but runs once per basis
    while (p >= N - 1 - a) {
      p -= N - 1 - a;
      ++a;
    }
    pair_ab[t] = (a << 16) | (a + 1 + (int)p);
  }
  double* c = tab;
  double* lc = tab + N;
  double* c2 = tab + 2 * N;
  double* inv = tab + 3 * N;
  if (t <= N) {
    if (t >= 1) inv[t] = 1.0 / (double)t;
    else inv[0] = 0.0;
  }
  if (t < N) {
    if (t == 0) {
      c[0] = lc[0] = c2[0] = 0.0;
    } else {
      double l = (double)t;
      double cl = 1.0 / sqrt(l * (l + 1.0));
      c[t] = cl;
      lc[t] = -l * cl;
      c2[t] = 1.0 / (l * (l + 1.0));
    }
  }
}

// Visit the canonical triples (m, n, s) with m fixed, in (n, s) order.
template <class Emit>
__host__ __device__ void for_each_canonical(const BasisView& B, int64_t m, int which, Emit& emit) {
  const Elem em = decode(B, m);
  const int N = B.N;
  if (em.kind == kD) {
    if (which != LB_D) return;
    const int l = em.a;
    for (int r = l; r < N; ++r) {
      if (l == 1 && r == 1) continue;
      emit(m, m, d_index(B, r), 2.0 * trace_ddd(B, l, l, r));
    }
    return;
  }
  const int a = em.a, b = em.b;
  for (int tn = kS; tn <= kJ; ++tn) {
    auto visit = [&](int u, int v) {
      const int64_t n = (int64_t)tn * B.P + pair_index(N, u, v);
      if (n < m) return;
      const Elem en = make_pair(tn, u, v);
      if (u == a && v == b) {  // same edge: the third element is a D_l
        if (which == LB_F && tn != em.kind) {
          for (int l = imax(a, 1); l <= b; ++l) {
            double f, d;
            fd_value(B, em, en, make_d(l), f, d);
            emit(m, n, d_index(B, l), f);
          }
        } else if (which == LB_D && tn == em.kind) {
          for (int l = imax(a, 1); l < N; ++l) {
            if (a == 0 && b == 1 && l == 1) continue;
            double f, d;
            fd_value(B, em, en, make_d(l), f, d);
            emit(m, n, d_index(B, l), d);
          }
        }
        return;
      }
      const int cv = common_vertex(em, en);
      int lo, hi;
      third_edge(em, en, cv, lo, hi);
      const int t3 = which == LB_F ? (1 ^ em.kind ^ tn) : (em.kind ^ tn);
      const int64_t s = (int64_t)t3 * B.P + pair_index(N, lo, hi);
      if (s < n) return;
      double f, d;
      fd_value(B, em, en, make_pair(t3, lo, hi), f, d);
      emit(m, n, s, which == LB_F ? f : d);
    };
    // edges sharing a vertex with (a,b), and (a,b) itself, in lexicographic order
    for (int x = 0; x < N - 1 && x <= b; ++x) {
      if (x < a) {
        visit(x, a);
        visit(x, b);
      } else if (x == a) {
        for (int y = a + 1; y < N; ++y) visit(a, y);
      } else if (x < b) {
        visit(x, b);
      } else {  // x == b
        for (int y = b + 1; y < N; ++y) visit(b, y);
      }
    }
  }
}

struct CountEmit {
  int64_t n = 0;
  __host__ __device__ void operator()(int64_t, int64_t, int64_t, double v) { n += (v != 0.0); }
};

struct FillEmit {
  int32_t* idx;
  double* val;
  int64_t off;
  __host__ __device__ void operator()(int64_t m, int64_t n, int64_t s, double v) {
    if (v == 0.0) return;
    idx[3 * off] = (int32_t)m;
    idx[3 * off + 1] = (int32_t)n;
    idx[3 * off + 2] = (int32_t)s;
    val[off] = v;
    ++off;
  }
};

__global__ void k_count(BasisView B, int which, int64_t* per_m) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= B.M) return;
  CountEmit e;
  for_each_canonical(B, m, which, e);
  per_m[m] = e.n;
}

__global__ void k_fill(BasisView B, int which, const int64_t* off, int32_t* idx, double* val) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= B.M) return;
  FillEmit e{idx, val, off[m]};
  for_each_canonical(B, m, which, e);
}

// Eq. (02): coef_j = Tr(F_j A) = sum_pq (F_j)_pq A_qp.
__global__ void k_expand(BasisView B, const double2* A, double2* coef) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= B.M) return;
  const int N = B.N;
  const Elem e = decode(B, j);
  double2 r;
  if (e.kind == kD) {
    const int l = e.a;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k <= l; ++k) {
      const double w = delta(B, k, l);
      const double2 x = A[(int64_t)k * N + k];
      sr += w * x.x;
      si += w * x.y;
    }
    r = make_double2(sr, si);
  } else {
    const double2 ab = A[(int64_t)e.a * N + e.b];  // A_ab
    const double2 ba = A[(int64_t)e.b * N + e.a];  // A_ba
    if (e.kind == kS) {
      // (A_ba + A_ab)/sqrt2
      r = make_double2(kInvSqrt2 * (ba.x + ab.x), kInvSqrt2 * (ba.y + ab.y));
    } else {
      // (-i A_ba + i A_ab)/sqrt2
      r = make_double2(kInvSqrt2 * (ba.y - ab.y), kInvSqrt2 * (ab.x - ba.x));
    }
  }
  coef[j] = r;
}

// Eq. (rho): rho = 1/N + sum_i v_i F_i.
__global__ void k_rho(BasisView B, const double* v, double2* out) {
  const int N = B.N;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int p = (int)(t / N), q = (int)(t % N);
  double2 r;
  if (p == q) {
    double s = 1.0 / N;
    for (int l = imax(p, 1); l < N; ++l) s += v[d_index(B, l)] * delta(B, p, l);
    r = make_double2(s, 0.0);
  } else {
    const int64_t pi = pair_index_any(N, p, q);
    const double vs = v[pi], vj = v[B.P + pi];
    // S contributes v_S/sqrt2 at (p,q) and (q,p); J_ab contributes -i v_J/sqrt2 at (a,b), +i at (b,a)
    const double sg = p < q ? -1.0 : 1.0;
    r = make_double2(kInvSqrt2 * vs, sg * kInvSqrt2 * vj);
  }
  out[t] = r;
}

inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

namespace lbi {

cudaError_t build_tables(int N, int32_t* pair_ab, double* tab, cudaStream_t st) {
  int64_t P = (int64_t)N * (N - 1) / 2;
  int64_t n = P > N + 1 ? P : N + 1;
  k_tables<<<nblocks(n, 256), 256, 0, st>>>(N, pair_ab, tab);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t structure_count(const lb::BasisView& B, int which, int64_t* per_m, cudaStream_t st) {
  k_count<<<nblocks(B.M, 128), 128, 0, st>>>(B, which, per_m);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t structure_fill(const lb::BasisView& B, int which, const int64_t* offsets,
                           int32_t* idx3, double* val, cudaStream_t st) {
  k_fill<<<nblocks(B.M, 128), 128, 0, st>>>(B, which, offsets, idx3, val);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t expand(const lb::BasisView& B, const double2* A, double2* coef, cudaStream_t st) {
  k_expand<<<nblocks(B.M, 256), 256, 0, st>>>(B, A, coef);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t rho(const lb::BasisView& B, const double* v, double2* out, cudaStream_t st) {
  k_rho<<<nblocks((int64_t)B.N * B.N, 256), 256, 0, st>>>(B, v, out);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace lbi

// lb_basis.cu -- kernel (a): index-arithmetic enumeration of the nonzero
// structure constants f_mns, d_mns (Eq. (05); Table 1 step 2.2), plus the
// basis index tables, the expansion of Eq. (02) and the reconstruction of
// Eq. (rho).
//
// Canonical lists hold each unordered triple once as m <= n <= s, sorted by
// (m, n, s).  Row m's partners n come in increasing index order and for each
// the third indices s >= n in increasing order, so a count pass, an
// exclusive scan over m and a fill pass give the sorted list without any
// sort.  The nonzero triples fall into three classes:
//   * three pair elements whose edges form a triangle a-b-c: for given
//     types of two of them the type of the third is fixed by parity (f: odd
//     number of J's, d: even);
//   * two pair elements on one edge (a,b) and D_l: f(S_ab, J_ab, D_l) != 0
//     for max(a,1) <= l <= b; d(S_ab, S_ab, D_l) = d(J_ab, J_ab, D_l) != 0
//     for l >= max(a,1) except (a,b,l) = (0,1,1);
//   * d(D_l, D_l, D_r) for r >= l except l = r = 1 (canonical form of the
//     "two smallest equal" rule).
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

// One warp per row m.  The candidates of a row are laid out as a sequence of
// slots whose (n, s) order is the canonical order; the warp takes 32 slots at
// a time, each lane evaluates one, and a ballot gives each nonzero its place,
// so the output of a row is written in order by consecutive lanes.
//
// Pair row m = (k, a, b).  For each partner type tn >= k (tn < k gives n < m)
// the partners are the 2N-3 edges that share a vertex with (a,b) or equal it,
// in lexicographic order:
//   e <  2a           : (e/2, a) for even e, (e/2, b) for odd e
//   2a <= e < a+N-1   : (a, e-a+1)           -- holds (a,b) itself at e = a+b-1
//   a+N-1 <= e < N+b-2: (e-N+2, b)
//   N+b-2 <= e < 2N-3 : (b, e-N+3)
// The slot of (a,b) itself is replaced by the run of D_l it pairs with:
// f(S_ab, J_ab, D_l) for max(a,1) <= l <= b when tn != k, d(X_ab, X_ab, D_l)
// for max(a,1) <= l < N when tn == k (the zero at (a,b,l) = (0,1,1) is
// dropped by the value test).  With tn == k the row starts at (a,b).
// A shared-vertex partner fixes the third edge and, by parity, its type; the
// triple is canonical when s >= n.
//
// Diagonal row m = D_l (d only): d(D_l, D_l, D_r) for r >= l; the zero at
// l = r = 1 is dropped by the value test.
struct PairPlan {
  int pab;    // slot of the edge (a,b): a + b - 1
  int first;  // first slot of the row
  int lo, nl; // D run l = lo .. lo + nl - 1
  int total;  // slots: 2N-4 edges + nl
};

__device__ __forceinline__ PairPlan pair_plan(int N, const Elem& em, int tn, int which) {
  PairPlan p;
  p.pab = em.a + em.b - 1;
  p.first = tn == em.kind ? p.pab : 0;
  p.lo = imax(em.a, 1);
  if (which == LB_F) p.nl = tn != em.kind ? em.b - p.lo + 1 : 0;
  else p.nl = tn == em.kind ? N - p.lo : 0;
  p.total = 2 * N - 4 + p.nl;
  return p;
}

__device__ __forceinline__ void edge_of_slot(int N, int a, int b, int e, int& u, int& v) {
  if (e < 2 * a) {
    u = e >> 1;
    v = (e & 1) ? b : a;
  } else if (e < a + N - 1) {
    u = a;
    v = e - a + 1;
  } else if (e < N + b - 2) {
    u = e - N + 2;
    v = b;
  } else {
    u = b;
    v = e - N + 3;
  }
}

// Evaluate slot j of a pair row: (n, s, value); false when the slot holds no
// canonical triple.
__device__ __forceinline__ bool pair_slot(const BasisView& B, const Elem& em, int tn, int which,
                                          const PairPlan& p, int j, int64_t& n, int64_t& s, double& val) {
  const int N = B.N;
  double f, d;
  if (j >= p.pab && j < p.pab + p.nl) {
    const int l = p.lo + (j - p.pab);
    n = (int64_t)tn * B.P + pair_index(N, em.a, em.b);
    s = d_index(B, l);
    fd_value(B, em, make_pair(tn, em.a, em.b), make_d(l), f, d);
  } else {
    int u, v;
    edge_of_slot(N, em.a, em.b, j < p.pab ? j : j - p.nl + 1, u, v);
    n = (int64_t)tn * B.P + pair_index(N, u, v);
    const Elem en = make_pair(tn, u, v);
    int lo, hi;
    third_edge(em, en, common_vertex(em, en), lo, hi);
    const int t3 = which == LB_F ? (1 ^ em.kind ^ tn) : (em.kind ^ tn);
    s = (int64_t)t3 * B.P + pair_index(N, lo, hi);
    if (s < n) return false;
    fd_value(B, em, en, make_pair(t3, lo, hi), f, d);
  }
  val = which == LB_F ? f : d;
  return val != 0.0;
}

// FILL = false: per_m[m] = number of nonzero canonical triples of row m.
// FILL = true : write row m's triples from offset off[m].
template <bool FILL>
__global__ void __launch_bounds__(256) k_rows(BasisView B, int which, int64_t* per_m, const int64_t* off,
                                              int32_t* idx, double* val) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (m >= B.M) return;  // whole warps leave together
  const Elem em = decode(B, m);
  const int N = B.N;
  int64_t pos = FILL ? off[m] : 0;
  auto take = [&](bool nz, int64_t n, int64_t s, double v) {
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (FILL && nz) {
      const int64_t o = pos + __popc(bal & below);
      idx[3 * o] = (int32_t)m;
      idx[3 * o + 1] = (int32_t)n;
      idx[3 * o + 2] = (int32_t)s;
      val[o] = v;
    }
    pos += __popc(bal);
  };
  if (em.kind == kD) {
    if (which == LB_D) {
      const int l = em.a;
      for (int r0 = l; r0 < N; r0 += 32) {
        const int r = r0 + lane;
        const double v = r < N ? 2.0 * trace_ddd(B, l, l, r) : 0.0;
        take(v != 0.0, m, d_index(B, r < N ? r : l), v);
      }
    }
  } else {
    for (int tn = em.kind; tn <= kJ; ++tn) {
      const PairPlan p = pair_plan(N, em, tn, which);
      for (int j0 = p.first; j0 < p.total; j0 += 32) {
        const int j = j0 + lane;
        int64_t n = 0, s = 0;
        double v = 0.0;
        const bool nz = j < p.total && pair_slot(B, em, tn, which, p, j, n, s, v);
        take(nz, n, s, v);
      }
    }
  }
  if (!FILL && lane == 0) per_m[m] = pos;
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
__global__ void k_rho(BasisView B, const double* v, double2* out, double id) {
  const int N = B.N;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int p = (int)(t / N), q = (int)(t % N);
  double2 r;
  if (p == q) {
    double s = id;
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
  k_rows<false><<<nblocks(B.M * 32, 256), 256, 0, st>>>(B, which, per_m, nullptr, nullptr, nullptr);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t structure_fill(const lb::BasisView& B, int which, const int64_t* offsets,
                           int32_t* idx3, double* val, cudaStream_t st) {
  k_rows<true><<<nblocks(B.M * 32, 256), 256, 0, st>>>(B, which, nullptr, offsets, idx3, val);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t expand(const lb::BasisView& B, const double2* A, double2* coef, cudaStream_t st) {
  k_expand<<<nblocks(B.M, 256), 256, 0, st>>>(B, A, coef);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t rho(const lb::BasisView& B, const double* v, double2* out, cudaStream_t st) {
  k_rho<<<nblocks((int64_t)B.N * B.N, 256), 256, 0, st>>>(B, v, out, 1.0 / B.N);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t synth(const lb::BasisView& B, const double* v, double2* out, cudaStream_t st) {
  k_rho<<<nblocks((int64_t)B.N * B.N, 256), 256, 0, st>>>(B, v, out, 0.0);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace lbi

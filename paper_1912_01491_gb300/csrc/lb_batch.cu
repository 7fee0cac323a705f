// lb_batch.cu -- the batched form: many independent realizations of mixed N
// (the paper's Sec. 6 ensemble of random Lindbladians: one sample per group
// of processors, trivially parallel), assembled and then integrated by one
// persistent launch per cluster-size group.
//
// Integration: a thread-block cluster owns one realization at a time (taken
// from a global counter by the cluster's rank-0 block).  Each block of the
// cluster owns a contiguous slice of rows; its slice of the FP32 matrix stays
// in shared memory for the whole 4 x nsteps stages when it fits, else it is
// re-read from global memory (L2) every stage.  Each block keeps the whole
// stage vector in its shared memory, double-buffered: while it reads one copy
// for the product, the epilogue of every row stores the row's next-stage
// value into the other copy of every block of the cluster (distributed
// shared memory stores, one lane per destination block), and one cluster
// barrier per stage orders those stores before the next stage reads them.
// State, stage combination and the FP64 defect correction stay FP64, as in
// the single-system kernels.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lb_internal.h"

namespace cg = cooperative_groups;

namespace {

using BItem = lbi::BatchItem;

struct SmemLayout {
  int64_t slice, mmax;
  bool resident;
  size_t off_x32, off_x64, off_v, off_acc, off_keff, off_r, off_item, total;
};

inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

SmemLayout layout(int64_t mmax, int C, bool resident) {
  SmemLayout L;
  L.mmax = mmax;
  L.slice = (mmax + C - 1) / C;
  L.resident = resident;
  size_t o = 0;
  L.off_item = o; o = a16(o + 16);
  L.off_x32 = o; o = a16(o + sizeof(float) * 2 * mmax);
  L.off_x64 = o; o = a16(o + sizeof(double) * mmax);
  L.off_v = o; o = a16(o + sizeof(double) * L.slice);
  L.off_acc = o; o = a16(o + sizeof(double) * L.slice);
  L.off_keff = o; o = a16(o + sizeof(double) * L.slice);
  L.off_r = o;
  if (resident) o = a16(o + sizeof(float) * L.slice * mmax);
  L.total = o;
  return L;
}

// Classical RK4 stage epilogue for one row (Table 1 step 3.1): k = A x + K,
// acc and the next stage input as in the single-system kernels.
__device__ __forceinline__ double stage_update(int stage, double k, double vi, double acci, double dt,
                                               double* acc_out, double* v_out) {
  if (stage == 1) {
    *acc_out = k;
    return vi + 0.5 * dt * k;
  }
  if (stage == 2) {
    *acc_out = acci + 2.0 * k;
    return vi + 0.5 * dt * k;
  }
  if (stage == 3) {
    *acc_out = acci + 2.0 * k;
    return vi + dt * k;
  }
  const double nx = vi + (dt / 6.0) * (acci + k);
  *v_out = nx;
  return nx;
}

// Lanes per row: small rows are shared by fewer lanes so that one warp
// instruction of the FP64 epilogue serves 32 / W rows.
__device__ __forceinline__ int row_group_width(int64_t M) {
  return M >= 256 ? 32 : M >= 96 ? 16 : M >= 32 ? 8 : 4;
}

// Multiply-add in the element type (an explicit FP32 FMA for float, so that
// no operand is promoted to FP64).
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }

// Partial dot product of one lane of a W-lane row group.  Full-warp rows use
// a compile-time stride, which the compiler unrolls with the loads of several
// iterations in flight (long rows stream from L2); short rows use W lanes.
template <class T>
__device__ __forceinline__ T group_dot(const T* __restrict__ row, const T* __restrict__ x, int64_t M, int sub,
                                       int W) {
  T a = T(0);
  if (W == 32) {
    for (int64_t n = sub; n < M; n += 32) a = mad(row[n], x[n], a);
  } else {
    for (int64_t n = sub; n < M; n += W) a = mad(row[n], x[n], a);
  }
  return a;
}

// Takes the next realization for this cluster; every block returns the same
// queue position.
__device__ __forceinline__ int next_item(cg::cluster_group& cluster, int rank, int* item_slot, int* counter) {
  if (rank == 0 && threadIdx.x == 0) *item_slot = atomicAdd(counter, 1);
  cluster.sync();
  const int qi = *cluster.map_shared_rank(item_slot, 0);
  cluster.sync();  // every block has read the slot before rank 0 may overwrite it
  return qi;
}

__global__ void __launch_bounds__(256, 4) k_rk4_batch(const BItem* __restrict__ items, const int* __restrict__ order,
                                                   int nitems, int* __restrict__ counter, int64_t nsteps, double dt,
                                                   int correct_every, SmemLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  int* item_slot = reinterpret_cast<int*>(smem + L.off_item);
  float* x32 = reinterpret_cast<float*>(smem + L.off_x32);  // [2][mmax]
  double* x64 = reinterpret_cast<double*>(smem + L.off_x64);
  double* vv = reinterpret_cast<double*>(smem + L.off_v);
  double* acc = reinterpret_cast<double*>(smem + L.off_acc);
  double* keff = reinterpret_cast<double*>(smem + L.off_keff);
  float* Rs = reinterpret_cast<float*>(smem + L.off_r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t mmax = L.mmax;
  while (true) {
    const int qi = next_item(cluster, rank, item_slot, counter);
    if (qi >= nitems) break;
    const BItem it = items[order[qi]];
    const int64_t M = it.M;
    const int64_t slice = (M + C - 1) / C;
    const int64_t r0 = rank * slice, r1 = r0 + slice < M ? r0 + slice : M;
    const int64_t nrow = r1 > r0 ? r1 - r0 : 0;
    const bool resident = L.resident;
    const bool correct = correct_every > 0 && it.A64 != nullptr;
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) {
      vv[i] = it.v[r0 + i];
      keff[i] = it.K[r0 + i];
    }
    if (resident)
      for (int64_t e = threadIdx.x; e < nrow * M; e += blockDim.x) Rs[e] = it.A32[r0 * M + e];
    for (int64_t n = threadIdx.x; n < M; n += blockDim.x) {
      x32[n] = (float)it.v[n];
      x64[n] = it.v[n];
    }
    __syncthreads();
    for (int64_t t = 0; t < nsteps; ++t) {
      if (correct && t % correct_every == 0) {
        // FP64 defect c = (A64 - A32) v on own rows, with the full current v in x64
        for (int64_t i = warp; i < nrow; i += nw) {
          const int64_t s = r0 + i;
          double c = 0.0;
          for (int64_t n = lane; n < M; n += 32)
            c = fma(it.A64[s * M + n] - (double)it.A32[s * M + n], x64[n], c);
          for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
          if (lane == 0) keff[i] = it.K[s] + c;
        }
        __syncthreads();
      }
      const bool push64 = correct && (t + 1) % correct_every == 0;
      const int W = row_group_width(M), G = 32 / W, g = lane / W, sub = lane % W;
      for (int stage = 1; stage <= 4; ++stage) {
        const float* xc = x32 + ((stage - 1) & 1) * mmax;
        float* xn = x32 + (stage & 1) * mmax;
        for (int64_t i0 = (int64_t)warp * G; i0 < nrow; i0 += (int64_t)nw * G) {
          const int64_t i = i0 + g;
          const bool valid = i < nrow;  // every lane reaches the shuffles
          float a = 0.f;
          if (valid) {
            const float* row = resident ? Rs + i * M : it.A32 + (r0 + i) * M;
            a = group_dot(row, xc, M, sub, W);
          }
          for (int o = W >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          // every lane of the group holds the row sum: all form the update,
          // lane 0 of the group keeps the state, lanes store the value into
          // blocks sub, sub + W, ...
          const double vi = valid ? vv[i] : 0.0, ai = valid ? acc[i] : 0.0, ki = valid ? keff[i] : 0.0;
          __syncwarp();
          if (valid) {
            double acc_new = ai, v_new = vi;
            const double nx = stage_update(stage, (double)a + ki, vi, ai, dt, &acc_new, &v_new);
            if (sub == 0) {
              acc[i] = acc_new;
              vv[i] = v_new;
            }
            for (int q = sub; q < C; q += W) {
              *cluster.map_shared_rank(xn + r0 + i, q) = (float)nx;
              if (stage == 4 && push64) *cluster.map_shared_rank(x64 + r0 + i, q) = nx;
            }
          }
        }
        cluster.sync();  // every block's copy of the next stage vector is complete
      }
    }
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) it.v[r0 + i] = vv[i];
    cluster.sync();  // all blocks are done with this realization's buffers
  }
}

// FP64 form of the same kernel: the matrix slice (resident or streamed) and
// the exchanged stage vector are FP64, products are FP64 FMAs and there is
// no correction.  For small M the per-stage work is a few microseconds, so
// one persistent launch replaces 4 launches per step.
struct SmemLayout64 {
  int64_t slice, mmax;
  bool resident;
  size_t off_item, off_x, off_v, off_acc, off_keff, off_r, total;
};

SmemLayout64 layout64(int64_t mmax, int C, bool resident) {
  SmemLayout64 L;
  L.mmax = mmax;
  L.slice = (mmax + C - 1) / C;
  L.resident = resident;
  size_t o = 0;
  L.off_item = o; o = a16(o + 16);
  L.off_x = o; o = a16(o + sizeof(double) * 2 * mmax);
  L.off_v = o; o = a16(o + sizeof(double) * L.slice);
  L.off_acc = o; o = a16(o + sizeof(double) * L.slice);
  L.off_keff = o; o = a16(o + sizeof(double) * L.slice);
  L.off_r = o;
  if (resident) o = a16(o + sizeof(double) * L.slice * mmax);
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(256, 4) k_rk4_batch64(const BItem* __restrict__ items, const int* __restrict__ order,
                                                     int nitems, int* __restrict__ counter, int64_t nsteps,
                                                     double dt, SmemLayout64 L) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  int* item_slot = reinterpret_cast<int*>(smem + L.off_item);
  double* x = reinterpret_cast<double*>(smem + L.off_x);  // [2][mmax]
  double* vv = reinterpret_cast<double*>(smem + L.off_v);
  double* acc = reinterpret_cast<double*>(smem + L.off_acc);
  double* keff = reinterpret_cast<double*>(smem + L.off_keff);
  double* Rs = reinterpret_cast<double*>(smem + L.off_r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t mmax = L.mmax;
  while (true) {
    const int qi = next_item(cluster, rank, item_slot, counter);
    if (qi >= nitems) break;
    const BItem it = items[order[qi]];
    const int64_t M = it.M;
    const int64_t slice = (M + C - 1) / C;
    const int64_t r0 = rank * slice, r1 = r0 + slice < M ? r0 + slice : M;
    const int64_t nrow = r1 > r0 ? r1 - r0 : 0;
    const bool resident = L.resident;
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) {
      vv[i] = it.v[r0 + i];
      keff[i] = it.K[r0 + i];
    }
    if (resident)
      for (int64_t e = threadIdx.x; e < nrow * M; e += blockDim.x) Rs[e] = it.A64[r0 * M + e];
    for (int64_t n = threadIdx.x; n < M; n += blockDim.x) x[n] = it.v[n];
    __syncthreads();
    const int W = row_group_width(M), G = 32 / W, g = lane / W, sub = lane % W;
    for (int64_t t = 0; t < nsteps; ++t) {
      for (int stage = 1; stage <= 4; ++stage) {
        const double* xc = x + ((stage - 1) & 1) * mmax;
        double* xn = x + (stage & 1) * mmax;
        for (int64_t i0 = (int64_t)warp * G; i0 < nrow; i0 += (int64_t)nw * G) {
          const int64_t i = i0 + g;
          const bool valid = i < nrow;
          double a = 0.0;
          if (valid) {
            const double* row = resident ? Rs + i * M : it.A64 + (r0 + i) * M;
            a = group_dot(row, xc, M, sub, W);
          }
          for (int o = W >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          const double vi = valid ? vv[i] : 0.0, ai = valid ? acc[i] : 0.0, ki = valid ? keff[i] : 0.0;
          __syncwarp();
          if (valid) {
            double acc_new = ai, v_new = vi;
            const double nx = stage_update(stage, a + ki, vi, ai, dt, &acc_new, &v_new);
            if (sub == 0) {
              acc[i] = acc_new;
              vv[i] = v_new;
            }
            for (int q = sub; q < C; q += W) *cluster.map_shared_rank(xn + r0 + i, q) = nx;
          }
        }
        cluster.sync();
      }
    }
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) it.v[r0 + i] = vv[i];
    cluster.sync();
  }
}


// ---------------------------------------------------------------------------
// Propagator form (lb_prop.cu): one step is v <- v + h (D' v + c'), one
// product with the matrix and one exchange of the state per step.  The
// cluster layout is that of k_rk4_batch: each block owns a slice of rows and
// keeps its slice of D' in shared memory when it fits.
//   FP32: D' stored in FP32 (D32 = fl(A32 + R32), R32 = D' - A in FP32),
//     products FP32 FMAs of the FP32-rounded state, state FP64.  Every
//     correct_every steps the FP64 defect d = (A64 + R32 - D32) v is formed
//     from the FP64 state and added to c' until the next one: A64 - A32 is
//     the storage error of A and A32 + R32 - D32 the rounding of the sum,
//     the two FP32 errors of D' to first order (R32's own rounding is h|A|
//     times smaller).
//   FP64: D' in FP64, FP64 products, no correction.
struct PItem {
  int64_t M;
  const float* D32;   // FP32 form: D' (M x M)
  const float* R32;   // FP32 form: D' - A in FP32, for the correction
  const double* A64;  // FP32 form with correction: A; FP64 form: D' (FP64)
  const double* cp;   // c' (M)
  double* v;          // M, in/out
};

struct SmemLayoutP {
  int64_t slice, mmax;
  bool resident;
  size_t off_item, off_x32, off_x64, off_v, off_keff, off_r, total;
};

SmemLayoutP layoutP(int64_t mmax, int C, bool resident, bool f64) {
  SmemLayoutP L;
  L.mmax = mmax;
  L.slice = (mmax + C - 1) / C;
  L.resident = resident;
  size_t o = 0;
  L.off_item = o; o = a16(o + 16);
  L.off_x32 = o; o = a16(o + (f64 ? 0 : sizeof(float) * 2 * mmax));
  L.off_x64 = o; o = a16(o + sizeof(double) * (f64 ? 2 : 1) * mmax);
  L.off_v = o; o = a16(o + sizeof(double) * L.slice);
  L.off_keff = o; o = a16(o + sizeof(double) * L.slice);
  L.off_r = o;
  if (resident) o = a16(o + (f64 ? sizeof(double) : sizeof(float)) * L.slice * mmax);
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(256, 4) k_prop_batch(const PItem* __restrict__ items, const int* __restrict__ order,
                                                    int nitems, int* __restrict__ counter, int64_t nsteps, double h,
                                                    int correct_every, SmemLayoutP L) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  int* item_slot = reinterpret_cast<int*>(smem + L.off_item);
  float* x32 = reinterpret_cast<float*>(smem + L.off_x32);  // [2][mmax]
  double* x64 = reinterpret_cast<double*>(smem + L.off_x64);
  double* vv = reinterpret_cast<double*>(smem + L.off_v);
  double* keff = reinterpret_cast<double*>(smem + L.off_keff);
  float* Ds = reinterpret_cast<float*>(smem + L.off_r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t mmax = L.mmax;
  while (true) {
    const int qi = next_item(cluster, rank, item_slot, counter);
    if (qi >= nitems) break;
    const PItem it = items[order[qi]];
    const int64_t M = it.M;
    const int64_t slice = (M + C - 1) / C;
    const int64_t r0 = rank * slice, r1 = r0 + slice < M ? r0 + slice : M;
    const int64_t nrow = r1 > r0 ? r1 - r0 : 0;
    const bool resident = L.resident;
    const bool correct = correct_every > 0 && it.A64 != nullptr && it.R32 != nullptr;
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) {
      vv[i] = it.v[r0 + i];
      keff[i] = it.cp[r0 + i];
    }
    if (resident)
      for (int64_t e = threadIdx.x; e < nrow * M; e += blockDim.x) Ds[e] = it.D32[r0 * M + e];
    for (int64_t n = threadIdx.x; n < M; n += blockDim.x) {
      x32[n] = (float)it.v[n];
      x64[n] = it.v[n];
    }
    __syncthreads();
    const int W = row_group_width(M), G = 32 / W, g = lane / W, sub = lane % W;
    for (int64_t t = 0; t < nsteps; ++t) {
      if (correct && t % correct_every == 0) {
        // FP64 defect d = (A64 + R32 - D32) v on own rows
        for (int64_t i = warp; i < nrow; i += nw) {
          const int64_t s = r0 + i;
          double d = 0.0;
          for (int64_t n = lane; n < M; n += 32) {
            const int64_t q = s * M + n;
            d = fma((it.A64[q] + (double)it.R32[q]) - (double)it.D32[q], x64[n], d);
          }
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          if (lane == 0) keff[i] = it.cp[s] + d;
        }
        __syncthreads();
      }
      const bool push64 = correct && (t + 1) % correct_every == 0;
      const float* xc = x32 + (t & 1) * mmax;
      float* xn = x32 + ((t + 1) & 1) * mmax;
      for (int64_t i0 = (int64_t)warp * G; i0 < nrow; i0 += (int64_t)nw * G) {
        const int64_t i = i0 + g;
        const bool valid = i < nrow;  // every lane reaches the shuffles
        float a = 0.f;
        if (valid) {
          const float* row = resident ? Ds + i * M : it.D32 + (r0 + i) * M;
          a = group_dot(row, xc, M, sub, W);
        }
        for (int o = W >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const double vi = valid ? vv[i] : 0.0, ki = valid ? keff[i] : 0.0;
        __syncwarp();
        if (valid) {
          const double nx = fma(h, (double)a + ki, vi);
          if (sub == 0) vv[i] = nx;
          for (int q = sub; q < C; q += W) {
            *cluster.map_shared_rank(xn + r0 + i, q) = (float)nx;
            if (push64) *cluster.map_shared_rank(x64 + r0 + i, q) = nx;
          }
        }
      }
      cluster.sync();  // every block's copy of the next state is complete
    }
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) it.v[r0 + i] = vv[i];
    cluster.sync();  // all blocks are done with this realization's buffers
  }
}

__global__ void __launch_bounds__(256, 4) k_prop_batch64(const PItem* __restrict__ items,
                                                      const int* __restrict__ order, int nitems,
                                                      int* __restrict__ counter, int64_t nsteps, double h,
                                                      SmemLayoutP L) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  int* item_slot = reinterpret_cast<int*>(smem + L.off_item);
  double* x = reinterpret_cast<double*>(smem + L.off_x64);  // [2][mmax]
  double* vv = reinterpret_cast<double*>(smem + L.off_v);
  double* keff = reinterpret_cast<double*>(smem + L.off_keff);
  double* Ds = reinterpret_cast<double*>(smem + L.off_r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t mmax = L.mmax;
  while (true) {
    const int qi = next_item(cluster, rank, item_slot, counter);
    if (qi >= nitems) break;
    const PItem it = items[order[qi]];
    const int64_t M = it.M;
    const int64_t slice = (M + C - 1) / C;
    const int64_t r0 = rank * slice, r1 = r0 + slice < M ? r0 + slice : M;
    const int64_t nrow = r1 > r0 ? r1 - r0 : 0;
    const bool resident = L.resident;
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) {
      vv[i] = it.v[r0 + i];
      keff[i] = it.cp[r0 + i];
    }
    if (resident)
      for (int64_t e = threadIdx.x; e < nrow * M; e += blockDim.x) Ds[e] = it.A64[r0 * M + e];
    for (int64_t n = threadIdx.x; n < M; n += blockDim.x) x[n] = it.v[n];
    __syncthreads();
    const int W = row_group_width(M), G = 32 / W, g = lane / W, sub = lane % W;
    for (int64_t t = 0; t < nsteps; ++t) {
      const double* xc = x + (t & 1) * mmax;
      double* xn = x + ((t + 1) & 1) * mmax;
      for (int64_t i0 = (int64_t)warp * G; i0 < nrow; i0 += (int64_t)nw * G) {
        const int64_t i = i0 + g;
        const bool valid = i < nrow;
        double a = 0.0;
        if (valid) {
          const double* row = resident ? Ds + i * M : it.A64 + (r0 + i) * M;
          a = group_dot(row, xc, M, sub, W);
        }
        for (int o = W >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const double vi = valid ? vv[i] : 0.0, ki = valid ? keff[i] : 0.0;
        __syncwarp();
        if (valid) {
          const double nx = fma(h, a + ki, vi);
          if (sub == 0) vv[i] = nx;
          for (int q = sub; q < C; q += W) *cluster.map_shared_rank(xn + r0 + i, q) = nx;
        }
      }
      cluster.sync();
    }
    for (int64_t i = threadIdx.x; i < nrow; i += blockDim.x) it.v[r0 + i] = vv[i];
    cluster.sync();
  }
}
}  // namespace

struct lb_batch {
  int count = 0;
  std::vector<int> N;
  std::vector<int64_t> M;
  std::vector<const double*> a, h;  // caller-owned device inputs
  std::vector<double*> v;           // caller-owned device state
  std::vector<lb_basis_t*> basis;   // one per distinct N (owned)
  std::vector<int> basis_of;
  std::vector<double*> A64, K;
  std::vector<float*> A32;
  std::vector<int> cluster;  // chosen cluster size per realization
  int precision = LB_FP32;   // storage and arithmetic of the integration
  int form = LB_FORM_RK4;    // stage-by-stage RK4 or the propagator form
  // propagator form, made for step prop_dt and precision prop_prec
  double prop_dt = 0.0;
  int prop_prec = -1;
  std::vector<float*> D32, R32;  // FP32: D' and D' - A
  std::vector<double*> D64, cp;  // FP64: D'; both: c'
  float prop_ms = 0.f;           // device time of the last formation
  BItem* d_items = nullptr;
  int* d_order = nullptr;
  int* d_counter = nullptr;
  void* d_prop_items = nullptr;
};

namespace lbi {

cudaError_t batch_alloc(lb_batch* b) {
  for (int r = 0; r < b->count; ++r) {
    const size_t mm = (size_t)b->M[r] * (size_t)b->M[r];
    cudaError_t e;
    if ((e = cudaMalloc(&b->A64[r], 8 * mm)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b->A32[r], 4 * mm)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b->K[r], 8 * (size_t)b->M[r])) != cudaSuccess) return e;
  }
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_items, sizeof(BItem) * b->count)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&b->d_order, sizeof(int) * b->count)) != cudaSuccess) return e;
  return cudaMalloc(&b->d_counter, sizeof(int) * 8);
}

void prop_free(lb_batch* b) {
  for (auto* p : b->D32) cudaFree(p);
  for (auto* p : b->R32) cudaFree(p);
  for (auto* p : b->D64) cudaFree(p);
  for (auto* p : b->cp) cudaFree(p);
  b->D32.clear();
  b->R32.clear();
  b->D64.clear();
  b->cp.clear();
  cudaFree(b->d_prop_items);
  b->d_prop_items = nullptr;
  b->prop_prec = -1;
}

void batch_free(lb_batch* b) {
  prop_free(b);
  for (int r = 0; r < b->count; ++r) {
    cudaFree(b->A64[r]);
    cudaFree(b->A32[r]);
    cudaFree(b->K[r]);
  }
  cudaFree(b->d_items);
  cudaFree(b->d_order);
  cudaFree(b->d_counter);
}

cudaError_t batch_assemble(lb_batch* b, const std::vector<lb::BasisView>& views, int algorithm, cudaStream_t st) {
  for (int r = 0; r < b->count; ++r) {
    const lb::BasisView& B = views[b->basis_of[r]];
    cudaError_t e = assemble_dense(B, b->h[r], reinterpret_cast<const double2*>(b->a[r]), b->A64[r], nullptr,
                                   nullptr, b->K[r], algorithm, st);
    if (e != cudaSuccess) return e;
    if ((e = pack_fp32(b->M[r], b->A64[r], b->A32[r], st)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// D' and c' of every realization for step h in the batch's precision
// (lb_prop.cu): G0 = A + (h/4) A A, G1 = A + (h/3) A G0, R' = (h/2) A G1,
// D' = A + R' (FP32 from A32, or FP64 from A64); c' from A64 in FP64.
cudaError_t batch_form_propagator(lb_batch* b, double h, cudaStream_t st) {
  const bool f64 = b->precision == LB_FP64;
  if (b->prop_prec != -1 && b->prop_prec == b->precision && b->prop_dt == h) return cudaSuccess;
  prop_free(b);
  const int n = b->count;
  cudaError_t e = cudaSuccess;
  b->cp.assign(n, nullptr);
  if (f64) {
    b->D64.assign(n, nullptr);
  } else {
    b->D32.assign(n, nullptr);
    b->R32.assign(n, nullptr);
  }
  std::vector<void*> tmp;
  auto scratch_free = [&]() {
    for (auto* p : tmp) cudaFree(p);
    tmp.clear();
  };
  for (int r = 0; r < n && e == cudaSuccess; ++r) {
    const size_t mm = (size_t)b->M[r] * (size_t)b->M[r];
    e = cudaMalloc(&b->cp[r], 8 * (size_t)b->M[r]);
    if (e == cudaSuccess) e = f64 ? cudaMalloc(&b->D64[r], 8 * mm) : cudaMalloc(&b->D32[r], 4 * mm);
    if (e == cudaSuccess && !f64) e = cudaMalloc(&b->R32[r], 4 * mm);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_prop_items, sizeof(PItem) * n);
  // scratch: G0, G1 per realization, the job lists, the GEMV vectors
  std::vector<void*> G0(n, nullptr), G1(n, nullptr), u(n, nullptr);
  const size_t esz = f64 ? 8 : 4;
  for (int r = 0; r < n && e == cudaSuccess; ++r) {
    const size_t mm = (size_t)b->M[r] * (size_t)b->M[r];
    if ((e = cudaMalloc(&G0[r], esz * mm)) == cudaSuccess) tmp.push_back(G0[r]);
    if (e == cudaSuccess && (e = cudaMalloc(&G1[r], esz * mm)) == cudaSuccess) tmp.push_back(G1[r]);
    if (e == cudaSuccess && (e = cudaMalloc(&u[r], 16 * (size_t)b->M[r])) == cudaSuccess) tmp.push_back(u[r]);
  }
  const size_t sb = std::max(batch_gemm_scratch_bytes(b->M), sizeof(GemvJob) * (size_t)n + 256);
  void* js = nullptr;
  if (e == cudaSuccess && (e = cudaMalloc(&js, sb)) == cudaSuccess) tmp.push_back(js);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(t0, st);
  // the three products
  for (int step = 0; step < 3 && e == cudaSuccess; ++step) {
    const double alpha = step == 0 ? h / 4.0 : step == 1 ? h / 3.0 : h / 2.0;
    if (f64) {
      std::vector<GemmJob<double>> jobs;
      for (int r = 0; r < n; ++r) {
        const double* A = b->A64[r];
        const double* G = step == 0 ? A : step == 1 ? static_cast<double*>(G0[r]) : static_cast<double*>(G1[r]);
        double* Y = step == 0 ? static_cast<double*>(G0[r]) : step == 1 ? static_cast<double*>(G1[r]) : b->D64[r];
        jobs.push_back(GemmJob<double>{b->M[r], A, G, step == 2 ? nullptr : A, Y, alpha});
      }
      e = batch_gemm<double>(jobs, js, sb, st);
    } else {
      std::vector<GemmJob<float>> jobs;
      for (int r = 0; r < n; ++r) {
        const float* A = b->A32[r];
        const float* G = step == 0 ? A : step == 1 ? static_cast<float*>(G0[r]) : static_cast<float*>(G1[r]);
        float* Y = step == 0 ? static_cast<float*>(G0[r]) : step == 1 ? static_cast<float*>(G1[r]) : b->R32[r];
        jobs.push_back(GemmJob<float>{b->M[r], A, G, step == 2 ? nullptr : A, Y, (float)alpha});
      }
      e = batch_gemm<float>(jobs, js, sb, st);
    }
  }
  // D' = A + R'
  for (int r = 0; r < n && e == cudaSuccess; ++r) {
    const int64_t mm = b->M[r] * b->M[r];
    e = f64 ? add64(b->A64[r], b->D64[r], b->D64[r], mm, st) : add32(b->A32[r], b->R32[r], b->D32[r], mm, st);
  }
  // c' = K + (h/2) A (K + (h/3) A (K + (h/4) A K)) in FP64
  for (int step = 0; step < 3 && e == cudaSuccess; ++step) {
    const double alpha = step == 0 ? h / 4.0 : step == 1 ? h / 3.0 : h / 2.0;
    std::vector<GemvJob> jobs;
    for (int r = 0; r < n; ++r) {
      double* ua = static_cast<double*>(u[r]);
      double* ub = ua + b->M[r];
      const double* x = step == 0 ? b->K[r] : step == 1 ? ua : ub;
      double* y = step == 0 ? ua : step == 1 ? ub : b->cp[r];
      jobs.push_back(GemvJob{b->M[r], b->A64[r], x, b->K[r], y, alpha});
    }
    e = batch_gemv64(jobs, js, sb, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(t1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&b->prop_ms, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  scratch_free();
  if (e != cudaSuccess) {
    prop_free(b);
    return e;
  }
  b->prop_dt = h;
  b->prop_prec = b->precision;
  return cudaSuccess;
}

int smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Shared-memory layout for (mmax, C): resident when the slice fits, else
// streamed; total 0 if even the streamed layout does not fit.
SmemLayout pick_layout(int64_t mmax, int C) {
  const size_t cap = (size_t)smem_optin();
  SmemLayout L = layout(mmax, C, true);
  if (L.total > cap) L = layout(mmax, C, false);
  if (L.total > cap) L.total = 0;
  return L;
}

SmemLayoutP pick_layoutP(int64_t mmax, int C, bool f64) {
  const size_t cap = (size_t)smem_optin();
  SmemLayoutP L = layoutP(mmax, C, true, f64);
  if (L.total > cap) L = layoutP(mmax, C, false, f64);
  if (L.total > cap) L.total = 0;
  return L;
}

SmemLayout64 pick_layout64(int64_t mmax, int C) {
  const size_t cap = (size_t)smem_optin();
  SmemLayout64 L = layout64(mmax, C, true);
  if (L.total > cap) L = layout64(mmax, C, false);
  if (L.total > cap) L.total = 0;
  return L;
}

// Launch configuration of a batched kernel (func) for n items at cluster size
// C with smem bytes of dynamic shared memory; the number of clusters is what
// the device can hold at once, capped at n.  The dynamic shared-memory limit
// is raised to the device maximum (the same value from every thread), so
// concurrent launches never see a smaller limit.
cudaError_t configure(const void* func, int C, size_t smem, int n, cudaStream_t st, cudaLaunchConfig_t* cfg,
                      cudaLaunchAttribute* attr) {
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  *cfg = cudaLaunchConfig_t{};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->blockDim = dim3(256, 1, 1);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = st;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  cfg->gridDim = dim3((unsigned)C, 1, 1);
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, func, cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  clusters = std::min<int>(clusters, n);
  cfg->gridDim = dim3((unsigned)(clusters * C), 1, 1);
  return cudaSuccess;
}

// The propagator form of batch_run_group (formed for dt beforehand).
cudaError_t batch_run_group_prop(lb_batch* b, const std::vector<int>& ids, int C, int64_t mmax, int64_t nsteps,
                                 double dt, int correct_every, cudaStream_t st, float* ms) {
  const bool f64 = b->precision == LB_FP64;
  cudaError_t e = batch_form_propagator(b, dt, st);
  if (e != cudaSuccess) return e;
  const SmemLayoutP L = pick_layoutP(mmax, C, f64);
  if (L.total == 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  e = f64 ? configure((const void*)k_prop_batch64, C, L.total, (int)ids.size(), st, &cfg, attr)
          : configure((const void*)k_prop_batch, C, L.total, (int)ids.size(), st, &cfg, attr);
  if (e != cudaSuccess) return e;
  std::vector<int> ord(ids.begin(), ids.end());
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return b->M[x] > b->M[y]; });
  std::vector<PItem> host(b->count);
  for (int r = 0; r < b->count; ++r) {
    if (f64)
      host[r] = PItem{b->M[r], nullptr, nullptr, b->D64[r], b->cp[r], b->v[r]};
    else
      host[r] = PItem{b->M[r], b->D32[r], b->R32[r], correct_every > 0 ? b->A64[r] : nullptr, b->cp[r], b->v[r]};
  }
  if ((e = cudaMemcpyAsync(b->d_prop_items, host.data(), sizeof(PItem) * b->count, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b->d_order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  const PItem* items = static_cast<const PItem*>(b->d_prop_items);
  if (f64)
    e = cudaLaunchKernelEx(&cfg, k_prop_batch64, items, (const int*)b->d_order, (int)ord.size(), b->d_counter, nsteps,
                           dt, L);
  else
    e = cudaLaunchKernelEx(&cfg, k_prop_batch, items, (const int*)b->d_order, (int)ord.size(), b->d_counter, nsteps,
                           dt, correct_every, L);
  note_launch(1);
  if (ms) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (e != cudaSuccess) return e;
  // the item list is read by the kernel: keep it until the launch is done
  return cudaStreamSynchronize(st);
}

// Run the realizations `ids` (one cluster size C) for nsteps; synchronous when
// ms is requested.  A cluster size the device cannot place with the needed
// shared memory fails with cudaErrorInvalidConfiguration before any launch.
cudaError_t batch_run_group(lb_batch* b, const std::vector<int>& ids, int C, int64_t nsteps, double dt,
                            int correct_every, cudaStream_t st, float* ms) {
  if (ids.empty()) {
    if (ms) *ms = 0.f;
    return cudaSuccess;
  }
  int64_t mmax = 0;
  for (int r : ids) mmax = std::max<int64_t>(mmax, b->M[r]);
  const bool f64 = b->precision == LB_FP64;
  if (b->form == LB_FORM_PROPAGATOR) return batch_run_group_prop(b, ids, C, mmax, nsteps, dt, correct_every, st, ms);
  const SmemLayout L = f64 ? SmemLayout{} : pick_layout(mmax, C);
  const SmemLayout64 L64 = f64 ? pick_layout64(mmax, C) : SmemLayout64{};
  if ((f64 ? L64.total : L.total) == 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = f64 ? configure((const void*)k_rk4_batch64, C, L64.total, (int)ids.size(), st, &cfg, attr)
                      : configure((const void*)k_rk4_batch, C, L.total, (int)ids.size(), st, &cfg, attr);
  if (e != cudaSuccess) return e;
  // items in decreasing order of work (largest first)
  std::vector<int> ord(ids.begin(), ids.end());
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return b->M[x] > b->M[y]; });
  std::vector<BItem> host(b->count);
  for (int r = 0; r < b->count; ++r)
    host[r] = BItem{b->M[r], b->A32[r], (correct_every > 0 || f64) ? b->A64[r] : nullptr, b->K[r], b->v[r]};
  if ((e = cudaMemcpyAsync(b->d_items, host.data(), sizeof(BItem) * b->count, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b->d_order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  if (f64)
    e = cudaLaunchKernelEx(&cfg, k_rk4_batch64, (const BItem*)b->d_items, (const int*)b->d_order, (int)ord.size(),
                           b->d_counter, nsteps, dt, L64);
  else
    e = cudaLaunchKernelEx(&cfg, k_rk4_batch, (const BItem*)b->d_items, (const int*)b->d_order, (int)ord.size(),
                           b->d_counter, nsteps, dt, correct_every, L);
  note_launch(1);
  if (ms) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int batch_default_cluster(int64_t M) {
  const size_t cap = (size_t)smem_optin();
  for (int C : {1, 2, 4, 8, 16})
    if (layout(M, C, true).total <= cap) return C;
  return 16;
}

cudaError_t batch_launch_async(const BatchItem* items, int n, int C, int64_t nsteps, double dt, int correct_every,
                               cudaMemPool_t pool, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t mmax = 0;
  for (int i = 0; i < n; ++i) mmax = std::max<int64_t>(mmax, items[i].M);
  const SmemLayout L = pick_layout(mmax, C);
  if (L.total == 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = configure((const void*)k_rk4_batch, C, L.total, n, st, &cfg, attr);
  if (e != cudaSuccess) return e;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return items[x].M > items[y].M; });
  // one block: items, then order, then the counter
  const size_t bi = sizeof(BItem) * (size_t)n, bo = sizeof(int) * (size_t)n;
  const size_t off_o = (bi + 255) & ~size_t(255), off_c = (off_o + bo + 255) & ~size_t(255);
  std::vector<unsigned char> host(off_c + sizeof(int), 0);
  std::memcpy(host.data(), items, bi);
  std::memcpy(host.data() + off_o, ord.data(), bo);
  void* d = nullptr;
  if ((e = cudaMallocFromPoolAsync(&d, host.size(), pool, st)) != cudaSuccess) return e;
  unsigned char* db = static_cast<unsigned char*>(d);
  e = cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaLaunchKernelEx(&cfg, k_rk4_batch, reinterpret_cast<const BItem*>(db),
                           reinterpret_cast<const int*>(db + off_o), n, reinterpret_cast<int*>(db + off_c), nsteps,
                           dt, correct_every, L);
  note_launch(1);
  const cudaError_t ef = cudaFreeAsync(d, st);
  if (e != cudaSuccess) return e;
  if (ef != cudaSuccess) return ef;
  return cudaGetLastError();
}

}  // namespace lbi

// ------------------------------------------------------------------ ABI

extern "C" {

int lb_batch_create(int count, const int* Ns, lb_batch_t** out) {
  if (!out || !Ns || count <= 0) {
    lbi::set_error("lb_batch_create: bad arguments");
    return LB_EINVAL;
  }
  *out = nullptr;
  lb_batch* b = new lb_batch;
  b->count = count;
  b->N.assign(Ns, Ns + count);
  b->M.resize(count);
  b->a.assign(count, nullptr);
  b->h.assign(count, nullptr);
  b->v.assign(count, nullptr);
  b->A64.assign(count, nullptr);
  b->A32.assign(count, nullptr);
  b->K.assign(count, nullptr);
  b->cluster.assign(count, 1);
  b->basis_of.assign(count, -1);
  std::vector<int> distinct;
  for (int r = 0; r < count; ++r) {
    if (Ns[r] < 2 || Ns[r] > lbi::kBatchMaxN) {
      lbi::set_error("lb_batch_create: N = %d outside [2, %d]", Ns[r], lbi::kBatchMaxN);
      delete b;
      return LB_EINVAL;
    }
    b->M[r] = (int64_t)Ns[r] * Ns[r] - 1;
    auto it = std::find(distinct.begin(), distinct.end(), Ns[r]);
    if (it == distinct.end()) {
      distinct.push_back(Ns[r]);
      b->basis_of[r] = (int)distinct.size() - 1;
    } else {
      b->basis_of[r] = (int)(it - distinct.begin());
    }
  }
  for (int n : distinct) {
    lb_basis_t* bb = nullptr;
    int rc = lb_basis_create(n, nullptr, &bb);
    if (rc != LB_OK) {
      for (auto* x : b->basis) lb_basis_destroy(x);
      delete b;
      return rc;
    }
    b->basis.push_back(bb);
  }
  cudaError_t e = lbi::batch_alloc(b);
  if (e != cudaSuccess) {
    lbi::batch_free(b);
    for (auto* x : b->basis) lb_basis_destroy(x);
    delete b;
    cudaGetLastError();
    lbi::set_error("lb_batch_create: device allocation failed (%s)", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;
  }
  *out = b;
  return LB_OK;
}

int lb_batch_set(lb_batch_t* b, int r, const double* a, const double* h, double* v) {
  if (!b || r < 0 || r >= b->count || !a || !v) {
    lbi::set_error("lb_batch_set: bad arguments");
    return LB_EINVAL;
  }
  b->a[r] = a;
  b->h[r] = h;
  b->v[r] = v;
  return LB_OK;
}

int lb_batch_assemble(lb_batch_t* b, int algorithm, void* stream) {
  if (!b) {
    lbi::set_error("lb_batch_assemble: NULL batch");
    return LB_EINVAL;
  }
  for (int r = 0; r < b->count; ++r)
    if (!b->a[r] || !b->v[r]) {
      lbi::set_error("lb_batch_assemble: realization %d has no inputs (lb_batch_set)", r);
      return LB_EINVAL;
    }
  std::vector<lb::BasisView> views;
  for (auto* x : b->basis) views.push_back(x->view());
  cudaError_t e = lbi::batch_assemble(b, views, algorithm, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_batch_assemble");
  return LB_OK;
}

int lb_batch_set_cluster(lb_batch_t* b, int r, int C) {
  if (!b || r < 0 || r >= b->count || !(C == 1 || C == 2 || C == 4 || C == 8 || C == 16)) {
    lbi::set_error("lb_batch_set_cluster: bad arguments");
    return LB_EINVAL;
  }
  b->cluster[r] = C;
  return LB_OK;
}

int lb_batch_set_precision(lb_batch_t* b, int precision) {
  if (!b || (precision != LB_FP32 && precision != LB_FP64)) {
    lbi::set_error("lb_batch_set_precision: bad arguments (LB_FP32 or LB_FP64)");
    return LB_EINVAL;
  }
  b->precision = precision;
  return LB_OK;
}

int lb_batch_set_form(lb_batch_t* b, int form) {
  if (!b || (form != LB_FORM_RK4 && form != LB_FORM_PROPAGATOR)) {
    lbi::set_error("lb_batch_set_form: bad arguments (LB_FORM_RK4 or LB_FORM_PROPAGATOR)");
    return LB_EINVAL;
  }
  b->form = form;
  return LB_OK;
}

int lb_batch_form_propagator(lb_batch_t* b, double dt, void* stream, float* ms) {
  if (!b || !(dt > 0.0) || !std::isfinite(dt)) {
    lbi::set_error("lb_batch_form_propagator: bad arguments");
    return LB_EINVAL;
  }
  cudaError_t e = lbi::batch_form_propagator(b, dt, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      lbi::set_error("lb_batch_form_propagator: device memory exhausted");
      return LB_ENOMEM;
    }
    return lbi::cuda_fail(e, "lb_batch_form_propagator");
  }
  if (ms) *ms = b->prop_ms;
  return LB_OK;
}

int lb_batch_integrate(lb_batch_t* b, int correct_every, double dt, int64_t nsteps, void* stream, float* ms) {
  if (!b || nsteps < 0 || correct_every < 0) {
    lbi::set_error("lb_batch_integrate: bad arguments");
    return LB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float total = 0.f;
  for (int C : {16, 8, 4, 2, 1}) {
    std::vector<int> ids;
    for (int r = 0; r < b->count; ++r)
      if (b->cluster[r] == C) ids.push_back(r);
    float m = 0.f;
    cudaError_t e = lbi::batch_run_group(b, ids, C, nsteps, dt, correct_every, st, ms ? &m : nullptr);
    if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_batch_integrate");
    total += m;
  }
  if (ms) *ms = total;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_batch_integrate");
  return LB_OK;
}

// Autotuner: realizations are bucketed by N (bucket width `width`); for each
// bucket every cluster size of {1, 2, 4, 8, 16} that the device can place
// runs the bucket's realizations for probe_steps steps (timed with CUDA
// events), the states are restored, and the size with the shortest time is
// kept.  choice (optional, one per realization) receives the result.
int lb_batch_tune(lb_batch_t* b, int width, int probe_steps, double dt, void* stream, int* choice) {
  if (!b || width < 1 || probe_steps < 1) {
    lbi::set_error("lb_batch_tune: bad arguments");
    return LB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // save the states
  std::vector<double*> saved(b->count, nullptr);
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < b->count && e == cudaSuccess; ++r) {
    if (!b->v[r]) {
      lbi::set_error("lb_batch_tune: realization %d has no state (lb_batch_set)", r);
      for (auto* p : saved) cudaFree(p);
      return LB_EINVAL;
    }
    e = cudaMalloc(&saved[r], 8 * (size_t)b->M[r]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved[r], b->v[r], 8 * (size_t)b->M[r], cudaMemcpyDeviceToDevice, st);
  }
  int nmax = 0;
  for (int n : b->N) nmax = std::max(nmax, n);
  for (int lo = 2; lo <= nmax && e == cudaSuccess; lo += width) {
    std::vector<int> ids;
    for (int r = 0; r < b->count; ++r)
      if (b->N[r] >= lo && b->N[r] < lo + width) ids.push_back(r);
    if (ids.empty()) continue;
    float best = 3.4e38f;
    int bestC = 1;
    for (int C : {1, 2, 4, 8, 16}) {
      float ms = 0.f;
      cudaError_t ec = lbi::batch_run_group(b, ids, C, probe_steps, dt, 0, st, &ms);
      if (ec != cudaSuccess) {  // size not placeable with this shared memory: skip it
        cudaGetLastError();
        continue;
      }
      if (ms < best) {
        best = ms;
        bestC = C;
      }
      for (int r : ids)
        e = cudaMemcpyAsync(b->v[r], saved[r], 8 * (size_t)b->M[r], cudaMemcpyDeviceToDevice, st);
    }
    for (int r : ids) b->cluster[r] = bestC;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (auto* p : saved) cudaFree(p);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_batch_tune");
  if (choice)
    for (int r = 0; r < b->count; ++r) choice[r] = b->cluster[r];
  return LB_OK;
}

int lb_batch_system(const lb_batch_t* b, int r, const double** A64, const float** A32, const double** K,
                    int64_t* M) {
  if (!b || r < 0 || r >= b->count) {
    lbi::set_error("lb_batch_system: bad arguments");
    return LB_EINVAL;
  }
  if (A64) *A64 = b->A64[r];
  if (A32) *A32 = b->A32[r];
  if (K) *K = b->K[r];
  if (M) *M = b->M[r];
  return LB_OK;
}

int lb_batch_copy_system(const lb_batch_t* b, int r, double* A64, double* K, void* stream) {
  if (!b || r < 0 || r >= b->count) {
    lbi::set_error("lb_batch_copy_system: bad arguments");
    return LB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t M = (size_t)b->M[r];
  cudaError_t e = cudaSuccess;
  if (A64) e = cudaMemcpyAsync(A64, b->A64[r], 8 * M * M, cudaMemcpyDefault, st);
  if (K && e == cudaSuccess) e = cudaMemcpyAsync(K, b->K[r], 8 * M, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_batch_copy_system");
  return LB_OK;
}

int lb_batch_destroy(lb_batch_t* b) {
  if (!b) return LB_OK;
  lbi::batch_free(b);
  for (auto* x : b->basis) lb_basis_destroy(x);
  delete b;
  return LB_OK;
}

}  // extern "C"

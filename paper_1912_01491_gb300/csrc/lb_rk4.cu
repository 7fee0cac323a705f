// lb_rk4.cu -- kernel (c): classical fourth-order Runge-Kutta for
// dv/dt = A v + K (Eq. (04) with time-independent Q and R; Table 1 step 3.1,
// Sec. 4 item 3), as one fused GEMV + stage-update kernel per RK stage.
//
// Stage i computes k_i = A x_i + K row by row (one warp per row) and, in the
// same kernel's epilogue, forms the next stage input and the running
// combination:
//   stage 1: acc  = k1,     x2 = v + h/2 k1
//   stage 2: acc += 2 k2,   x3 = v + h/2 k2
//   stage 3: acc += 2 k3,   x4 = v + h k3
//   stage 4: v   += h/6 (acc + k4),  x1' = v
// so each stage reads A once and O(M) vectors, and nothing else.
//
// Storage precisions (a6): FP64; FP32 (A32 = fl32(A)); BF16 with per-row
// scales r_s = max_n |A_sn|.  For FP32/BF16 the products use FP32 multiply-
// adds on an FP32 copy of the stage vector, per-lane partial sums are FP32
// and the 32 lane sums are combined in FP64; state and stage combination
// stay FP64.  Optional FP64 defect correction (a8): every k steps
// c = (A64 - A_lp) v at the current v, added to K until the next one.
#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>

#include "lb_internal.h"

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ float bf16_bits_to_float(uint16_t u) {
  return __uint_as_float(((uint32_t)u) << 16);
}

template <int PREC>
__device__ __forceinline__ double row_dot(int64_t M, int64_t s, const void* __restrict__ Ap,
                                          const float* __restrict__ scale,
                                          const double* __restrict__ x,
                                          const float* __restrict__ x32, int64_t xstride, int lane) {
  if (PREC == LB_FP64) {
    const double* __restrict__ row = static_cast<const double*>(Ap) + s * M;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t n = lane;
    for (; n + 96 < M; n += 128) {
      a0 = fma(__ldcs(row + n), __ldg(x + n), a0);
      a1 = fma(__ldcs(row + n + 32), __ldg(x + n + 32), a1);
      a2 = fma(__ldcs(row + n + 64), __ldg(x + n + 64), a2);
      a3 = fma(__ldcs(row + n + 96), __ldg(x + n + 96), a3);
    }
    for (; n < M; n += 32) a0 = fma(__ldcs(row + n), __ldg(x + n), a0);
    double t = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
  } else if (PREC == LB_FP32) {
    // Lane k reads A as float4 at element head + 4k (a scalar head up to the
    // first 16-byte boundary; rows start anywhere for odd M) and x as the
    // matching float4 of the shifted copy o = head mod 4, so a warp reads
    // 512 contiguous bytes of each per instruction.
    const float* __restrict__ row = static_cast<const float*>(Ap) + s * M;
    const int64_t h4 = (int64_t)(((16 - ((uintptr_t)row & 15)) & 15) >> 2);
    const int head = (int)(h4 < M ? h4 : M);
    const int o = head & 3;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (lane < head) a0 = fmaf(__ldcs(row + lane), __ldg(x32 + lane), a0);
    const float4* __restrict__ rv = reinterpret_cast<const float4*>(row + head);
    const float4* __restrict__ xv = reinterpret_cast<const float4*>(x32 + o * xstride + head - o);
    const int64_t nv = (M - head) >> 2;
    int64_t k = lane;
    for (; k + 32 < nv; k += 64) {
      const float4 u = __ldcs(rv + k), w = __ldcs(rv + k + 32);
      const float4 xu = __ldg(xv + k), xw = __ldg(xv + k + 32);
      a0 = fmaf(u.x, xu.x, a0);
      a1 = fmaf(u.y, xu.y, a1);
      a2 = fmaf(u.z, xu.z, a2);
      a3 = fmaf(u.w, xu.w, a3);
      a0 = fmaf(w.x, xw.x, a0);
      a1 = fmaf(w.y, xw.y, a1);
      a2 = fmaf(w.z, xw.z, a2);
      a3 = fmaf(w.w, xw.w, a3);
    }
    for (; k < nv; k += 32) {
      const float4 u = __ldcs(rv + k), xu = __ldg(xv + k);
      a0 = fmaf(u.x, xu.x, a0);
      a1 = fmaf(u.y, xu.y, a1);
      a2 = fmaf(u.z, xu.z, a2);
      a3 = fmaf(u.w, xu.w, a3);
    }
    for (int64_t n = head + 4 * nv + lane; n < M; n += 32) a0 = fmaf(__ldcs(row + n), __ldg(x32 + n), a0);
    double t = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
    for (int o2 = 16; o2 > 0; o2 >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o2);
    return t;
  } else {
    // BF16: lane k reads four values (8 bytes) of A at element head + 4k
    // (head up to the first 8-byte boundary) and the matching float4 of the
    // shifted copy o = head mod 4 of x: 256 contiguous bytes of A and 512 of
    // x per warp instruction.
    const uint16_t* __restrict__ row = static_cast<const uint16_t*>(Ap) + s * M;
    const int64_t h2 = (int64_t)(((8 - ((uintptr_t)row & 7)) & 7) >> 1);
    const int head = (int)(h2 < M ? h2 : M);
    const int o = head & 3;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (lane < head)
      a0 = fmaf(bf16_bits_to_float(__ldcs(reinterpret_cast<const unsigned short*>(row + lane))), __ldg(x32 + lane), a0);
    const uint2* __restrict__ rv = reinterpret_cast<const uint2*>(row + head);
    const float4* __restrict__ xv = reinterpret_cast<const float4*>(x32 + o * xstride + head - o);
    const int64_t nv = (M - head) >> 2;
    int64_t k = lane;
    for (; k + 96 < nv; k += 128) {
      uint2 u[4];
      float4 xu[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        u[i] = __ldcs(rv + k + 32 * i);
        xu[i] = __ldg(xv + k + 32 * i);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a0 = fmaf(__uint_as_float(u[i].x << 16), xu[i].x, a0);
        a1 = fmaf(__uint_as_float(u[i].x & 0xffff0000u), xu[i].y, a1);
        a2 = fmaf(__uint_as_float(u[i].y << 16), xu[i].z, a2);
        a3 = fmaf(__uint_as_float(u[i].y & 0xffff0000u), xu[i].w, a3);
      }
    }
    for (; k < nv; k += 32) {
      const uint2 u = __ldcs(rv + k);
      const float4 xu = __ldg(xv + k);
      a0 = fmaf(__uint_as_float(u.x << 16), xu.x, a0);
      a1 = fmaf(__uint_as_float(u.x & 0xffff0000u), xu.y, a1);
      a2 = fmaf(__uint_as_float(u.y << 16), xu.z, a2);
      a3 = fmaf(__uint_as_float(u.y & 0xffff0000u), xu.w, a3);
    }
    for (int64_t n = head + 4 * nv + lane; n < M; n += 32)
      a0 = fmaf(bf16_bits_to_float(__ldcs(reinterpret_cast<const unsigned short*>(row + n))), __ldg(x32 + n), a0);
    double t = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
    for (int o2 = 16; o2 > 0; o2 >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o2);
    return t * (double)__ldg(scale + s);
  }
}

template <int PREC, int STAGE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_stage(int64_t M, const void* __restrict__ Ap, const float* __restrict__ scale,
            const double* __restrict__ Keff, const double* __restrict__ x,
            const float* __restrict__ x32, double* __restrict__ xn, float* __restrict__ xn32,
            int64_t xstride, double* __restrict__ acc, double* __restrict__ v, double h) {
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const double y = row_dot<PREC>(M, s, Ap, scale, x, x32, xstride, lane);
  if (lane != 0) return;
  const double k = y + Keff[s];
  double nx;
  if (STAGE == 1) {
    acc[s] = k;
    nx = v[s] + 0.5 * h * k;
  } else if (STAGE == 2) {
    acc[s] += 2.0 * k;
    nx = v[s] + 0.5 * h * k;
  } else if (STAGE == 3) {
    acc[s] += 2.0 * k;
    nx = v[s] + h * k;
  } else {
    nx = v[s] + (h / 6.0) * (acc[s] + k);
    v[s] = nx;
  }
  xn[s] = nx;
  if (PREC != LB_FP64) {  // the four shifted copies: copy o holds x[j + o] at j
    const float f = (float)nx;
#pragma unroll
    for (int o = 0; o < 4; ++o)
      if (s >= o) xn32[o * xstride + (s - o)] = f;
  }
}

// c = (A64 - A_lp) v in FP64;  Keff = K + c.
template <int PREC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_correction(int64_t M, const double* __restrict__ A64, const void* __restrict__ Ap,
                 const float* __restrict__ scale, const double* __restrict__ v,
                 const double* __restrict__ K, double* __restrict__ Keff) {
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const double* __restrict__ r64 = A64 + s * M;
  double t = 0.0;
  if (PREC == LB_FP32) {
    const float* __restrict__ r = static_cast<const float*>(Ap) + s * M;
    for (int64_t n = lane; n < M; n += 32) t = fma(__ldcs(r64 + n) - (double)__ldcs(r + n), v[n], t);
  } else {
    // sum_n A64_sn v_n - r_s sum_n q_sn v_n: two FP64 dot products (the
    // difference is formed once per row, not per entry)
    const uint16_t* __restrict__ r = static_cast<const uint16_t*>(Ap) + s * M;
    double tq = 0.0;
    for (int64_t n = lane; n < M; n += 32) {
      const double vn = v[n];
      t = fma(__ldcs(r64 + n), vn, t);
      tq = fma((double)bf16_bits_to_float(__ldcs(reinterpret_cast<const unsigned short*>(r + n))), vn, tq);
    }
    for (int o = 16; o > 0; o >>= 1) tq += __shfl_xor_sync(0xffffffffu, tq, o);
    if (lane == 0) t -= (double)scale[s] * tq;  // once, before the lane sum below
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) Keff[s] = K[s] + t;
}

// ---------------------------------------------------------------- CSR
// Block-staged form, for short rows (about seven entries for the ladder
// model): the block's 256 consecutive rows own one contiguous range of the
// column and value arrays, which the block first copies into shared memory
// with coalesced loads; then every thread walks its own row there, gathers x
// (FP32 copy in FP32 mode, which stays in L2) and runs the stage epilogue.  A
// block whose range exceeds the staging capacity `cap` walks its rows in
// global memory instead (the same arithmetic in the same order).  In FP32
// mode the row sum is FP32 and only the FP32 copy of the next stage vector is
// written (the FP64 copy is not read by the FP32 product).
template <int PREC, int STAGE>
__global__ void __launch_bounds__(256)
    k_stage_csr_blk(int64_t M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                    const void* __restrict__ val, int cap, const double* __restrict__ Keff,
                    const double* __restrict__ x, const float* __restrict__ x32, double* __restrict__ xn,
                    float* __restrict__ xn32, double* __restrict__ acc, double* __restrict__ v, double h) {
  using V = typename std::conditional<PREC == LB_FP64, double, float>::type;
  extern __shared__ __align__(16) unsigned char csr_stage[];
  V* sval = reinterpret_cast<V*>(csr_stage);
  int32_t* scol = reinterpret_cast<int32_t*>(csr_stage + sizeof(V) * (size_t)cap);
  const V* __restrict__ vv = static_cast<const V*>(val);
  const int64_t r0 = (int64_t)blockIdx.x * 256;
  const int64_t r1 = r0 + 256 < M ? r0 + 256 : M;
  const int64_t base = __ldg(rowptr + r0), n = __ldg(rowptr + r1) - base;
  const bool staged = n <= cap;
  if (staged)
    for (int64_t i = threadIdx.x; i < n; i += 256) {
      sval[i] = __ldcs(vv + base + i);
      scol[i] = __ldcs(col + base + i);
    }
  __syncthreads();
  const int64_t s = r0 + threadIdx.x;
  if (s >= M) return;
  const double kf = __ldcs(Keff + s), vs = __ldcs(v + s);
  const double ac = STAGE > 1 ? __ldcs(acc + s) : 0.0;
  const int64_t b = __ldg(rowptr + s), e = __ldg(rowptr + s + 1);
  double y;
  if (PREC == LB_FP64) {
    double t = 0.0;
    if (staged) {
      for (int64_t q = b - base; q < e - base; ++q) t = fma((double)sval[q], __ldg(x + scol[q]), t);
    } else {
#pragma unroll 4
      for (int64_t q = b; q < e; ++q) t = fma((double)__ldcs(vv + q), __ldg(x + __ldcs(col + q)), t);
    }
    y = t;
  } else {
    float t = 0.f;
    if (staged) {
      for (int64_t q = b - base; q < e - base; ++q) t = fmaf((float)sval[q], __ldg(x32 + scol[q]), t);
    } else {
#pragma unroll 4
      for (int64_t q = b; q < e; ++q) t = fmaf((float)__ldcs(vv + q), __ldg(x32 + __ldcs(col + q)), t);
    }
    y = (double)t;
  }
  const double k = y + kf;
  double nx;
  if (STAGE == 1) {
    acc[s] = k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 2) {
    acc[s] = ac + 2.0 * k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 3) {
    acc[s] = ac + 2.0 * k;
    nx = vs + h * k;
  } else {
    nx = vs + (h / 6.0) * (ac + k);
    v[s] = nx;
  }
  if (PREC == LB_FP64)
    xn[s] = nx;
  else
    xn32[s] = (float)nx;
}

// ---------------------------------------------------------------- CSR, pipelined
// Persistent form of the block-staged stage: each block walks the chunks of
// 256 rows c = blockIdx.x, blockIdx.x + gridDim.x, ... and, while it sums
// chunk i out of one shared-memory buffer, the bulk-copy engine (TMA,
// cp.async.bulk) fills the other with the column and value range of chunk
// i + 1; the rows' own state (row pointers, Keff, v, acc) of chunk i + 1 is
// loaded into registers during chunk i.  A copy starts at the range's first
// entry rounded down to 16 bytes and ends at its last rounded up (up to three
// entries of the neighbouring chunks on either side; never past nnz): a
// chunk whose rounded range would pass nnz, or that exceeds `cap`, is summed
// from global memory instead.  Every wait on a copy is bounded (about two
// seconds of clock): on a timeout the block sets *err, waits (bounded) for its
// other copy in flight and returns.
constexpr long long kCopyWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bulk copy global -> shared, completing on the mbarrier; `policy` is an L2
// cache policy (the streamed arrays are marked evict-first, so that the
// gathered vector stays in L2)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// true once the phase of the given parity has completed; false after about
// kCopyWaitCycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kCopyWaitCycles) return false;
  }
}

// *out = the largest entry count of a chunk of 256 rows (clamped to int).
__global__ void k_chunk_max_range(int64_t M, const int64_t* __restrict__ rowptr, int* __restrict__ out) {
  const int64_t cc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((cc << 8) >= M) return;
  const int64_t r0 = cc << 8, r1 = r0 + 256 < M ? r0 + 256 : M;
  const int64_t n = rowptr[r1] - rowptr[r0];
  atomicMax(out, n < 0x7fffffff ? (int)n : 0x7fffffff);
}

// Shared-memory layout of one buffer of k_stage_csr_pipe: the chunk's row
// pointers (258 entries), Keff, v and acc (256 each), then its values and
// columns (cap + 8 entries each: the range rounded out to 16 bytes).
constexpr size_t kPipeRowBytes = 258 * 8 + 3 * 256 * 8;
template <class V>
__host__ __device__ inline size_t csr_pipe_vbytes(int cap) {
  return ((sizeof(V) * (size_t)(cap + 8)) + 15) & ~size_t(15);
}
template <class V>
__host__ __device__ inline size_t csr_pipe_buf_bytes(int cap) {
  return kPipeRowBytes + csr_pipe_vbytes<V>(cap) + ((sizeof(int32_t) * (size_t)(cap + 8) + 15) & ~size_t(15));
}

template <int PREC, int STAGE>
__global__ void __launch_bounds__(256)
    k_stage_csr_pipe(int64_t M, int64_t nnz, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const void* __restrict__ val, int cap, const double* __restrict__ Keff,
                     const double* __restrict__ x, const float* __restrict__ x32, double* __restrict__ xn,
                     float* __restrict__ xn32, double* __restrict__ acc, double* __restrict__ v, double h,
                     int* __restrict__ err) {
  using V = typename std::conditional<PREC == LB_FP64, double, float>::type;
  constexpr int64_t kVA = 16 / (int64_t)sizeof(V);  // entries per 16 bytes
  extern __shared__ __align__(128) unsigned char csr_pipe[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int64_t s_base[2];
  __shared__ int s_offv[2], s_offc[2], s_staged[2], s_rows[2];
  const size_t vbytes = csr_pipe_vbytes<V>(cap), buf_bytes = csr_pipe_buf_bytes<V>(cap);
  const V* __restrict__ vv = static_cast<const V*>(val);
  const int64_t nch = (M + 255) >> 8, G = gridDim.x;
  int64_t c = blockIdx.x;
  if (c >= nch) return;
  const uint32_t bars[2] = {smem_u32(&bar[0]), smem_u32(&bar[1])};
  // thread 0: stage chunk cc, whose entries are [base, end), into buffer b:
  // its row arrays when the chunk is whole (and its 258th row pointer
  // exists), its column and value range when within cap and nnz
  auto issue = [&](int b, int64_t cc, int64_t base, int64_t end) {
    const int64_t r0 = cc << 8;
    const bool rows = r0 + 258 <= M + 1;
    const int64_t a0c = base & ~int64_t(3), a1c = (end + 3) & ~int64_t(3);
    const int64_t a0v = base & ~(kVA - 1), a1v = (end + kVA - 1) & ~(kVA - 1);
    const bool st = end - base <= cap && a1c <= nnz;
    s_base[b] = base;
    s_offc[b] = (int)(base - a0c);
    s_offv[b] = (int)(base - a0v);
    s_staged[b] = st ? 1 : 0;
    s_rows[b] = rows ? 1 : 0;
    const uint32_t bc = st ? (uint32_t)(sizeof(int32_t) * (a1c - a0c)) : 0u;
    const uint32_t bv = st ? (uint32_t)(sizeof(V) * (a1v - a0v)) : 0u;
    const uint32_t br = rows ? (uint32_t)(258 * 8 + (STAGE > 1 ? 3 : 2) * 256 * 8) : 0u;
    unsigned char* buf = csr_pipe + b * buf_bytes;
    const uint64_t pol = l2_evict_first();
    // the buffer was last read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bars[b], bc + bv + br);
    if (rows) {
      bulk_g2s(smem_u32(buf), rowptr + r0, 258 * 8, bars[b], pol);
      bulk_g2s(smem_u32(buf + 258 * 8), Keff + r0, 256 * 8, bars[b], pol);
      bulk_g2s(smem_u32(buf + 258 * 8 + 2048), v + r0, 256 * 8, bars[b], pol);
      if (STAGE > 1) bulk_g2s(smem_u32(buf + 258 * 8 + 4096), acc + r0, 256 * 8, bars[b], pol);
    }
    if (bv) bulk_g2s(smem_u32(buf + kPipeRowBytes), vv + a0v, bv, bars[b], pol);
    if (bc) bulk_g2s(smem_u32(buf + kPipeRowBytes + vbytes), col + a0c, bc, bars[b], pol);
  };
  auto range = [&](int64_t cc, int64_t& base, int64_t& end) {
    const int64_t r0 = cc << 8, r1 = r0 + 256 < M ? r0 + 256 : M;
    base = __ldg(rowptr + r0);
    end = __ldg(rowptr + r1);
  };
  if (threadIdx.x == 0) {
    mbar_init(bars[0], 1);
    mbar_init(bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t base, end;
    range(c, base, end);
    issue(0, c, base, end);
    if (c + G < nch) {
      range(c + G, base, end);
      issue(1, c + G, base, end);
    }
  }
  int64_t nb = 0, ne = 0;
  for (int64_t i = 0; c < nch; ++i, c += G) {
    const int b = (int)(i & 1);
    // thread 0: the range of the chunk after the next, in flight during this one
    if (threadIdx.x == 0 && c + 2 * G < nch) range(c + 2 * G, nb, ne);
    const bool ok = mbar_wait(bars[b], (uint32_t)((i >> 1) & 1));
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {  // the copies still in flight, bounded again
        atomicExch(err, 1);
        mbar_wait(bars[b], (uint32_t)((i >> 1) & 1));
        if (c + G < nch) mbar_wait(bars[b ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
      }
      return;
    }
    const unsigned char* buf = csr_pipe + b * buf_bytes;
    const int64_t s = (c << 8) + threadIdx.x;
    if (s < M) {
      int64_t rb, re;
      double kf, vs, ac = 0.0;
      if (s_rows[b]) {
        const int64_t* srp = reinterpret_cast<const int64_t*>(buf);
        const double* sk = reinterpret_cast<const double*>(buf + 258 * 8);
        rb = srp[threadIdx.x];
        re = srp[threadIdx.x + 1];
        kf = sk[threadIdx.x];
        vs = sk[256 + threadIdx.x];
        if (STAGE > 1) ac = sk[512 + threadIdx.x];
      } else {
        rb = __ldg(rowptr + s);
        re = __ldg(rowptr + s + 1);
        kf = __ldcs(Keff + s);
        vs = __ldcs(v + s);
        if (STAGE > 1) ac = __ldcs(acc + s);
      }
      double y;
      if (s_staged[b]) {
        // entry q of the range sits at index q - base + offset of its array
        const V* sval = reinterpret_cast<const V*>(buf + kPipeRowBytes);
        const int32_t* scol = reinterpret_cast<const int32_t*>(buf + kPipeRowBytes + vbytes);
        const int qv = (int)(rb - s_base[b]) + s_offv[b], qc = (int)(rb - s_base[b]) + s_offc[b];
        const int len = (int)(re - rb);
        if (PREC == LB_FP64) {
          double t = 0.0;
          for (int q = 0; q < len; ++q) t = fma((double)sval[qv + q], __ldg(x + scol[qc + q]), t);
          y = t;
        } else {
          float t = 0.f;
          for (int q = 0; q < len; ++q) t = fmaf((float)sval[qv + q], __ldg(x32 + scol[qc + q]), t);
          y = (double)t;
        }
      } else if (PREC == LB_FP64) {
        double t = 0.0;
#pragma unroll 4
        for (int64_t q = rb; q < re; ++q) t = fma((double)__ldcs(vv + q), __ldg(x + __ldcs(col + q)), t);
        y = t;
      } else {
        float t = 0.f;
#pragma unroll 4
        for (int64_t q = rb; q < re; ++q) t = fmaf((float)__ldcs(vv + q), __ldg(x32 + __ldcs(col + q)), t);
        y = (double)t;
      }
      const double k = y + kf;
      double nx;
      if (STAGE == 1) {
        acc[s] = k;
        nx = vs + 0.5 * h * k;
      } else if (STAGE == 2) {
        acc[s] = ac + 2.0 * k;
        nx = vs + 0.5 * h * k;
      } else if (STAGE == 3) {
        acc[s] = ac + 2.0 * k;
        nx = vs + h * k;
      } else {
        nx = vs + (h / 6.0) * (ac + k);
        v[s] = nx;
      }
      if (PREC == LB_FP64)
        xn[s] = nx;
      else
        xn32[s] = (float)nx;
    }
    __syncthreads();  // buffer b is free
    if (threadIdx.x == 0 && c + 2 * G < nch) issue(b, c + 2 * G, nb, ne);
  }
}

// Row-group form, for long rows: W consecutive lanes share a row, so the
// row's columns and values are read by consecutive lanes (coalesced), the
// products are summed by W-lane shuffles, and every lane of the group forms
// the FP64 epilogue (lane 0 of the group stores it).  The state loads of
// the row are issued before the walk.
template <int PREC, int STAGE, int W>
__global__ void __launch_bounds__(256)
    k_stage_csr_grp(int64_t M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                    const void* __restrict__ val, const double* __restrict__ Keff, const double* __restrict__ x,
                    const float* __restrict__ x32, double* __restrict__ xn, float* __restrict__ xn32,
                    double* __restrict__ acc, double* __restrict__ v, double h) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = gt / W;
  const int sub = (int)(gt % W);
  const bool valid = s < M;
  double kf = 0.0, vs = 0.0, ac = 0.0;
  int64_t b = 0, e = 0;
  if (valid) {
    b = __ldg(rowptr + s);
    e = __ldg(rowptr + s + 1);
    if (sub == 0) {
      kf = __ldcs(Keff + s);
      vs = __ldcs(v + s);
      if (STAGE > 1) ac = __ldcs(acc + s);
    }
  }
  double y;
  if (PREC == LB_FP64) {
    const double* __restrict__ vv = static_cast<const double*>(val);
    double t = 0.0;
    for (int64_t q = b + sub; q < e; q += W) t = fma(__ldcs(vv + q), __ldg(x + __ldcs(col + q)), t);
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o, W);
    y = t;
  } else {
    const float* __restrict__ vv = static_cast<const float*>(val);
    float t = 0.f;
    for (int64_t q = b + sub; q < e; q += W) t = fmaf(__ldcs(vv + q), __ldg(x32 + __ldcs(col + q)), t);
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o, W);
    y = (double)t;
  }
  if (!valid || sub != 0) return;
  const double k = y + kf;
  double nx;
  if (STAGE == 1) {
    acc[s] = k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 2) {
    acc[s] = ac + 2.0 * k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 3) {
    acc[s] = ac + 2.0 * k;
    nx = vs + h * k;
  } else {
    nx = vs + (h / 6.0) * (ac + k);
    v[s] = nx;
  }
  if (PREC == LB_FP64)
    xn[s] = nx;
  else
    xn32[s] = (float)nx;
}

// Time-dependent form (Sec. 3, the rocked dimer: Q(t) = Q0 + eps(t) Q1): the
// FP64 stage for A0 = Q0 + R plus eps Q1 x, both row sums formed before the
// epilogue, each in the order of k_stage_csr_blk.  One thread per row.
template <int STAGE>
__global__ void __launch_bounds__(256)
    k_stage_csr_td(int64_t M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                   const double* __restrict__ val, const int64_t* __restrict__ rowptr1,
                   const int32_t* __restrict__ col1, const double* __restrict__ val1, double eps,
                   const double* __restrict__ K, const double* __restrict__ x, double* __restrict__ xn,
                   double* __restrict__ acc, double* __restrict__ v, double h) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const double kf = __ldcs(K + s), vs = __ldcs(v + s);
  const double ac = STAGE > 1 ? __ldcs(acc + s) : 0.0;
  const int64_t b = __ldg(rowptr + s), e = __ldg(rowptr + s + 1);
  const int64_t b1 = __ldg(rowptr1 + s), e1 = __ldg(rowptr1 + s + 1);
  double t = 0.0, t1 = 0.0;
#pragma unroll 4
  for (int64_t q = b; q < e; ++q) t = fma(__ldcs(val + q), __ldg(x + __ldcs(col + q)), t);
  for (int64_t q = b1; q < e1; ++q) t1 = fma(__ldcs(val1 + q), __ldg(x + __ldcs(col1 + q)), t1);
  const double k = fma(eps, t1, t) + kf;
  double nx;
  if (STAGE == 1) {
    acc[s] = k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 2) {
    acc[s] = ac + 2.0 * k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 3) {
    acc[s] = ac + 2.0 * k;
    nx = vs + h * k;
  } else {
    nx = vs + (h / 6.0) * (ac + k);
    v[s] = nx;
  }
  xn[s] = nx;
}

// Row-group form of k_stage_csr_td: W lanes per row, the row sums of A0 and
// of Q1 formed in the lane order and shuffle tree of k_stage_csr_grp, so that
// eps = 0 gives the bits of the autonomous step.
template <int STAGE, int W>
__global__ void __launch_bounds__(256)
    k_stage_csr_td_grp(int64_t M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const int64_t* __restrict__ rowptr1,
                       const int32_t* __restrict__ col1, const double* __restrict__ val1, double eps,
                       const double* __restrict__ K, const double* __restrict__ x, double* __restrict__ xn,
                       double* __restrict__ acc, double* __restrict__ v, double h) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = gt / W;
  const int sub = (int)(gt % W);
  const bool valid = s < M;
  double kf = 0.0, vs = 0.0, ac = 0.0;
  int64_t b = 0, e = 0, b1 = 0, e1 = 0;
  if (valid) {
    b = __ldg(rowptr + s);
    e = __ldg(rowptr + s + 1);
    b1 = __ldg(rowptr1 + s);
    e1 = __ldg(rowptr1 + s + 1);
    if (sub == 0) {
      kf = __ldcs(K + s);
      vs = __ldcs(v + s);
      if (STAGE > 1) ac = __ldcs(acc + s);
    }
  }
  double t = 0.0, t1 = 0.0;
  for (int64_t q = b + sub; q < e; q += W) t = fma(__ldcs(val + q), __ldg(x + __ldcs(col + q)), t);
  for (int64_t q = b1 + sub; q < e1; q += W) t1 = fma(__ldcs(val1 + q), __ldg(x + __ldcs(col1 + q)), t1);
#pragma unroll
  for (int o = W >> 1; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o, W);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o, W);
  }
  if (!valid || sub != 0) return;
  const double k = fma(eps, t1, t) + kf;
  double nx;
  if (STAGE == 1) {
    acc[s] = k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 2) {
    acc[s] = ac + 2.0 * k;
    nx = vs + 0.5 * h * k;
  } else if (STAGE == 3) {
    acc[s] = ac + 2.0 * k;
    nx = vs + h * k;
  } else {
    nx = vs + (h / 6.0) * (ac + k);
    v[s] = nx;
  }
  xn[s] = nx;
}

// c = (A64 - A32) v on the CSR pattern;  Keff = K + c.  One thread per row.
__global__ void __launch_bounds__(256)
    k_correction_csr(int64_t M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const double* __restrict__ v64, const float* __restrict__ v32, const double* __restrict__ x,
                     const double* __restrict__ K, double* __restrict__ Keff) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int64_t b = rowptr[s], e = rowptr[s + 1];
  double t = 0.0;
  for (int64_t q = b; q < e; ++q) t = fma(v64[q] - (double)v32[q], x[col[q]], t);
  Keff[s] = K[s] + t;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) b[i] = (float)a[i];
}

// The four shifted FP32 copies of x: copy o holds x[j + o] at index j.
__global__ void k_to_f32_shifted(int64_t M, const double* __restrict__ x, float* __restrict__ y, int64_t xstride) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float f = (float)x[j];
#pragma unroll
  for (int o = 0; o < 4; ++o)
    if (j >= o) y[o * xstride + (j - o)] = f;
}

// One warp per row: r_s = max |A_sn| (as float), then bf16(A_sn / r_s).
__global__ void k_pack_bf16(int64_t M, const double* __restrict__ A, uint16_t* __restrict__ Ab,
                            float* __restrict__ scale) {
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= M) return;
  const double* row = A + s * M;
  double mx = 0.0;
  for (int64_t n = lane; n < M; n += 32) mx = fmax(mx, fabs(row[n]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float r = (float)mx;
  if (!(r > 0.f)) r = 1.f;
  const double inv = 1.0 / (double)r;
  uint16_t* out = Ab + s * M;
  for (int64_t n = lane; n < M; n += 32) {
    __nv_bfloat16 q = __double2bfloat16(row[n] * inv);
    out[n] = *reinterpret_cast<uint16_t*>(&q);
  }
  if (lane == 0) scale[s] = r;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// RK4 workspace: FP64 stage vectors X, Y, the running combination and
// K + correction, and the FP32 stage vectors X32, Y32, each as four copies
// shifted by 0..3 elements (xstride floats apart, 256-byte aligned) so that
// every row of a dense FP32/BF16 product reads x with aligned 16-byte loads.
struct Work {
  double *X, *Y, *acc, *Keff;
  float *X32, *Y32;
  int64_t xstride;
  int* err;  // set by a kernel whose bounded wait ran out
};

inline int64_t x32_stride(int64_t M) { return (M + 63) & ~int64_t(63); }

Work carve(void* base, int64_t M) {
  char* p = static_cast<char*>(base);
  Work w;
  w.xstride = x32_stride(M);
  size_t d = align256(sizeof(double) * (size_t)M), f = sizeof(float) * 4 * (size_t)w.xstride;
  w.X = reinterpret_cast<double*>(p); p += d;
  w.Y = reinterpret_cast<double*>(p); p += d;
  w.acc = reinterpret_cast<double*>(p); p += d;
  w.Keff = reinterpret_cast<double*>(p); p += d;
  w.X32 = reinterpret_cast<float*>(p); p += f;
  w.Y32 = reinterpret_cast<float*>(p); p += f;
  w.err = reinterpret_cast<int*>(p);
  return w;
}

template <int PREC>
cudaError_t run_steps(int64_t M, const void* Ap, const float* scale, const double* A64,
                      int correct_every, const double* K, double* v, double dt, int64_t nsteps,
                      double* snaps, int64_t snap_every, const Work& w, cudaStream_t st) {
  const unsigned grid = (unsigned)((M + kWarpsPerBlock - 1) / kWarpsPerBlock);
  const unsigned bs = kWarpsPerBlock * 32;
  cudaError_t e;
  e = cudaMemcpyAsync(w.X, v, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(w.Keff, K, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (PREC != LB_FP64) {
    k_to_f32_shifted<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, v, w.X32, w.xstride);
    lbi::note_launch(1);
  }
  const bool correct = PREC != LB_FP64 && correct_every > 0 && A64 != nullptr;
  const int64_t xs = w.xstride;
  for (int64_t t = 0; t < nsteps; ++t) {
    if (correct && t % correct_every == 0) {
      k_correction<PREC><<<grid, bs, 0, st>>>(M, A64, Ap, scale, v, K, w.Keff);
      lbi::note_launch(1);
    }
    k_stage<PREC, 1><<<grid, bs, 0, st>>>(M, Ap, scale, w.Keff, w.X, w.X32, w.Y, w.Y32, xs, w.acc, v, dt);
    k_stage<PREC, 2><<<grid, bs, 0, st>>>(M, Ap, scale, w.Keff, w.Y, w.Y32, w.X, w.X32, xs, w.acc, v, dt);
    k_stage<PREC, 3><<<grid, bs, 0, st>>>(M, Ap, scale, w.Keff, w.X, w.X32, w.Y, w.Y32, xs, w.acc, v, dt);
    k_stage<PREC, 4><<<grid, bs, 0, st>>>(M, Ap, scale, w.Keff, w.Y, w.Y32, w.X, w.X32, xs, w.acc, v, dt);
    lbi::note_launch(4);
    if (snaps && snap_every > 0 && (t + 1) % snap_every == 0) {
      e = cudaMemcpyAsync(snaps + ((t + 1) / snap_every - 1) * M, v, sizeof(double) * M,
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

// Lanes per CSR row: the largest power of two W <= 32 with four or more
// entries per lane on average (W = 1: the block-staged thread-per-row form).
// Short rows favour one thread per row, which keeps 32 rows' loads in flight
// per warp instruction; long rows favour lanes that share a row's entries.
int csr_group_width(int64_t nnz, int64_t M) {
  const double mean = M > 0 ? (double)nnz / (double)M : 0.0;
  int w = 1;
  while (w < 32 && 4.0 * (2 * w) <= mean) w *= 2;
  return w;
}

// Staging capacity (entries) of k_stage_csr_blk: 1.5 times a block's mean
// range plus one row of slack, within 48 KB of shared memory.
int csr_stage_cap(int64_t nnz, int64_t M, size_t entry_bytes) {
  const double mean = M > 0 ? (double)nnz / (double)M : 0.0;
  const int64_t lim = (int64_t)((48 * 1024) / entry_bytes);
  int64_t cap = (int64_t)(1.5 * mean * 256.0) + 256;
  cap = (cap + 31) & ~int64_t(31);
  return (int)(cap < lim ? cap : lim);
}

template <int PREC>
cudaError_t run_steps_csr(int64_t M, const int64_t* rowptr, const int32_t* col, const void* val,
                          const double* val64, int correct_every, const double* K, double* v, double dt,
                          int64_t nsteps, const Work& w, cudaStream_t st) {
  const unsigned grid = (unsigned)((M + 255) / 256);
  cudaError_t e;
  e = cudaMemcpyAsync(w.X, v, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(w.Keff, K, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (PREC != LB_FP64) {
    k_to_f32<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, v, w.X32);
    lbi::note_launch(1);
  }
  const bool correct = PREC == LB_FP32 && correct_every > 0 && val64 != nullptr;
  // lanes per row from the mean row length; W = 1: the block-staged kernel
  int64_t nnz = 0;
  e = cudaMemcpyAsync(&nnz, rowptr + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const int W = csr_group_width(nnz, M);
  const unsigned ggrid = (unsigned)((M * W + 255) / 256);
  using V = typename std::conditional<PREC == LB_FP64, double, float>::type;
  const int cap = csr_stage_cap(nnz, M, sizeof(V) + sizeof(int32_t));
  const size_t smem = (sizeof(V) + sizeof(int32_t)) * (size_t)cap;
  // short rows: the pipelined kernel when the arrays allow 16-byte bulk
  // copies (the library's own arrays always do), else the block-staged one
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool pipe = W == 1 && al16(col) && al16(val) && al16(rowptr) && al16(v);
  // its staging capacity: the largest range of a chunk of 256 rows, when two
  // buffers of it stay within 112 KB (chunks above the capacity are summed
  // from global memory)
  int pcap = 0;
  if (pipe) {
    e = cudaMemsetAsync(w.err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      k_chunk_max_range<<<(unsigned)(((M + 255) / 256 + 255) / 256), 256, 0, st>>>(M, rowptr, w.err);
      lbi::note_launch(1);
      int mx = 0;
      e = cudaMemcpyAsync(&mx, w.err, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      const int lim = (int)((56 * 1024 - kPipeRowBytes) / (sizeof(V) + sizeof(int32_t))) - 16;
      pcap = ((mx < lim ? mx : lim) + 7) & ~7;
    }
    if (e != cudaSuccess) return e;
  }
  const size_t psmem = 2 * csr_pipe_buf_bytes<V>(pcap);
  unsigned pgrid = 0;
  if (W == 1) {
    auto attr = [&](const void* k, size_t bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    if (pipe) {
      attr((const void*)k_stage_csr_pipe<PREC, 1>, psmem);
      attr((const void*)k_stage_csr_pipe<PREC, 2>, psmem);
      attr((const void*)k_stage_csr_pipe<PREC, 3>, psmem);
      attr((const void*)k_stage_csr_pipe<PREC, 4>, psmem);
      int dev = 0, sms = 0, per = 0;
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage_csr_pipe<PREC, 1>, 256, psmem);
      const int64_t nch = (M + 255) / 256, resident = (int64_t)sms * (per > 0 ? per : 1);
      pgrid = (unsigned)(nch < resident ? nch : resident);
    } else {
      attr((const void*)k_stage_csr_blk<PREC, 1>, smem);
      attr((const void*)k_stage_csr_blk<PREC, 2>, smem);
      attr((const void*)k_stage_csr_blk<PREC, 3>, smem);
      attr((const void*)k_stage_csr_blk<PREC, 4>, smem);
    }
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(w.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  auto stage = [&](auto stage_c, const double* xc, const float* xc32, double* xn, float* xn32) {
    constexpr int S = decltype(stage_c)::value;
    switch (W) {
      case 2:
        k_stage_csr_grp<PREC, S, 2><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, w.Keff, xc, xc32, xn, xn32, w.acc, v, dt);
        break;
      case 4:
        k_stage_csr_grp<PREC, S, 4><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, w.Keff, xc, xc32, xn, xn32, w.acc, v, dt);
        break;
      case 8:
        k_stage_csr_grp<PREC, S, 8><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, w.Keff, xc, xc32, xn, xn32, w.acc, v, dt);
        break;
      case 16:
        k_stage_csr_grp<PREC, S, 16><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, w.Keff, xc, xc32, xn, xn32, w.acc, v, dt);
        break;
      case 32:
        k_stage_csr_grp<PREC, S, 32><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, w.Keff, xc, xc32, xn, xn32, w.acc, v, dt);
        break;
      default:
        if (pipe)
          k_stage_csr_pipe<PREC, S><<<pgrid, 256, psmem, st>>>(M, nnz, rowptr, col, val, pcap, w.Keff, xc, xc32, xn,
                                                               xn32, w.acc, v, dt, w.err);
        else
          k_stage_csr_blk<PREC, S><<<grid, 256, smem, st>>>(M, rowptr, col, val, cap, w.Keff, xc, xc32, xn, xn32,
                                                            w.acc, v, dt);
    }
  };
  for (int64_t t = 0; t < nsteps; ++t) {
    if (correct && t % correct_every == 0) {
      k_correction_csr<<<grid, 256, 0, st>>>(M, rowptr, col, val64, static_cast<const float*>(val), v, K, w.Keff);
      lbi::note_launch(1);
    }
    stage(std::integral_constant<int, 1>{}, w.X, w.X32, w.Y, w.Y32);
    stage(std::integral_constant<int, 2>{}, w.Y, w.Y32, w.X, w.X32);
    stage(std::integral_constant<int, 3>{}, w.X, w.X32, w.Y, w.Y32);
    stage(std::integral_constant<int, 4>{}, w.Y, w.Y32, w.X, w.X32);
    lbi::note_launch(4);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !pipe) return e;
  // a bounded wait of the pipelined kernel that ran out
  int flag = 0;
  e = cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && flag) e = cudaErrorLaunchTimeout;
  return e;
}

// eps(t) periodic with period T: seg_eps[k] for (t mod T) in
// [seg_start[k], seg_start[k + 1]).
double eps_at(double t, int nseg, const double* seg_start, const double* seg_eps, double T) {
  double u = std::fmod(t, T);
  if (u < 0) u += T;
  int k = 0;
  while (k + 1 < nseg && u >= seg_start[k + 1]) ++k;
  return seg_eps[k];
}

}  // namespace

namespace lbi {

// RK4 for dv/dt = (A0 + eps(t) Q1) v + K, each stage with eps at its own
// time, the end stages taken 1e-6 dt inside the step (so that a step between
// two switches sees one value whatever the rounding of its end times).
cudaError_t rk4_csr_td(int64_t M, const int64_t* rowptr, const int32_t* col, const double* val,
                       const int64_t* rowptr1, const int32_t* col1, const double* val1, const double* K, int nseg,
                       const double* seg_start, const double* seg_eps, double T, double t0, double* v, double dt,
                       int64_t nsteps, void* work, cudaStream_t st) {
  Work w = carve(work, M);
  const unsigned grid = (unsigned)((M + 255) / 256);
  int64_t nnz = 0;
  cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const int W = csr_group_width(nnz, M);
  const unsigned ggrid = (unsigned)((M * W + 255) / 256);
  auto stage = [&](auto stage_c, double eps, const double* xc, double* xn) {
    constexpr int S = decltype(stage_c)::value;
    switch (W) {
      case 2:
        k_stage_csr_td_grp<S, 2><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
        break;
      case 4:
        k_stage_csr_td_grp<S, 4><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
        break;
      case 8:
        k_stage_csr_td_grp<S, 8><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
        break;
      case 16:
        k_stage_csr_td_grp<S, 16><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
        break;
      case 32:
        k_stage_csr_td_grp<S, 32><<<ggrid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
        break;
      default:
        k_stage_csr_td<S><<<grid, 256, 0, st>>>(M, rowptr, col, val, rowptr1, col1, val1, eps, K, xc, xn, w.acc, v, dt);
    }
  };
  e = cudaMemcpyAsync(w.X, v, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
  for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
    const double t = t0 + (double)n * dt;
    const double e1 = eps_at(t + 1e-6 * dt, nseg, seg_start, seg_eps, T);
    const double e2 = eps_at(t + 0.5 * dt, nseg, seg_start, seg_eps, T);
    const double e4 = eps_at(t + dt - 1e-6 * dt, nseg, seg_start, seg_eps, T);
    stage(std::integral_constant<int, 1>{}, e1, w.X, w.Y);
    stage(std::integral_constant<int, 2>{}, e2, w.Y, w.X);
    stage(std::integral_constant<int, 3>{}, e2, w.X, w.Y);
    stage(std::integral_constant<int, 4>{}, e4, w.Y, w.X);
    lbi::note_launch(4);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t rk4_csr(int64_t M, int precision, const int64_t* rowptr, const int32_t* col, const void* val,
                    const double* val64, int correct_every, const double* K, double* v, double dt, int64_t nsteps,
                    void* work, cudaStream_t st) {
  Work w = carve(work, M);
  if (precision == LB_FP64)
    return run_steps_csr<LB_FP64>(M, rowptr, col, val, val64, correct_every, K, v, dt, nsteps, w, st);
  if (precision == LB_FP32)
    return run_steps_csr<LB_FP32>(M, rowptr, col, val, val64, correct_every, K, v, dt, nsteps, w, st);
  return cudaErrorInvalidValue;
}

cudaError_t to_f32(int64_t n, const double* x, float* y, cudaStream_t st) {
  k_to_f32<<<4 * 152 * 8, 256, 0, st>>>(n, x, y);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t pack_fp32(int64_t M, const double* A, float* A32, cudaStream_t st) {
  const int64_t n = M * M;
  k_to_f32<<<4 * 152 * 8, 256, 0, st>>>(n, A, A32);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t pack_bf16(int64_t M, const double* A, uint16_t* Ab, float* scale, cudaStream_t st) {
  k_pack_bf16<<<(unsigned)((M + kWarpsPerBlock - 1) / kWarpsPerBlock), kWarpsPerBlock * 32, 0, st>>>(
      M, A, Ab, scale);
  note_launch(1);
  return cudaGetLastError();
}

size_t rk4_workspace_bytes(int64_t M) {
  return 4 * align256(sizeof(double) * (size_t)M) + 2 * sizeof(float) * 4 * (size_t)x32_stride(M) + 256;
}

cudaError_t rk4_dense(int64_t M, int precision, const void* Ap, const float* scale,
                      const double* A64, int correct_every, const double* K, double* v, double dt,
                      int64_t nsteps, double* snaps, int64_t snap_every, void* work,
                      cudaStream_t st) {
  Work w = carve(work, M);
  switch (precision) {
    case LB_FP64:
      return run_steps<LB_FP64>(M, Ap, scale, A64, correct_every, K, v, dt, nsteps, snaps, snap_every, w, st);
    case LB_FP32:
      return run_steps<LB_FP32>(M, Ap, scale, A64, correct_every, K, v, dt, nsteps, snaps, snap_every, w, st);
    case LB_BF16:
      return run_steps<LB_BF16>(M, Ap, scale, A64, correct_every, K, v, dt, nsteps, snaps, snap_every, w, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lbi

// lb_noalloc.cu -- a variant of lb_structure_export for callers that cannot
// allocate device memory per call: processes whose host framework's caching
// allocator has reserved the device memory (a cudaMalloc there fails or
// fragments the pool, and a cudaFree synchronizes the whole device, stalling
// every other stream), and real-time or embedded callers that reserve all
// memory once at start-up and may not allocate afterwards.  The export's
// scratch (the per-m counts and their exclusive scan) lives in a file-scope
// __device__ array of fixed size instead of buffers allocated per call.  The
// paper has no counterpart: it is a deployment concern of this library.
#include "lb_internal.h"

namespace {

// Largest M the static scratch covers: N <= 256 (M = N^2 - 1 = 65535).
constexpr int64_t kNoAllocMaxM = 65535;

// [0, kNoAllocMaxM + 1): per-m counts; [kNoAllocMaxM + 1, 2 (kNoAllocMaxM + 1)):
// offsets (exclusive scan, M + 1 entries).  1 MiB per device, held by every
// GPU that loads the library until the process exits.  In host code this
// name is only a stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) int64_t g_export_scratch[2 * (kNoAllocMaxM + 1)];

constexpr int kScanThreads = 1024;

// Exclusive scan of per[0, M) into off[0, M], off[M] = total, by one block:
// thread t sums a contiguous chunk, the block scans the chunk sums, and each
// thread writes its chunk's prefixes.  Every word of off[0, M] is written, so
// nothing in the scratch has to start at zero.
__global__ void __launch_bounds__(kScanThreads) k_scan_single_block(const int64_t* __restrict__ per, int64_t M,
                                                                    int64_t* __restrict__ off) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t chunk = (M + kScanThreads - 1) / kScanThreads;
  const int64_t b0 = t * chunk < M ? t * chunk : M;
  const int64_t b1 = b0 + chunk < M ? b0 + chunk : M;
  int64_t s = 0;
  for (int64_t i = b0; i < b1; ++i) s += per[i];
  // inclusive warp scan of the chunk sums
  int64_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t x = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int64_t run = inc - s + (w > 0 ? warp_tot[w - 1] : 0);  // exclusive prefix of this chunk
  for (int64_t i = b0; i < b1; ++i) {
    off[i] = run;
    run += per[i];
  }
  if (t == kScanThreads - 1) off[M] = warp_tot[kScanThreads / 32 - 1];
}

// Device address of g_export_scratch in the current device's context, looked
// up on every call (cheap next to the count and fill kernels).  A cached
// address would outlive a cudaDeviceReset or a recreated primary context, in
// which the module, and with it the array, is loaded again elsewhere.
cudaError_t scratch_address(int64_t** out) {
  int64_t* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_export_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" {

int lb_structure_export_noalloc(const lb_basis_t* b, int which, int32_t* idx3, double* val, int64_t capacity,
                                int64_t* nnz, void* stream) {
  if (b == nullptr || nnz == nullptr) {
    lbi::set_error("lb_structure_export_noalloc: NULL argument");
    return LB_EINVAL;
  }
  if (which != LB_F && which != LB_D) {
    lbi::set_error("lb_structure_export_noalloc: which = %d", which);
    return LB_EINVAL;
  }
  if (b->M > kNoAllocMaxM) {
    lbi::set_error("lb_structure_export_noalloc: M = %lld (N = %d) exceeds the static scratch maximum "
                   "M = %lld (N = 256); use lb_structure_export",
                   (long long)b->M, b->N, (long long)kNoAllocMaxM);
    return LB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_structure_export_noalloc: scratch address");
  int64_t* per = scratch;
  int64_t* off = scratch + (kNoAllocMaxM + 1);
  const lb::BasisView B = b->view();
  if ((e = lbi::structure_count(B, which, per, st)) != cudaSuccess)
    return lbi::cuda_fail(e, "lb_structure_export_noalloc: count");
  k_scan_single_block<<<1, kScanThreads, 0, st>>>(per, b->M, off);
  lbi::note_launch(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return lbi::cuda_fail(e, "lb_structure_export_noalloc: scan");
  int64_t total = 0;
  if ((e = cudaMemcpyAsync(&total, off + b->M, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return lbi::cuda_fail(e, "lb_structure_export_noalloc: total");
  *nnz = total;
  if (idx3 == nullptr || val == nullptr) {
    lbi::set_error("lb_structure_export_noalloc: NULL output buffer");
    return LB_EINVAL;
  }
  if (capacity < total) {
    lbi::set_error("lb_structure_export_noalloc: capacity %lld < %lld triples", (long long)capacity,
                   (long long)total);
    return LB_EINVAL;
  }
  if ((e = lbi::structure_fill(B, which, off, idx3, val, st)) != cudaSuccess)
    return lbi::cuda_fail(e, "lb_structure_export_noalloc: fill");
  // the next call reuses the scratch: wait for the fill that reads the offsets
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return lbi::cuda_fail(e, "lb_structure_export_noalloc: fill");
  return LB_OK;
}

}  // extern "C"

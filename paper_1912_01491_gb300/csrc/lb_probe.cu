// lb_probe.cu -- FP64 fused multiply-add throughput probe (the roofline
// denominator of the FP64-bound kernels), and the process-wide count of
// kernels this library has launched.
#include <atomic>

#include "lb_internal.h"

namespace {

std::atomic<long long> g_launches{0};

// Eight independent FMA chains per thread keep the FP64 pipe busy.
__global__ void k_fp64_fma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

}  // namespace

namespace lbi {
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace lbi

extern "C" {

long long lb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int lb_probe_fp64(double* tflops) {
  if (!tflops) {
    lbi::set_error("lb_probe_fp64: NULL output");
    return LB_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_probe_fp64");
  const int blocks = sms * 4, threads = 256, iters = 20000;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fp64_fma<<<blocks, threads>>>(out, 100, 0.999, 1e-3);  // warm-up
    cudaEventRecord(e0);
    k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999, 1e-3);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    lbi::note_launch(2);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return lbi::cuda_fail(e, "lb_probe_fp64");
  *tflops = 2.0 * 8.0 * (double)blocks * threads * iters / (ms * 1e-3) / 1e12;
  return LB_OK;
}

}  // extern "C"

// fe_devrate.cu -- issue rate of the FP64 unit of the device (not in the paper): the
// denominator of the roofline of the FP64 kernels, which are bound by FP64 arithmetic, not
// by memory.  Each thread runs eight independent dependency chains of one FP64 operation
// (fused multiply-add, add or multiply), enough warps per SM to hide the pipeline latency;
// every block times its loop with the SM clock, so the rate comes out in operations per
// clock per SM whatever clock the GPU runs at, and the event time of the launch gives the
// clock it ran at.
#include <algorithm>
#include <vector>

#include "fe_internal.cuh"

namespace fe {
namespace {

constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSM = 4;
constexpr int kRateChains = 8;

template <int OP>
__global__ void __launch_bounds__(kRateThreads) k_fp64_rate(int iters, double seed, double* sink,
                                                            long long* cycles) {
  double a[kRateChains];
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) a[k] = seed + 1e-3 * (threadIdx.x + k);
  const double m = 1.0 - 1e-12, c = 1e-15;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) {
      if (OP == FE_RATE_DFMA) a[k] = fma(a[k], m, c);
      else if (OP == FE_RATE_DADD) a[k] = a[k] + c;
      else a[k] = a[k] * m;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) s += a[k];
  if (s == 1234.5) sink[0] = s;   // never true; keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_fp64_rate(int device, int op, double* per_clock_per_sm, double* sm_ghz) {
  if (!per_clock_per_sm || op < FE_RATE_DFMA || op > FE_RATE_DMUL) return set_error(FE_EINVAL, "bad arguments");
  int prev = -1;
  cudaGetDevice(&prev);
  fe_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (st) return st;
  const int sms = sm_count(device);
  const int blocks = sms * kRateBlocksPerSM;
  const int iters = 1 << 12;
  double* sink = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<long long> hc(blocks);
  float ms = 0.f;
  auto launch = [&] {
    if (op == FE_RATE_DFMA) k_fp64_rate<FE_RATE_DFMA><<<blocks, kRateThreads>>>(iters, 1.0, sink, cyc);
    else if (op == FE_RATE_DADD) k_fp64_rate<FE_RATE_DADD><<<blocks, kRateThreads>>>(iters, 1.0, sink, cyc);
    else k_fp64_rate<FE_RATE_DMUL><<<blocks, kRateThreads>>>(iters, 1.0, sink, cyc);
  };
  if (!st) st = cuda_check(cudaMalloc((void**)&sink, sizeof(double)), "cudaMalloc");
  if (!st) st = cuda_check(cudaMalloc((void**)&cyc, sizeof(long long) * blocks), "cudaMalloc");
  if (!st) st = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  if (!st) {
    launch();   // warm-up (clocks ramp up, code loaded)
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    st = cuda_check(cudaEventSynchronize(e1), "rate kernel");
  }
  if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  if (!st) st = cuda_check(cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (!st) {
    // blocks run kRateBlocksPerSM to an SM at once: the SM's operations over the longest of
    // its blocks' loops
    const long long cmax = *std::max_element(hc.begin(), hc.end());
    const double ops_per_sm = (double)kRateBlocksPerSM * kRateThreads * (double)iters * kRateChains;
    *per_clock_per_sm = ops_per_sm / (double)cmax;
    if (sm_ghz) *sm_ghz = (double)cmax / (ms * 1e6);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

}  // extern "C"

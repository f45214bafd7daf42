// fe_debug.cu -- the host side of the bounds-checking build (bounds.cuh; not in the paper):
// the registry of the per-unit error words, the call that reads and clears them, and a
// self-test that makes one checked access out of range on purpose.  In the ordinary build the
// calls report that the checks are not compiled in.
#include <mutex>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

#ifdef FE_DEBUG_BOUNDS

namespace {

std::vector<BoundsReader>& bounds_readers() {
  static std::vector<BoundsReader> v;
  return v;
}

std::mutex& bounds_mutex() {
  static std::mutex m;
  return m;
}

// One checked read of buf[index] (buf holds n doubles): out of range, the check records the
// index and reads buf[0] instead.
__global__ void k_bounds_selftest(const double* __restrict__ buf, int64_t n, int64_t index, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = buf[FE_CHK(index, n, kSiteSelfTest)];
}

}  // namespace

void register_bounds_reader(BoundsReader f) {
  std::lock_guard<std::mutex> lock(bounds_mutex());
  bounds_readers().push_back(f);
}

#endif

}  // namespace fe

using namespace fe;

extern "C" {

int fe_debug_bounds_enabled(void) {
#ifdef FE_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}

fe_status fe_debug_bounds(int device, int* site, int64_t* index) {
  if (!site || !index) return set_error(FE_EINVAL, "null argument");
  *site = 0;
  *index = 0;
#ifdef FE_DEBUG_BOUNDS
  int prev = -1;
  cudaGetDevice(&prev);
  fe_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (st) return st;
  unsigned long long first = 0;
  {
    std::lock_guard<std::mutex> lock(bounds_mutex());
    for (BoundsReader f : bounds_readers()) {
      unsigned long long w = 0;
      if ((st = cuda_check(f(&w), "bounds word"))) break;
      if (!first) first = w;
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (st) return st;
  if (first) {
    *site = (int)(first >> 48);
    const unsigned long long lo = first & 0xffffffffffffULL;   // 48 bits, sign-extended
    *index = (int64_t)((lo & 0x800000000000ULL) ? (lo | 0xffff000000000000ULL) : lo);
  }
#else
  (void)device;
#endif
  return FE_OK;
}

fe_status fe_debug_bounds_selftest(int device, int64_t index, int64_t n) {
#ifdef FE_DEBUG_BOUNDS
  if (n < 1 || n > 1024) return set_error(FE_EINVAL, "n must be in [1, 1024]");
  int prev = -1;
  cudaGetDevice(&prev);
  fe_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (st) return st;
  double* buf = nullptr;
  if (!(st = cuda_check(cudaMalloc((void**)&buf, sizeof(double) * (size_t)(n + 1)), "cudaMalloc"))) {
    cudaMemset(buf, 0, sizeof(double) * (size_t)(n + 1));
    k_bounds_selftest<<<1, 32>>>(buf, n, index, buf + n);
    st = cuda_check(cudaDeviceSynchronize(), "bounds self-test");
    cudaFree(buf);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return st;
#else
  (void)device;
  (void)index;
  (void)n;
  return set_error(FE_EINVAL, "not a bounds-checking build (FE_DEBUG_BOUNDS)");
#endif
}

}  // extern "C"

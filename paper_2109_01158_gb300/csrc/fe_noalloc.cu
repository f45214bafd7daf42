// fe_noalloc.cu -- fe_energy_noalloc: the energy evaluation for callers that cannot let
// this library allocate device memory.
//
// The regular entry points keep a context whose buffers (mesh copies, precompute, work
// arrays, reduction partials) the library allocates with cudaMalloc.  Some host programs
// cannot allow that: their GPU memory is entirely owned by their own pool allocator, or
// their time-critical loop must not call cudaMalloc (which can synchronise the device).
// This entry point takes every input and the output from the caller and allocates nothing.
// Its only scratch -- the per-block partial sums of the energy and of b.v, and the ticket
// that elects the block finishing the reduction -- lives in the file-scope device array
// below, of fixed size (2 * 1216 + 2 doubles = 19,472 bytes), which every GPU that loads
// the library holds until the process exits.
//
// Set-up: the first call on a device looks up the device address of that array with
// cudaGetSymbolAddress (with the device current) and caches it; make that first call
// before any stream capture.  Every call uses the same array and leaves its contents
// behind; each call clears the ticket before its kernel.  Calls that overlap on the GPU
// (on different streams, or from different host threads) race on the array and give wrong
// results: serialise them.
#include <mutex>

#include "density_f64.cuh"  // W of eqs. neoHook / pLaplacian in FP64
#include "fe_internal.cuh"

namespace fe {
namespace {

constexpr int kNoAllocBlocks = 1216;
constexpr int kNoAllocScratchDoubles = 2 * kNoAllocBlocks + 2;
constexpr unsigned kNoAllocBadIndex = 1u, kNoAllocDomain = 2u;

// [0, B): element partial sums, [B, 2B): partial sums of b.v, [2B]: ticket (as uint32),
// [2B + 1]: flags (as uint32: an element named a node outside [0, nn); some det F <= 0).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
fe_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(FE_EINVAL, "device index too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    fe_status st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    if (st) return st;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return FE_OK;
}

__device__ __forceinline__ double nsum_warp(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double nsum_block(double x, double* sh) {
  x = nsum_warp(x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  x = (threadIdx.x < kThreads / 32) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) x = nsum_warp(x);
  __syncthreads();
  return x;
}

// One launch: each block sums |T| W over a grid-stride range of elements and b.v over a
// grid-stride range of dofs; the last block to finish adds the partials in a fixed order.
// Inputs in the paper's layouts: coords[i*DIM+m], elems[e*(DIM+1)+l],
// dphi[(e*(DIM+1)+l)*DIM+m], vol[e], b[i*D+j], v[i*D+j].  W is evaluated as in the context
// kernels: F = I + H with H = sum_{l>=1} (u_l - u_0) grad(phi_l)^T, u = v - X (Neo-Hookean,
// displacement form of eq. neoHook) or u = v (p-Laplacians).  An element with det F <= 0 adds
// nothing and sets the domain flag (J = +Inf at the end, also for an element of volume 0);
// an element naming a node outside [0, nn) is skipped without reading it and sets the index
// flag (J = NaN).
template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_energy_noalloc(
    int64_t nn, int64_t ne, const double* __restrict__ coords, const int32_t* __restrict__ elems,
    const double* __restrict__ dphi, const double* __restrict__ vol, const double* __restrict__ b,
    const double* __restrict__ v, ModelParams mp, double* scratch, double* J) {
  constexpr int K = DIM + 1;
  __shared__ double sh[kThreads / 32];
  __shared__ bool am_last;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + 2 * kNoAllocBlocks);
  unsigned* flags = reinterpret_cast<unsigned*>(scratch + 2 * kNoAllocBlocks + 1);
  double acc = 0.0;
  unsigned fl = 0u;
  for (int64_t e = tid; e < ne; e += stride) {
    int64_t n[K];
    bool inside = true;
#pragma unroll
    for (int l = 0; l < K; ++l) {
      n[l] = elems[e * K + l];
      inside = inside && (uint64_t)n[l] < (uint64_t)nn;
    }
    if (!inside) {
      fl |= kNoAllocBadIndex;
      continue;
    }
    double ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
      for (int j = 0; j < D; ++j)
        ul[l][j] = (MODEL == FE_NEOHOOKE) ? v[n[l] * D + j] - coords[n[l] * DIM + j] : v[n[l] * D + j];
    double H[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double s = 0.0;
#pragma unroll
        for (int l = 1; l < K; ++l) s = fma(ul[l][j] - ul[0][j], dphi[(e * K + l) * DIM + m], s);
        H[j][m] = s;
      }
    double W;
    if constexpr (MODEL == FE_NEOHOOKE) {
      bool bad = false;
      W = nh_density_disp<DIM>(H, mp, bad);
      if (bad) {
        fl |= kNoAllocDomain;
        continue;
      }
    } else if constexpr (MODEL == FE_PLAPLACE_LP) {
      double sp = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double ap, ap2;
        plap_lp_terms(H[0][m], mp, &ap, &ap2);
        sp += ap;
      }
      W = sp / mp.p;
    } else {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) s = fma(H[0][m], H[0][m], s);
      W = plap_density(s, mp);
    }
    acc = fma(vol[e], W, acc);
  }
  double dot = 0.0;
  if (b)
    for (int64_t k = tid; k < nn * D; k += stride) dot = fma(b[k], v[k], dot);
  acc = nsum_block(acc, sh);
  dot = nsum_block(dot, sh);
  // the block's flags reach the word before its ticket is taken
  const int any_index = __syncthreads_or((int)(fl & kNoAllocBadIndex));
  const int any_domain = __syncthreads_or((int)(fl & kNoAllocDomain));
  if (threadIdx.x == 0) {
    const unsigned bf = (any_index ? kNoAllocBadIndex : 0u) | (any_domain ? kNoAllocDomain : 0u);
    if (bf) atomicOr(flags, bf);
    scratch[blockIdx.x] = acc;
    scratch[kNoAllocBlocks + blockIdx.x] = dot;
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double s = 0.0, t = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += kThreads) {
    s += __ldcg(scratch + k);
    t += __ldcg(scratch + kNoAllocBlocks + k);
  }
  s = nsum_block(s, sh);
  t = nsum_block(t, sh);
  if (threadIdx.x == 0) {
    const unsigned f = atomicOr(flags, 0u);
    *J = (f & kNoAllocBadIndex) ? CUDART_NAN : (f & kNoAllocDomain) ? CUDART_INF : s - t;
    *ticket = 0u;
    *flags = 0u;
  }
}

// Makes `dev` current for the scope of a call and restores the caller's device after it.
struct NoAllocGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit NoAllocGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) err = cudaSetDevice(dev);
  }
  ~NoAllocGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" fe_status fe_energy_noalloc(int device, void* cuda_stream, int dim, int d, int model,
                                       double p, double C1, double D1, int64_t n_nodes,
                                       const double* coords_dev, int64_t n_elems,
                                       const int32_t* elems_dev, const double* dphi_dev,
                                       const double* vol_dev, const double* b_dev,
                                       const double* v_dev, double* J_dev) {
  if (dim != 2 && dim != 3) return set_error(FE_EINVAL, "fe_energy_noalloc: dim must be 2 or 3");
  if (model != FE_NEOHOOKE && model != FE_PLAPLACE && model != FE_PLAPLACE_LP)
    return set_error(FE_EINVAL, "fe_energy_noalloc: unknown model");
  if (model == FE_NEOHOOKE ? d != dim : d != 1)
    return set_error(FE_EINVAL, "fe_energy_noalloc: model and d do not match (Neo-Hookean d = dim, p-Laplacians d = 1)");
  if (model != FE_NEOHOOKE && !(p > 1.0)) return set_error(FE_EINVAL, "fe_energy_noalloc: p must be > 1");
  if (n_nodes < 0 || n_elems < 0) return set_error(FE_EINVAL, "fe_energy_noalloc: negative size");
  if (n_elems * (dim + 1) >= ((int64_t)1 << 31) || n_nodes * d >= ((int64_t)1 << 31))
    return set_error(FE_EINVAL,
                     "fe_energy_noalloc: size beyond the maximum (n_elems*(dim+1) and n_nodes*d must be < 2^31)");
  if (!v_dev || !J_dev || (n_elems > 0 && (!coords_dev || !elems_dev || !dphi_dev || !vol_dev)))
    return set_error(FE_EINVAL, "fe_energy_noalloc: null input or output");
  int n_dev = 0;
  fe_status st = cuda_check(cudaGetDeviceCount(&n_dev), "cudaGetDeviceCount");
  if (st) return st;
  if (device < 0 || device >= n_dev) return set_error(FE_EINVAL, "fe_energy_noalloc: no such device");
  NoAllocGuard guard(device);
  if (guard.err != cudaSuccess) return cuda_check(guard.err, "cudaSetDevice");
  double* scratch = nullptr;
  st = scratch_address(device, &scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the ticket and the flags must start at zero (a call that was interrupted could leave
  // them set)
  st = cuda_check(cudaMemsetAsync(scratch + 2 * kNoAllocBlocks, 0, 2 * sizeof(double), s), "cudaMemsetAsync");
  if (st) return st;
  ModelParams mp;
  mp.p = p;
  mp.C1 = C1;
  mp.D1 = D1;
  mp.twoC1 = 2.0 * C1;
  mp.twoD1 = 2.0 * D1;
  mp.pcase = (p == 2.0) ? 2 : (p == 3.0) ? 3 : 0;
  const int64_t work = n_elems > n_nodes * d ? n_elems : n_nodes * d;
  const int grid = grid_for(work, kNoAllocBlocks);
#define FE_NOALLOC(DIM_, D_, M_)                                                                        \
  k_energy_noalloc<DIM_, D_, M_><<<grid, kThreads, 0, s>>>(n_nodes, n_elems, coords_dev, elems_dev, dphi_dev, \
                                                          vol_dev, b_dev, v_dev, mp, scratch, J_dev)
  if (model == FE_NEOHOOKE) {
    if (dim == 2) FE_NOALLOC(2, 2, FE_NEOHOOKE);
    else FE_NOALLOC(3, 3, FE_NEOHOOKE);
  } else if (model == FE_PLAPLACE_LP) {
    if (dim == 2) FE_NOALLOC(2, 1, FE_PLAPLACE_LP);
    else FE_NOALLOC(3, 1, FE_PLAPLACE_LP);
  } else {
    if (dim == 2) FE_NOALLOC(2, 1, FE_PLAPLACE);
    else FE_NOALLOC(3, 1, FE_PLAPLACE);
  }
#undef FE_NOALLOC
  return cuda_check(cudaGetLastError(), "fe_energy_noalloc launch");
}

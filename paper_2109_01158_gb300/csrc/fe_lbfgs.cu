// fe_lbfgs.cu -- the limited-memory BFGS inverse Hessian on the device (not in the paper,
// whose minimiser is a closed trust-region toolbox; the minimiser driven by the kernels).
//
// The m most recent pairs s_i = v_{i+1} - v_i, y_i = g_{i+1} - g_i (oldest first) define
// H = gamma I + [S gamma Y] M [S^T; gamma Y^T] in the compact representation of Byrd,
// Nocedal & Schnabel (Math. Prog. 63, 1994, Thm. 2.2), with
//   M = [[R^-T (D + gamma Y^T Y) R^-1, -R^-T], [-R^-1, 0]],
//   R_ij = s_i.y_j (i <= j), D = diag(s_i.y_i), gamma = s.y / y.y of the newest pair,
// which equals the two-loop recursion in exact arithmetic.  With a = S^T g, b = Y^T g,
// t = R^-1 a and p = R^-T ((D + gamma Y^T Y) t - gamma b) the direction is
//   d = -H g = -gamma g - S p + gamma Y t,
// and with no pairs d = -g / ||g|| (a first step of unit length).
//
// Device data: m + 1 slots of s and y (the pairs in use plus one spare that receives the
// next pair), the small matrices s_i.y_j and y_i.y_j between slots, and the direction's
// coefficients.  A direction is two passes over the slots:
//   k_lb_project  a, b and g.g in one fixed-order reduction; its last block solves for the
//                 coefficients (O(k^2), one thread)
//   k_lb_combine  d from g and the slots, and g.d (read by the host)
// An update writes s and y into the spare slot and, in the same pass, their products with
// the slots in use; the host keeps the pair when s.y > 0 (the spare joins the ring and the
// oldest slot becomes the spare when the memory is full).
#include <new>
#include <vector>

#include "fe_internal.cuh"
#include "reduce.cuh"
#include "trace.h"

namespace {
constexpr int kMaxPairs = 16;
}

struct fe_lbfgs {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  int m = 0;
  double* S = nullptr;      // (m + 1) slots of n
  double* Y = nullptr;      // (m + 1) slots of n
  double* SY = nullptr;     // (m + 1)^2: SY[i * (m + 1) + j] = s_i . y_j
  double* YY = nullptr;     // (m + 1)^2: y_i . y_j
  double* coef = nullptr;   // 1 + 2 kMaxPairs direction coefficients
  double* scal = nullptr;   // [0] s.y of the last update, [1] g.d of the last direction, [2] max |g|
  double* part = nullptr;   // partial sums
  unsigned* ticket = nullptr;
  double* host = nullptr;   // page-locked copy of scal
  int count = 0;            // pairs in use
  int ring[kMaxPairs];      // slots of the pairs in use, oldest first
  int spare = 0;
};

namespace fe {
namespace {

struct LbSlots {
  int s[kMaxPairs];
};

// Slots of the K pairs in use (S, Y) against the new pair in the spare slot: s_i.y_new,
// y_i.y_new, s_new.y_new, y_new.y_new.
template <int K>
__global__ void __launch_bounds__(kThreads) k_lb_update(int64_t n, const double* __restrict__ v_new,
                                                        const double* __restrict__ v, const double* __restrict__ g_new,
                                                        const double* __restrict__ g, double* __restrict__ S,
                                                        double* __restrict__ Y, LbSlots sl, int spare, int ld,
                                                        double* SY, double* YY, double* scal, double* part,
                                                        unsigned* ticket) {
  constexpr int NV = 2 * K + 2;
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  double* sp = S + (int64_t)spare * n;
  double* yp = Y + (int64_t)spare * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double s = v_new[e] - v[e], y = g_new[e] - g[e];
    sp[e] = s;
    yp[e] = y;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      acc[i] = fma(S[(int64_t)sl.s[i] * n + e], y, acc[i]);
      acc[K + i] = fma(Y[(int64_t)sl.s[i] * n + e], y, acc[K + i]);
    }
    acc[2 * K] = fma(s, y, acc[2 * K]);
    acc[2 * K + 1] = fma(y, y, acc[2 * K + 1]);
  }
  double tot[NV];
  if (red_finish<NV>(acc, part, ticket, tot)) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      SY[sl.s[i] * ld + spare] = tot[i];
      YY[sl.s[i] * ld + spare] = tot[K + i];
      YY[spare * ld + sl.s[i]] = tot[K + i];
    }
    SY[spare * ld + spare] = tot[2 * K];
    YY[spare * ld + spare] = tot[2 * K + 1];
    scal[0] = tot[2 * K];
  }
}

// a_i = s_i.g, b_i = y_i.g, g.g; the last block solves for the direction's coefficients.
template <int K>
__global__ void __launch_bounds__(kThreads) k_lb_project(int64_t n, const double* __restrict__ g,
                                                         const double* __restrict__ S, const double* __restrict__ Y,
                                                         LbSlots sl, int ld, const double* SY, const double* YY,
                                                         double* coef, double* part, unsigned* ticket) {
  constexpr int NV = 2 * K + 1;
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double ge = g[e];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      acc[i] = fma(S[(int64_t)sl.s[i] * n + e], ge, acc[i]);
      acc[K + i] = fma(Y[(int64_t)sl.s[i] * n + e], ge, acc[K + i]);
    }
    acc[2 * K] = fma(ge, ge, acc[2 * K]);
  }
  double tot[NV];
  if (!red_finish<NV>(acc, part, ticket, tot)) return;
  if (K == 0) {
    coef[0] = tot[2 * K] > 0.0 ? -1.0 / sqrt(tot[2 * K]) : -1.0;
    return;
  }
  const int kn = sl.s[K > 0 ? K - 1 : 0];
  const double gamma = SY[kn * ld + kn] / YY[kn * ld + kn];
  // t = R^-1 a (R upper triangular, R_ij = s_i.y_j)
  double t[K > 0 ? K : 1], w[K > 0 ? K : 1];
  for (int i = K - 1; i >= 0; --i) {
    double x = tot[i];
    for (int j = i + 1; j < K; ++j) x -= SY[sl.s[i] * ld + sl.s[j]] * t[j];
    t[i] = x / SY[sl.s[i] * ld + sl.s[i]];
  }
  // w = (D + gamma Y^T Y) t - gamma b
  for (int i = 0; i < K; ++i) {
    double x = SY[sl.s[i] * ld + sl.s[i]] * t[i] - gamma * tot[K + i];
    for (int j = 0; j < K; ++j) x += gamma * YY[sl.s[i] * ld + sl.s[j]] * t[j];
    w[i] = x;
  }
  // p = R^-T w (R^T lower triangular), written over w
  for (int i = 0; i < K; ++i) {
    double x = w[i];
    for (int j = 0; j < i; ++j) x -= SY[sl.s[j] * ld + sl.s[i]] * w[j];
    w[i] = x / SY[sl.s[i] * ld + sl.s[i]];
  }
  coef[0] = -gamma;
  for (int i = 0; i < K; ++i) {
    coef[1 + i] = -w[i];
    coef[1 + K + i] = gamma * t[i];
  }
}

// d = coef_0 g + sum_i coef_{1+i} s_i + coef_{1+K+i} y_i, and g.d.
template <int K>
__global__ void __launch_bounds__(kThreads) k_lb_combine(int64_t n, const double* __restrict__ g,
                                                         const double* __restrict__ S, const double* __restrict__ Y,
                                                         LbSlots sl, const double* coef, double* __restrict__ d,
                                                         double* scal, double* part, unsigned* ticket) {
  double c[2 * K + 1];
#pragma unroll
  for (int j = 0; j < 2 * K + 1; ++j) c[j] = coef[j];
  double acc[1] = {0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const double ge = g[e];
    double x = c[0] * ge;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      x = fma(c[1 + i], S[(int64_t)sl.s[i] * n + e], x);
      x = fma(c[1 + K + i], Y[(int64_t)sl.s[i] * n + e], x);
    }
    d[e] = x;
    acc[0] = fma(ge, x, acc[0]);
  }
  double tot[1];
  if (red_finish<1>(acc, part, ticket, tot)) scal[1] = tot[0];
}

// max_e |g_e| (order-independent), finished by the last block into scal[2].
__global__ void __launch_bounds__(kThreads) k_lb_maxabs(int64_t n, const double* __restrict__ g, double* scal,
                                                        double* part, unsigned* ticket) {
  __shared__ double sh[kThreads / 32];
  __shared__ bool am_last;
  double x = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) x = fmax(x, fabs(g[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sh[0];
    for (int w = 1; w < kThreads / 32; ++w) b = fmax(b, sh[w]);
    part[blockIdx.x] = b;
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!am_last || threadIdx.x != 0) return;
  __threadfence();
  double m = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) m = fmax(m, __ldcg(part + b));
  scal[2] = m;
  *ticket = 0u;
}

template <int K>
void lb_launch_update(fe_lbfgs* L, const double* v_new, const double* v, const double* g_new, const double* g,
                      const LbSlots& sl, int nb) {
  k_lb_update<K><<<nb, kThreads, 0, L->stream>>>(L->n, v_new, v, g_new, g, L->S, L->Y, sl, L->spare, L->m + 1,
                                                 L->SY, L->YY, L->scal, L->part, L->ticket);
}

template <int K>
void lb_launch_direction(fe_lbfgs* L, const double* g, double* d, const LbSlots& sl, int nb) {
  k_lb_project<K><<<nb, kThreads, 0, L->stream>>>(L->n, g, L->S, L->Y, sl, L->m + 1, L->SY, L->YY, L->coef, L->part,
                                                  L->ticket);
  k_lb_combine<K><<<nb, kThreads, 0, L->stream>>>(L->n, g, L->S, L->Y, sl, L->coef, d, L->scal, L->part, L->ticket);
}

// Runtime pair count -> compiled kernels (0..kMaxPairs).
template <int K = 0>
void lb_dispatch(int k, fe_lbfgs* L, const double* a, const double* b, const double* c, const double* e,
                 double* d, const LbSlots& sl, int nb, bool update) {
  if constexpr (K <= kMaxPairs) {
    if (k == K) {
      if (update) lb_launch_update<K>(L, a, b, c, e, sl, nb);
      else lb_launch_direction<K>(L, a, d, sl, nb);
      return;
    }
    lb_dispatch<K + 1>(k, L, a, b, c, e, d, sl, nb, update);
  }
}

struct LbDeviceGuard {
  int prev = -1;
  explicit LbDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~LbDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

LbSlots slots_of(const fe_lbfgs* L) {
  LbSlots sl{};
  for (int i = 0; i < L->count; ++i) sl.s[i] = L->ring[i];
  return sl;
}

fe_status lb_read_scalars(fe_lbfgs* L) {
  fe_status st = cuda_check(cudaMemcpyAsync(L->host, L->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream),
                            "lbfgs scalars");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(L->stream), "lbfgs sync");
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_lbfgs_create(fe_lbfgs** out, int device, void* stream, int64_t n, int m) {
  if (!out) return set_error(FE_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1) return set_error(FE_EINVAL, "n must be >= 1");
  if (m < 1 || m > kMaxPairs) return set_error(FE_EINVAL, "m must be in 1..16");
  fe_lbfgs* L = new (std::nothrow) fe_lbfgs();
  if (!L) return set_error(FE_ENOMEM, "host allocation");
  L->device = device;
  L->stream = (cudaStream_t)stream;
  L->n = n;
  L->m = m;
  L->spare = 0;
  LbDeviceGuard g(device);
  const size_t slots = (size_t)(m + 1) * (size_t)n, ld2 = (size_t)(m + 1) * (m + 1);
  const size_t part = (size_t)(2 * kMaxPairs + 2) * kMaxNodeBlocks;
  fe_status st = FE_OK;
  if ((st = cuda_check(cudaMalloc((void**)&L->S, slots * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->Y, slots * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->SY, ld2 * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->YY, ld2 * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->coef, (1 + 2 * kMaxPairs) * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->scal, 3 * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->part, part * sizeof(double)), "cudaMalloc")) ||
      (st = cuda_check(cudaMalloc((void**)&L->ticket, sizeof(unsigned)), "cudaMalloc")) ||
      (st = cuda_check(cudaMemset(L->ticket, 0, sizeof(unsigned)), "cudaMemset")) ||
      (st = cuda_check(cudaMallocHost((void**)&L->host, 3 * sizeof(double)), "cudaMallocHost"))) {
    fe_lbfgs_destroy(L);
    return st;
  }
  *out = L;
  return FE_OK;
}

fe_status fe_lbfgs_destroy(fe_lbfgs* L) {
  if (!L) return FE_OK;
  LbDeviceGuard g(L->device);
  cudaStreamSynchronize(L->stream);
  cudaFree(L->S);
  cudaFree(L->Y);
  cudaFree(L->SY);
  cudaFree(L->YY);
  cudaFree(L->coef);
  cudaFree(L->scal);
  cudaFree(L->part);
  cudaFree(L->ticket);
  if (L->host) cudaFreeHost(L->host);
  delete L;
  return FE_OK;
}

fe_status fe_lbfgs_reset(fe_lbfgs* L) {
  if (!L) return set_error(FE_EINVAL, "null argument");
  L->count = 0;
  L->spare = 0;
  return FE_OK;
}

fe_status fe_lbfgs_pairs(const fe_lbfgs* L, int* count) {
  if (!L || !count) return set_error(FE_EINVAL, "null argument");
  *count = L->count;
  return FE_OK;
}

}  // extern "C"

namespace {

// The spare slot (holding the last offered pair) joins the pairs in use.
void lb_keep_spare(fe_lbfgs* L) {
  if (L->count < L->m) {
    // the next spare is a slot none of the pairs in use holds (m + 1 slots, at most m pairs)
    L->ring[L->count++] = L->spare;
    bool used[kMaxPairs + 1] = {false};
    for (int i = 0; i < L->count; ++i) used[L->ring[i]] = true;
    for (int i = 0; i <= L->m; ++i)
      if (!used[i]) {
        L->spare = i;
        break;
      }
  } else {
    const int oldest = L->ring[0];
    for (int i = 0; i + 1 < L->m; ++i) L->ring[i] = L->ring[i + 1];
    L->ring[L->m - 1] = L->spare;
    L->spare = oldest;
  }
}

}  // namespace

extern "C" {

fe_status fe_lbfgs_step(fe_lbfgs* L, const double* v_new, const double* v, const double* g_new, const double* g,
                        double* d, double* out3) {
  FE_TRACE("fe_lbfgs_step");
  if (!L || !v_new || !v || !g_new || !g || !d || !out3) return set_error(FE_EINVAL, "null argument");
  LbDeviceGuard guard(L->device);
  const int nb = grid_for(L->n, kMaxNodeBlocks);
  // offer the pair, keep it provisionally, and compute the next direction and max |g_new|
  const int count0 = L->count, spare0 = L->spare;
  int ring0[kMaxPairs];
  for (int i = 0; i < count0; ++i) ring0[i] = L->ring[i];
  lb_dispatch(L->count, L, v_new, v, g_new, g, nullptr, slots_of(L), nb, true);
  lb_keep_spare(L);
  lb_dispatch(L->count, L, g_new, nullptr, nullptr, nullptr, d, slots_of(L), nb, false);
  k_lb_maxabs<<<nb, kThreads, 0, L->stream>>>(L->n, g_new, L->scal, L->part, L->ticket);
  fe_status st = cuda_check(cudaGetLastError(), "lbfgs step launch");
  if (st || (st = lb_read_scalars(L))) return st;
  if (!(L->host[0] > 0.0)) {
    // s.y <= 0: drop the pair and compute the direction from the pairs kept before
    L->count = count0;
    L->spare = spare0;
    for (int i = 0; i < count0; ++i) L->ring[i] = ring0[i];
    const double sy = L->host[0], gmax = L->host[2];
    lb_dispatch(L->count, L, g_new, nullptr, nullptr, nullptr, d, slots_of(L), nb, false);
    if ((st = cuda_check(cudaGetLastError(), "lbfgs direction launch")) || (st = lb_read_scalars(L))) return st;
    L->host[0] = sy;
    L->host[2] = gmax;
  }
  out3[0] = L->host[0];
  out3[1] = L->host[1];
  out3[2] = L->host[2];
  return FE_OK;
}

}  // extern "C"

extern "C" {

fe_status fe_lbfgs_update(fe_lbfgs* L, const double* v_new, const double* v, const double* g_new, const double* g,
                          double* sy) {
  FE_TRACE("fe_lbfgs_update");
  if (!L || !v_new || !v || !g_new || !g || !sy) return set_error(FE_EINVAL, "null argument");
  LbDeviceGuard guard(L->device);
  const LbSlots sl = slots_of(L);
  const int nb = grid_for(L->n, kMaxNodeBlocks);
  lb_dispatch(L->count, L, v_new, v, g_new, g, nullptr, sl, nb, true);
  fe_status st = cuda_check(cudaGetLastError(), "lbfgs update launch");
  if (st || (st = lb_read_scalars(L))) return st;
  *sy = L->host[0];
  if (*sy > 0.0) lb_keep_spare(L);
  return FE_OK;
}

fe_status fe_lbfgs_direction(fe_lbfgs* L, const double* g, double* d, double* gd) {
  FE_TRACE("fe_lbfgs_direction");
  if (!L || !g || !d || !gd) return set_error(FE_EINVAL, "null argument");
  LbDeviceGuard guard(L->device);
  const LbSlots sl = slots_of(L);
  const int nb = grid_for(L->n, kMaxNodeBlocks);
  lb_dispatch(L->count, L, g, nullptr, nullptr, nullptr, d, sl, nb, false);
  fe_status st = cuda_check(cudaGetLastError(), "lbfgs direction launch");
  if (st || (st = lb_read_scalars(L))) return st;
  *gd = L->host[1];
  return FE_OK;
}

}  // extern "C"

// ---- checkpoint / resume ----------------------------------------------------------------------
// The memory of a minimisation can be saved to the host and restored into another memory of
// the same size: the pairs in use (oldest first) and their products s_i.y_j and y_i.y_j are
// copied as they are, so the directions computed after a restore are bitwise those the saved
// memory would have given (the kernels read pairs and products in pair order, whatever slots
// hold them).

extern "C" {

fe_status fe_lbfgs_save(const fe_lbfgs* L, double* s_host, double* y_host, double* sy_host, double* yy_host,
                        int* count) {
  if (!L || !count || (L->count > 0 && (!s_host || !y_host || !sy_host || !yy_host)))
    return set_error(FE_EINVAL, "null argument");
  LbDeviceGuard guard(L->device);
  fe_status st = cuda_check(cudaStreamSynchronize(L->stream), "lbfgs sync");
  if (st) return st;
  const int k = L->count, ld = L->m + 1;
  const size_t n = (size_t)L->n;
  std::vector<double> sy((size_t)ld * ld), yy((size_t)ld * ld);
  if (k > 0 && ((st = cuda_check(cudaMemcpy(sy.data(), L->SY, sizeof(double) * sy.size(), cudaMemcpyDeviceToHost),
                                 "lbfgs save")) ||
                (st = cuda_check(cudaMemcpy(yy.data(), L->YY, sizeof(double) * yy.size(), cudaMemcpyDeviceToHost),
                                 "lbfgs save"))))
    return st;
  for (int i = 0; i < k; ++i) {
    const int a = L->ring[i];
    if ((st = cuda_check(cudaMemcpy(s_host + i * n, L->S + (size_t)a * n, sizeof(double) * n, cudaMemcpyDeviceToHost),
                         "lbfgs save")) ||
        (st = cuda_check(cudaMemcpy(y_host + i * n, L->Y + (size_t)a * n, sizeof(double) * n, cudaMemcpyDeviceToHost),
                         "lbfgs save")))
      return st;
    for (int j = 0; j < k; ++j) {
      sy_host[i * k + j] = sy[(size_t)a * ld + L->ring[j]];
      yy_host[i * k + j] = yy[(size_t)a * ld + L->ring[j]];
    }
  }
  *count = k;
  return FE_OK;
}

fe_status fe_lbfgs_restore(fe_lbfgs* L, const double* s_host, const double* y_host, const double* sy_host,
                           const double* yy_host, int count) {
  if (!L || count < 0 || count > L->m || (count > 0 && (!s_host || !y_host || !sy_host || !yy_host)))
    return set_error(FE_EINVAL, "bad arguments");
  LbDeviceGuard guard(L->device);
  fe_status st = cuda_check(cudaStreamSynchronize(L->stream), "lbfgs sync");
  if (st) return st;
  const int ld = L->m + 1;
  const size_t n = (size_t)L->n;
  std::vector<double> sy((size_t)ld * ld, 0.0), yy((size_t)ld * ld, 0.0);
  for (int i = 0; i < count; ++i) {
    if ((st = cuda_check(cudaMemcpy(L->S + i * n, s_host + i * n, sizeof(double) * n, cudaMemcpyHostToDevice),
                         "lbfgs restore")) ||
        (st = cuda_check(cudaMemcpy(L->Y + i * n, y_host + i * n, sizeof(double) * n, cudaMemcpyHostToDevice),
                         "lbfgs restore")))
      return st;
    for (int j = 0; j < count; ++j) {
      sy[(size_t)i * ld + j] = sy_host[i * count + j];
      yy[(size_t)i * ld + j] = yy_host[i * count + j];
    }
  }
  if ((st = cuda_check(cudaMemcpy(L->SY, sy.data(), sizeof(double) * sy.size(), cudaMemcpyHostToDevice),
                       "lbfgs restore")) ||
      (st = cuda_check(cudaMemcpy(L->YY, yy.data(), sizeof(double) * yy.size(), cudaMemcpyHostToDevice),
                       "lbfgs restore")))
    return st;
  for (int i = 0; i < count; ++i) L->ring[i] = i;
  L->count = count;
  L->spare = count;
  return FE_OK;
}

}  // extern "C"

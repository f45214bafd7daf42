// gather_bulk.cuh -- warp-cooperative patch gather with bulk (TMA) copies.
//
// g_i = sum over the CSR segment of node i of the local forces r_{T,l} (written by the
// element kernel to the CSR positions), minus b_i (when a load is given), and 0 on Dirichlet
// dofs (Sec. 6.2, Remark 1).  Each warp owns 32 consecutive nodes; their segments form one contiguous range
// of r, which lane 0 copies into the warp's shared-memory buffer with one cp.async.bulk
// completing on an mbarrier.  Each lane then sums its node's segment in a fixed rotated order
// (below), so results do not depend on the launch shape.  A range larger than the buffer is
// read directly from global memory in slot order.
#pragma once

#include <type_traits>

#include "async_copy.cuh"
#include "fe_internal.cuh"

namespace fe {

constexpr int kGatherWarps = 11;  // 11 x 20 KB = 220 KB of shared memory: one block per SM
constexpr int kGatherCap = 20480;   // bytes of shared memory per warp
constexpr int kGatherSmem = kGatherWarps * kGatherCap;

// Double slots, FP64 sums (the FP64 path).
struct AccF64 {
  using T = double;
  double s = 0.0;
  __device__ __forceinline__ void set(double x) { s = x; }
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// Double-float slots (float2 per component), double-float sums.
struct AccDF {
  using T = float2;
  df s = {0.f, 0.f};
  __device__ __forceinline__ void set(float2 x) { s = df{x.x, x.y}; }
  __device__ __forceinline__ void add(float2 x) { s = df_add(s, df{x.x, x.y}); }
  __device__ __forceinline__ double value() const { return df_to_double(s); }
};

// A node's FP64 segment, staged in shared memory, summed in 64-bit fixed point: every term is
// made an integer relative to the segment's largest exponent (keeping ceil(log2 len) + 1 bits
// of headroom, so the integer sum cannot overflow), the integers are added exactly on the
// integer pipes, and the sum goes back to FP64 with one rounding.  A term loses less than
// 2^-(62 - headroom) of the largest term, so the result is as accurate as a sequential FP64
// sum, and it does not depend on the order of the terms.  It replaces len FP64 additions per
// component, which run at 1/64 of the FP32 rate on this GPU, by integer work and one
// conversion.  Subnormal terms count as zero.  Returns false, and the caller adds in FP64,
// for a segment longer than 512 terms or with an Inf or NaN term or no normal term.
// Both passes walk the segment in the same rotated order as the FP64 sum (distinct banks).
template <int D>
__device__ __forceinline__ bool fixed_point_sum(const double* sbuf, int64_t q0, int32_t len, int lane,
                                                double (&out)[D]) {
  if (len < 1 || len > 512) return false;
  unsigned emax[D];
#pragma unroll
  for (int j = 0; j < D; ++j) emax[j] = 0u;
  int32_t pos = lane % len;
  for (int32_t t = 0; t < len; ++t) {
    const int64_t q = q0 + pos;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const unsigned e = (unsigned)((unsigned long long)__double_as_longlong(sbuf[q * D + j]) >> 52) & 0x7ffu;
      emax[j] = e > emax[j] ? e : emax[j];
    }
    pos = (pos + 1 == len) ? 0 : pos + 1;
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < D; ++j) ok = ok && emax[j] != 0u && emax[j] != 0x7ffu;
  if (!ok) return false;
  const int up = 9 - (len > 1 ? 32 - __clz(len - 1) : 0);   // 62 - (ceil(log2 len) + 1) - 52
  long long acc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) acc[j] = 0;
  pos = lane % len;
  for (int32_t t = 0; t < len; ++t) {
    const int64_t q = q0 + pos;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(sbuf[q * D + j]);
      const unsigned e = (unsigned)(bits >> 52) & 0x7ffu;
      const unsigned long long m = (bits & 0xfffffffffffffULL) | (1ULL << 52);
      const unsigned d = emax[j] - e;
      const long long x = (e == 0u || d > 63u) ? 0LL : (long long)((m << up) >> d);
      acc[j] += (bits >> 63) ? -x : x;
    }
    pos = (pos + 1 == len) ? 0 : pos + 1;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) out[j] = ldexp((double)acc[j], (int)emax[j] - 1075 - up);
  return true;
}

// The kernel and its launcher have internal linkage: every translation unit that uses them
// compiles its own copy of the kernel, and the launcher's once-per-device attribute mask must
// belong to that copy.
namespace {

template <int D, class Acc>
__global__ void __launch_bounds__(kGatherWarps * 32) k_gather_bulk(
    int64_t nn, const int32_t* __restrict__ row_ptr, const typename Acc::T* __restrict__ r,
    const double* __restrict__ b, const uint8_t* __restrict__ dir, const int32_t* __restrict__ perm,
    double* __restrict__ g, int* status, const int* skip, long long wait_limit) {
  using T = typename Acc::T;
  if (skip && *skip) return;  // a solver loop enqueued this launch after it had finished
  extern __shared__ __align__(128) unsigned char gsmem[];
  __shared__ __align__(8) uint64_t bars[kGatherWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = gsmem + warp * kGatherCap;
  uint64_t* bar = &bars[warp];
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncwarp();
  uint32_t phase = 0;
  const int64_t nchunks = (nn + 31) / 32;
  const int64_t wstride = (int64_t)gridDim.x * kGatherWarps;
  for (int64_t c = (int64_t)blockIdx.x * kGatherWarps + warp; c < nchunks; c += wstride) {
    const int64_t n0 = c * 32;
    const int64_t n1 = (n0 + 32 < nn) ? n0 + 32 : nn;
    const int64_t s0 = __ldg(row_ptr + n0), s1 = __ldg(row_ptr + n1);
    const int64_t byte0 = s0 * D * (int64_t)sizeof(T), byte1 = s1 * D * (int64_t)sizeof(T);
    const int64_t a0 = byte0 & ~15LL, a1 = (byte1 + 15) & ~15LL;
    const bool staged = (a1 > a0) && (a1 - a0 <= kGatherCap);
    if (staged) {
      if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)(a1 - a0));
        bulk_g2s(buf, reinterpret_cast<const unsigned char*>(r) + a0, (uint32_t)(a1 - a0), bar);
      }
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, phase, wait_limit));
      if (!ok) {
        // give up: record it, wait (with the full limit) for the copy still in flight, so
        // that nothing is written to shared memory after the block has left, and stop
        if (lane == 0) atomicOr(status, kStatusTimeout);
        mbar_wait_bounded(bar, phase);
        return;
      }
      phase ^= 1u;
    }
    const int64_t i = n0 + lane;
    if (i < nn) {
#ifdef FE_DEBUG_BOUNDS
      int32_t q0 = __ldg(row_ptr + i), q1 = __ldg(row_ptr + i + 1);
      if (!(s0 <= q0 && q0 <= q1 && q1 <= s1)) {   // the row must lie in the warp's range
        (void)FE_CHK(q1, 0, kSiteGatherRow);
        q0 = q1 = (int32_t)s0;
      }
#else
      const int32_t q0 = __ldg(row_ptr + i), q1 = __ldg(row_ptr + i + 1);
#endif
      Acc acc[D];
      if (staged) {
        // element k of r is at sbuf[k - k0] (a0 is a multiple of 16, so of sizeof(T)).
        // Lane k walks its segment starting at position k (mod its length) and wraps around:
        // with the common 24-slot patches, a plain walk puts every lane's reads on two
        // shared-memory banks, while the rotated walk makes them distinct.  The order is
        // still fixed by the mesh alone.
        const T* sbuf = reinterpret_cast<const T*>(buf) - a0 / (int64_t)sizeof(T);
        const int32_t len = q1 - q0;
        bool done = false;
        if constexpr (std::is_same<T, double>::value) {   // FP64 slots: fixed-point sums
          double fx[D];
          done = fixed_point_sum<D>(reinterpret_cast<const double*>(sbuf), (int64_t)q0, len, lane, fx);
          if (done) {
#pragma unroll
            for (int j = 0; j < D; ++j) acc[j].set(fx[j]);
          }
        }
        int32_t pos = len > 0 ? lane % len : 0;
        for (int32_t t = 0; t < len && !done; ++t) {
          const int64_t q = (int64_t)q0 + pos;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            if (t == 0) acc[j].set(sbuf[q * D + j]);   // (adding it to zero would return it unchanged)
            else acc[j].add(sbuf[q * D + j]);
          }
          pos = (pos + 1 == len) ? 0 : pos + 1;
        }
      } else {
        for (int32_t q = q0; q < q1; ++q)
#pragma unroll
          for (int j = 0; j < D; ++j) {
            if (q == q0) acc[j].set(__ldg(r + (int64_t)q * D + j));
            else acc[j].add(__ldg(r + (int64_t)q * D + j));
          }
      }
      const int64_t dst = perm ? (int64_t)FE_CHK(__ldg(perm + i), nn, kSiteGatherPerm) : i;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const double val = b ? acc[j].value() - b[i * D + j] : acc[j].value();
        g[dst * D + j] = dir[i * D + j] ? 0.0 : val;
      }
    }
    __syncwarp();
  }
}

// Launch on the context stream: one block of 11 warps per SM (220 KB of shared memory each;
// 8 warps, 160 KB, were measured 13% slower on the FP64 gather of 128^3 x 6).
// b: the load vector subtracted from the sums (the context's b unless given; nullptr = 0).
// skip: nullptr, or a device flag; the launch does nothing when it is nonzero.
template <int D, class Acc>
inline fe_status launch_gather_bulk(fe_ctx* c, const typename Acc::T* r, double* g, const double* b,
                                    const int* skip = nullptr) {
  static std::atomic<uint64_t> smem_set{0};
  fe_status st = ensure_smem((const void*)k_gather_bulk<D, Acc>, c->device, kGatherSmem, smem_set);
  if (st) return st;
  const int sms = sm_count(c->device);
  const int64_t nchunks = (c->nn + 31) / 32;
  int64_t blocks = (nchunks + kGatherWarps - 1) / kGatherWarps;
  if (blocks > sms) blocks = sms;
  if (blocks < 1) blocks = 1;
  k_gather_bulk<D, Acc><<<(unsigned)blocks, kGatherWarps * 32, kGatherSmem, c->stream>>>(
      c->nn, c->row_ptr, r, b, c->dir, io_perm(c), g, c->status, skip, c->wait_limit);
  return cuda_check(cudaGetLastError(), "gather launch");
}

template <int D, class Acc>
inline fe_status launch_gather_bulk(fe_ctx* c, const typename Acc::T* r, double* g) {
  return launch_gather_bulk<D, Acc>(c, r, g, c->b);
}

}  // namespace

}  // namespace fe

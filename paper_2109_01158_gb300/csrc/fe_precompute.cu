// fe_precompute.cu -- per-mesh precompute on the device (Sec. 4.1-4.2 of the paper):
// element volumes |T| and P1 shape-function gradients, the nodal-patch CSR and b = M f.
//
// The floating-point steps use the _rn intrinsics so that no multiply-add is contracted:
// every value is produced by the same sequence of correctly rounded operations as the
// plain definition, which makes this one-off step reproducible bit for bit.
#include <cmath>
#include <vector>

#include "fe_internal.cuh"

namespace fe {
namespace {

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// Shape-function gradients and volume of each element.  With B = [x_1-x_0, ..., x_dim-x_0]
// (columns), grad(phi_l) for l >= 1 is row l of B^{-1} (barycentric coordinates are
// B^{-1}(x - x_0)), grad(phi_0) = -sum_l grad(phi_l), and |T| = |det B| / dim!.
// Only l = 1..dim is stored: dphi[((l-1)*DIM + m)*ne + e].
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_shape(int64_t ne, const int32_t* __restrict__ elems,
                                                    const double* __restrict__ X,
                                                    double* __restrict__ dphi,
                                                    double* __restrict__ vol, int* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    int n0 = elems[e];
    double x0[DIM], B[DIM][DIM], inv[DIM][DIM], det;
#pragma unroll
    for (int m = 0; m < DIM; ++m) x0[m] = X[(int64_t)n0 * DIM + m];
#pragma unroll
    for (int k = 1; k <= DIM; ++k) {
      int nk = elems[(int64_t)k * ne + e];
#pragma unroll
      for (int m = 0; m < DIM; ++m) B[m][k - 1] = sub(X[(int64_t)nk * DIM + m], x0[m]);
    }
    if (DIM == 2) {
      det = sub(mul(B[0][0], B[1][1]), mul(B[0][1], B[1][0]));
      inv[0][0] = B[1][1] / det;
      inv[0][1] = -B[0][1] / det;
      inv[1][0] = -B[1][0] / det;
      inv[1][1] = B[0][0] / det;
      vol[e] = fabs(det) / 2.0;
    } else {
      double C[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int r0 = (a + 1) % 3, r1 = (a + 2) % 3, c0 = (c + 1) % 3, c1 = (c + 2) % 3;
          C[a][c] = sub(mul(B[r0][c0], B[r1][c1]), mul(B[r0][c1], B[r1][c0]));
        }
      det = add(add(mul(B[0][0], C[0][0]), mul(B[0][1], C[0][1])), mul(B[0][2], C[0][2]));
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) inv[a][c] = C[c][a] / det;
      vol[e] = fabs(det) / 6.0;
    }
    if (det == 0.0 || !isfinite(det)) atomicOr(status, kStatusDegenerate);
#pragma unroll
    for (int l = 1; l <= DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) dphi[((int64_t)(l - 1) * DIM + m) * ne + e] = inv[l - 1][m];
  }
}

// ---- nodal-patch CSR -----------------------------------------------------------------

template <int K>
__global__ void __launch_bounds__(kThreads) k_count(int64_t ne, const int32_t* __restrict__ elems,
                                                    int32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride)
#pragma unroll
    for (int l = 0; l < K; ++l) atomicAdd(&cnt[elems[(int64_t)l * ne + e] + 1], 1);
}

// In-place inclusive scan of a[0..n): per-tile scan, scan of tile totals, tile offsets.
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t* sh, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < kThreads / 32) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kThreads / 32) sh[lane] = w;
  }
  __syncthreads();
  int32_t excl = v - x + (warp > 0 ? sh[warp - 1] : 0);
  *total = sh[kThreads / 32 - 1];
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(kThreads) k_scan_tiles(int32_t* a, int64_t n, int32_t* tile_sum) {
  __shared__ int32_t sh[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t loc[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = (base + k < n) ? a[base + k] : 0;
    s += loc[k];
  }
  int32_t total;
  int32_t run = block_exclusive_scan(s, sh, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    run += loc[k];
    if (base + k < n) a[base + k] = run;
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_scan_totals(int32_t* tile_sum, int64_t ntiles) {
  __shared__ int32_t sh[kThreads / 32];
  int32_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += kThreads) {
    int64_t i = base + threadIdx.x;
    int32_t x = (i < ntiles) ? tile_sum[i] : 0, total;
    int32_t ex = block_exclusive_scan(x, sh, &total);
    if (i < ntiles) tile_sum[i] = carry + ex;   // exclusive offset of tile i
    carry += total;
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_add(int32_t* a, int64_t n, const int32_t* tile_off) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int32_t off = tile_off[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kThreads)
    if (base + k < n) a[base + k] += off;
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_fill(int64_t ne, const int32_t* __restrict__ elems,
                                                   int32_t* __restrict__ cursor,
                                                   int32_t* __restrict__ ent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride)
#pragma unroll
    for (int l = 0; l < K; ++l) {
      int32_t pos = atomicAdd(&cursor[elems[(int64_t)l * ne + e]], 1);
      ent[pos] = (int32_t)(e * K + l);
    }
}

// Order each patch by element id (insertion sort: patches are short).
__global__ void __launch_bounds__(kThreads) k_sort_rows(int64_t nn, const int32_t* __restrict__ row_ptr,
                                                        int32_t* __restrict__ ent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const int32_t a = row_ptr[i], b = row_ptr[i + 1];
    for (int32_t q = a + 1; q < b; ++q) {
      int32_t key = ent[q], t = q - 1;
      while (t >= a && ent[t] > key) {
        ent[t + 1] = ent[t];
        --t;
      }
      ent[t + 1] = key;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_slots(int64_t nn, int64_t ne, const int32_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ ent,
                                                    int32_t* __restrict__ slot) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride)
    for (int32_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      int32_t en = ent[q];
      slot[(int64_t)(en % K) * ne + en / K] = q;
    }
}

// b^(j)_i = sum over the patch of i (element order) of sum_c M^T_{l c} f^(j)_c with the P1
// element mass matrix M^T_{lc} = |T| (1 + delta_lc) / ((dim+1)(dim+2))  (eq. mass2D).
template <int DIM, int D>
__global__ void __launch_bounds__(kThreads) k_load(int64_t nn, int64_t ne, const int32_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ ent,
                                                   const int32_t* __restrict__ elems,
                                                   const double* __restrict__ vol,
                                                   const double* __restrict__ f,
                                                   double* __restrict__ b) {
  constexpr int K = DIM + 1;
  const double denom = (double)((DIM + 1) * (DIM + 2));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    double s[D];
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = 0.0;
    for (int32_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int32_t en = ent[q];
      const int64_t e = en / K;
      const int l = en % K;
      const double w = vol[e] / denom;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < K; ++c)
          t = add(t, mul(c == l ? 2.0 : 1.0, f[(int64_t)elems[(int64_t)c * ne + e] * D + j]));
        s[j] = add(s[j], mul(w, t));
      }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) b[i * D + j] = s[j];
  }
}

template <int DIM>
fe_status precompute_dim(fe_ctx* c) {
  constexpr int K = DIM + 1;
  cudaStream_t s = c->stream;
  const int64_t ne = c->ne, nn = c->nn;
  fe_status st;
  if (ne > 0) {
    k_shape<DIM><<<grid_for(ne, 4 * kMaxElemBlocks), kThreads, 0, s>>>(ne, c->elems, c->X, c->dphi,
                                                                         c->vol, c->status);
    c->launches++;
  }
  // CSR: counts at row_ptr[i+1], inclusive scan, fill, order rows, slot map
  if ((st = cuda_check(cudaMemsetAsync(c->row_ptr, 0, sizeof(int32_t) * (nn + 1), s), "memset")))
    return st;
  if (ne > 0) {
    k_count<K><<<grid_for(ne, 4 * kMaxElemBlocks), kThreads, 0, s>>>(ne, c->elems, c->row_ptr);
    c->launches++;
  }
  const int64_t ntiles = (nn + 1 + kScanTile - 1) / kScanTile;
  int32_t* tiles = nullptr;
  if ((st = cuda_check(cudaMallocAsync((void**)&tiles, sizeof(int32_t) * ntiles, s), "alloc scan")))
    return st;
  k_scan_tiles<<<(unsigned)ntiles, kThreads, 0, s>>>(c->row_ptr, nn + 1, tiles);
  k_scan_totals<<<1, kThreads, 0, s>>>(tiles, ntiles);
  k_scan_add<<<(unsigned)ntiles, kThreads, 0, s>>>(c->row_ptr, nn + 1, tiles);
  c->launches += 3;
  cudaFreeAsync(tiles, s);
  if (ne > 0) {
    int32_t* cursor = nullptr;
    if ((st = cuda_check(cudaMallocAsync((void**)&cursor, sizeof(int32_t) * nn, s), "alloc cursor")))
      return st;
    cudaMemcpyAsync(cursor, c->row_ptr, sizeof(int32_t) * nn, cudaMemcpyDeviceToDevice, s);
    k_fill<K><<<grid_for(ne, 4 * kMaxElemBlocks), kThreads, 0, s>>>(ne, c->elems, cursor, c->ent);
    cudaFreeAsync(cursor, s);
    k_sort_rows<<<grid_for(nn, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(nn, c->row_ptr, c->ent);
    k_slots<K><<<grid_for(nn, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(nn, ne, c->row_ptr, c->ent, c->slot);
    c->launches += 3;
  }
  if ((c->pre_mask & (1u << FE_F32_COMP)) && ne > 0 && (st = launch_tile_blocks_f32(c))) return st;
  return cuda_check(cudaGetLastError(), "precompute launch");
}

template <int DIM>
fe_status load_vector_dim(fe_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t ne = c->ne, nn = c->nn;
  fe_status st;
  // b = M f (load given in the caller's order; permuted to device order on the host side)
  if ((st = cuda_check(cudaMemsetAsync(c->b, 0, sizeof(double) * nn * c->d, s), "memset b"))) return st;
  if (!c->f_host.empty() && ne > 0) {
    double* fdev = nullptr;
    if ((st = cuda_check(cudaMallocAsync((void**)&fdev, sizeof(double) * nn * c->d, s), "alloc f")))
      return st;
    std::vector<double> fdevorder(c->f_host.size());
    for (int64_t i = 0; i < nn; ++i) {
      int64_t src = c->perm_h.empty() ? i : c->perm_h[i];
      for (int j = 0; j < c->d; ++j) fdevorder[i * c->d + j] = c->f_host[src * c->d + j];
    }
    cudaMemcpyAsync(fdev, fdevorder.data(), sizeof(double) * nn * c->d, cudaMemcpyHostToDevice, s);
    if (c->d == 1)
      k_load<DIM, 1><<<grid_for(nn, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(nn, ne, c->row_ptr, c->ent,
                                                                          c->elems, c->vol, fdev, c->b);
    else
      k_load<DIM, DIM><<<grid_for(nn, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(nn, ne, c->row_ptr, c->ent,
                                                                            c->elems, c->vol, fdev, c->b);
    c->launches++;
    cudaFreeAsync(fdev, s);
    // the host copy of the reordered load must outlive the async copy
    if ((st = cuda_check(cudaStreamSynchronize(s), "load vector"))) return st;
  }
  return cuda_check(cudaGetLastError(), "load vector launch");
}

}  // namespace

fe_status launch_precompute(fe_ctx* c) {
  return c->dim == 2 ? precompute_dim<2>(c) : precompute_dim<3>(c);
}

// b.X for vector problems (d = dim): the constant part of b.v when the caller passes the
// Neo-Hookean displacement u = v - X.  Neumaier sum in device node order on the host.
static fe_status compute_bX(fe_ctx* c) {
  c->bX = 0.0;
  if (c->d != c->dim || c->nn == 0) return FE_OK;
  const size_t n = (size_t)c->nn * c->d;
  std::vector<double> bh(n), xh((size_t)c->nn * c->dim);
  cudaMemcpyAsync(bh.data(), c->b, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(xh.data(), c->X, sizeof(double) * xh.size(), cudaMemcpyDeviceToHost, c->stream);
  fe_status st = cuda_check(cudaStreamSynchronize(c->stream), "b.X read back");
  if (st) return st;
  double s = 0.0, comp = 0.0;
  for (int64_t i = 0; i < c->nn; ++i)
    for (int j = 0; j < c->d; ++j) {
      const double t = bh[(size_t)i * c->d + j] * xh[(size_t)i * c->dim + j];
      const double y = s + t;
      comp += (std::fabs(s) >= std::fabs(t)) ? (s - y) + t : (t - y) + s;
      s = y;
    }
  c->bX = s + comp;
  return FE_OK;
}

fe_status launch_load_vector(fe_ctx* c) {
  const fe_status st = c->dim == 2 ? load_vector_dim<2>(c) : load_vector_dim<3>(c);
  return st ? st : compute_bX(c);
}

}  // namespace fe

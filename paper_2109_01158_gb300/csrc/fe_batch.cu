// fe_batch.cu -- batched energy + exact gradient over many resident meshes (serving).
//
// One call evaluates J and grad J (Sec. 5 and 6.2, double-float arithmetic as FE_DF64) for a
// list of independent requests, each on its own precomputed mesh, with three launches in
// total whatever the number of requests:
//   k_batch_prep     one block per 256-node tile of any request: u = v - X (or u = v when the
//                    mesh takes displacements) as double-floats
//                    into the request's scratch, per-tile partial sums of b.v
//   k_batch_elem     one block per 256-element tile of any request: W and the local forces
//                    (elem_df_one, the same code as the single-mesh kernels), per-tile partial
//                    sums of |T| W
//   k_batch_gather   one block per 256-node tile: per-node patch sums in slot order, - b, 0 on
//                    Dirichlet dofs; the block of tile 0 of each request adds the request's
//                    tile partials in a fixed order and writes J
// Every partial sum belongs to one request and is reduced in an order fixed by that
// request's own mesh, so a request gets bitwise the same J and g alone and in any mix.
#include <algorithm>
#include <vector>

#include "elem_df.cuh"
#include "fe_internal.cuh"

namespace fe {
namespace {

constexpr int kBT = 256;   // threads per block = elements or nodes per tile

struct BItem {
  const int32_t* elems;
  const float2* dphi;
  const float2* vol;
  const int32_t* slot;
  const int32_t* row_ptr;
  const double* X;
  const double* b;
  const uint8_t* dir;
  const int32_t* perm;
  int64_t nn, ne;
  int dim, d, model, disp;   // disp: v is the Neo-Hookean displacement u = v - X
  double shift;             // b.X, added to the b.u partial of tile 0 when disp
  ModelDF md;
  const double* v;
  double* J;
  double* g;
  float2* u;
  float2* r;
  double* epart;
  double* npart;
  int64_t etile0, ntile0;   // first global element tile and node tile of this request
  int64_t netiles, nntiles;
};

// Index of the request owning global tile t (first0 is increasing over requests).
__device__ __forceinline__ int find_item(const BItem* __restrict__ items, int n, int64_t t, bool elem) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t f = elem ? items[mid].etile0 : items[mid].ntile0;
    if (f <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double bwarp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double bblock_sum(double x, double* sh) {
  x = bwarp_sum(x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  x = (threadIdx.x < kBT / 32) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) x = bwarp_sum(x);
  __syncthreads();
  return x;
}

template <int D, bool NH, int DIM>
__device__ __forceinline__ double prep_node(const BItem& it, int64_t i) {
  constexpr int DP = D == 3 ? 4 : D;
  const int64_t src = it.perm ? (int64_t)it.perm[i] : i;
  df w[DP];
  double dot = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double vj = it.v[src * D + j];
    dot += it.b[i * D + j] * vj;
    w[j] = df_from_double((NH && !it.disp) ? vj - it.X[i * DIM + j] : vj);
  }
  if (DP == 4) w[3] = {0.f, 0.f};
  if (DP == 1) {
    it.u[i] = make_float2(w[0].hi, w[0].lo);
  } else {
    float4* o = reinterpret_cast<float4*>(it.u) + i * (DP / 2);
    o[0] = make_float4(w[0].hi, w[0].lo, w[1].hi, w[1].lo);
    if (DP == 4) o[1] = make_float4(w[2].hi, w[2].lo, w[3].hi, w[3].lo);
  }
  return dot;
}

__global__ void __launch_bounds__(kBT) k_batch_prep(const BItem* __restrict__ items, int n) {
  __shared__ double sh[kBT / 32];
  const int k = find_item(items, n, blockIdx.x, false);
  const BItem& it = items[k];
  const int64_t t = blockIdx.x - it.ntile0;
  const int64_t i = t * kBT + threadIdx.x;
  double dot = 0.0;
  if (i < it.nn) {
    if (it.model == FE_NEOHOOKE) dot = (it.dim == 3) ? prep_node<3, true, 3>(it, i) : prep_node<2, true, 2>(it, i);
    else dot = (it.dim == 3) ? prep_node<1, false, 3>(it, i) : prep_node<1, false, 2>(it, i);
  }
  dot = bblock_sum(dot, sh);
  if (threadIdx.x == 0) it.npart[t] = (t == 0 && it.disp) ? dot + it.shift : dot;
}

__global__ void __launch_bounds__(kBT) k_batch_elem(const BItem* __restrict__ items, int n,
                                                    const LogEntry* __restrict__ tab, int* status) {
  __shared__ double sh[kBT / 32];
  const int k = find_item(items, n, blockIdx.x, true);
  const BItem& it = items[k];
  const int64_t t = blockIdx.x - it.etile0;
  const int64_t e = t * kBT + threadIdx.x;
  double w = 0.0;
  bool bad = false;
  if (e < it.ne) {
    df vT, W;
    if (it.model == FE_NEOHOOKE) {
      if (it.dim == 3)
        W = elem_df_one<3, 3, FE_NEOHOOKE, true, true>(e, it.ne, it.elems, it.dphi, it.vol, it.u, it.slot, it.md,
                                                       tab, it.r, bad, vT);
      else
        W = elem_df_one<2, 2, FE_NEOHOOKE, true, true>(e, it.ne, it.elems, it.dphi, it.vol, it.u, it.slot, it.md,
                                                       tab, it.r, bad, vT);
    } else {
      if (it.dim == 3)
        W = elem_df_one<3, 1, FE_PLAPLACE, true, true>(e, it.ne, it.elems, it.dphi, it.vol, it.u, it.slot, it.md,
                                                       tab, it.r, bad, vT);
      else
        W = elem_df_one<2, 1, FE_PLAPLACE, true, true>(e, it.ne, it.elems, it.dphi, it.vol, it.u, it.slot, it.md,
                                                       tab, it.r, bad, vT);
    }
    w = isinf(W.hi) ? CUDART_INF : df_to_double(df_mul(vT, W));   // keep +Inf out of the pair product
  }
  if (bad) atomicOr(status, kStatusDomain);
  w = bblock_sum(w, sh);
  if (threadIdx.x == 0) it.epart[t] = w;
}

template <int D>
__device__ __forceinline__ void gather_node(const BItem& it, int64_t i) {
  df s[D];
  const int32_t q0 = it.row_ptr[i], q1 = it.row_ptr[i + 1];
  // the first slot starts the sum (adding it to {0, 0} would return it unchanged)
#pragma unroll
  for (int j = 0; j < D; ++j) s[j] = (q1 > q0) ? ld_df(it.r, (int64_t)q0 * D + j) : df{0.f, 0.f};
  for (int32_t q = q0 + 1; q < q1; ++q)
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = df_add(s[j], ld_df(it.r, (int64_t)q * D + j));
  const int64_t dst = it.perm ? (int64_t)it.perm[i] : i;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double val = df_to_double(s[j]) - it.b[i * D + j];
    it.g[dst * D + j] = it.dir[i * D + j] ? 0.0 : val;
  }
}

__global__ void __launch_bounds__(kBT) k_batch_gather(const BItem* __restrict__ items, int n) {
  __shared__ double sh[kBT / 32];
  const int k = find_item(items, n, blockIdx.x, false);
  const BItem& it = items[k];
  const int64_t t = blockIdx.x - it.ntile0;
  const int64_t i = t * kBT + threadIdx.x;
  if (i < it.nn) {
    if (it.d == 3) gather_node<3>(it, i);
    else if (it.d == 2) gather_node<2>(it, i);
    else gather_node<1>(it, i);
  }
  if (t == 0) {   // the request's energy: its tile partials in a fixed order
    double s = 0.0, q = 0.0;
    for (int64_t m = threadIdx.x; m < it.netiles; m += kBT) s += it.epart[m];
    for (int64_t m = threadIdx.x; m < it.nntiles; m += kBT) q += it.npart[m];
    s = bblock_sum(s, sh);
    q = bblock_sum(q, sh);
    if (threadIdx.x == 0) *it.J = s - q;
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WorkLayout {
  size_t u, r, ep, np, total;
};

WorkLayout work_layout(const fe_ctx* m) {
  WorkLayout L;
  const size_t nn = (size_t)m->nn, ne = (size_t)m->ne, k = (size_t)m->dim + 1;
  const size_t netiles = (ne + kBT - 1) / kBT, nntiles = (nn + kBT - 1) / kBT;
  L.u = 0;
  L.r = align256(L.u + sizeof(float2) * nn * padded_d(m->d));
  L.ep = align256(L.r + sizeof(float2) * ne * k * m->d);
  L.np = align256(L.ep + sizeof(double) * (netiles > 0 ? netiles : 1));
  L.total = align256(L.np + sizeof(double) * (nntiles > 0 ? nntiles : 1)) + 256;
  return L;
}

ModelDF model_df_of(const fe_ctx* c) {
  ModelDF m;
  auto split = [](double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
  };
  m.C1 = split(c->C1);
  m.D1 = split(c->D1);
  m.twoC1 = split(2.0 * c->C1);
  m.twoD1 = split(2.0 * c->D1);
  m.negTwoC1 = split(-2.0 * c->C1);
  m.p = c->p;
  m.pcase = (c->p == 2.0) ? 2 : (c->p == 3.0) ? 3 : (c->p == 4.0) ? 4 : (c->p == 1.5) ? 15 : 0;
  return m;
}

}  // namespace

size_t batch_item_bytes() { return sizeof(BItem); }

size_t batch_work_bytes(const fe_ctx* m) { return work_layout(m).total; }

fe_status batch_enqueue(cudaStream_t s, const fe_batch_item* items, int n, void* host_stage, void* dev_stage,
                        int* status) {
  BItem* host = static_cast<BItem*>(host_stage);
  BItem* dev = static_cast<BItem*>(dev_stage);
  const LogEntry* tab = nullptr;
  int64_t et = 0, nt = 0;
  for (int k = 0; k < n; ++k) {
    const fe_batch_item& q = items[k];
    const fe_ctx* m = q.mesh;
    if (!m || !m->have_pre || !m->model_set || !(m->pre_mask & (1u << FE_DF64)))
      return set_error(FE_EINVAL, "batch item: mesh must be precomputed with FE_DF64 and have a model");
    if (m->model != FE_PLAPLACE && m->model != FE_NEOHOOKE)
      return set_error(FE_EINVAL, "batch item: the batched kernels evaluate FE_PLAPLACE and FE_NEOHOOKE");
    if (!q.v || !q.J || !q.g || !q.work) return set_error(FE_EINVAL, "batch item: null v, J, g or work");
    if (reinterpret_cast<uintptr_t>(q.work) & 255u) return set_error(FE_EINVAL, "batch item: work not 256-byte aligned");
    const WorkLayout L = work_layout(m);
    unsigned char* w = static_cast<unsigned char*>(q.work);
    BItem& it = host[k];
    it.elems = m->elems;
    it.dphi = m->dphi_df;
    it.vol = m->vol_df;
    it.slot = m->slot;
    it.row_ptr = m->row_ptr;
    it.X = m->X;
    it.b = m->b;
    it.dir = m->dir;
    it.perm = m->perm;
    it.nn = m->nn;
    it.ne = m->ne;
    it.dim = m->dim;
    it.d = m->d;
    it.model = m->model;
    it.disp = input_is_disp(m) ? 1 : 0;
    it.shift = it.disp ? m->bX : 0.0;
    it.md = model_df_of(m);
    it.v = q.v;
    it.J = q.J;
    it.g = q.g;
    it.u = reinterpret_cast<float2*>(w + L.u);
    it.r = reinterpret_cast<float2*>(w + L.r);
    it.epart = reinterpret_cast<double*>(w + L.ep);
    it.npart = reinterpret_cast<double*>(w + L.np);
    it.netiles = std::max<int64_t>((m->ne + kBT - 1) / kBT, 1);
    it.nntiles = std::max<int64_t>((m->nn + kBT - 1) / kBT, 1);
    it.etile0 = et;
    it.ntile0 = nt;
    et += it.netiles;
    nt += it.nntiles;
    tab = m->log_tab;
  }
  if (et >= (1ll << 31) || nt >= (1ll << 31)) return set_error(FE_EINVAL, "batch too large");
  cudaMemcpyAsync(dev, host, sizeof(BItem) * n, cudaMemcpyHostToDevice, s);
  k_batch_prep<<<(unsigned)nt, kBT, 0, s>>>(dev, n);
  k_batch_elem<<<(unsigned)et, kBT, 0, s>>>(dev, n, tab, status);
  k_batch_gather<<<(unsigned)nt, kBT, 0, s>>>(dev, n);
  return cuda_check(cudaGetLastError(), "batch launch");
}

}  // namespace fe

struct fe_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  fe::BItem* host = nullptr;   // pinned staging of the request descriptors
  fe::BItem* dev = nullptr;
  int cap = 0;
  int* status = nullptr;
  int64_t launches = 0;
};

using namespace fe;

extern "C" {

fe_status fe_batch_work_bytes(const fe_ctx* mesh, size_t* bytes) {
  if (!mesh || !bytes) return set_error(FE_EINVAL, "null argument");
  if (!mesh->have_pre) return set_error(FE_EINVAL, "mesh is not precomputed");
  *bytes = work_layout(mesh).total;
  return FE_OK;
}

fe_status fe_batch_create(fe_batch** out, int device, void* stream) {
  if (!out) return set_error(FE_EINVAL, "null argument");
  *out = nullptr;
  fe_batch* b = new (std::nothrow) fe_batch();
  if (!b) return set_error(FE_ENOMEM, "host allocation");
  b->device = device;
  b->stream = (cudaStream_t)stream;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  fe_status st = cuda_check(cudaMalloc((void**)&b->status, sizeof(int)), "cudaMalloc");
  if (!st) st = cuda_check(cudaMemset(b->status, 0, sizeof(int)), "cudaMemset");
  if (prev >= 0) cudaSetDevice(prev);
  if (st) {
    delete b;
    return st;
  }
  *out = b;
  return FE_OK;
}

fe_status fe_batch_destroy(fe_batch* b) {
  if (!b) return FE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->host) cudaFreeHost(b->host);
  if (b->dev) cudaFree(b->dev);
  if (b->status) cudaFree(b->status);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return FE_OK;
}

fe_status fe_batch_energy_gradient(fe_batch* b, const fe_batch_item* items, int n) {
  if (!b || (n > 0 && !items) || n < 0) return set_error(FE_EINVAL, "bad arguments");
  if (n == 0) return FE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, b->device};
  fe_status st;
  if (n > b->cap) {
    cudaStreamSynchronize(b->stream);
    if (b->host) cudaFreeHost(b->host);
    if (b->dev) cudaFree(b->dev);
    b->host = nullptr;
    b->dev = nullptr;
    b->cap = 0;
    const int cap = std::max(n, 64);
    if ((st = cuda_check(cudaMallocHost((void**)&b->host, sizeof(BItem) * cap), "cudaMallocHost"))) return st;
    if ((st = cuda_check(cudaMalloc((void**)&b->dev, sizeof(BItem) * cap), "cudaMalloc"))) return st;
    b->cap = cap;
  }
  // the staging buffer may still be read by the previous call's copy
  if ((st = cuda_check(cudaStreamSynchronize(b->stream), "batch sync"))) return st;
  for (int k = 0; k < n; ++k)
    if (items[k].mesh && items[k].mesh->device != b->device) return set_error(FE_EINVAL, "batch item on another device");
  if ((st = batch_enqueue(b->stream, items, n, b->host, b->dev, b->status))) return st;
  b->launches += 3;
  return FE_OK;
}

fe_status fe_batch_sync_status(fe_batch* b) {
  if (!b) return set_error(FE_EINVAL, "null batch");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  int hs = 0;
  cudaMemcpyAsync(&hs, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  fe_status st = cuda_check(cudaStreamSynchronize(b->stream), "batch sync");
  if (!st && hs) {
    cudaMemsetAsync(b->status, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
  }
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  if (st) return st;
  if (hs & kStatusDomain) return set_error(FE_EDOMAIN, "an element has det F <= 0");
  return FE_OK;
}

fe_status fe_batch_launch_count(const fe_batch* b, int64_t* count) {
  if (!b || !count) return set_error(FE_EINVAL, "null argument");
  *count = b->launches;
  return FE_OK;
}

}  // extern "C"

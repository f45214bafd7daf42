// fe_batch.cu -- batched energy + exact gradient over many resident meshes (serving).
//
// One call evaluates J and grad J (Sec. 5 and 6.2, double-float arithmetic as FE_DF64) for a
// list of independent requests, each on its own precomputed mesh, in ONE persistent launch
// whatever the number of requests.  Every request has three steps, each a range of tiles:
//   prep tiles     (1024 nodes, four per thread) u = v - X (or u = v when the mesh takes
//                  displacements) as double-floats into the request's scratch, and per-tile
//                  partial sums of b.v;
//   element tiles  (256 x ept elements, ept = 1, 2 or 4 elements per thread: more for large
//                  requests, whose tiles then amortise the per-tile work of the schedule,
//                  fewer for small ones, whose elements then spread over more blocks) W and
//                  the local forces (elem_df_one, the same code as the single-mesh kernels),
//                  per-tile partial sums of |T| W;
//   gather tiles   (1024 nodes) per-node patch sums in slot order, - b, 0 on Dirichlet dofs.
// The host lays the ranges out in one work list, software-pipelined over waves of requests
// (a wave: consecutive requests with at least four tiles per resident block in all):
//   P(0) | P(1) E(0) | P(2) E(1) G(0) | P(3) E(2) G(1) | ...
// so that the tiles a step depends on were handed out a wave earlier and have normally
// finished when it starts.  Every block takes the next item from a counter (claiming its
// following item while it works on the current one, so the claim's latency is hidden), so
// no block idles at a step boundary and no grid-wide barrier separates the steps.  An element tile
// still checks that all prep tiles of its request are done, a gather tile that all its
// element tiles are: per-request counters, polled by one thread of the block, with a clock
// limit after which the block records a timeout in the status word and carries on (an item
// only ever depends on items earlier in the list, handed out to blocks that are already
// running, so the waits end; the limit only guards against a fault elsewhere).  The block
// that completes the last gather tile of a request adds the request's tile partials in a
// fixed order, writes J and then, if the caller asked for one, raises the request's
// completion flag -- the caller can take each request's result as soon as it is ready, not
// at the end of the launch.
//
// Prep and gather tiles run over the nodes in the caller's numbering, so the vector read and
// the gradient written are contiguous: v, J, g and the flag can live in page-locked host
// memory, which the kernel then reads and writes directly over the host link (no copies).
//
// Every partial sum belongs to one request and is reduced in an order fixed by that
// request's own mesh, so a request gets bitwise the same J and g alone and in any mix.
#include <algorithm>
#include <atomic>
#include <vector>

#include "elem_df.cuh"
#include "fe_internal.cuh"
#include "trace.h"

namespace fe {
namespace {

constexpr int kBT = 256;          // threads per block = elements per element tile
constexpr int kNPT = 4;           // nodes per thread in the prep and gather tiles
constexpr int kNT = kBT * kNPT;   // nodes per prep or gather tile

struct BItem {
  const int32_t* elems;
  const float2* dphi;
  const float2* vol;
  const int32_t* slot;
  const int32_t* row_ptr;
  const double* X;
  const double* b;
  const uint8_t* dir;
  const int32_t* iperm;     // caller node -> device node (null = identity)
  int64_t nn, ne;
  int dim, d, model, disp;  // disp: v is the Neo-Hookean displacement u = v - X
  double shift;             // b.X, added to the b.u partial of tile 0 when disp
  ModelDF md;
  const double* v;
  double* J;
  double* g;
  int* done;                // completion flag (null = none)
  float2* u;
  float2* r;
  double* epart;
  double* npart;
  int64_t netiles, nntiles;
  int ept;                  // elements per thread in the element tiles
};

// Head of the descriptor block: the work counter and the number of items.
struct BHead {
  unsigned long long next;
  long long total;
};

// Per-request progress: prep, element and gather tiles done; err = a wait gave up.
struct BCount {
  int prep, elem, gather, err;
};

// One step of one request: its tiles are the work items [start, start + tiles).
struct BRange {
  long long start;
  int k;       // request
  int step;    // 0 prep, 1 element, 2 gather
};

// Descriptor block: [BHead][BItem x n][BCount x n][BRange x 3n], 16-byte aligned pieces.
inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
inline size_t stage_items_off() { return align16(sizeof(BHead)); }
inline size_t stage_counts_off(int n) { return align16(stage_items_off() + sizeof(BItem) * (size_t)n); }
inline size_t stage_ranges_off(int n) { return align16(stage_counts_off(n) + sizeof(BCount) * (size_t)n); }

// The range holding work item w (ranges sorted by start, the first at 0).
__device__ __forceinline__ int find_range(const BRange* __restrict__ rg, int nr, long long w) {
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&rg[mid].start) <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double bwarp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Block sum, valid in thread 0.
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

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *c >= target (bounded by `limit` SM clocks); then the block proceeds.
__device__ __forceinline__ void wait_count(const int* c, int target, long long limit, int* err, int* status) {
  if (threadIdx.x == 0 && ld_acquire(c) < target) {
    const long long t0 = clock64();
    while (ld_acquire(c) < target) {
      if (clock64() - t0 > limit) {
        atomicOr(err, 1);
        atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
}

// Every thread's writes of this tile become visible (to the host too when sys), then thread
// 0 counts the tile; returns the count before it (valid in thread 0).
__device__ __forceinline__ int signal_tile(int* c, bool sys) {
  if (sys) __threadfence_system();
  else __threadfence();
  __syncthreads();
  return threadIdx.x == 0 ? atomicAdd(c, 1) : 0;
}

// Nodes c = t*kNT + q*kBT + threadIdx.x (q < kNPT) of the caller's numbering: u at device
// node i, and the sum of b_i . v_c over them (q-major).  Every load is issued before the
// first store, so the loads of the four nodes are in flight together.
template <int D, bool NH, int DIM>
__device__ __forceinline__ double prep_nodes(const BItem& it, int64_t t) {
  constexpr int DP = D == 3 ? 4 : D;
  const bool sub = NH && !it.disp;
  int64_t c[kNPT], i[kNPT];
  double v[kNPT][D], b[kNPT][D], x[kNPT][D];
#pragma unroll
  for (int q = 0; q < kNPT; ++q) {
    c[q] = t * kNT + q * kBT + threadIdx.x;
    i[q] = c[q] < it.nn ? (it.iperm ? (int64_t)__ldg(it.iperm + c[q]) : c[q]) : -1;
  }
#pragma unroll
  for (int q = 0; q < kNPT; ++q)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const bool ok = i[q] >= 0;
      v[q][j] = ok ? it.v[c[q] * D + j] : 0.0;
      b[q][j] = ok ? __ldg(it.b + i[q] * D + j) : 0.0;
      x[q][j] = (ok && sub) ? __ldg(it.X + i[q] * DIM + j) : 0.0;
    }
  double dot = 0.0;
#pragma unroll
  for (int q = 0; q < kNPT; ++q) {
    if (i[q] < 0) continue;
    df w[DP];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      dot += b[q][j] * v[q][j];
      w[j] = df_from_double(sub ? v[q][j] - x[q][j] : v[q][j]);
    }
    if (DP == 4) w[3] = {0.f, 0.f};
    if (DP == 1) {
      it.u[i[q]] = make_float2(w[0].hi, w[0].lo);
    } else {
      float4* o = reinterpret_cast<float4*>(it.u) + i[q] * (DP / 2);
      o[0] = make_float4(w[0].hi, w[0].lo, w[1].hi, w[1].lo);
      if (DP == 4) o[1] = make_float4(w[2].hi, w[2].lo, w[3].hi, w[3].lo);
    }
  }
  return dot;
}

__device__ __forceinline__ void prep_tile(const BItem& it, int64_t t, double* sh) {
  double dot;
  if (it.model == FE_NEOHOOKE) dot = (it.dim == 3) ? prep_nodes<3, true, 3>(it, t) : prep_nodes<2, true, 2>(it, t);
  else dot = (it.dim == 3) ? prep_nodes<1, false, 3>(it, t) : prep_nodes<1, false, 2>(it, t);
  dot = bblock_sum(dot, sh);
  if (threadIdx.x == 0) it.npart[t] = (t == 0 && it.disp) ? dot + it.shift : dot;
}

template <int DIM, int D, int MODEL>
__device__ __forceinline__ double elem_range(const BItem& it, int64_t e0, const LogEntry* tab, bool& bad) {
  double w = 0.0;
  for (int q = 0; q < it.ept; ++q) {
    const int64_t e = e0 + q * kBT + threadIdx.x;
    if (e >= it.ne) break;
    df vT;
    const df W = elem_df_one<DIM, D, MODEL, true, true, true>(e, it.ne, it.elems, it.dphi, it.vol, it.u, it.slot, it.md,
                                                               tab, it.r, bad, vT);
    w += isinf(W.hi) ? CUDART_INF : df_to_double(df_mul(vT, W));   // keep +Inf out of the pair product
  }
  return w;
}

__device__ __forceinline__ void elem_tile(const BItem& it, int64_t t, const LogEntry* tab, int* status, double* sh) {
  const int64_t e0 = t * kBT * it.ept;
  bool bad = false;
  double w;
  if (it.model == FE_NEOHOOKE)
    w = (it.dim == 3) ? elem_range<3, 3, FE_NEOHOOKE>(it, e0, tab, bad) : elem_range<2, 2, FE_NEOHOOKE>(it, e0, tab, bad);
  else
    w = (it.dim == 3) ? elem_range<3, 1, FE_PLAPLACE>(it, e0, tab, bad) : elem_range<2, 1, FE_PLAPLACE>(it, e0, tab, bad);
  if (bad) atomicOr(status, kStatusDomain);
  w = bblock_sum(w, sh);
  if (threadIdx.x == 0) it.epart[t] = w;
}

// Nodes c = t*kNT + q*kBT + threadIdx.x (q < kNPT) of the caller's numbering: the sum of
// the local forces of device node i's patch in slot order, - b_i, 0 on Dirichlet dofs.  The
// four nodes' slot runs are walked side by side, so their loads are in flight together;
// each node's own sum keeps the slot order.
template <int D>
__device__ __forceinline__ void gather_nodes(const BItem& it, int64_t t) {
  int64_t c[kNPT], i[kNPT];
  int32_t q0[kNPT], n[kNPT];
#pragma unroll
  for (int q = 0; q < kNPT; ++q) {
    c[q] = t * kNT + q * kBT + threadIdx.x;
    i[q] = c[q] < it.nn ? (it.iperm ? (int64_t)__ldg(it.iperm + c[q]) : c[q]) : -1;
  }
  int len = 0;
#pragma unroll
  for (int q = 0; q < kNPT; ++q) {
    q0[q] = i[q] >= 0 ? __ldg(it.row_ptr + i[q]) : 0;
    n[q] = i[q] >= 0 ? __ldg(it.row_ptr + i[q] + 1) - q0[q] : 0;
    len = max(len, n[q]);
  }
  // the first slot starts each sum (adding it to {0, 0} would return it unchanged)
  df s[kNPT][D];
#pragma unroll
  for (int q = 0; q < kNPT; ++q)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float2 a = n[q] > 0 ? __ldca(it.r + (int64_t)q0[q] * D + j) : make_float2(0.f, 0.f);
      s[q][j] = {a.x, a.y};
    }
  for (int m = 1; m < len; ++m) {
    float2 a[kNPT][D];
#pragma unroll
    for (int q = 0; q < kNPT; ++q)
#pragma unroll
      for (int j = 0; j < D; ++j) a[q][j] = m < n[q] ? __ldca(it.r + (int64_t)(q0[q] + m) * D + j) : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kNPT; ++q)
      if (m < n[q])
#pragma unroll
        for (int j = 0; j < D; ++j) s[q][j] = df_add(s[q][j], df{a[q][j].x, a[q][j].y});
  }
#pragma unroll
  for (int q = 0; q < kNPT; ++q) {
    if (i[q] < 0) continue;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double val = df_to_double(s[q][j]) - __ldg(it.b + i[q] * D + j);
      it.g[c[q] * D + j] = __ldg(it.dir + i[q] * D + j) ? 0.0 : val;
    }
  }
}

__device__ __forceinline__ void gather_tile(const BItem& it, int64_t t) {
  if (it.d == 3) gather_nodes<3>(it, t);
  else if (it.d == 2) gather_nodes<2>(it, t);
  else gather_nodes<1>(it, t);
}

// The request's energy from its tile partials, in a fixed order; then its completion flag.
__device__ __forceinline__ void finish_request(const BItem& it, const BCount* cnt, double* sh) {
  double s = 0.0, q = 0.0;
  for (int64_t m = threadIdx.x; m < it.netiles; m += kBT) s += __ldcg(it.epart + m);
  for (int64_t m = threadIdx.x; m < it.nntiles; m += kBT) q += __ldcg(it.npart + m);
  s = bblock_sum(s, sh);
  q = bblock_sum(q, sh);
  if (threadIdx.x == 0) {
    *it.J = s - q;
    if (it.done) {
      const int err = ld_acquire(&cnt->err);
      __threadfence_system();
      *reinterpret_cast<volatile int*>(it.done) = err ? 3 : 1;
    }
  }
}

__global__ void __launch_bounds__(kBT) k_batch_persistent(const BItem* __restrict__ items, const BRange* __restrict__ rg,
                                                          int nr, BHead* head, BCount* cnt,
                                                          const LogEntry* __restrict__ log_tab, int* status,
                                                          long long limit) {
  __shared__ double sh[kBT / 32];
  __shared__ LogEntry tab[kLogTable];
  __shared__ long long s_w;
  __shared__ int s_last;
  for (int i = threadIdx.x; i < kLogTable; i += kBT) tab[i] = log_tab[i];
  const long long total = head->total;
  // thread 0 claims the block's next item while the block works on the current one (an item
  // only depends on earlier items, so the smallest unfinished item can always proceed)
  long long next = threadIdx.x == 0 ? (long long)atomicAdd(&head->next, 1ull) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_w = next;
      if (next < total) next = (long long)atomicAdd(&head->next, 1ull);
    }
    __syncthreads();
    const long long w = s_w;
    if (w >= total) break;   // the same w in every thread
    const int ri = find_range(rg, nr, w);
    const int k = __ldg(&rg[ri].k), step = __ldg(&rg[ri].step);
    const int64_t t = w - __ldg(&rg[ri].start);
    const BItem& it = items[k];
    BCount* ck = cnt + k;
    if (step == 0) {
      prep_tile(it, t, sh);
      signal_tile(&ck->prep, false);
    } else if (step == 1) {
      wait_count(&ck->prep, (int)it.nntiles, limit, &ck->err, status);
      elem_tile(it, t, tab, status, sh);
      signal_tile(&ck->elem, false);
    } else {
      wait_count(&ck->elem, (int)it.netiles, limit, &ck->err, status);
      gather_tile(it, t);
      const int before = signal_tile(&ck->gather, true);
      if (threadIdx.x == 0) {
        s_last = before == (int)it.nntiles - 1;
        if (s_last) __threadfence();   // acquire: the other blocks' partials and forces
      }
      __syncthreads();
      if (s_last) finish_request(it, ck, sh);
    }
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WorkLayout {
  size_t u, r, ep, np, total;
};

WorkLayout work_layout(const fe_ctx* m) {
  WorkLayout L;
  const size_t nn = (size_t)m->nn, ne = (size_t)m->ne, k = (size_t)m->dim + 1;
  // element tiles: at most one per 256 elements, whatever the elements per thread
  const size_t netiles = (ne + kBT - 1) / kBT, nntiles = (nn + kNT - 1) / kNT;
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

// Resident blocks of the persistent kernel per SM, once per device.
int persistent_blocks(int device) {
  static std::atomic<int> cache[64];
  if (device < 0 || device >= 64) return 1;
  int b = cache[device].load(std::memory_order_relaxed);
  if (b > 0) return b;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_persistent, kBT, 0) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  cache[device].store(b, std::memory_order_relaxed);
  return b;
}

// The work list: waves of consecutive requests with at least four tiles per resident block in
// all, pipelined as P(s), E(s-1), G(s-2) at stage s (P, E, G: the prep, element and gather
// ranges of the wave's requests, in request order); out[3n] receives the ranges in list
// order.  Returns the number of items.
int64_t plan_work(int n, const int64_t* nnt, const int64_t* net, int64_t resident, BRange* out) {
  std::vector<int> wb{0};
  int64_t acc = 0;
  for (int k = 0; k < n; ++k) {
    acc += 2 * nnt[k] + net[k];
    if (acc >= 4 * resident || k == n - 1) {
      wb.push_back(k + 1);
      acc = 0;
    }
  }
  const int nw = (int)wb.size() - 1;
  int nr = 0;
  int64_t w = 0;
  auto emit = [&](int wave, int step) {
    if (wave < 0 || wave >= nw) return;
    for (int k = wb[wave]; k < wb[wave + 1]; ++k) {
      out[nr++] = BRange{(long long)w, k, step};
      w += step == 1 ? net[k] : nnt[k];
    }
  };
  for (int st = 0; st < nw + 2; ++st) {
    emit(st, 0);
    emit(st - 1, 1);
    emit(st - 2, 2);
  }
  return w;
}

}  // namespace

size_t batch_stage_bytes(int n) { return stage_ranges_off(n) + sizeof(BRange) * 3 * (size_t)(n > 0 ? n : 1); }

size_t batch_work_bytes(const fe_ctx* m) { return work_layout(m).total; }

fe_status batch_enqueue(cudaStream_t s, int device, const fe_batch_item* items, int n, void* host_stage,
                        void* dev_stage, int* status, long long wait_limit) {
  unsigned char* hs = static_cast<unsigned char*>(host_stage);
  unsigned char* ds = static_cast<unsigned char*>(dev_stage);
  BHead* head = reinterpret_cast<BHead*>(hs);
  BItem* host = reinterpret_cast<BItem*>(hs + stage_items_off());
  BCount* hcnt = reinterpret_cast<BCount*>(hs + stage_counts_off(n));
  BRange* hr = reinterpret_cast<BRange*>(hs + stage_ranges_off(n));
  const int64_t resident = (int64_t)sm_count(device) * persistent_blocks(device);
  const LogEntry* tab = nullptr;
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
    unsigned char* wk = static_cast<unsigned char*>(q.work);
    BItem& it = host[k];
    it.elems = m->elems;
    it.dphi = m->dphi_df;
    it.vol = m->vol_df;
    it.slot = m->slot;
    it.row_ptr = m->row_ptr;
    it.X = m->X;
    it.b = m->b;
    it.dir = m->dir;
    it.iperm = m->iperm;
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
    it.done = q.done;
    it.u = reinterpret_cast<float2*>(wk + L.u);
    it.r = reinterpret_cast<float2*>(wk + L.r);
    it.epart = reinterpret_cast<double*>(wk + L.ep);
    it.npart = reinterpret_cast<double*>(wk + L.np);
    // elements per thread: 2 or 4 when the request still has two tiles per resident block
    it.ept = 1;
    while (it.ept < 4 && (m->ne + 2 * kBT * it.ept - 1) / (2 * kBT * it.ept) >= 2 * resident) it.ept *= 2;
    it.netiles = std::max<int64_t>((m->ne + kBT * it.ept - 1) / (kBT * it.ept), 1);
    it.nntiles = std::max<int64_t>((m->nn + kNT - 1) / kNT, 1);
    if (it.netiles >= (1ll << 31) || it.nntiles >= (1ll << 31)) return set_error(FE_EINVAL, "batch item too large");
    hcnt[k] = BCount{0, 0, 0, 0};
    tab = m->log_tab;
  }
  std::vector<int64_t> nnt(n), net(n);
  for (int k = 0; k < n; ++k) {
    nnt[k] = host[k].nntiles;
    net[k] = host[k].netiles;
  }
  const int64_t w = plan_work(n, nnt.data(), net.data(), resident, hr);
  const int nr = 3 * n;
  if (w >= (1ll << 40)) return set_error(FE_EINVAL, "batch too large");
  head->next = 0;
  head->total = w;
  const size_t bytes = batch_stage_bytes(n);
  fe_status st = cuda_check(cudaMemcpyAsync(ds, hs, bytes, cudaMemcpyHostToDevice, s), "batch descriptors");
  if (st) return st;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(w, resident));
  k_batch_persistent<<<grid, kBT, 0, s>>>(reinterpret_cast<const BItem*>(ds + stage_items_off()),
                                          reinterpret_cast<const BRange*>(ds + stage_ranges_off(n)), nr,
                                          reinterpret_cast<BHead*>(ds),
                                          reinterpret_cast<BCount*>(ds + stage_counts_off(n)), tab, status,
                                          wait_limit > 0 ? wait_limit : 2000000000LL);
  return cuda_check(cudaGetLastError(), "batch launch");
}

}  // namespace fe

// Descriptor blocks of the last kRing calls: a call reuses the block of the call kRing
// before it once that call's descriptor copy has completed (its event), so enqueueing does
// not wait for the GPU.
constexpr int kRing = 4;

struct fe_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  unsigned char* host[kRing] = {};   // pinned staging of the descriptor block
  unsigned char* dev[kRing] = {};
  cudaEvent_t copied[kRing] = {};
  bool pending[kRing] = {};
  int cap = 0;
  int* status = nullptr;
  long long wait_limit = 2000000000LL;
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
  fe_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (!st) st = cuda_check(cudaMalloc((void**)&b->status, sizeof(int)), "cudaMalloc");
  if (!st) st = cuda_check(cudaMemset(b->status, 0, sizeof(int)), "cudaMemset");
  if (prev >= 0) cudaSetDevice(prev);
  if (st) {
    if (b->status) cudaFree(b->status);
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
  for (int i = 0; i < kRing; ++i) {
    if (b->host[i]) cudaFreeHost(b->host[i]);
    if (b->dev[i]) cudaFree(b->dev[i]);
    if (b->copied[i]) cudaEventDestroy(b->copied[i]);
  }
  if (b->status) cudaFree(b->status);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return FE_OK;
}

fe_status fe_batch_set_wait_limit(fe_batch* b, int64_t cycles) {
  if (!b || cycles < 0) return set_error(FE_EINVAL, "bad arguments");
  b->wait_limit = cycles == 0 ? 2000000000LL : (long long)cycles;
  return FE_OK;
}

fe_status fe_batch_energy_gradient(fe_batch* b, const fe_batch_item* items, int n) {
  FE_TRACE("fe_batch_energy_gradient");
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
  for (int k = 0; k < n; ++k)
    if (items[k].mesh && items[k].mesh->device != b->device) return set_error(FE_EINVAL, "batch item on another device");
  if (n > b->cap) {
    // every block may still be read by an enqueued copy
    if ((st = cuda_check(cudaStreamSynchronize(b->stream), "batch sync"))) return st;
    const int cap = std::max(n, 64);
    const size_t bytes = batch_stage_bytes(cap);
    for (int i = 0; i < kRing; ++i) {
      if (b->host[i]) cudaFreeHost(b->host[i]);
      if (b->dev[i]) cudaFree(b->dev[i]);
      b->host[i] = b->dev[i] = nullptr;
      b->pending[i] = false;
    }
    b->cap = 0;
    for (int i = 0; i < kRing; ++i) {
      if (!b->copied[i] &&
          (st = cuda_check(cudaEventCreateWithFlags(&b->copied[i], cudaEventDisableTiming), "cudaEventCreate")))
        return st;
      if ((st = cuda_check(cudaMallocHost((void**)&b->host[i], bytes), "cudaMallocHost"))) return st;
      if ((st = cuda_check(cudaMalloc((void**)&b->dev[i], bytes), "cudaMalloc"))) return st;
    }
    b->cap = cap;
  }
  const int slot = (int)(b->launches % kRing);
  if (b->pending[slot] && (st = cuda_check(cudaEventSynchronize(b->copied[slot]), "batch staging"))) return st;
  b->pending[slot] = false;
  if ((st = batch_enqueue(b->stream, b->device, items, n, b->host[slot], b->dev[slot], b->status, b->wait_limit)))
    return st;
  // the host block is free once the copy has run; the device block once the kernel has, and
  // the next copy into it is ordered after that kernel on the stream
  if ((st = cuda_check(cudaEventRecord(b->copied[slot], b->stream), "cudaEventRecord"))) return st;
  b->pending[slot] = true;
  b->launches += 1;
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
  if (hs & kStatusTimeout) return set_error(FE_ETIMEOUT, "a bounded wait of the batched kernel gave up");
  if (hs & kStatusDomain) return set_error(FE_EDOMAIN, "an element has det F <= 0");
  return FE_OK;
}

fe_status fe_batch_plan(int n, const int64_t* prep_tiles, const int64_t* elem_tiles, int64_t resident_blocks,
                        int64_t* start_out, int32_t* request_out, int32_t* step_out, int64_t* total_out) {
  if (n < 0 || (n > 0 && (!prep_tiles || !elem_tiles || !start_out || !request_out || !step_out)) || !total_out ||
      resident_blocks < 1)
    return set_error(FE_EINVAL, "bad arguments");
  for (int k = 0; k < n; ++k)
    if (prep_tiles[k] < 1 || elem_tiles[k] < 1) return set_error(FE_EINVAL, "every request has at least one tile per step");
  std::vector<BRange> r((size_t)3 * n);
  *total_out = n > 0 ? plan_work(n, prep_tiles, elem_tiles, resident_blocks, r.data()) : 0;
  for (int q = 0; q < 3 * n; ++q) {
    start_out[q] = r[q].start;
    request_out[q] = r[q].k;
    step_out[q] = r[q].step;
  }
  return FE_OK;
}

fe_status fe_batch_launch_count(const fe_batch* b, int64_t* count) {
  if (!b || !count) return set_error(FE_EINVAL, "null argument");
  *count = b->launches;
  return FE_OK;
}

}  // extern "C"

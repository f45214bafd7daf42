// fe_api.cu -- host side of the C ABI declared in include/femenergy.h: argument checks,
// mesh upload and internal renumbering, device buffer management, dispatch of the
// precompute and evaluation kernels, and read-back helpers.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "async_copy.cuh"  // kWaitCycles
#include "fe_internal.cuh"
#include "trace.h"

namespace fe {

static thread_local std::string g_err;

fe_status set_error(fe_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

fe_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FE_OK;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FE_ENOMEM : FE_ECUDA;
}

int sm_count(int device) {
  static std::atomic<int> cache[64];
  if (device >= 0 && device < 64) {
    const int v = cache[device].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) sms = 1;
  if (device >= 0 && device < 64) cache[device].store(sms, std::memory_order_relaxed);
  return sms;
}

void prof_begin(fe_ctx* c, int stage) {
  if (!c->prof) return;
  auto& ev = c->prof_ev[stage];
  const size_t need = 2 * (size_t)c->prof_n[stage] + 2;
  while (ev.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ev.push_back(e);
  }
  cudaEventRecord(ev[2 * c->prof_n[stage]], c->stream);
}

void prof_end(fe_ctx* c, int stage) {
  if (!c->prof) return;
  auto& ev = c->prof_ev[stage];
  if (ev.size() < 2 * (size_t)c->prof_n[stage] + 2) return;
  cudaEventRecord(ev[2 * c->prof_n[stage] + 1], c->stream);
  c->prof_n[stage]++;
}

namespace {

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Release the slots of the pipelined host evaluations (after their copies have drained);
// the streams and events stay until fe_destroy.
void pipe_free(fe_ctx* c) {
  if (c->pipe_in) cudaStreamSynchronize(c->pipe_in);
  if (c->pipe_out) cudaStreamSynchronize(c->pipe_out);
  const size_t n = (size_t)c->nn * c->d;
  for (int s = 0; s < 2; ++s) {
    dev_free(c, &c->pipe_v[s], n);
    dev_free(c, &c->pipe_g[s], n);
  }
  dev_free(c, &c->pipe_J, 2);
  c->pipe_k = 0;
}

void free_precompute(fe_ctx* c) {
  const size_t ne = (size_t)c->ne, nn = (size_t)c->nn, k = (size_t)c->dim + 1;
  dev_free(c, &c->dphi, ne * c->dim * c->dim);
  dev_free(c, &c->vol, ne);
  dev_free(c, &c->row_ptr, nn + 1);
  dev_free(c, &c->ent, ne * k);
  dev_free(c, &c->slot, ne * k);
  dev_free(c, &c->b, nn * c->d);
  dev_free(c, &c->blk32, (size_t)c->n_tiles * tile_block_bytes_f32(c->dim));
  dev_free(c, &c->dphi_df, ne * c->dim * c->dim);
  dev_free(c, &c->vol_df, ne);
  dev_free(c, &c->log_tab, kLogTable);
  dev_free(c, &c->u_df, nn * padded_d(c->d));
  dev_free(c, &c->r_df, ne * k * c->d);
  dev_free(c, &c->u, nn * padded_d(c->d));
  dev_free(c, &c->w_hvp, nn * padded_d(c->d));
  dev_free(c, &c->r, ne * k * c->d);
  free_tiles(c);
  dev_free(c, &c->stage_v, nn * c->d);
  dev_free(c, &c->stage_g, nn * c->d);
  pipe_free(c);
  dev_free(c, &c->cg_vec, 3 * nn * c->d);
  dev_free(c, &c->hvp_cache, hvp_cache_doubles(c));
  c->have_pre = false;
  c->pre_mask = 0;
}

void free_mesh(fe_ctx* c) {
  free_precompute(c);
  const size_t ne = (size_t)c->ne, nn = (size_t)c->nn, k = (size_t)c->dim + 1;
  dev_free(c, &c->X, nn * c->dim);
  dev_free(c, &c->elems, ne * k);
  dev_free(c, &c->dir, nn * c->d);
  dev_free(c, &c->perm, nn);
  dev_free(c, &c->iperm, nn);
  dev_free(c, &c->eperm, ne);
  c->perm_h.clear();
  c->eperm_h.clear();
  c->have_mesh = false;
}

// Spread the low `bits` bits of x so that consecutive bits land `stride` apart.
uint64_t spread_bits(uint64_t x, int bits, int stride) {
  uint64_t r = 0;
  for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1ull) << (b * stride);
  return r;
}

// Morton (Z-order) renumbering of the nodes; perm[new] = old.  Every axis is quantised on
// the scale of the largest extent of the bounding box, so that the key follows distance in
// space also on elongated domains (a per-axis scale would stretch the short axis to full
// range and let its bits dominate the key).
std::vector<int32_t> morton_order(int dim, int64_t nn, const double* X) {
  std::vector<double> lo(dim, 0.0), hi(dim, 0.0);
  for (int m = 0; m < dim; ++m) {
    lo[m] = hi[m] = nn > 0 ? X[m] : 0.0;
  }
  for (int64_t i = 0; i < nn; ++i)
    for (int m = 0; m < dim; ++m) {
      lo[m] = std::min(lo[m], X[i * dim + m]);
      hi[m] = std::max(hi[m], X[i * dim + m]);
    }
  const int bits = dim == 3 ? 21 : 31;
  const double scale = (double)((1ull << bits) - 1);
  double ext = 0.0;
  for (int m = 0; m < dim; ++m) ext = std::max(ext, hi[m] - lo[m]);
  std::vector<uint64_t> key(nn);
  for (int64_t i = 0; i < nn; ++i) {
    uint64_t k = 0;
    for (int m = 0; m < dim; ++m) {
      double t = ext > 0 ? (X[i * dim + m] - lo[m]) / ext : 0.0;
      uint64_t q = (uint64_t)(t * scale);
      k |= spread_bits(q, bits, dim) << m;
    }
    key[i] = k;
  }
  std::vector<int32_t> perm(nn);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  return perm;
}

// Device order of the elements (eperm[new] = old): stable sort by the Morton key of the
// centroid, quantised like morton_order's keys (the largest extent of the bounding box of the
// nodes).  Empty when that order is the identity.
std::vector<int32_t> element_order(int dim, int64_t nn, const double* X, int64_t ne, const int32_t* elems) {
  if (ne <= 1 || nn <= 0) return {};
  const int k = dim + 1;
  std::vector<double> lo(dim), hi(dim);
  for (int m = 0; m < dim; ++m) lo[m] = hi[m] = X[m];
  for (int64_t i = 0; i < nn; ++i)
    for (int m = 0; m < dim; ++m) {
      lo[m] = std::min(lo[m], X[i * dim + m]);
      hi[m] = std::max(hi[m], X[i * dim + m]);
    }
  const int bits = dim == 3 ? 21 : 31;
  const double scale = (double)((1ull << bits) - 1);
  double ext = 0.0;
  for (int m = 0; m < dim; ++m) ext = std::max(ext, hi[m] - lo[m]);
  std::vector<uint64_t> key(ne);
  for (int64_t e = 0; e < ne; ++e) {
    uint64_t kk = 0;
    for (int m = 0; m < dim; ++m) {
      double cm = 0.0;
      for (int l = 0; l < k; ++l) cm += X[(int64_t)elems[e * k + l] * dim + m];
      const double t = ext > 0 ? (cm / k - lo[m]) / ext : 0.0;
      const double tq = std::min(std::max(t, 0.0), 1.0);
      kk |= spread_bits((uint64_t)(tq * scale), bits, dim) << m;
    }
    key[e] = kk;
  }
  std::vector<int32_t> perm(ne);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  bool id = true;
  for (int64_t e = 0; e < ne && id; ++e) id = perm[e] == (int32_t)e;
  if (id) return {};
  return perm;
}

// Node adjacency of a P1 mesh (two nodes are adjacent when they share an element), as a
// CSR whose rows are sorted and free of duplicates.
void node_graph(int k, int64_t nn, int64_t ne, const int32_t* elems, std::vector<int64_t>& ptr,
                std::vector<int32_t>& adj) {
  ptr.assign(nn + 1, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int l = 0; l < k; ++l) ptr[elems[e * k + l] + 1] += k - 1;
  for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
  adj.resize(ptr[nn]);
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t e = 0; e < ne; ++e)
    for (int l = 0; l < k; ++l)
      for (int m = 0; m < k; ++m)
        if (m != l) adj[fill[elems[e * k + l]]++] = elems[e * k + m];
  // sort and deduplicate each row, compacting in place
  int64_t out = 0;
  for (int64_t i = 0; i < nn; ++i) {
    const int64_t b = ptr[i], end = ptr[i + 1];
    std::sort(adj.begin() + b, adj.begin() + end);
    const int64_t start = out;
    for (int64_t q = b; q < end; ++q)
      if (q == b || adj[q] != adj[q - 1]) adj[out++] = adj[q];
    ptr[i] = start;
  }
  ptr[nn] = out;
  adj.resize(out);
}

// Reverse Cuthill-McKee renumbering of the node graph (Cuthill & McKee 1969; reversed as
// proposed by George 1971); perm[new] = old.  Each connected component is numbered from a
// pseudo-peripheral node (George & Liu: restart the level structure from a node of least
// degree in its last level while its depth grows), visiting the unnumbered neighbours of
// each node in order of increasing degree (ties by id); the whole sequence is then reversed.
// Components are taken in order of their least-degree, least-id node.
std::vector<int32_t> rcm_order(int k, int64_t nn, int64_t ne, const int32_t* elems) {
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
  node_graph(k, nn, ne, elems, ptr, adj);
  auto deg = [&](int32_t i) { return ptr[i + 1] - ptr[i]; };
  auto by_degree = [&](int32_t a, int32_t b) {
    return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
  };
  std::vector<int32_t> seeds(nn);
  std::iota(seeds.begin(), seeds.end(), 0);
  std::stable_sort(seeds.begin(), seeds.end(), by_degree);

  std::vector<int32_t> order;
  order.reserve(nn);
  std::vector<uint8_t> numbered(nn, 0);
  std::vector<int64_t> stamp(nn, -1);   // the last search that reached each node
  std::vector<int32_t> queue;
  int64_t bfs_id = 0;
  // Level structure rooted at r within r's component: returns its depth and a node of
  // least degree (then least id) in its last level.
  auto levels = [&](int32_t r, int32_t* last_min) {
    ++bfs_id;
    queue.assign(1, r);
    stamp[r] = bfs_id;
    int depth = 0;
    size_t head = 0;
    while (true) {
      const size_t level_end = queue.size();
      int32_t best = queue[head];
      for (size_t q = head; q < level_end; ++q) {
        if (by_degree(queue[q], best)) best = queue[q];
        const int32_t u = queue[q];
        for (int64_t a = ptr[u]; a < ptr[u + 1]; ++a)
          if (stamp[adj[a]] != bfs_id) {
            stamp[adj[a]] = bfs_id;
            queue.push_back(adj[a]);
          }
      }
      if (queue.size() == level_end) {
        *last_min = best;
        return depth;
      }
      head = level_end;
      ++depth;
    }
  };
  std::vector<int32_t> nb;
  for (int32_t s0 : seeds) {
    if (numbered[s0]) continue;
    int32_t root = s0, cand;
    int depth = levels(root, &cand);
    for (int it = 0; it < 16 && cand != root; ++it) {
      int32_t next;
      const int dc = levels(cand, &next);
      if (dc <= depth) break;
      root = cand;
      depth = dc;
      cand = next;
    }
    size_t head = order.size();
    order.push_back(root);
    numbered[root] = 1;
    while (head < order.size()) {
      const int32_t u = order[head++];
      nb.clear();
      for (int64_t a = ptr[u]; a < ptr[u + 1]; ++a)
        if (!numbered[adj[a]]) {
          numbered[adj[a]] = 1;
          nb.push_back(adj[a]);
        }
      std::sort(nb.begin(), nb.end(), by_degree);
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// Checks shared by fe_mesh_upload and fe_node_order.
fe_status check_mesh(int dim, int64_t nn, const double* coords, int64_t ne, const int32_t* elems,
                     int order) {
  if (dim != 2 && dim != 3) return set_error(FE_EINVAL, "dim must be 2 or 3");
  if (nn < 0 || ne < 0) return set_error(FE_EINVAL, "negative size");
  if (nn >= (int64_t)1 << 31 || ne * (dim + 1) >= (int64_t)1 << 31)
    return set_error(FE_EINVAL, "mesh too large: n_nodes and n_elems*(dim+1) must be < 2^31");
  if ((nn > 0 && !coords) || (ne > 0 && !elems)) return set_error(FE_EINVAL, "null mesh array");
  if (order != FE_ORDER_NONE && order != FE_ORDER_MORTON && order != FE_ORDER_RCM)
    return set_error(FE_EINVAL, "bad order");
  const int k = dim + 1;
  for (int64_t e = 0; e < ne; ++e)
    for (int l = 0; l < k; ++l) {
      int32_t i = elems[e * k + l];
      if (i < 0 || i >= nn) return set_error(FE_EINVAL, "element node id out of range");
      for (int l2 = 0; l2 < l; ++l2)
        if (elems[e * k + l2] == i) return set_error(FE_EINVAL, "repeated node in an element");
    }
  return FE_OK;
}

// The node renumbering of `order` (perm[new] = old); empty for FE_ORDER_NONE.
std::vector<int32_t> node_order(int dim, int64_t nn, const double* coords, int64_t ne,
                                const int32_t* elems, int order) {
  if (order == FE_ORDER_MORTON) return morton_order(dim, nn, coords);
  if (order == FE_ORDER_RCM) return rcm_order(dim + 1, nn, ne, elems);
  return {};
}

fe_status check_ready(fe_ctx* c, bool need_model = true) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (!c->have_mesh) return set_error(FE_EINVAL, "no mesh uploaded");
  if (!c->have_pre) return set_error(FE_EINVAL, "fe_precompute has not been called");
  if (need_model && !c->model_set) return set_error(FE_EINVAL, "fe_set_model has not been called");
  return FE_OK;
}

fe_status eval(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
               bool want_grad) {
  if (c->model == FE_PLAPLACE_LP && c->precision != FE_F64)
    return set_error(FE_EINVAL, "the componentwise p-Laplacian is evaluated in FP64 only");
  if (c->precision == FE_F32_COMP) return launch_eval_f32(c, v, J, dens, g, want_energy, want_grad);
  if (c->precision == FE_DF64) return launch_eval_df64(c, v, J, dens, g, want_energy, want_grad);
  return launch_eval_f64(c, v, J, dens, g, want_energy, want_grad);
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" {

int fe_version(void) { return 10000; }

fe_status fe_node_order(int dim, int64_t nn, const double* coords, int64_t ne,
                        const int32_t* elems, int order, int32_t* perm) {
  fe_status st = check_mesh(dim, nn, coords, ne, elems, order);
  if (st) return st;
  if (nn > 0 && !perm) return set_error(FE_EINVAL, "perm is null");
  std::vector<int32_t> p = node_order(dim, nn, coords, ne, elems, order);
  if (p.empty()) {
    for (int64_t i = 0; i < nn; ++i) perm[i] = (int32_t)i;
  } else {
    std::copy(p.begin(), p.end(), perm);
  }
  return FE_OK;
}

const char* fe_last_error(void) { return g_err.c_str(); }

fe_status fe_create(fe_ctx** out, int device, void* cuda_stream) {
  if (!out) return set_error(FE_EINVAL, "out is null");
  *out = nullptr;
  int ndev = 0;
  fe_status st = cuda_check(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
  if (st) return st;
  if (device < 0 || device >= ndev) return set_error(FE_EINVAL, "bad device index");
  fe_ctx* c = new (std::nothrow) fe_ctx();
  if (!c) return set_error(FE_ENOMEM, "host allocation");
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  DeviceGuard g(device);
  if (!g.ok) {
    delete c;
    return set_error(FE_ECUDA, "cudaSetDevice failed");
  }
  if ((st = dev_alloc(c, &c->partials, kMaxElemBlocks + kMaxNodeBlocks)) ||
      (st = dev_alloc(c, &c->counter, 1)) || (st = dev_alloc(c, &c->status, 1)) ||
      (st = dev_alloc(c, &c->stage_J, 1))) {
    fe_destroy(c);
    return st;
  }
  cudaMemset(c->counter, 0, sizeof(unsigned));
  cudaMemset(c->status, 0, sizeof(int));
  if ((st = cuda_check(cudaDeviceSynchronize(), "fe_create"))) {
    fe_destroy(c);
    return st;
  }
  *out = c;
  return FE_OK;
}

fe_status fe_destroy(fe_ctx* c) {
  if (!c) return FE_OK;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& pool : c->prof_ev)
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  free_mesh(c);
  dev_free(c, &c->partials, kMaxElemBlocks + kMaxNodeBlocks);
  dev_free(c, &c->counter, 1);
  dev_free(c, &c->status, 1);
  dev_free(c, &c->stage_J, 1);
  if (c->pipe_in) cudaStreamDestroy(c->pipe_in);
  if (c->pipe_out) cudaStreamDestroy(c->pipe_out);
  for (auto& pair : c->pipe_ev)
    for (cudaEvent_t e : pair)
      if (e) cudaEventDestroy(e);
  dev_free(c, &c->cg_part, 2 * kMaxNodeBlocks);
  dev_free(c, &c->cg_ticket, 1);
  dev_free(c, &c->cg_state, 1);
  if (c->cg_host) cudaFreeHost(c->cg_host);
  delete c;
  return FE_OK;
}

fe_status fe_set_stream(fe_ctx* c, void* cuda_stream) {
  if (!c) return set_error(FE_EINVAL, "null context");
  c->stream = (cudaStream_t)cuda_stream;
  return FE_OK;
}

fe_status fe_mesh_upload(fe_ctx* c, int dim, int d, int64_t nn, const double* coords, int64_t ne,
                         const int32_t* elems, const uint8_t* dirichlet, int order) {
  FE_TRACE("fe_mesh_upload");
  if (!c) return set_error(FE_EINVAL, "null context");
  if (d != 1 && d != dim) return set_error(FE_EINVAL, "d must be 1 or dim");
  fe_status st0 = check_mesh(dim, nn, coords, ne, elems, order);
  if (st0) return st0;
  const int k = dim + 1;
  DeviceGuard g(c->device);
  if (!g.ok) return set_error(FE_ECUDA, "cudaSetDevice failed");
  cudaStreamSynchronize(c->stream);
  free_mesh(c);
  c->dim = dim;
  c->d = d;
  c->nn = nn;
  c->ne = ne;
  c->order = order;

  // internal numbering: nodes as `order` asks; elements always along the Morton curve of
  // their centroids, so that a contiguous range of elements is a compact piece of the mesh
  // (the tiles of the fused element + patch kernels are such ranges)
  std::vector<int32_t> iperm;  // caller node -> device node
  if (order != FE_ORDER_NONE && nn > 0) {
    c->perm_h = node_order(dim, nn, coords, ne, elems, order);
    iperm.resize(nn);
    for (int64_t i = 0; i < nn; ++i) iperm[c->perm_h[i]] = (int32_t)i;
  }
  c->eperm_h = element_order(dim, nn, coords, ne, elems);
  const bool ident = c->perm_h.empty();
  const bool eident = c->eperm_h.empty();
  std::vector<double> Xd(nn * dim);
  std::vector<uint8_t> dd(nn * d, 0);
  for (int64_t i = 0; i < nn; ++i) {
    const int64_t src = ident ? i : c->perm_h[i];
    for (int m = 0; m < dim; ++m) Xd[i * dim + m] = coords[src * dim + m];
    if (dirichlet)
      for (int j = 0; j < d; ++j) dd[i * d + j] = dirichlet[src * d + j] ? 1 : 0;
  }
  std::vector<int32_t> Ed(ne * k);
  for (int64_t e = 0; e < ne; ++e) {
    const int64_t src = eident ? e : c->eperm_h[e];
    for (int l = 0; l < k; ++l) {
      int32_t n = elems[src * k + l];
      Ed[(int64_t)l * ne + e] = ident ? n : iperm[n];
    }
  }
  fe_status st;
  if ((st = dev_alloc(c, &c->X, nn * dim)) || (st = dev_alloc(c, &c->elems, ne * k)) ||
      (st = dev_alloc(c, &c->dir, nn * d))) {
    free_mesh(c);
    return st;
  }
  cudaMemcpy(c->X, Xd.data(), sizeof(double) * nn * dim, cudaMemcpyHostToDevice);
  cudaMemcpy(c->elems, Ed.data(), sizeof(int32_t) * ne * k, cudaMemcpyHostToDevice);
  cudaMemcpy(c->dir, dd.data(), nn * d, cudaMemcpyHostToDevice);
  if (!ident) {
    if ((st = dev_alloc(c, &c->perm, nn)) || (st = dev_alloc(c, &c->iperm, nn))) {
      free_mesh(c);
      return st;
    }
    cudaMemcpy(c->perm, c->perm_h.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice);
    cudaMemcpy(c->iperm, iperm.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice);
  }
  if (!eident) {
    if ((st = dev_alloc(c, &c->eperm, ne))) {
      free_mesh(c);
      return st;
    }
    cudaMemcpy(c->eperm, c->eperm_h.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice);
  }
  if ((st = cuda_check(cudaDeviceSynchronize(), "mesh upload"))) {
    free_mesh(c);
    return st;
  }
  c->have_mesh = true;
  if (!c->f_host.empty() && (int64_t)c->f_host.size() != nn * d) c->f_host.clear();
  if (c->model_set && ((c->model == FE_NEOHOOKE && d != dim) || (c->model == FE_PLAPLACE && d != 1)))
    c->model_set = false;
  return FE_OK;
}

fe_status fe_set_model(fe_ctx* c, int model, double p, double C1, double D1) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (!c->have_mesh) return set_error(FE_EINVAL, "upload the mesh before the model");
  if (model == FE_PLAPLACE || model == FE_PLAPLACE_LP) {
    if (c->d != 1) return set_error(FE_EINVAL, "the p-Laplacian needs d = 1");
    if (!(p > 1.0) || !std::isfinite(p)) return set_error(FE_EINVAL, "p must be > 1");
  } else if (model == FE_NEOHOOKE) {
    if (c->d != c->dim) return set_error(FE_EINVAL, "Neo-Hookean needs d = dim");
    if (!std::isfinite(C1) || !std::isfinite(D1)) return set_error(FE_EINVAL, "bad C1/D1");
  } else {
    return set_error(FE_EINVAL, "unknown model");
  }
  c->model = model;
  c->p = p;
  c->C1 = C1;
  c->D1 = D1;
  c->model_set = true;
  return FE_OK;
}

fe_status fe_set_load(fe_ctx* c, const double* f_host) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (!c->have_mesh) return set_error(FE_EINVAL, "upload the mesh before the load");
  if (!f_host) {
    c->f_host.clear();
  } else {
    c->f_host.assign(f_host, f_host + c->nn * c->d);
  }
  if (c->have_pre) {
    DeviceGuard g(c->device);
    fe_status st = launch_load_vector(c);
    if (st) return st;
    return cuda_check(cudaStreamSynchronize(c->stream), "load vector");
  }
  return FE_OK;
}

fe_status fe_precompute(fe_ctx* c, unsigned precisions) {
  FE_TRACE("fe_precompute");
  if (!c) return set_error(FE_EINVAL, "null context");
  if (!c->have_mesh) return set_error(FE_EINVAL, "no mesh uploaded");
  if (precisions == 0 || (precisions & ~7u)) return set_error(FE_EINVAL, "bad precision mask");
  DeviceGuard g(c->device);
  if (!g.ok) return set_error(FE_ECUDA, "cudaSetDevice failed");
  cudaStreamSynchronize(c->stream);
  free_precompute(c);
  const size_t ne = (size_t)c->ne, nn = (size_t)c->nn, k = (size_t)c->dim + 1;
  const int dp = padded_d(c->d);
  fe_status st;
  if ((st = dev_alloc(c, &c->dphi, ne * c->dim * c->dim)) || (st = dev_alloc(c, &c->vol, ne)) ||
      (st = dev_alloc(c, &c->row_ptr, nn + 1)) || (st = dev_alloc(c, &c->ent, ne * k)) ||
      (st = dev_alloc(c, &c->slot, ne * k)) || (st = dev_alloc(c, &c->b, nn * c->d))) {
    free_precompute(c);
    return st;
  }
  if (precisions & (1u << FE_F64)) {
    if ((st = dev_alloc(c, &c->u, nn * dp)) || (st = dev_alloc(c, &c->r, ne * k * c->d))) {
      free_precompute(c);
      return st;
    }
  }
  if (precisions & (1u << FE_F32_COMP)) {
    if ((st = build_tiles(c)) || (st = dev_alloc(c, &c->blk32, (size_t)c->n_tiles * tile_block_bytes_f32(c->dim)))) {
      free_precompute(c);
      return st;
    }
  }
  if ((precisions & ((1u << FE_DF64) | (1u << FE_F32_COMP))) && (st = dev_alloc(c, &c->u_df, nn * dp))) {
    free_precompute(c);
    return st;
  }
  if (precisions & (1u << FE_DF64)) {
    if ((st = dev_alloc(c, &c->dphi_df, ne * c->dim * c->dim)) || (st = dev_alloc(c, &c->vol_df, ne)) ||
        (st = dev_alloc(c, &c->log_tab, kLogTable)) || (st = dev_alloc(c, &c->r_df, ne * k * c->d))) {
      free_precompute(c);
      return st;
    }
  }
  c->pre_mask = precisions;
  cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if ((st = launch_precompute(c)) || (st = launch_load_vector(c)) ||
      ((precisions & (1u << FE_DF64)) && (st = launch_precompute_df(c)))) {
    free_precompute(c);
    return st;
  }
  int hs = 0;
  cudaMemcpyAsync(&hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if ((st = cuda_check(cudaStreamSynchronize(c->stream), "precompute"))) {
    free_precompute(c);
    return st;
  }
  cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (hs & kStatusDegenerate) {
    free_precompute(c);
    return set_error(FE_EINVAL, "degenerate element (zero volume)");
  }
  // the per-element local ids / slots are in the FP32 tile blocks now (copied there by the
  // precompute, which the synchronisation above finished): their own array is not read again
  dev_free(c, &c->tile_elem, (size_t)c->ne);
  c->have_pre = true;
  c->precision = (precisions & 1u) ? FE_F64 : (precisions & 4u) ? FE_DF64 : FE_F32_COMP;
  return FE_OK;
}

fe_status fe_set_precision(fe_ctx* c, int precision) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (precision != FE_F64 && precision != FE_F32_COMP && precision != FE_DF64)
    return set_error(FE_EINVAL, "bad precision");
  if (!c->have_pre || !(c->pre_mask & (1u << precision)))
    return set_error(FE_EINVAL, "precision was not precomputed");
  c->precision = precision;
  return FE_OK;
}

fe_status fe_set_input(fe_ctx* c, int input) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (input != FE_INPUT_DEFORMATION && input != FE_INPUT_DISPLACEMENT) return set_error(FE_EINVAL, "bad input kind");
  c->input = input;
  return FE_OK;
}

fe_status fe_footprint(const fe_ctx* c, size_t* bytes) {
  if (!c || !bytes) return set_error(FE_EINVAL, "null argument");
  *bytes = c->bytes;
  return FE_OK;
}

fe_status fe_energy(fe_ctx* c, const double* v, double* J, double* dens) {
  FE_TRACE("fe_energy");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !J) return set_error(FE_EINVAL, "null v or J");
  DeviceGuard g(c->device);
  return eval(c, v, J, dens, nullptr, true, false);
}

fe_status fe_gradient_exact(fe_ctx* c, const double* v, double* gout) {
  FE_TRACE("fe_gradient_exact");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !gout) return set_error(FE_EINVAL, "null v or g");
  DeviceGuard g(c->device);
  return eval(c, v, nullptr, nullptr, gout, false, true);
}

fe_status fe_energy_gradient(fe_ctx* c, const double* v, double* J, double* gout) {
  FE_TRACE("fe_energy_gradient");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !J || !gout) return set_error(FE_EINVAL, "null v, J or g");
  DeviceGuard g(c->device);
  return eval(c, v, J, nullptr, gout, true, true);
}

fe_status fe_hessian_vector(fe_ctx* c, const double* v, const double* w, double* Hw) {
  FE_TRACE("fe_hessian_vector");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !w || !Hw) return set_error(FE_EINVAL, "null v, w or Hw");
  if (!(c->pre_mask & (1u << FE_F64)))
    return set_error(FE_EINVAL, "the Hessian-vector product needs the FP64 precompute");
  DeviceGuard g(c->device);
  if (!c->w_hvp && (st = dev_alloc(c, &c->w_hvp, (size_t)c->nn * padded_d(c->d)))) return st;
  return launch_hvp_f64(c, v, w, Hw);
}

namespace fe {
namespace {
// Dof vectors between the caller's numbering and the device numbering (perm: device -> caller).
__global__ void __launch_bounds__(kThreads) k_permute_dofs(int64_t nn, int d, const int32_t* __restrict__ perm,
                                                           const double* __restrict__ in, double* __restrict__ out,
                                                           bool to_device) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const int64_t p = perm[i];
    for (int j = 0; j < d; ++j) {
      if (to_device) out[i * d + j] = in[p * d + j];
      else out[p * d + j] = in[i * d + j];
    }
  }
}
}  // namespace
}  // namespace fe

fe_status fe_set_vector_order(fe_ctx* c, int order) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (order != FE_VECTORS_CALLER && order != FE_VECTORS_DEVICE) return set_error(FE_EINVAL, "unknown vector order");
  c->vector_order = order;
  return FE_OK;
}

static fe_status permute_dofs(fe_ctx* c, const double* in, double* out, bool to_device) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (!c->have_mesh) return set_error(FE_EINVAL, "no mesh uploaded");
  if (!in || !out) return set_error(FE_EINVAL, "null vector");
  if (in == out) return set_error(FE_EINVAL, "the two vectors must not overlap");
  DeviceGuard g(c->device);
  const int64_t n = c->nn * c->d;
  if (!c->perm)
    return cuda_check(cudaMemcpyAsync(out, in, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream),
                      "vector copy");
  k_permute_dofs<<<grid_for(c->nn, kMaxNodeBlocks), kThreads, 0, c->stream>>>(c->nn, c->d, c->perm, in, out,
                                                                                 to_device);
  c->launches++;
  return cuda_check(cudaGetLastError(), "vector permutation");
}

fe_status fe_to_device_order(fe_ctx* c, const double* x, double* y) { return permute_dofs(c, x, y, true); }
fe_status fe_from_device_order(fe_ctx* c, const double* y, double* x) { return permute_dofs(c, y, x, false); }

fe_status fe_cg_steihaug(fe_ctx* c, const double* v, const double* g, double radius, double tol, int max_cg,
                         double* z, double* Hz, int* iters, int* boundary) {
  FE_TRACE("fe_cg_steihaug");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !g || !z || !Hz || !iters || !boundary) return set_error(FE_EINVAL, "null argument");
  if (!(radius > 0.0) || !std::isfinite(radius)) return set_error(FE_EINVAL, "radius must be finite and > 0");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return set_error(FE_EINVAL, "tol must be finite and >= 0");
  if (max_cg < 0) return set_error(FE_EINVAL, "negative max_cg");
  if (!(c->pre_mask & (1u << FE_F64)))
    return set_error(FE_EINVAL, "the Hessian-vector product needs the FP64 precompute");
  DeviceGuard dg(c->device);
  const size_t n = (size_t)c->nn * c->d;
  if (!c->w_hvp && (st = dev_alloc(c, &c->w_hvp, (size_t)c->nn * padded_d(c->d)))) return st;
  if (!c->cg_vec && (st = dev_alloc(c, &c->cg_vec, 3 * n))) return st;
  if (!c->hvp_cache && (st = dev_alloc(c, &c->hvp_cache, hvp_cache_doubles(c)))) return st;
  if (!c->cg_part && (st = dev_alloc(c, &c->cg_part, 2 * kMaxNodeBlocks))) return st;
  if (!c->cg_ticket) {
    if ((st = dev_alloc(c, &c->cg_ticket, 1))) return st;
    if ((st = cuda_check(cudaMemsetAsync(c->cg_ticket, 0, sizeof(unsigned), c->stream), "cg ticket"))) return st;
  }
  if (!c->cg_state && (st = dev_alloc(c, &c->cg_state, 1))) return st;
  if (!c->cg_host && (st = cuda_check(cudaMallocHost((void**)&c->cg_host, sizeof(CgState)), "cg host state"))) {
    c->cg_host = nullptr;
    return st;
  }
  return launch_cg_steihaug(c, v, g, radius, tol, max_cg, z, Hz, iters, boundary);
}

fe_status fe_gradient_fd(fe_ctx* c, const double* v, double eps, double* gout, const int64_t* dofs,
                         int64_t ndofs) {
  FE_TRACE("fe_gradient_fd");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v || !gout) return set_error(FE_EINVAL, "null v or g");
  if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(FE_EINVAL, "eps must be > 0");
  if (dofs && ndofs < 0) return set_error(FE_EINVAL, "negative n_dofs");
  if (!(c->pre_mask & (1u << FE_F64)))
    return set_error(FE_EINVAL, "the central-difference gradient needs the FP64 precompute");
  DeviceGuard g(c->device);
  return launch_fd_f64(c, v, eps, gout, dofs, ndofs);
}

// Device address of page-locked host memory mapped into the device's address space, or
// nullptr (pageable memory, or a registration without a mapping).
static void* mapped_device_ptr(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

fe_status fe_energy_gradient_host(fe_ctx* c, const double* v_host, double* J_host, double* g_host) {
  FE_TRACE("fe_energy_gradient_host");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v_host || !J_host || !g_host) return set_error(FE_EINVAL, "null argument");
  DeviceGuard g(c->device);
  const size_t n = (size_t)c->nn * c->d;
  // Page-locked buffers are read (v, by the node preparation) and written (g, by the patch
  // gather) by the kernels directly over the host link; pageable ones are staged through
  // device buffers with one copy each way.
  const double* vin = static_cast<const double*>(mapped_device_ptr(v_host));
  double* gout = static_cast<double*>(mapped_device_ptr(g_host));
  if ((!vin || !gout) && !c->stage_v && ((st = dev_alloc(c, &c->stage_v, n)) || (st = dev_alloc(c, &c->stage_g, n))))
    return st;
  if (!vin) {
    cudaMemcpyAsync(c->stage_v, v_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
    vin = c->stage_v;
  }
  if ((st = eval(c, vin, c->stage_J, nullptr, gout ? gout : c->stage_g, true, true))) return st;
  cudaMemcpyAsync(J_host, c->stage_J, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!gout) cudaMemcpyAsync(g_host, c->stage_g, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  return fe_sync_status(c);
}

fe_status fe_energy_gradient_host_async(fe_ctx* c, const double* v_host, double* J_host, double* g_host) {
  FE_TRACE("fe_energy_gradient_host_async");
  fe_status st = check_ready(c);
  if (st) return st;
  if (!v_host || !J_host || !g_host) return set_error(FE_EINVAL, "null argument");
  DeviceGuard g(c->device);
  const size_t n = (size_t)c->nn * c->d;
  if (!c->pipe_in) {
    if ((st = cuda_check(cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking), "copy stream")) ||
        (st = cuda_check(cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking), "copy stream")))
      return st;
    for (auto& pair : c->pipe_ev)
      for (cudaEvent_t& e : pair)
        if ((st = cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event"))) return st;
  }
  if (!c->pipe_J) {
    for (int s = 0; s < 2; ++s)
      if ((st = dev_alloc(c, &c->pipe_v[s], n)) || (st = dev_alloc(c, &c->pipe_g[s], n))) {
        pipe_free(c);
        return st;
      }
    if ((st = dev_alloc(c, &c->pipe_J, 2))) {
      pipe_free(c);
      return st;
    }
    c->pipe_k = 0;
  }
  const int s = (int)(c->pipe_k & 1);
  cudaEvent_t in_done = c->pipe_ev[0][s], eval_done = c->pipe_ev[1][s], out_done = c->pipe_ev[2][s];
  const bool reuse = c->pipe_k >= 2;   // slot s held evaluation k - 2
  // v into slot s once evaluation k - 2 has finished reading it
  if (reuse) cudaStreamWaitEvent(c->pipe_in, eval_done, 0);
  cudaMemcpyAsync(c->pipe_v[s], v_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->pipe_in);
  cudaEventRecord(in_done, c->pipe_in);
  // evaluate once v has arrived and the slot's previous J and g have been copied out
  cudaStreamWaitEvent(c->stream, in_done, 0);
  if (reuse) cudaStreamWaitEvent(c->stream, out_done, 0);
  if ((st = eval(c, c->pipe_v[s], c->pipe_J + s, nullptr, c->pipe_g[s], true, true))) return st;
  cudaEventRecord(eval_done, c->stream);
  cudaStreamWaitEvent(c->pipe_out, eval_done, 0);
  cudaMemcpyAsync(J_host, c->pipe_J + s, sizeof(double), cudaMemcpyDeviceToHost, c->pipe_out);
  cudaMemcpyAsync(g_host, c->pipe_g[s], sizeof(double) * n, cudaMemcpyDeviceToHost, c->pipe_out);
  cudaEventRecord(out_done, c->pipe_out);
  ++c->pipe_k;
  return cuda_check(cudaGetLastError(), "fe_energy_gradient_host_async");
}

fe_status fe_host_wait(fe_ctx* c) {
  if (!c) return set_error(FE_EINVAL, "null context");
  DeviceGuard g(c->device);
  if (c->pipe_out) {
    fe_status st = cuda_check(cudaStreamSynchronize(c->pipe_out), "copy stream");
    if (st) return st;
  }
  return fe_sync_status(c);
}

fe_status fe_set_wait_limit(fe_ctx* c, int64_t cycles) {
  if (!c) return set_error(FE_EINVAL, "null context");
  if (cycles < 0) return set_error(FE_EINVAL, "negative wait limit");
  c->wait_limit = cycles > 0 ? (long long)cycles : kWaitCycles;
  return FE_OK;
}

fe_status fe_sync_status(fe_ctx* c) {
  if (!c) return set_error(FE_EINVAL, "null context");
  DeviceGuard g(c->device);
  int hs = 0;
  cudaMemcpyAsync(&hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  fe_status st = cuda_check(cudaStreamSynchronize(c->stream), "stream");
  if (st) return st;
  if (hs) {
    cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
  }
  if (hs & kStatusTimeout) return set_error(FE_ETIMEOUT, "a bounded device wait gave up");
  if (hs & kStatusDomain) return set_error(FE_EDOMAIN, "an element has det F <= 0");
  return FE_OK;
}

fe_status fe_get_shape_gradients(fe_ctx* c, double* dphi_host, double* vol_host) {
  fe_status st = check_ready(c, false);
  if (st) return st;
  if (!dphi_host || !vol_host) return set_error(FE_EINVAL, "null argument");
  DeviceGuard g(c->device);
  const size_t nd = (size_t)c->ne * (c->dim + 1) * c->dim;
  double *dd = nullptr, *vv = nullptr;
  if ((st = cuda_check(cudaMalloc((void**)&dd, sizeof(double) * (nd ? nd : 1)), "alloc"))) return st;
  if ((st = cuda_check(cudaMalloc((void**)&vv, sizeof(double) * (c->ne ? c->ne : 1)), "alloc"))) {
    cudaFree(dd);
    return st;
  }
  st = launch_expand_dphi(c, dd, vv);
  if (!st) {
    cudaMemcpyAsync(dphi_host, dd, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(vol_host, vv, sizeof(double) * c->ne, cudaMemcpyDeviceToHost, c->stream);
    st = cuda_check(cudaStreamSynchronize(c->stream), "read back");
  }
  cudaFree(dd);
  cudaFree(vv);
  return st;
}

fe_status fe_get_patches(fe_ctx* c, int64_t* row_ptr_host, int64_t* ent_host) {
  fe_status st = check_ready(c, false);
  if (st) return st;
  if (!row_ptr_host || !ent_host) return set_error(FE_EINVAL, "null argument");
  DeviceGuard g(c->device);
  const int64_t nn = c->nn, ne = c->ne, k = c->dim + 1;
  std::vector<int32_t> rp(nn + 1), en(ne * k);
  cudaMemcpyAsync(rp.data(), c->row_ptr, sizeof(int32_t) * (nn + 1), cudaMemcpyDeviceToHost, c->stream);
  if (ne > 0)
    cudaMemcpyAsync(en.data(), c->ent, sizeof(int32_t) * ne * k, cudaMemcpyDeviceToHost, c->stream);
  if ((st = cuda_check(cudaStreamSynchronize(c->stream), "read back"))) return st;
  if (c->perm_h.empty() && c->eperm_h.empty()) {
    for (int64_t i = 0; i <= nn; ++i) row_ptr_host[i] = rp[i];
    for (int64_t q = 0; q < ne * k; ++q) ent_host[q] = en[q];
    return FE_OK;
  }
  // translate to the caller's numbering: caller node iu is device node iperm[iu], device
  // element e is caller element eperm[e]; rows are listed in caller element order
  std::vector<int32_t> iperm(nn);
  for (int64_t i = 0; i < nn; ++i) iperm[c->perm_h.empty() ? i : c->perm_h[i]] = (int32_t)i;
  row_ptr_host[0] = 0;
  for (int64_t iu = 0; iu < nn; ++iu) {
    const int32_t i = iperm[iu];
    const int64_t len = rp[i + 1] - rp[i];
    int64_t* out = ent_host + row_ptr_host[iu];
    for (int64_t t = 0; t < len; ++t) {
      const int32_t v = en[rp[i] + t];
      out[t] = (int64_t)(c->eperm_h.empty() ? v / k : c->eperm_h[v / k]) * k + v % k;
    }
    std::sort(out, out + len);
    row_ptr_host[iu + 1] = row_ptr_host[iu] + len;
  }
  return FE_OK;
}

fe_status fe_get_load_vector(fe_ctx* c, double* b_host) {
  fe_status st = check_ready(c, false);
  if (st) return st;
  if (!b_host) return set_error(FE_EINVAL, "null argument");
  DeviceGuard g(c->device);
  const int64_t nn = c->nn, d = c->d;
  std::vector<double> bd(nn * d);
  cudaMemcpyAsync(bd.data(), c->b, sizeof(double) * nn * d, cudaMemcpyDeviceToHost, c->stream);
  if ((st = cuda_check(cudaStreamSynchronize(c->stream), "read back"))) return st;
  for (int64_t i = 0; i < nn; ++i) {
    const int64_t dst = c->perm_h.empty() ? i : c->perm_h[i];
    for (int j = 0; j < d; ++j) b_host[dst * d + j] = bd[i * d + j];
  }
  return FE_OK;
}

fe_status fe_profile_enable(fe_ctx* c, int enable) {
  if (!c) return set_error(FE_EINVAL, "null context");
  c->prof = enable != 0;
  for (int k = 0; k < FE_PROFILE_STAGES; ++k) c->prof_n[k] = 0;
  return FE_OK;
}

fe_status fe_profile_read(fe_ctx* c, double* ms, int64_t* launches, int n_stages) {
  if (!c || !ms || !launches) return set_error(FE_EINVAL, "null argument");
  if (n_stages < 0 || n_stages > FE_PROFILE_STAGES) return set_error(FE_EINVAL, "bad n_stages");
  DeviceGuard g(c->device);
  fe_status st = cuda_check(cudaStreamSynchronize(c->stream), "profile sync");
  if (st) return st;
  for (int k = 0; k < n_stages; ++k) {
    double tot = 0.0;
    for (int i = 0; i < c->prof_n[k]; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->prof_ev[k][2 * i], c->prof_ev[k][2 * i + 1]) == cudaSuccess) tot += t;
    }
    ms[k] = tot;
    launches[k] = c->prof_n[k];
  }
  for (int k = 0; k < FE_PROFILE_STAGES; ++k) c->prof_n[k] = 0;
  return FE_OK;
}

fe_status fe_diag_df64_log(fe_ctx* c, const double* x, double* y, int64_t n) {
  fe_status st = check_ready(c, false);
  if (st) return st;
  if (!c->log_tab) return set_error(FE_EINVAL, "needs the FE_DF64 precompute");
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(FE_EINVAL, "bad arguments");
  DeviceGuard g(c->device);
  return launch_diag_df_log(c->log_tab, x, y, n, c->stream);
}

fe_status fe_launch_count(const fe_ctx* c, int64_t* count) {
  if (!c || !count) return set_error(FE_EINVAL, "null argument");
  *count = c->launches;
  return FE_OK;
}

}  // extern "C"

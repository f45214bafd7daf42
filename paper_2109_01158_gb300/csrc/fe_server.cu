// fe_server.cu -- continuous-batching server over resident meshes: the host runtime around
// the batched kernels of fe_batch.cu (energy + exact gradient, double-float arithmetic).
//
// Threads:
//   worker     waits for arrived requests; admits them FIFO while their device bytes fit in
//              one contiguous region of the arena ring; stages their vectors in pinned memory
//              (one host-to-device copy per batch; vectors the caller keeps in page-locked
//              memory are copied straight from it); enqueues the three batch kernels and the
//              device-to-host copies of the results; records a completion event.  It prepares
//              the next batch while earlier ones run (up to kSlots batches in flight).
//   completer  waits for the batches in launch order, copies each request's J and g into the
//              caller's buffers, stamps the completion time, frees the arena region and the
//              batch slot.
// Device layout of one batch region: [v_1 .. v_n][g_1 .. g_n][J_1 .. J_n][work_1 .. work_n],
// every piece 256-byte aligned; the v block is copied in, the g and J blocks copied out.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fe_internal.cuh"

namespace fe {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kSlots = 3;

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Req {
  const fe_ctx* mesh = nullptr;
  const double* v = nullptr;
  double* J = nullptr;
  double* g = nullptr;
  int64_t ticket = 0;
  size_t nvals = 0;   // n_nodes * d
  size_t work = 0;    // batch scratch bytes
  size_t bytes = 0;   // device bytes in a batch region
  double t_arrival = 0.0, t_start = 0.0, t_done = 0.0;
  int status = FE_OK;
  bool done = false;
  bool v_pinned = false, g_pinned = false;   // page-locked caller buffers: copied by DMA directly
};

struct Slot {
  std::vector<Req*> reqs;
  std::vector<size_t> voff, goff, Joff;   // offsets inside the region
  size_t off = 0, bytes = 0, vbytes = 0, obytes = 0, obase = 0;
  unsigned char* pin_in = nullptr;
  unsigned char* pin_out = nullptr;
  size_t pin_in_cap = 0, pin_out_cap = 0;
  void* items_host = nullptr;
  void* items_dev = nullptr;
  int items_cap = 0;
  std::vector<fe_batch_item> items;
  cudaEvent_t done = nullptr;
  fe_status launch_status = FE_OK;
};

// Grow a pinned host buffer to at least `need` bytes (geometrically after the first
// allocation; only a request larger than the staging size set at creation grows it).
fe_status grow_pinned(unsigned char** p, size_t* cap, size_t need) {
  if (need <= *cap) return FE_OK;
  size_t n = *cap ? std::max(need, *cap * 2) : need;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  fe_status st = cuda_check(cudaMallocHost((void**)p, n), "server pinned staging");
  if (!st) *cap = n;
  return st;
}

// True for page-locked host memory (cudaMallocHost / cudaHostAlloc / cudaHostRegister).
bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace
}  // namespace fe

using namespace fe;

struct fe_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  int* status = nullptr;        // device status word of the batch kernels (domain bits)
  size_t budget = 0;
  size_t staging = 0;           // pinned bytes per slot and direction (vectors in, results out)
  int max_batch = 1;
  unsigned char* arena = nullptr;
  Clock::time_point epoch;

  std::mutex mu;
  std::condition_variable cv;   // signalled on every state change
  std::deque<Req*> pending;     // submitted, not admitted (arrival order)
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_ticket = 0;
  double last_arrival = -1.0;
  bool stop = false, worker_done = false;

  std::deque<std::pair<size_t, size_t>> regions;   // arena regions in flight, launch order
  Slot slot_store[kSlots];
  std::deque<Slot*> free_slots;
  std::deque<Slot*> inflight;

  std::thread worker, completer;
  int64_t batches = 0, maxb = 0, launches = 0, completed = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }

  // Largest contiguous region available in the ring (caller holds mu).
  size_t ring_avail() const {
    if (regions.empty()) return budget;
    const size_t tail = regions.front().first;
    const size_t head = regions.back().first + regions.back().second;
    if (regions.back().first < tail) return tail - head;   // wrapped: free is [head, tail)
    return std::max(budget - head, tail);                    // free is [head, budget) + [0, tail)
  }

  // Allocate `bytes` (<= ring_avail()) at the ring head (caller holds mu).
  size_t ring_alloc(size_t bytes) {
    size_t off = 0;
    if (!regions.empty()) {
      const size_t tail = regions.front().first;
      const size_t head = regions.back().first + regions.back().second;
      if (regions.back().first < tail) off = head;
      else off = (budget - head >= bytes) ? head : 0;
    }
    regions.emplace_back(off, bytes);
    return off;
  }

  void worker_loop();
  void completer_loop();
  fe_status launch(Slot* S);
};

fe_status fe_server::launch(Slot* S) {
  const int n = (int)S->reqs.size();
  // layout of the region
  S->voff.resize(n);
  S->goff.resize(n);
  S->Joff.resize(n);
  size_t o = 0;
  for (int k = 0; k < n; ++k) {
    S->voff[k] = o;
    o += al256(sizeof(double) * S->reqs[k]->nvals);
  }
  S->vbytes = o;
  S->obase = o;
  for (int k = 0; k < n; ++k) {
    S->goff[k] = o;
    o += al256(sizeof(double) * S->reqs[k]->nvals);
  }
  for (int k = 0; k < n; ++k) {
    S->Joff[k] = o;
    o += 256;
  }
  S->obytes = o - S->obase;
  fe_status st;
  if ((st = grow_pinned(&S->pin_in, &S->pin_in_cap, S->vbytes))) return st;
  if ((st = grow_pinned(&S->pin_out, &S->pin_out_cap, S->obytes))) return st;
  if (n > S->items_cap) {
    if (S->items_host) cudaFreeHost(S->items_host);
    if (S->items_dev) cudaFree(S->items_dev);
    S->items_host = S->items_dev = nullptr;
    S->items_cap = 0;
    const int cap = std::max(n, 64);
    if ((st = cuda_check(cudaMallocHost(&S->items_host, batch_item_bytes() * cap), "server descriptors"))) return st;
    if ((st = cuda_check(cudaMalloc(&S->items_dev, batch_item_bytes() * cap), "server descriptors"))) return st;
    S->items_cap = cap;
  }
  unsigned char* base = arena + S->off;
  S->items.resize(n);
  bool staged_in = false, staged_out = false;
  for (int k = 0; k < n; ++k) {
    Req* r = S->reqs[k];
    if (!r->v_pinned) {
      std::memcpy(S->pin_in + S->voff[k], r->v, sizeof(double) * r->nvals);
      staged_in = true;
    }
    if (!r->g_pinned) staged_out = true;
    fe_batch_item& it = S->items[k];
    it.mesh = r->mesh;
    it.v = reinterpret_cast<const double*>(base + S->voff[k]);
    it.g = reinterpret_cast<double*>(base + S->goff[k]);
    it.J = reinterpret_cast<double*>(base + S->Joff[k]);
    it.work = nullptr;
  }
  size_t w = o;
  for (int k = 0; k < n; ++k) {
    S->items[k].work = base + w;
    w += S->reqs[k]->work;
  }
  // inputs: one copy of the staged block, then the page-locked vectors straight from the callers
  if (staged_in &&
      (st = cuda_check(cudaMemcpyAsync(base, S->pin_in, S->vbytes, cudaMemcpyHostToDevice, stream), "server copy in")))
    return st;
  for (int k = 0; k < n; ++k) {
    Req* r = S->reqs[k];
    if (r->v_pinned && (st = cuda_check(cudaMemcpyAsync(base + S->voff[k], r->v, sizeof(double) * r->nvals,
                                                        cudaMemcpyHostToDevice, stream), "server copy in")))
      return st;
  }
  if ((st = batch_enqueue(stream, S->items.data(), n, S->items_host, S->items_dev, status))) return st;
  // outputs: the staged block (all g's and J's, or the J's only), page-locked g's directly
  const size_t jbase = S->Joff.empty() ? S->obytes : S->Joff[0] - S->obase;
  const size_t from = staged_out ? 0 : jbase;
  if ((st = cuda_check(cudaMemcpyAsync(S->pin_out + from, base + S->obase + from, S->obytes - from,
                                       cudaMemcpyDeviceToHost, stream), "server copy out")))
    return st;
  for (int k = 0; k < n; ++k) {
    Req* r = S->reqs[k];
    if (r->g_pinned && (st = cuda_check(cudaMemcpyAsync(r->g, base + S->goff[k], sizeof(double) * r->nvals,
                                                        cudaMemcpyDeviceToHost, stream), "server copy out")))
      return st;
  }
  return cuda_check(cudaEventRecord(S->done, stream), "server event");
}

void fe_server::worker_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    if (pending.empty()) {
      if (stop) break;
      cv.wait(lk);
      continue;
    }
    const double t = now();
    const double ta = pending.front()->t_arrival;
    if (ta > t) {
      // sleep until shortly before the arrival, then spin (timed waits wake tens of
      // microseconds late, which is the scale of a request)
      if (ta - t > 2e-4) {
        cv.wait_for(lk, std::chrono::duration<double>(ta - t - 1e-4));
      } else {
        lk.unlock();
        while (now() < ta) std::this_thread::yield();
        lk.lock();
      }
      continue;
    }
    if (free_slots.empty()) {
      cv.wait(lk);
      continue;
    }
    // admit arrived requests FIFO while they fit in one contiguous region of the ring
    const size_t avail = ring_avail();
    size_t total = 0, vin = 0, vout = 0;
    int n = 0;
    for (Req* r : pending) {
      if (n >= max_batch || r->t_arrival > t || total + r->bytes > avail) break;
      const size_t vb = al256(sizeof(double) * r->nvals);
      // the staging buffers bound a batch too (a single larger request grows them)
      if (n > 0 && (vin + vb > staging || vout + vb + 256 > staging)) break;
      total += r->bytes;
      vin += vb;
      vout += vb + 256;
      ++n;
    }
    if (n == 0) {   // the oldest request waits for arena space
      cv.wait(lk);
      continue;
    }
    Slot* S = free_slots.front();
    free_slots.pop_front();
    S->reqs.assign(pending.begin(), pending.begin() + n);
    pending.erase(pending.begin(), pending.begin() + n);
    S->bytes = total;
    S->off = ring_alloc(total);
    lk.unlock();
    const double ts = now();
    for (Req* r : S->reqs) r->t_start = ts;
    S->launch_status = launch(S);
    lk.lock();
    inflight.push_back(S);
    batches += 1;
    maxb = std::max<int64_t>(maxb, n);
    if (!S->launch_status) launches += 3;
    cv.notify_all();
  }
  worker_done = true;
  cv.notify_all();
}

void fe_server::completer_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    if (inflight.empty()) {
      if (worker_done) break;
      cv.wait(lk);
      continue;
    }
    Slot* S = inflight.front();
    lk.unlock();
    fe_status st = S->launch_status;
    if (!st) st = cuda_check(cudaEventSynchronize(S->done), "server batch");
    for (size_t k = 0; k < S->reqs.size(); ++k) {
      Req* r = S->reqs[k];
      if (st) {
        r->status = st;
        continue;
      }
      if (!r->g_pinned) std::memcpy(r->g, S->pin_out + (S->goff[k] - S->obase), sizeof(double) * r->nvals);
      double J;
      std::memcpy(&J, S->pin_out + (S->Joff[k] - S->obase), sizeof(double));
      *r->J = J;
      r->status = std::isinf(J) && J > 0 ? FE_EDOMAIN : FE_OK;
    }
    const double td = now();
    lk.lock();
    for (Req* r : S->reqs) {
      r->t_done = td;
      r->done = true;
    }
    completed += (int64_t)S->reqs.size();
    S->reqs.clear();
    inflight.pop_front();
    regions.pop_front();
    free_slots.push_back(S);
    cv.notify_all();
  }
}

extern "C" {

fe_status fe_server_create(fe_server** out, int device, size_t hbm_budget, int max_batch) {
  if (!out || max_batch < 1 || hbm_budget < 4096) return set_error(FE_EINVAL, "bad server arguments");
  *out = nullptr;
  fe_server* s = new (std::nothrow) fe_server();
  if (!s) return set_error(FE_ENOMEM, "host allocation");
  s->device = device;
  s->budget = hbm_budget & ~(size_t)255;
  s->max_batch = max_batch;
  s->epoch = Clock::now();
  int prev = -1;
  cudaGetDevice(&prev);
  fe_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (!st) st = cuda_check(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "server stream");
  if (!st) st = cuda_check(cudaMalloc((void**)&s->status, sizeof(int)), "server status");
  if (!st) st = cuda_check(cudaMemset(s->status, 0, sizeof(int)), "server status");
  if (!st) st = cuda_check(cudaMalloc((void**)&s->arena, s->budget), "server arena");
  // pinned staging and descriptors of every slot are allocated here, so that serving
  // allocates nothing (allocating pinned memory costs milliseconds)
  s->staging = std::min<size_t>(std::max<size_t>(s->budget / 16, 1 << 20), (size_t)256 << 20);
  for (int k = 0; k < kSlots && !st; ++k) {
    Slot& S = s->slot_store[k];
    st = cuda_check(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming), "server event");
    if (!st) st = grow_pinned(&S.pin_in, &S.pin_in_cap, s->staging);
    if (!st) st = grow_pinned(&S.pin_out, &S.pin_out_cap, s->staging);
    if (!st) st = cuda_check(cudaMallocHost(&S.items_host, batch_item_bytes() * max_batch), "server descriptors");
    if (!st) st = cuda_check(cudaMalloc(&S.items_dev, batch_item_bytes() * max_batch), "server descriptors");
    if (!st) S.items_cap = max_batch;
    s->free_slots.push_back(&S);
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (st) {
    fe_server_destroy(s);
    return st;
  }
  s->worker = std::thread([s] { s->worker_loop(); });
  s->completer = std::thread([s] { s->completer_loop(); });
  *out = s;
  return FE_OK;
}

fe_status fe_server_destroy(fe_server* s) {
  if (!s) return FE_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  else s->worker_done = true;
  if (s->completer.joinable()) s->completer.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (Slot& S : s->slot_store) {
    if (S.pin_in) cudaFreeHost(S.pin_in);
    if (S.pin_out) cudaFreeHost(S.pin_out);
    if (S.items_host) cudaFreeHost(S.items_host);
    if (S.items_dev) cudaFree(S.items_dev);
    if (S.done) cudaEventDestroy(S.done);
  }
  if (s->arena) cudaFree(s->arena);
  if (s->status) cudaFree(s->status);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (prev >= 0) cudaSetDevice(prev);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return FE_OK;
}

fe_status fe_server_submit(fe_server* s, const fe_ctx* mesh, const double* v_host, double* J_host,
                           double* g_host, double t_arrival, int64_t* ticket) {
  if (!s || !mesh || !v_host || !J_host || !g_host || !ticket) return set_error(FE_EINVAL, "null argument");
  if (!mesh->have_pre || !mesh->model_set || !(mesh->pre_mask & (1u << FE_DF64)))
    return set_error(FE_EINVAL, "server request: mesh must be precomputed with FE_DF64 and have a model");
  if (mesh->device != s->device) return set_error(FE_EINVAL, "server request: mesh on another device");
  if (mesh->model != FE_PLAPLACE && mesh->model != FE_NEOHOOKE)
    return set_error(FE_EINVAL, "server request: the batched kernels evaluate FE_PLAPLACE and FE_NEOHOOKE");
  Req* r = new (std::nothrow) Req();
  if (!r) return set_error(FE_ENOMEM, "host allocation");
  r->mesh = mesh;
  r->v = v_host;
  r->J = J_host;
  r->g = g_host;
  r->nvals = (size_t)mesh->nn * mesh->d;
  r->work = batch_work_bytes(mesh);
  r->v_pinned = is_pinned(v_host);
  r->g_pinned = is_pinned(g_host);
  r->bytes = 2 * al256(sizeof(double) * r->nvals) + 256 + r->work;
  if (r->bytes > s->budget) {
    delete r;
    return set_error(FE_EINVAL, "server request larger than the HBM budget");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const double t = s->now();
  r->t_arrival = t_arrival < 0.0 ? t : t_arrival;
  if (r->t_arrival < s->last_arrival) r->t_arrival = s->last_arrival;   // keep FIFO = arrival order
  s->last_arrival = r->t_arrival;
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  s->pending.push_back(r);
  *ticket = r->ticket;
  s->cv.notify_all();
  return FE_OK;
}

fe_status fe_server_wait(fe_server* s, int64_t ticket, double* t_arrival, double* t_start, double* t_done) {
  if (!s) return set_error(FE_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(FE_EINVAL, "unknown ticket");
  Req* r = it->second;
  s->cv.wait(lk, [r] { return r->done; });
  if (t_arrival) *t_arrival = r->t_arrival;
  if (t_start) *t_start = r->t_start;
  if (t_done) *t_done = r->t_done;
  const fe_status st = (fe_status)r->status;
  s->reqs.erase(it);
  delete r;
  if (st == FE_EDOMAIN) return set_error(FE_EDOMAIN, "request: an element has det F <= 0");
  if (st) return set_error(st, "request failed on the device");
  return FE_OK;
}

fe_status fe_server_now(const fe_server* s, double* t) {
  if (!s || !t) return set_error(FE_EINVAL, "null argument");
  *t = s->now();
  return FE_OK;
}

fe_status fe_server_stats(const fe_server* s, int64_t* batches, int64_t* max_batch, int64_t* launches,
                          int64_t* completed) {
  if (!s) return set_error(FE_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(const_cast<fe_server*>(s)->mu);
  if (batches) *batches = s->batches;
  if (max_batch) *max_batch = s->maxb;
  if (launches) *launches = s->launches;
  if (completed) *completed = s->completed;
  return FE_OK;
}

fe_status fe_server_reset_stats(fe_server* s) {
  if (!s) return set_error(FE_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->batches = s->maxb = s->launches = s->completed = 0;
  return FE_OK;
}

}  // extern "C"

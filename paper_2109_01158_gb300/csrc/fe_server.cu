// fe_server.cu -- continuous-batching server over resident meshes: the host runtime around
// the persistent batched kernel of fe_batch.cu (energy + exact gradient, double-float
// arithmetic).
//
// Threads:
//   worker     waits for arrived requests; admits them FIFO while their device scratch fits
//              in one contiguous region of the arena ring; orders the batch smallest mesh
//              first (so that small requests sharing a batch with a large one finish early);
//              enqueues the descriptor copy and the one persistent launch.  The kernel reads
//              each request's vector and writes its gradient directly in page-locked host
//              memory (the caller's, or the server's staging for pageable buffers), and
//              raises a per-request completion flag there.  The worker prepares the next batch
//              while earlier ones run (up to kSlots batches in flight).  With max_batch > 1
//              every slot has its own stream, so a batch's blocks start on the SMs that the
//              batch before it frees during its last tiles; with max_batch = 1 (one request
//              at a time) all batches run in order on one stream.
//   completer  polls the completion flags of the batches in flight and completes each
//              request as soon as its flag is up (copies out of the staging where the caller's
//              buffer is pageable, stamps the completion time), not at the end of its batch;
//              frees a batch's arena region and slot once all its requests are complete.
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
#include "trace.h"

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
  const double* v_dev = nullptr;   // device address of a page-locked v (null: pageable)
  double* g_dev = nullptr;         // device address of a page-locked g (null: pageable)
  int64_t ticket = 0;
  size_t nvals = 0;   // n_nodes * d
  size_t bytes = 0;   // device scratch of the batched kernel (arena bytes)
  double t_arrival = 0.0, t_start = 0.0, t_done = 0.0;
  int status = FE_OK;
  bool done = false;
};

struct Slot {
  std::vector<Req*> reqs;
  std::vector<size_t> voff, goff;    // offsets in the pinned staging (pageable buffers)
  std::vector<char> fin;             // request k completed (completer only)
  std::vector<Req*> newly;           // completed by the last poll, not yet published
  int nfin = 0;
  size_t off = 0, bytes = 0;         // arena region
  unsigned char* pin_in = nullptr;   // staging of pageable vectors
  unsigned char* pin_out = nullptr;  // J of every request, then staging of pageable gradients
  unsigned char* pin_in_dev = nullptr;
  unsigned char* pin_out_dev = nullptr;
  size_t pin_in_cap = 0, pin_out_cap = 0;
  int* flags = nullptr;              // page-locked completion flags, one per request
  int* flags_dev = nullptr;
  void* stage_host = nullptr;        // descriptor block (pinned) and its device copy
  void* stage_dev = nullptr;
  std::vector<fe_batch_item> items;
  cudaStream_t stream = nullptr;     // the server's stream, or the slot's own (max_batch > 1)
  bool own_stream = false;
  bool any_error = false;            // a request of the batch ended with an error flag
  cudaEvent_t done = nullptr;
  fe_status launch_status = FE_OK;
};

// Device address of page-locked host memory, or null (pageable, or not mapped).
template <class T>
T* mapped(T* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost) return nullptr;
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, const_cast<void*>(static_cast<const void*>(p)), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<T*>(d);
}

// Grow a pinned host buffer to at least `need` bytes (geometrically after the first
// allocation; only a request larger than the staging size set at creation grows it) and
// look up its device address.
fe_status grow_pinned(unsigned char** p, unsigned char** pd, size_t* cap, size_t need) {
  if (need <= *cap && *p) return FE_OK;
  size_t n = *cap ? std::max(need, *cap * 2) : std::max<size_t>(need, 256);
  if (*p) cudaFreeHost(*p);
  *p = *pd = nullptr;
  *cap = 0;
  fe_status st = cuda_check(cudaMallocHost((void**)p, n), "server pinned staging");
  if (st) return st;
  *cap = n;
  return cuda_check(cudaHostGetDevicePointer((void**)pd, *p, 0), "server pinned staging address");
}

}  // namespace
}  // namespace fe

using namespace fe;

struct fe_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  int* status = nullptr;        // device status word of the batched kernel
  size_t budget = 0;
  size_t staging = 0;           // pinned bytes per slot and direction (pageable vectors)
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
  bool poll(Slot* S);
  fe_status launch(Slot* S);
};

fe_status fe_server::launch(Slot* S) {
  FE_TRACE("fe_server_launch");
  const int n = (int)S->reqs.size();
  // smallest mesh first: the tiles of a batch are handed out in this order
  std::stable_sort(S->reqs.begin(), S->reqs.end(), [](const Req* a, const Req* b) { return a->mesh->ne < b->mesh->ne; });
  S->voff.assign(n, 0);
  S->goff.assign(n, 0);
  S->fin.assign(n, 0);
  S->newly.clear();
  S->nfin = 0;
  size_t vin = 0, out = al256(sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    const Req* r = S->reqs[k];
    if (!r->v_dev) {
      S->voff[k] = vin;
      vin += al256(sizeof(double) * r->nvals);
    }
    if (!r->g_dev) {
      S->goff[k] = out;
      out += al256(sizeof(double) * r->nvals);
    }
  }
  fe_status st;
  if ((st = grow_pinned(&S->pin_in, &S->pin_in_dev, &S->pin_in_cap, vin))) return st;
  if ((st = grow_pinned(&S->pin_out, &S->pin_out_dev, &S->pin_out_cap, out))) return st;
  std::memset(S->flags, 0, sizeof(int) * n);
  unsigned char* base = arena + S->off;
  S->items.resize(n);
  size_t w = 0;
  for (int k = 0; k < n; ++k) {
    Req* r = S->reqs[k];
    if (!r->v_dev) std::memcpy(S->pin_in + S->voff[k], r->v, sizeof(double) * r->nvals);
    fe_batch_item& it = S->items[k];
    it.mesh = r->mesh;
    it.v = r->v_dev ? r->v_dev : reinterpret_cast<const double*>(S->pin_in_dev + S->voff[k]);
    it.g = r->g_dev ? r->g_dev : reinterpret_cast<double*>(S->pin_out_dev + S->goff[k]);
    it.J = reinterpret_cast<double*>(S->pin_out_dev) + k;
    it.done = S->flags_dev + k;
    it.work = base + w;
    w += r->bytes;
  }
  if ((st = batch_enqueue(S->stream, device, S->items.data(), n, S->stage_host, S->stage_dev, status, 0))) return st;
  return cuda_check(cudaEventRecord(S->done, S->stream), "server event");
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
      const size_t in = r->v_dev ? 0 : vb, outb = r->g_dev ? 0 : vb;
      // the staging buffers bound a batch of pageable requests too (a single larger request
      // grows them)
      if (n > 0 && (vin + in > staging || vout + outb > staging)) break;
      total += r->bytes;
      vin += in;
      vout += outb;
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
    if (!S->launch_status) launches += 1;
    cv.notify_all();
  }
  worker_done = true;
  cv.notify_all();
}

// Complete the requests of S whose flags are up (without the lock); true if any.  A batch
// whose launch failed, or whose kernel has ended (or failed) with flags still down after a
// last look at them, completes its remaining requests with an error.
bool fe_server::poll(Slot* S) {
  const int n = (int)S->reqs.size();
  auto scan = [&] {
    for (int k = 0; k < n; ++k) {
      if (S->fin[k]) continue;
      const int f = __atomic_load_n(S->flags + k, __ATOMIC_ACQUIRE);
      if (!f) continue;
      Req* r = S->reqs[k];
      double J;
      std::memcpy(&J, S->pin_out + sizeof(double) * k, sizeof(double));
      if (!r->g_dev) std::memcpy(r->g, S->pin_out + S->goff[k], sizeof(double) * r->nvals);
      *r->J = J;
      r->status = f != 1 ? FE_ETIMEOUT : (std::isinf(J) && J > 0) ? FE_EDOMAIN : FE_OK;
      if (f != 1) S->any_error = true;
      S->fin[k] = 1;
      S->nfin += 1;
      S->newly.push_back(r);
    }
  };
  fe_status fail = S->launch_status;
  if (!fail && S->nfin < n) {
    scan();
    if (S->nfin < n) {
      const cudaError_t q = cudaEventQuery(S->done);
      if (q == cudaSuccess) {
        scan();   // the kernel has ended: every flag it raised is visible now
        if (S->nfin < n) fail = set_error(FE_ECUDA, "server batch: the kernel ended without completing a request");
      } else if (q != cudaErrorNotReady) {
        fail = cuda_check(q, "server batch");
      }
    }
  }
  if (fail) S->any_error = true;
  if (fail)
    for (int k = 0; k < n; ++k)
      if (!S->fin[k]) {
        S->reqs[k]->status = fail;
        S->fin[k] = 1;
        S->nfin += 1;
        S->newly.push_back(S->reqs[k]);
      }
  return !S->newly.empty();
}

void fe_server::completer_loop() {
  cudaSetDevice(device);
  std::vector<Slot*> snap;
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    if (inflight.empty()) {
      if (worker_done) break;
      cv.wait(lk);
      continue;
    }
    snap.assign(inflight.begin(), inflight.end());
    lk.unlock();
    bool progress = false;
    for (Slot* S : snap) progress |= poll(S);
    const double td = now();
    lk.lock();
    if (progress) {
      for (Slot* S : snap) {
        for (Req* r : S->newly) {
          r->t_done = td;
          r->done = true;
        }
        completed += (int64_t)S->newly.size();
        S->newly.clear();
      }
      // a batch whose requests are all complete no longer touches its region, staging or
      // flags (later work on its stream runs after its kernel); after an error its kernel may
      // still run, so it is waited for first
      while (!inflight.empty() && inflight.front()->nfin == (int)inflight.front()->reqs.size()) {
        Slot* S = inflight.front();
        if (S->any_error) {
          lk.unlock();
          cudaEventSynchronize(S->done);
          lk.lock();
          S->any_error = false;
        }
        S->reqs.clear();
        inflight.pop_front();
        regions.pop_front();
        free_slots.push_back(S);
      }
      cv.notify_all();
    } else {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
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
  // pinned staging, flags and descriptors of every slot are allocated here, so that serving
  // allocates nothing (allocating pinned memory costs milliseconds)
  s->staging = std::min<size_t>(std::max<size_t>(s->budget / 16, 1 << 20), (size_t)256 << 20);
  for (int k = 0; k < kSlots && !st; ++k) {
    Slot& S = s->slot_store[k];
    S.stream = s->stream;
    if (max_batch > 1) {
      st = cuda_check(cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking), "server slot stream");
      S.own_stream = !st;
    }
    if (!st) st = cuda_check(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming), "server event");
    if (!st) st = grow_pinned(&S.pin_in, &S.pin_in_dev, &S.pin_in_cap, s->staging);
    if (!st) st = grow_pinned(&S.pin_out, &S.pin_out_dev, &S.pin_out_cap, s->staging);
    if (!st) st = cuda_check(cudaMallocHost((void**)&S.flags, sizeof(int) * max_batch), "server flags");
    if (!st) st = cuda_check(cudaHostGetDevicePointer((void**)&S.flags_dev, S.flags, 0), "server flags");
    if (!st) st = cuda_check(cudaMallocHost(&S.stage_host, batch_stage_bytes(max_batch)), "server descriptors");
    if (!st) st = cuda_check(cudaMalloc(&S.stage_dev, batch_stage_bytes(max_batch)), "server descriptors");
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
    if (S.own_stream) {
      cudaStreamSynchronize(S.stream);
      cudaStreamDestroy(S.stream);
    }
    if (S.pin_in) cudaFreeHost(S.pin_in);
    if (S.pin_out) cudaFreeHost(S.pin_out);
    if (S.flags) cudaFreeHost(S.flags);
    if (S.stage_host) cudaFreeHost(S.stage_host);
    if (S.stage_dev) cudaFree(S.stage_dev);
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
  FE_TRACE("fe_server_submit");
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
  r->v_dev = mapped(v_host);
  r->g_dev = mapped(g_host);
  r->bytes = batch_work_bytes(mesh);
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
  FE_TRACE("fe_server_wait");
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

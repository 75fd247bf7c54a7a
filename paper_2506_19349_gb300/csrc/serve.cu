// The serving runtime (host side of the continuous-batching path).
//
// Requests (graph, source) are submitted at any time. A pump thread admits
// them in arrival order while the result-buffer budget (a first-fit arena in
// one device allocation) and the request ring have room, publishes them to
// the serving kernel through mapped pinned memory, relaunches the kernel when
// work arrives after it went idle, and collects completions. A request joins
// the GPU as soon as a block group is free, while others are in flight; every
// result is the exact one (the same kernel body as eic_sssp).
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "graph.h"
#include "pool.h"
#include "serve.h"

namespace {

constexpr uint64_t kNone = ~0ull;
constexpr uint32_t kDefaultRing = 1024;
constexpr uint32_t kDefaultIdleUs = 2000;
constexpr uint32_t kMaxIdleUs = 100000;
constexpr uint32_t kPollUs = 20000;        // a leader's longest single wait, far below the group-barrier bound
constexpr uint32_t kServeSpinLog2 = 26;    // group-barrier bound while a leader idles
constexpr uint32_t kServeStepCap = 1u << 17;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation, in 256-byte units; freed
// ranges merge with free neighbours.
class Arena {
 public:
  int init(uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    if (cudaMalloc((void**)&base_, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      base_ = nullptr;
      return EIC_ENOMEM;
    }
    cap_ = bytes;
    free_.clear();
    free_[0] = bytes;
    used_ = 0;
    return EIC_OK;
  }
  void destroy() {
    cudaFree(base_);
    base_ = nullptr;
    free_.clear();
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = (bytes + 255) & ~255ull;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  unsigned char* base() const { return base_; }
  uint64_t capacity() const { return cap_; }
  uint64_t used() const { return used_; }

 private:
  unsigned char* base_ = nullptr;
  uint64_t cap_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

enum class State { Queued, Admitted, Done };

struct Request {
  uint32_t graph = 0, source = 0;
  State state = State::Queued;
  int status = EIC_OK;
  uint64_t off = 0, bytes = 0;  // result buffer in the arena
  uint64_t seq = kNone;         // admission number (ring sequence)
  double t_submit = 0, t_done = 0;
};

}  // namespace

struct eic_server {
  int device = 0;
  std::vector<const eic_graph*> graphs;
  std::vector<BatchQuery> hq;  // the resident graphs' table (host copy of d_graphs)
  BatchQuery* d_graphs = nullptr;
  eic_params p{};
  uint32_t groups = 0, nb = 0, block = 0, cap = 0;  // groups (slots) at most, blocks per group at that count
  uint32_t gmax = 0;                                 // co-resident blocks of the serving kernel
  uint32_t launch_groups = 0;                        // groups of the running (or last) launch
  uint64_t idle_ns = 0;
  SlotPool pool;
  Arena arena;
  ServeRing* ring = nullptr;   // host view
  ServeRing* dring = nullptr;  // device view
  unsigned long long* d_claim = nullptr;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t kdone = nullptr;
  bool running = false;
  int launch_error = EIC_OK;
  uint64_t launches = 0;

  std::mutex mu;
  std::condition_variable cv;
  std::thread pump;
  bool quit = false;
  std::deque<uint64_t> queue;                 // tickets waiting for admission
  std::unordered_map<uint64_t, Request> reqs;  // by ticket
  std::vector<uint64_t> entry_ticket;          // ring entry -> ticket, or kNone
  std::vector<uint64_t> admitted;              // tickets on the GPU
  uint64_t next_ticket = 0, seq = 0, completed = 0, max_inflight = 0, submitted = 0;
  std::vector<double> lat_ms;                  // completed requests' latencies

  // The launch's group count for a backlog of waiting requests: a few wide
  // groups while the backlog is short (a lone request runs on a quarter of
  // the GPU, not on one of many small groups), more and narrower groups as it
  // grows, up to every slot the server has.
  uint32_t launch_shape(uint64_t backlog) const {
    for (uint32_t g : {4u, 8u, 16u})
      if (g < groups && backlog <= g) return g;
    return groups;
  }

  ServeArgs args(uint32_t g) const {
    ServeArgs a;
    a.ring = dring;
    a.req = serve_requests(dring);
    a.done = (ServeDone*)((char*)dring + ((char*)serve_done(ring) - (char*)ring));
    a.claim = d_claim;
    a.graphs = d_graphs;
    a.slot = pool.d_slots;
    a.num_graphs = (uint32_t)graphs.size();
    a.cap = cap;
    a.nb = g == groups ? nb : gmax / g;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.st_num = p.st_num;
    a.gap_shift = p.gap_shift;
    a.heavy_min = p.heavy_min;
    a.flags = p.flags;
    a.step_cap = kServeStepCap;
    const uint32_t sl = p.max_spin_log2 > kServeSpinLog2 ? p.max_spin_log2 : kServeSpinLog2;
    a.max_spin = 1ull << sl;
    a.groups = g;
    a.idle_ns = idle_ns;
    a.poll_ns = kPollUs * 1000ull;
    a.widen_at = g < groups ? 2ull * g : 0ull;
    return a;
  }

  // One pass of the pump (mu held): completions, admissions, kernel liveness.
  bool step() {
    bool progress = false;
    ServeDone* done = serve_done(ring);
    for (size_t i = 0; i < admitted.size();) {
      Request& r = reqs[admitted[i]];
      const uint32_t e = (uint32_t)(r.seq & (cap - 1));
      if (__atomic_load_n(&done[e].ticket_plus1, __ATOMIC_ACQUIRE) == r.seq + 1) {
        r.status = *(volatile int*)&done[e].status;
        r.state = State::Done;
        r.t_done = now_s();
        lat_ms.push_back((r.t_done - r.t_submit) * 1e3);
        entry_ticket[e] = kNone;
        ++completed;
        admitted[i] = admitted.back();
        admitted.pop_back();
        progress = true;
      } else {
        ++i;
      }
    }
    ServeRequest* req = serve_requests(ring);
    while (!queue.empty()) {
      const uint64_t t = queue.front();
      Request& r = reqs[t];
      const uint32_t e = (uint32_t)(seq & (cap - 1));
      if (entry_ticket[e] != kNone) break;         // the ring is full
      if (!arena.alloc(r.bytes, &r.off)) break;     // wait for result memory (arrival order)
      req[e].ticket = seq;
      req[e].out = (uint32_t*)(arena.base() + r.off);
      req[e].graph = r.graph;
      req[e].source = r.source;
      r.seq = seq;
      r.state = State::Admitted;
      entry_ticket[e] = t;
      admitted.push_back(t);
      ++seq;
      __atomic_store_n(&ring->head, (unsigned long long)seq, __ATOMIC_RELEASE);
      queue.pop_front();
      max_inflight = std::max<uint64_t>(max_inflight, admitted.size());
      progress = true;
    }
    if (running) {
      const cudaError_t q = cudaEventQuery(kdone);
      if (q == cudaSuccess) {
        running = false;
      } else if (q != cudaErrorNotReady) {
        (void)cudaGetLastError();
        running = false;
        launch_error = EIC_ECUDA;
      }
    }
    if (!running && !admitted.empty() && launch_error == EIC_OK) {
      launch_groups = launch_shape(admitted.size());
      int rc = eic_serve_launch(args(launch_groups), launch_groups, block, kstream);
      if (rc == EIC_OK && cudaEventRecord(kdone, kstream) != cudaSuccess) rc = EIC_ECUDA;
      if (rc != EIC_OK) {
        (void)cudaGetLastError();
        launch_error = rc;
      } else {
        running = true;
        ++launches;
      }
      progress = true;
    }
    if (launch_error != EIC_OK) {  // no kernel can run: fail what waits
      for (uint64_t t : admitted) {
        Request& r = reqs[t];
        r.status = launch_error;
        r.state = State::Done;
        r.t_done = now_s();
        entry_ticket[(uint32_t)(r.seq & (cap - 1))] = kNone;
        ++completed;
      }
      admitted.clear();
    }
    return progress;
  }

  void pump_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!quit) {
      const bool progress = step();
      if (progress) cv.notify_all();
      if (!progress) cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
};

namespace {

void server_free(eic_server* s) {
  if (s->pump.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->quit = true;
    }
    s->cv.notify_all();
    s->pump.join();
  }
  if (s->ring) __atomic_store_n(&s->ring->stop, 1u, __ATOMIC_RELEASE);
  if (s->kstream) cudaStreamSynchronize(s->kstream);  // groups leave at the stop flag
  if (s->kdone) cudaEventDestroy(s->kdone);
  if (s->kstream) cudaStreamDestroy(s->kstream);
  if (s->cstream) cudaStreamDestroy(s->cstream);
  s->pool.release();
  s->arena.destroy();
  cudaFree(s->d_graphs);
  cudaFree(s->d_claim);
  if (s->ring) cudaFreeHost(s->ring);
  (void)cudaGetLastError();
  delete s;
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t k = (size_t)(q * (double)(v.size() - 1) + 0.5);
  return v[std::min(k, v.size() - 1)];
}

}  // namespace

extern "C" {

int eic_server_create(const eic_graph* const* graphs, uint32_t num_graphs, const eic_params* params,
                      const eic_server_config* config, eic_server** out) {
  if (!out) return EIC_EINVAL;
  *out = nullptr;
  if (!graphs || num_graphs == 0) return EIC_EINVAL;
  eic_server_config cfg{};
  if (config) cfg = *config;
  if (cfg.ring_entries == 0) cfg.ring_entries = kDefaultRing;
  if ((cfg.ring_entries & (cfg.ring_entries - 1)) != 0 || cfg.ring_entries > (1u << 20)) return EIC_EINVAL;
  if (cfg.idle_us == 0) cfg.idle_us = kDefaultIdleUs;
  if (cfg.idle_us > kMaxIdleUs) return EIC_EINVAL;
  int dev = -1;
  for (uint32_t i = 0; i < num_graphs; ++i) {
    if (!graphs[i]) return EIC_EINVAL;
    if (dev < 0) dev = graphs[i]->device;
    if (graphs[i]->device != dev) return EIC_EINVAL;
  }
  eic_params pr;
  eic_params_default(&pr);
  if (params) pr = *params;
  if (!(pr.beta > 0.0 && pr.beta < 1.0) || pr.st_num == 0 || pr.st_num > 65536 || pr.gap_shift > 16)
    return EIC_EINVAL;
  if (pr.block_threads != 0 && (pr.block_threads % 32 != 0 || pr.block_threads < 128 || pr.block_threads > 512))
    return EIC_EINVAL;
  if (pr.heavy_min == 0) pr.heavy_min = 32;
  if (pr.heavy_min < kHeavyMinFloor || pr.heavy_min > 4096) return EIC_EINVAL;
  if (pr.max_spin_log2 == 0) pr.max_spin_log2 = 22;
  if (pr.max_spin_log2 > 40) return EIC_EINVAL;

  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_ECUDA;
  }
  eic_server* s = new eic_server();
  s->device = dev;
  s->p = pr;
  s->cap = cfg.ring_entries;
  s->idle_ns = (uint64_t)cfg.idle_us * 1000ull;
  s->block = pr.block_threads ? pr.block_threads : 512;
  int rc = EIC_OK;
  std::vector<BatchQuery> hq;
  SlotCaps caps;
  uint64_t max_n = 0;
  for (uint32_t i = 0; i < num_graphs; ++i) {
    const DevGraph& G = graphs[i]->dg;
    s->graphs.push_back(graphs[i]);
    BatchQuery q{};
    q.G = G;
    uint32_t shift = 0;
    const uint32_t bits = ring_layout(G.maxw, &shift);
    q.ring_mask = (1u << bits) - 1u;
    q.ring_shift = shift;
    q.task_cap = (uint32_t)(G.two_m / kHeavyMinFloor + 2);
    q.gap_shift = pr.gap_shift;
    q.heavy_min = pr.heavy_min;
    q.fuse = fuse_ok(G, pr.heavy_min, pr.flags) ? 1u : 0u;
    hq.push_back(q);
    caps.ni = std::max<uint64_t>(caps.ni, G.ni);
    caps.two_m = std::max<uint64_t>(caps.two_m, G.two_m);
    caps.D = std::max(caps.D, G.D);
    caps.ring_bits = std::max(caps.ring_bits, bits);
    max_n = std::max<uint64_t>(max_n, G.n);
  }
  uint32_t gmax = 0;
  if ((rc = eic_serve_grid((int)s->block, &gmax))) goto fail;
  {
    uint32_t groups = cfg.groups ? cfg.groups : std::max(1u, gmax / 8);
    groups = std::min(groups, gmax);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
      const uint64_t per = slot_layout(caps).bytes;
      const uint64_t out_b = cfg.output_bytes ? cfg.output_bytes : 64ull * max_n * 4;
      const double avail = (double)fr * kBatchMemFrac - (double)out_b;
      const uint64_t fit = avail > 0 ? (uint64_t)(avail / (double)per) : 0;
      groups = (uint32_t)std::min<uint64_t>(groups, fit);
    }
    (void)cudaGetLastError();
    if (groups == 0) {
      rc = EIC_ENOMEM;
      goto fail;
    }
    s->groups = groups;
    s->nb = gmax / groups;
    s->gmax = gmax;
  }
  if ((rc = s->pool.ensure(caps, s->groups))) goto fail;
  if ((rc = s->arena.init(cfg.output_bytes ? cfg.output_bytes : 64ull * max_n * 4))) goto fail;
  {
    const uint64_t rbytes = sizeof(ServeRing) + (uint64_t)s->cap * (sizeof(ServeRequest) + sizeof(ServeDone));
    if (cudaHostAlloc((void**)&s->ring, rbytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&s->dring, s->ring, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = EIC_ENOMEM;
      goto fail;
    }
    memset(s->ring, 0, rbytes);
    s->ring->cap = s->cap;
  }
  if (cudaMalloc((void**)&s->d_graphs, hq.size() * sizeof(BatchQuery)) != cudaSuccess ||
      cudaMalloc((void**)&s->d_claim, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemcpy(s->d_graphs, hq.data(), hq.size() * sizeof(BatchQuery), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->d_claim, 0, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = EIC_ENOMEM;
    goto fail;
  }
  s->hq = hq;
  s->entry_ticket.assign(s->cap, kNone);
  s->pump = std::thread([s] { s->pump_loop(); });
  cudaSetDevice(prev);
  *out = s;
  return EIC_OK;
fail:
  server_free(s);
  cudaSetDevice(prev);
  return rc;
}

int eic_server_submit(eic_server* s, uint32_t graph, uint32_t source, uint64_t* ticket) {
  if (!s || !ticket || graph >= s->graphs.size() || source >= s->graphs[graph]->dg.n) return EIC_EINVAL;
  const uint64_t bytes = (uint64_t)s->graphs[graph]->dg.n * 4;
  if (((bytes + 255) & ~255ull) > s->arena.capacity()) return EIC_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    Request r;
    r.graph = graph;
    r.source = source;
    r.bytes = bytes;
    r.t_submit = now_s();
    s->reqs.emplace(t, r);
    s->queue.push_back(t);
    ++s->submitted;
    *ticket = t;
  }
  s->cv.notify_all();
  return EIC_OK;
}

int eic_server_poll(eic_server* s, uint64_t ticket, int* status) {
  if (!s) return EIC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return EIC_EINVAL;
  if (it->second.state != State::Done) return EIC_EBUSY;
  if (status) *status = it->second.status;
  return EIC_OK;
}

int eic_server_wait(eic_server* s, uint64_t ticket, uint32_t timeout_ms, int* status) {
  if (!s) return EIC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return EIC_EINVAL;
  const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    auto j = s->reqs.find(ticket);
    return j == s->reqs.end() || j->second.state == State::Done;
  });
  it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return EIC_EINVAL;
  if (!ok) return EIC_ETIMEOUT;
  if (status) *status = it->second.status;
  return EIC_OK;
}

int eic_server_result(eic_server* s, uint64_t ticket, uint32_t* host_dist, const uint32_t** device_dist,
                      double* latency_ms) {
  if (!s) return EIC_EINVAL;
  const uint32_t* dptr = nullptr;
  uint64_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EIC_EINVAL;
    const Request& r = it->second;
    if (r.state != State::Done) return EIC_EBUSY;
    if (latency_ms) *latency_ms = (r.t_done - r.t_submit) * 1e3;
    if (r.status != EIC_OK) return r.status;
    dptr = (const uint32_t*)(s->arena.base() + r.off);
    bytes = r.bytes;
  }
  if (device_dist) *device_dist = dptr;
  if (host_dist) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    const bool ok = cudaMemcpyAsync(host_dist, dptr, bytes, cudaMemcpyDeviceToHost, s->cstream) == cudaSuccess &&
                    cudaStreamSynchronize(s->cstream) == cudaSuccess;
    cudaSetDevice(prev);
    if (!ok) {
      (void)cudaGetLastError();
      return EIC_ECUDA;
    }
  }
  return EIC_OK;
}

int eic_server_release(eic_server* s, uint64_t ticket) {
  if (!s) return EIC_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EIC_EINVAL;
    if (it->second.state != State::Done) return EIC_EBUSY;
    if (it->second.seq != kNone) s->arena.release(it->second.off, it->second.bytes);
    s->reqs.erase(it);
  }
  s->cv.notify_all();  // memory freed: the pump may admit
  return EIC_OK;
}

int eic_server_stats(eic_server* s, eic_server_report* out) {
  if (!s || !out) return EIC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->admitted = s->seq;
  out->completed = s->completed;
  out->queued = s->queue.size();
  out->in_flight = s->admitted.size();
  out->max_in_flight = s->max_inflight;
  out->kernel_launches = s->launches;
  out->output_bytes_used = s->arena.used();
  out->output_bytes = s->arena.capacity();
  out->scratch_bytes = (uint64_t)s->pool.count * s->pool.slot_bytes;
  out->groups = s->groups;
  out->blocks_per_group = s->nb;
  out->latency_p50_ms = percentile(s->lat_ms, 0.50);
  out->latency_p99_ms = percentile(s->lat_ms, 0.99);
  double sum = 0;
  for (double v : s->lat_ms) sum += v;
  out->latency_mean_ms = s->lat_ms.empty() ? 0.0 : sum / (double)s->lat_ms.size();
  out->latency_count = s->lat_ms.size();
  return EIC_OK;
}

int eic_server_reset_stats(eic_server* s) {
  if (!s) return EIC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->max_inflight = s->admitted.size();
  return EIC_OK;
}

int eic_server_tune(eic_server* s, const uint32_t* sample_sources, uint32_t* gap_shifts) {
  if (!s || !sample_sources) return EIC_EINVAL;
  for (size_t k = 0; k < s->graphs.size(); ++k)
    if (sample_sources[k] >= s->graphs[k]->dg.n) return EIC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);  // submissions wait while the server tunes
  if (!s->queue.empty() || !s->admitted.empty()) {
    cudaSetDevice(prev);
    return EIC_EBUSY;
  }
  // let a resident serving kernel leave before timing other launches
  if (s->running && cudaStreamSynchronize(s->kstream) != cudaSuccess) (void)cudaGetLastError();
  s->running = false;
  int rc = EIC_OK;
  for (size_t k = 0; k < s->graphs.size() && rc == EIC_OK; ++k) {
    uint32_t best = s->p.gap_shift;
    double ms = 0;
    rc = eic_tune_step_width(s->graphs[k], sample_sources[k], s->groups, s->nb, s->p, s->p.gap_shift, s->cstream,
                             &best, &ms);
    if (rc == EIC_OK) s->hq[k].gap_shift = best;
    if (gap_shifts) gap_shifts[k] = s->hq[k].gap_shift;
  }
  if (rc == EIC_OK && cudaMemcpy(s->d_graphs, s->hq.data(), s->hq.size() * sizeof(BatchQuery),
                                 cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = EIC_ECUDA;
  }
  cudaSetDevice(prev);
  return rc;
}

int eic_server_destroy(eic_server* s) {
  if (!s) return EIC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  server_free(s);
  cudaSetDevice(prev);
  return EIC_OK;
}

}  // extern "C"

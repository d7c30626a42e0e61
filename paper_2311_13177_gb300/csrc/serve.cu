// Request server: continuous batching of independent reconstructions on one
// GPU (the C ABI's prop_serve_* calls).
//
// Each request is a full reconstruction problem (geometry, Adam and TV
// settings, blade data).  Admission workers admit queued requests in FIFO
// order while a slot is free and the request's device footprint fits the
// server's HBM budget, build its plan inside one pre-allocated device arena
// (so retiring a request never synchronises the device) and upload its data.
// The scheduler thread groups the running requests by kernel class (the
// same transform length 2N, bin stride and kernel width: one set of kernel
// instances) and advances every class with batched iterations: one launch
// per stage (column FFTs, interpolation, spread, fused row update) serves
// every request of the class in the batch, each on the CTAs its share of
// the work earns, at most two batched iterations in flight per class, the
// classes on their own streams so that they overlap too.  Requests of
// different blade counts, frame counts and data share a launch; requests
// join their class's next batched iteration as soon as they are admitted and
// leave it when they finish.  A finished request has its volume copied back
// on its own stream, its arena memory returned, and the next waiting request
// is admitted at once.  Every request's arithmetic runs in its own buffers
// with the same kernels' per-element work as a lone solve, so its result is
// bitwise the same alone or in any mix.  Latency is measured on the host from
// submission to the completion of the final copy.
#include "prop_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

namespace prop {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device arena (host-side bookkeeping only).
class Arena : public DeviceAllocator {
 public:
  static constexpr size_t kAlign = 256;
  cudaError_t init(size_t bytes) {
    size_ = (bytes + kAlign - 1) & ~(kAlign - 1);
    cudaError_t e = cudaMalloc(&base_, size_);
    if (e != cudaSuccess) {
      base_ = nullptr;
      return e;
    }
    free_[0] = size_;
    return cudaSuccess;
  }
  ~Arena() override {
    if (base_) cudaFree(base_);
  }
  cudaError_t allocate(void** ptr, size_t bytes) override {
    bytes = std::max<size_t>((bytes + kAlign - 1) & ~(kAlign - 1), kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        in_use_ += bytes;
        peak_ = std::max(peak_, in_use_);
        *ptr = static_cast<char*>(base_) + off;
        return cudaSuccess;
      }
    }
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  void release(void* ptr) override {
    if (!ptr) return;
    const size_t off = static_cast<size_t>(static_cast<char*>(ptr) - static_cast<char*>(base_));
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    in_use_ -= len;
    used_.erase(u);
    auto nx = free_.lower_bound(start);
    if (nx != free_.end() && nx->first == start + len) {  // merge with the next free range
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge with the previous free range
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        start = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = len;
  }
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }

 private:
  void* base_ = nullptr;
  size_t size_ = 0, in_use_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;  // offset -> length
};

// Serialises a shared allocator between threads.
class LockedAlloc : public DeviceAllocator {
 public:
  LockedAlloc(DeviceAllocator* a, std::mutex* m) : a_(a), m_(m) {}
  cudaError_t allocate(void** ptr, size_t bytes) override {
    std::lock_guard<std::mutex> lk(*m_);
    return a_->allocate(ptr, bytes);
  }
  void release(void* ptr) override {
    std::lock_guard<std::mutex> lk(*m_);
    a_->release(ptr);
  }

 private:
  DeviceAllocator* a_;
  std::mutex* m_;
};

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Request {
  prop_ticket id = 0;
  prop_plan_desc desc{};
  std::vector<double> delta, theta;
  std::vector<int> frames;
  prop_recon_params params{};
  std::vector<float2> y_host, v_host;  // inputs (v empty: start from zero)
  int state = kPending;
  bool cancel = false;
  prop_status status = PROP_OK;
  std::string error;
  size_t footprint = 0;
  // device state (scheduler thread only)
  Plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  float2* y_dev = nullptr;
  float2* v_dev = nullptr;
  float2* cur = nullptr;
  float2* nxt = nullptr;
  int k = 0;
  std::deque<cudaEvent_t> inflight;   // unused with batched iterations (kept empty)
  cudaEvent_t last_ev = nullptr;      // completes with the last batched iteration this request took part in
  cudaEvent_t done_ev = nullptr;
  bool copying = false;
  float2* pinned = nullptr;
  size_t pinned_bytes = 0;
  double* loss_pinned = nullptr;
  // results
  std::unique_ptr<LockedAlloc> alloc;
  std::vector<float2> result;
  double final_loss = 0.0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace
}  // namespace prop

struct prop_server_s {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  prop::Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<prop_ticket> pending;
  std::map<prop_ticket, std::unique_ptr<prop::Request>> reqs;
  std::vector<prop::Request*> active;
  // kernel classes of the running requests: (2N, bin stride, width) -> stream
  // and the events of its batched iterations in flight
  struct Klass {
    cudaStream_t hi = nullptr, lo = nullptr;  // high- and low-priority streams
    cudaStream_t last = nullptr;              // the stream of the class's latest batched iteration
    std::deque<cudaEvent_t> inflight;
  };
  std::map<std::tuple<int, int, int>, Klass> klasses;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<float2*, size_t>> pinned_pool;
  size_t reserved = 0;  // footprints of admitted requests
  int admitting = 0;     // requests whose plans are being built
  uint64_t next_id = 1;
  bool stop = false;
  std::mutex arena_mu;   // the arena is shared by the admission workers and the scheduler
  std::condition_variable cv_admit;
  std::thread thr;
  std::vector<std::thread> workers;
  long long completed = 0, failed = 0, cancelled = 0;
};

namespace prop {
namespace {

cudaEvent_t take_ev(prop_server_s* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

float2* take_pinned(prop_server_s* s, size_t bytes, size_t* got) {
  size_t best = (size_t)-1, bi = 0;
  for (size_t i = 0; i < s->pinned_pool.size(); ++i)
    if (s->pinned_pool[i].second >= bytes && s->pinned_pool[i].second < best) {
      best = s->pinned_pool[i].second;
      bi = i;
    }
  if (best != (size_t)-1) {
    float2* p = s->pinned_pool[bi].first;
    *got = s->pinned_pool[bi].second;
    s->pinned_pool.erase(s->pinned_pool.begin() + bi);
    return p;
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, bytes + 64, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *got = bytes + 64;
  return static_cast<float2*>(p);
}

// Frees a request's device state (scheduler thread, stream idle).
void release(prop_server_s* s, Request* r) {
  for (cudaEvent_t e : r->inflight) s->ev_pool.push_back(e);
  r->inflight.clear();
  if (r->done_ev) s->ev_pool.push_back(r->done_ev);
  r->done_ev = nullptr;
  r->last_ev = nullptr;  // owned by its class's in-flight list
  if (r->alloc) {
    r->alloc->release(r->y_dev);
    r->alloc->release(r->v_dev);
  }
  r->y_dev = r->v_dev = nullptr;
  if (r->plan) {
    plan_free(r->plan);
    r->plan = nullptr;
  }
  if (r->stream) cudaStreamDestroy(r->stream);
  r->stream = nullptr;
  if (r->pinned) s->pinned_pool.emplace_back(r->pinned, r->pinned_bytes);
  r->pinned = nullptr;
  s->reserved -= r->footprint;
  r->footprint = 0;
}

// Builds the request's plan and buffers in the arena and uploads its data.
prop_status admit(prop_server_s* s, Request* r) {
  prop_plan_desc d = r->desc;
  d.delta = r->delta.data();
  d.theta = r->theta.data();
  d.blade_frame = r->frames.empty() ? nullptr : r->frames.data();
  d.device = s->device;
  r->alloc.reset(new LockedAlloc(&s->arena, &s->arena_mu));
  prop_status st = plan_build(&d, &r->plan, r->alloc.get());
  if (st != PROP_OK) return st;
  Plan& p = *r->plan;
  if ((st = plan_ensure_recon(&p, std::max(r->params.iters, 1))) != PROP_OK) return st;
  const size_t vb = p.vol_elems() * sizeof(float2), yb = (size_t)p.M * sizeof(float2);
  if (r->alloc->allocate((void**)&r->y_dev, yb) != cudaSuccess ||
      r->alloc->allocate((void**)&r->v_dev, vb) != cudaSuccess)
    return fail(PROP_ERR_OOM, "serve: arena exhausted (fragmentation)");
  PROP_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->pinned = take_pinned(s, vb + sizeof(double), &r->pinned_bytes);
  }
  if (!r->pinned) return fail(PROP_ERR_OOM, "serve: pinned host allocation failed");
  r->loss_pinned = reinterpret_cast<double*>(reinterpret_cast<char*>(r->pinned) + vb);
  PROP_CUDA(cudaMemcpyAsync(r->y_dev, r->y_host.data(), yb, cudaMemcpyHostToDevice, r->stream));
  if (r->v_host.empty())
    PROP_CUDA(cudaMemsetAsync(r->v_dev, 0, vb, r->stream));
  else
    PROP_CUDA(cudaMemcpyAsync(r->v_dev, r->v_host.data(), vb, cudaMemcpyHostToDevice, r->stream));
  PROP_CUDA(cudaStreamSynchronize(r->stream));  // host copies may be released now
  r->cur = r->v_dev;
  r->nxt = p.vol2;
  r->k = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->done_ev = take_ev(s);
  }
  return PROP_OK;
}

void finish(prop_server_s* s, Request* r, int state, prop_status st, const std::string& msg) {
  r->state = state;
  r->status = st;
  r->error = msg;
  r->t_done = now_s();
  r->y_host.clear();
  r->y_host.shrink_to_fit();
  r->v_host.clear();
  r->v_host.shrink_to_fit();
  if (state == kDone) ++s->completed;
  if (state == kFailed) ++s->failed;
  if (state == kCancelled) ++s->cancelled;
}

// Footprint of a request in the arena (upper bound).
size_t footprint(Request* r) {
  prop_plan_desc d = r->desc;
  d.delta = r->delta.data();
  d.theta = r->theta.data();
  d.blade_frame = r->frames.empty() ? nullptr : r->frames.data();
  const size_t vb = (size_t)d.nframes * d.n * d.n * d.nf * sizeof(float2);
  const size_t yb = (size_t)d.nblades * d.lines * d.readout * sizeof(float2);
  return plan_estimate_bytes(&d, r->params.iters) + vb + yb + 4096;
}

// Admission worker: FIFO while a slot is free and the footprint fits; builds
// the plan (host tables + arena memory + uploads) off the scheduler thread.
void admission(prop_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->pending.empty()) break;
    if (s->pending.empty()) {
      s->cv_admit.wait(lk);
      continue;
    }
    Request* r = s->reqs[s->pending.front()].get();
    if (r->cancel || s->stop) {
      s->pending.pop_front();
      finish(s, r, kCancelled, PROP_ERR_CANCELLED, "cancelled before admission");
      s->cv_done.notify_all();
      continue;
    }
    const size_t need = footprint(r);
    if (need > s->budget) {
      s->pending.pop_front();
      finish(s, r, kFailed, PROP_ERR_OOM,
             "request needs " + std::to_string(need) + " device bytes, server budget is " + std::to_string(s->budget));
      s->cv_done.notify_all();
      continue;
    }
    if ((int)s->active.size() + s->admitting >= s->max_slots || s->reserved + need > s->budget) {
      s->cv_admit.wait(lk);  // a retirement frees a slot or memory (FIFO: no overtaking)
      continue;
    }
    s->pending.pop_front();
    s->reserved += need;
    r->footprint = need;
    r->t_admit = now_s();
    ++s->admitting;
    lk.unlock();
    const prop_status st = admit(s, r);
    const std::string msg = st == PROP_OK ? "" : prop_last_error();
    lk.lock();
    --s->admitting;
    if (st != PROP_OK) {
      release(s, r);
      finish(s, r, kFailed, st, "admission failed: " + msg);
      s->cv_done.notify_all();
      s->cv_admit.notify_all();
      continue;
    }
    r->state = kRunning;
    s->active.push_back(r);
    s->cv_work.notify_all();
  }
}

std::tuple<int, int, int> klass_of(const Plan& p) { return std::make_tuple(p.n, p.cs, p.W); }

void scheduler(prop_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->active.empty() && s->pending.empty() && s->admitting == 0) break;
    bool progressed = false;
    // completed batched iterations of every class
    for (auto& kv : s->klasses) {
      auto& q = kv.second.inflight;
      while (!q.empty() && cudaEventQuery(q.front()) == cudaSuccess) {
        for (Request* r : s->active)
          if (r->last_ev == q.front()) r->last_ev = nullptr;  // its iterations are all done
        s->ev_pool.push_back(q.front());
        q.pop_front();
      }
    }
    // retire, cancel, start result copies
    std::vector<Request*> still;
    for (Request* r : s->active) {
      const bool idle = !r->last_ev || cudaEventQuery(r->last_ev) == cudaSuccess;
      if (r->cancel) {
        if (!idle) {
          still.push_back(r);
          continue;
        }
        cudaStreamSynchronize(r->stream);
        release(s, r);
        finish(s, r, kCancelled, PROP_ERR_CANCELLED, "cancelled");
        s->cv_done.notify_all();
        progressed = true;
        continue;
      }
      if (r->copying) {
        const cudaError_t q = cudaEventQuery(r->done_ev);
        if (q == cudaErrorNotReady) {
          still.push_back(r);
          continue;
        }
        const size_t vb = r->plan->vol_elems() * sizeof(float2);
        if (q == cudaSuccess) {
          r->result.resize(r->plan->vol_elems());
          std::memcpy(r->result.data(), r->pinned, vb);
          r->final_loss = *r->loss_pinned;
        }
        release(s, r);
        if (q == cudaSuccess)
          finish(s, r, kDone, PROP_OK, "");
        else
          finish(s, r, kFailed, PROP_ERR_CUDA, std::string("request failed: ") + cudaGetErrorString(q));
        s->cv_done.notify_all();
        progressed = true;
        continue;
      }
      if (r->k >= r->params.iters) {
        // the result copy runs on the request's own stream after its last iteration
        if (r->last_ev) cudaStreamWaitEvent(r->stream, r->last_ev, 0);
        const size_t vb = r->plan->vol_elems() * sizeof(float2);
        cudaMemcpyAsync(r->pinned, r->cur, vb, cudaMemcpyDeviceToHost, r->stream);
        *r->loss_pinned = 0.0;
        if (r->params.iters > 0)
          cudaMemcpyAsync(r->loss_pinned, r->plan->loss_dev + (r->params.iters - 1), sizeof(double),
                          cudaMemcpyDeviceToHost, r->stream);
        cudaEventRecord(r->done_ev, r->stream);
        r->copying = true;
        progressed = true;
      }
      still.push_back(r);
    }
    if (still.size() != s->active.size()) s->cv_admit.notify_all();
    s->active.swap(still);
    // one batched iteration for every class with work and fewer than two in
    // flight; the class holding the oldest running request issues on a
    // high-priority stream, so that it keeps the GPU as a FIFO queue would
    // give it, and the others fill in behind
    std::map<std::tuple<int, int, int>, std::vector<Request*>> ready;
    const Request* oldest = nullptr;
    for (Request* r : s->active)
      if (!r->cancel && !r->copying && r->k < r->params.iters) {
        ready[klass_of(*r->plan)].push_back(r);
        if (!oldest || r->t_submit < oldest->t_submit) oldest = r;
      }
    for (auto& kv : ready) {
      prop_server_s::Klass& K = s->klasses[kv.first];
      if (K.inflight.size() >= 2) continue;
      if (!K.hi) {
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if (cudaStreamCreateWithPriority(&K.hi, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
            cudaStreamCreateWithPriority(&K.lo, cudaStreamNonBlocking, lo_prio) != cudaSuccess) {
          cudaGetLastError();
          if (K.hi) cudaStreamDestroy(K.hi);
          K.hi = K.lo = nullptr;
          continue;
        }
      }
      std::vector<Request*>& rs = kv.second;
      const bool first = std::find(rs.begin(), rs.end(), oldest) != rs.end();
      cudaStream_t stream = first ? K.hi : K.lo;
      if (K.last && K.last != stream && !K.inflight.empty())
        cudaStreamWaitEvent(stream, K.inflight.back(), 0);  // the class's iterations stay in order
      K.last = stream;
      // the requests furthest behind first (admission order among equals)
      std::stable_sort(rs.begin(), rs.end(), [](const Request* a, const Request* b) { return a->k < b->k; });
      const int n = std::min<int>((int)rs.size(), kMaxBatch);
      BatchMember mb[kMaxBatch];
      for (int i = 0; i < n; ++i) {
        Request* r = rs[i];
        Plan& p = *r->plan;
        const int k = r->k + 1;
        mb[i] = BatchMember{&p, r->y_dev, &r->params, k, r->cur, r->nxt, p.loss_dev + (k - 1), k > 1,
                            k < r->params.iters};
        // a request's first batched iteration follows its uploads
        if (r->k == 0) {
          cudaEvent_t up = take_ev(s);
          cudaEventRecord(up, r->stream);
          cudaStreamWaitEvent(stream, up, 0);
          s->ev_pool.push_back(up);
        }
      }
      const prop_status st = batch_step(mb, n, stream);
      if (st != PROP_OK) {
        const std::string msg = prop_last_error();
        cudaStreamSynchronize(stream);
        for (int i = 0; i < n; ++i) {
          Request* r = rs[i];
          release(s, r);
          finish(s, r, kFailed, st, msg);
          r->state = kFailed;
        }
        std::vector<Request*> keep;
        for (Request* r : s->active)
          if (r->state != kFailed) keep.push_back(r);
        s->active.swap(keep);
        s->cv_done.notify_all();
        s->cv_admit.notify_all();
        progressed = true;
        continue;
      }
      cudaEvent_t e = take_ev(s);
      cudaEventRecord(e, stream);
      K.inflight.push_back(e);
      for (int i = 0; i < n; ++i) {
        Request* r = rs[i];
        std::swap(r->cur, r->nxt);
        r->k += 1;
        r->last_ev = e;
      }
      progressed = true;
    }
    if (!progressed) {
      // Nothing to issue: wait briefly for the GPU or for new submissions.
      s->cv_work.wait_for(lk, std::chrono::microseconds(s->active.empty() ? 2000 : 20));
    }
  }
  for (auto& kv : s->klasses) {
    for (cudaStream_t st : {kv.second.hi, kv.second.lo})
      if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
      }
    for (cudaEvent_t e : kv.second.inflight) s->ev_pool.push_back(e);
    kv.second.inflight.clear();
    kv.second.hi = kv.second.lo = kv.second.last = nullptr;
  }
}

}  // namespace
}  // namespace prop

using namespace prop;

extern "C" {

prop_status prop_serve_create(size_t hbm_budget_bytes, int max_slots, int device, prop_server* out) {
  if (!out) return fail(PROP_ERR_INVALID_ARG, "serve_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20) || max_slots < 1)
    return fail(PROP_ERR_INVALID_ARG, "serve_create: need budget >= 1 MiB and max_slots >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(PROP_ERR_INVALID_ARG, "serve_create: no such CUDA device");
  }
  std::unique_ptr<prop_server_s> s(new (std::nothrow) prop_server_s());
  if (!s) return fail(PROP_ERR_OOM, "serve_create: host allocation failed");
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  {
    DeviceGuard g(device);
    cudaError_t e = s->arena.init(hbm_budget_bytes + ((size_t)64 << 20));  // slack for rounding
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PROP_ERR_OOM, std::string("serve_create: arena allocation failed: ") + cudaGetErrorString(e));
    }
  }
  prop_server_s* raw = s.get();
  raw->thr = std::thread([raw] { scheduler(raw); });
  for (int i = 0; i < 2; ++i) raw->workers.emplace_back([raw] { admission(raw); });
  *out = s.release();
  return PROP_OK;
}

prop_status prop_serve_submit(prop_server server, const prop_plan_desc* desc, const prop_recon_params* params,
                              const void* y_host, const void* v0_host, prop_ticket* out) {
  if (!server || !desc || !params || !y_host || !out) return fail(PROP_ERR_INVALID_ARG, "serve_submit: null argument");
  if (params->iters < 0) return fail(PROP_ERR_INVALID_ARG, "serve_submit: iters must be >= 0");
  if (desc->n < 8 || desc->nf < 1 || desc->nblades < 1 || desc->lines < 1 || desc->readout < 1 ||
      desc->nframes < 1 || !desc->delta || !desc->theta)
    return fail(PROP_ERR_INVALID_ARG, "serve_submit: invalid geometry");
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return fail(PROP_ERR_OOM, "serve_submit: host allocation failed");
  r->desc = *desc;
  r->delta.assign(desc->delta, desc->delta + desc->nf);
  r->theta.assign(desc->theta, desc->theta + desc->nblades);
  if (desc->blade_frame) r->frames.assign(desc->blade_frame, desc->blade_frame + desc->nblades);
  r->params = *params;
  const size_t M = (size_t)desc->nblades * desc->lines * desc->readout;
  const size_t V = (size_t)desc->nframes * desc->n * desc->n * desc->nf;
  const float2* y = static_cast<const float2*>(y_host);
  r->y_host.assign(y, y + M);
  if (v0_host) {
    const float2* v = static_cast<const float2*>(v0_host);
    r->v_host.assign(v, v + V);
  }
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(server->mu);
  if (server->stop) return fail(PROP_ERR_CANCELLED, "serve_submit: server is shutting down");
  r->id = server->next_id++;
  *out = r->id;
  server->pending.push_back(r->id);
  server->reqs[r->id] = std::move(r);
  server->cv_admit.notify_all();
  return PROP_OK;
}

prop_status prop_serve_poll(prop_server server, prop_ticket ticket, int* state) {
  if (!server || !state) return fail(PROP_ERR_INVALID_ARG, "serve_poll: null argument");
  std::lock_guard<std::mutex> lk(server->mu);
  auto it = server->reqs.find(ticket);
  if (it == server->reqs.end()) return fail(PROP_ERR_INVALID_ARG, "serve_poll: unknown ticket");
  *state = it->second->state;
  return PROP_OK;
}

prop_status prop_serve_wait(prop_server server, prop_ticket ticket, int timeout_ms, void* v_host_out,
                            double* latency_s, double* final_loss) {
  if (!server) return fail(PROP_ERR_INVALID_ARG, "serve_wait: null server");
  std::unique_lock<std::mutex> lk(server->mu);
  auto it = server->reqs.find(ticket);
  if (it == server->reqs.end()) return fail(PROP_ERR_INVALID_ARG, "serve_wait: unknown ticket");
  Request* r = it->second.get();
  auto ready = [r] { return r->state >= kDone; };
  if (timeout_ms < 0)
    server->cv_done.wait(lk, ready);
  else if (!server->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return fail(PROP_ERR_NOT_READY, "serve_wait: request not finished within the timeout");
  const prop_status st = r->status;
  const std::string msg = r->error;
  if (r->state == kDone) {
    if (v_host_out) std::memcpy(v_host_out, r->result.data(), r->result.size() * sizeof(float2));
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (final_loss) *final_loss = r->final_loss;
  }
  server->reqs.erase(it);
  if (st != PROP_OK) return fail(st, msg);
  return PROP_OK;
}

prop_status prop_serve_cancel(prop_server server, prop_ticket ticket) {
  if (!server) return fail(PROP_ERR_INVALID_ARG, "serve_cancel: null server");
  std::lock_guard<std::mutex> lk(server->mu);
  auto it = server->reqs.find(ticket);
  if (it == server->reqs.end()) return fail(PROP_ERR_INVALID_ARG, "serve_cancel: unknown ticket");
  it->second->cancel = true;
  server->cv_work.notify_all();
  server->cv_admit.notify_all();
  return PROP_OK;
}

prop_status prop_serve_stats(prop_server server, prop_serve_stats_t* out) {
  if (!server || !out) return fail(PROP_ERR_INVALID_ARG, "serve_stats: null argument");
  std::lock_guard<std::mutex> lk(server->mu);
  out->completed = server->completed;
  out->failed = server->failed;
  out->cancelled = server->cancelled;
  out->pending = (long long)server->pending.size();
  out->running = (long long)server->active.size();
  out->reserved_bytes = server->reserved;
  out->arena_bytes_in_use = server->arena.in_use();
  out->arena_peak_bytes = server->arena.peak();
  out->budget_bytes = server->budget;
  return PROP_OK;
}

prop_status prop_serve_destroy(prop_server server) {
  if (!server) return PROP_OK;
  {
    std::lock_guard<std::mutex> lk(server->mu);
    server->stop = true;
    for (Request* r : server->active) r->cancel = true;
    server->cv_work.notify_all();
    server->cv_admit.notify_all();
  }
  for (auto& w : server->workers)
    if (w.joinable()) w.join();
  {
    std::lock_guard<std::mutex> lk(server->mu);
    for (Request* r : server->active) r->cancel = true;  // admitted while stopping
  }
  if (server->thr.joinable()) server->thr.join();
  {
    DeviceGuard g(server->device);
    for (cudaEvent_t e : server->ev_pool) cudaEventDestroy(e);
    for (auto& pp : server->pinned_pool) cudaFreeHost(pp.first);
    server->reqs.clear();
  }
  {
    DeviceGuard g(server->device);
    delete server;
  }
  return PROP_OK;
}

}  // extern "C"

extern "C" prop_status prop_plan_estimate_bytes(const prop_plan_desc* desc, int iters, size_t* bytes) {
  if (!desc || !bytes) return prop::fail(PROP_ERR_INVALID_ARG, "plan_estimate_bytes: null argument");
  *bytes = prop::plan_estimate_bytes(desc, iters);
  if (*bytes == 0) return prop::fail(PROP_ERR_INVALID_ARG, "plan_estimate_bytes: invalid geometry");
  return PROP_OK;
}

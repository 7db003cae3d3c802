// Continuous-batching compression server: requests of mixed sizes are
// admitted as device memory frees up, uploaded while earlier batches
// compute, batched into the next fused-kernel launch on a free compute slot,
// downloaded, and completed.  Every request's result is independent of the
// batch it rode in (per-image tiles and a fixed per-image summation order).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/atdct16.h"
#include "atdct16_arena.h"
#include "atdct16_internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id;
  atdct16_request r;
  double t_arrival = 0, t_submit = 0, t_done = 0;
  cudaEvent_t ev_h2d_start = nullptr, ev_h2d_end = nullptr;  // timing events on the H2D stream
  int slot = -1;                                              // compute slot of its launch
  atdct16_request_timing timing{};
  size_t off = 0, bytes = 0;  // arena slice: src then dst
  double psnr = 0;
  bool done = false;
  int status = ATDCT16_OK;
};

struct Slot {
  atdct16_plan_t plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t computed = nullptr, downloaded = nullptr;
  cudaEvent_t started = nullptr;  // timing event before the launch
  double* d_psnr = nullptr;
  double* h_psnr = nullptr;  // pinned
  std::vector<Req*> reqs;
  bool busy = false;
};

}  // namespace

struct atdct16_server_st {
  atdct16_server_config cfg{};
  int device = 0;
  unsigned char* arena_base = nullptr;
  atdct16::Arena arena;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<Req*> incoming;                     // submitted, not yet seen by the scheduler
  std::deque<Req*> pending;                      // waiting for memory
  std::vector<std::pair<Req*, cudaEvent_t>> uploading;  // admitted, upload in flight
  std::unordered_map<uint64_t, Req*> all;
  std::vector<cudaEvent_t> event_pool;
  std::vector<cudaEvent_t> timing_pool;  // timing-enabled events for the request stage boundaries
  cudaEvent_t ev_ref = nullptr;          // reference event: recorded at creation, at host time host_ref
  double host_ref = 0;
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  // statistics
  uint64_t completed = 0, launches = 0;
  double pixels = 0, first_submit = -1, last_done = 0;
  int sticky_error = ATDCT16_OK;
};

namespace {

cudaEvent_t get_event(atdct16_server_st* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

cudaEvent_t get_timing_event(atdct16_server_st* s) {
  if (!s->timing_pool.empty()) {
    cudaEvent_t e = s->timing_pool.back();
    s->timing_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Host time of a completed timing event: the reference's host time plus the
// device time elapsed since the reference.
double event_time(const atdct16_server_st* s, cudaEvent_t e) {
  float ms = 0.f;
  if (!e || cudaEventElapsedTime(&ms, s->ev_ref, e) != cudaSuccess) return 0.0;
  return s->host_ref + 1e-3 * ms;
}

size_t req_bytes(const atdct16_request& r) { return 2 * (size_t)r.width * (size_t)r.height; }

// h rows of w bytes: one linear copy when both sides are contiguous (the
// copy engine moves pitched 2-D copies row by row, far below the link rate
// for short rows), else a pitched copy.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t w, size_t h,
                      cudaMemcpyKind kind, cudaStream_t stream) {
  if (dpitch == w && spitch == w) return cudaMemcpyAsync(dst, src, w * h, kind, stream);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, w, h, kind, stream);
}

// One pass of the scheduler: completions, admissions, launches.
bool scheduler_pass(atdct16_server_st* s) {
  bool progress = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->incoming.empty()) {
      s->pending.push_back(s->incoming.front());
      s->incoming.pop_front();
    }
  }
  // 1. completions
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.downloaded);
    if (q == cudaErrorNotReady) continue;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    const double t_start = event_time(s, sl.started), t_comp = event_time(s, sl.computed),
                 t_down = event_time(s, sl.downloaded);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      Req* rq = sl.reqs[i];
      rq->psnr = sl.h_psnr[i];
      rq->t_done = t;
      atdct16_request_timing& tm = rq->timing;
      tm.arrival = rq->t_arrival;
      tm.submit = rq->t_submit;
      tm.h2d_start = event_time(s, rq->ev_h2d_start);
      tm.h2d_end = event_time(s, rq->ev_h2d_end);
      tm.compute_start = t_start;
      tm.compute_end = t_comp;
      tm.d2h_end = t_down;
      tm.done = t;
      s->timing_pool.push_back(rq->ev_h2d_start);
      s->timing_pool.push_back(rq->ev_h2d_end);
      rq->ev_h2d_start = rq->ev_h2d_end = nullptr;
      rq->status = q == cudaSuccess ? ATDCT16_OK : ATDCT16_ECUDA;
      rq->done = true;
      s->arena.release(rq->off, rq->bytes);
      s->completed++;
      s->pixels += (double)rq->r.width * rq->r.height;
    }
    s->last_done = t;
    sl.reqs.clear();
    sl.busy = false;
    progress = true;
    s->cv_done.notify_all();
  }
  // 2. admissions (FIFO): allocate, upload on the H2D stream
  while (!s->pending.empty()) {
    Req* rq = s->pending.front();
    size_t off = 0;
    if (!s->arena.alloc(rq->bytes, &off)) break;
    s->pending.pop_front();
    rq->off = off;
    unsigned char* d_src = s->arena_base + off;
    const size_t w = rq->r.width, h = rq->r.height;
    rq->ev_h2d_start = get_timing_event(s);
    rq->ev_h2d_end = get_timing_event(s);
    cudaError_t e = cudaEventRecord(rq->ev_h2d_start, s->h2d);
    if (e == cudaSuccess) e = copy_rows(d_src, w, rq->r.h_src, rq->r.src_pitch, w, h, cudaMemcpyHostToDevice, s->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(rq->ev_h2d_end, s->h2d);
    cudaEvent_t ev = get_event(s);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s->h2d);
    if (e != cudaSuccess) s->sticky_error = ATDCT16_ECUDA;
    s->uploading.emplace_back(rq, ev);
    progress = true;
  }
  // 3. launch: every uploaded request goes into the next batch on a free slot
  if (!s->uploading.empty()) {
    Slot* free_slot = nullptr;
    for (Slot& sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (free_slot) {
      const int maxb = s->cfg.max_batch;
      std::vector<atdct16_image> ims;
      size_t take = 0;
      while (take < s->uploading.size() && (int)take < maxb) {
        // the compute stream waits for this request's upload
        cudaStreamWaitEvent(free_slot->stream, s->uploading[take].second, 0);
        ++take;
      }
      for (size_t i = 0; i < take; ++i) {
        Req* rq = s->uploading[i].first;
        const size_t w = rq->r.width, h = rq->r.height;
        atdct16_image im;
        std::memset(&im, 0, sizeof im);
        im.src = s->arena_base + rq->off;
        im.dst = s->arena_base + rq->off + w * h;
        im.src_pitch = (int64_t)w;
        im.dst_pitch = (int64_t)w;
        im.width = (int32_t)w;
        im.height = (int32_t)h;
        im.r_or_qp = rq->r.r;
        ims.push_back(im);
        free_slot->reqs.push_back(rq);
        s->event_pool.push_back(s->uploading[i].second);
      }
      s->uploading.erase(s->uploading.begin(), s->uploading.begin() + take);
      cudaEventRecord(free_slot->started, free_slot->stream);
      atdct16_status st =
          atdct16_compress_zonal(free_slot->plan, ims.data(), (int32_t)ims.size(), free_slot->d_psnr, nullptr,
                                 free_slot->stream);
      cudaError_t e = st == ATDCT16_OK ? cudaEventRecord(free_slot->computed, free_slot->stream) : cudaErrorUnknown;
      // download on the D2H stream once the batch is computed
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->d2h, free_slot->computed, 0);
      for (size_t i = 0; e == cudaSuccess && i < free_slot->reqs.size(); ++i) {
        Req* rq = free_slot->reqs[i];
        const size_t w = rq->r.width, h = rq->r.height;
        e = copy_rows(rq->r.h_dst, rq->r.dst_pitch, s->arena_base + rq->off + w * h, w, w, h,
                      cudaMemcpyDeviceToHost, s->d2h);
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(free_slot->h_psnr, free_slot->d_psnr, sizeof(double) * free_slot->reqs.size(),
                            cudaMemcpyDeviceToHost, s->d2h);
      if (e == cudaSuccess) e = cudaEventRecord(free_slot->downloaded, s->d2h);
      if (e != cudaSuccess) s->sticky_error = ATDCT16_ECUDA;
      free_slot->busy = true;
      s->launches++;
      progress = true;
    }
  }
  return progress;
}

void worker_main(atdct16_server_st* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    const bool progress = scheduler_pass(s);
    if (!progress) {
      bool idle;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        idle = s->incoming.empty() && s->pending.empty() && s->uploading.empty();
        for (Slot& sl : s->slots) idle = idle && !sl.busy;
      }
      if (idle) {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_submit.wait_for(lk, std::chrono::milliseconds(2),
                              [&] { return s->stop.load() || !s->incoming.empty(); });
      } else {
        std::this_thread::yield();
      }
    }
  }
}

void destroy_server(atdct16_server_st* s) {
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.plan) atdct16_plan_destroy(sl.plan);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.computed) cudaEventDestroy(sl.computed);
    if (sl.started) cudaEventDestroy(sl.started);
    if (sl.downloaded) cudaEventDestroy(sl.downloaded);
    cudaFree(sl.d_psnr);
    cudaFreeHost(sl.h_psnr);
  }
  if (s->h2d) {
    cudaStreamSynchronize(s->h2d);
    cudaStreamDestroy(s->h2d);
  }
  if (s->d2h) {
    cudaStreamSynchronize(s->d2h);
    cudaStreamDestroy(s->d2h);
  }
  for (auto& kv : s->uploading) cudaEventDestroy(kv.second);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : s->timing_pool) cudaEventDestroy(e);
  for (auto& kv : s->all) {
    if (kv.second->ev_h2d_start) cudaEventDestroy(kv.second->ev_h2d_start);
    if (kv.second->ev_h2d_end) cudaEventDestroy(kv.second->ev_h2d_end);
  }
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  for (auto& kv : s->all) delete kv.second;
  cudaFree(s->arena_base);
  delete s;
}

}  // namespace

extern "C" {

atdct16_status atdct16_server_create(const atdct16_server_config* cfg, atdct16_server_t* out) {
  if (!cfg || !out || cfg->memory_budget_bytes < 4096 || cfg->max_batch < 1 || cfg->compute_slots < 1 ||
      cfg->compute_slots > 16 || cfg->reserved != 0)
    return ATDCT16_EINVAL;
  *out = nullptr;
  atdct16_server_st* s = new (std::nothrow) atdct16_server_st();
  if (!s) return ATDCT16_ENOMEM;
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return ATDCT16_ECUDA;
  }
  cudaError_t e = cudaMalloc(&s->arena_base, cfg->memory_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return ATDCT16_ENOMEM;
  }
  s->arena.init(cfg->memory_budget_bytes);
  e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
  s->slots.resize(cfg->compute_slots);
  for (Slot& sl : s->slots) {
    if (e != cudaSuccess) break;
    if (atdct16_plan_create(&sl.plan, ATDCT16_U8, cfg->max_batch, 0, 0) != ATDCT16_OK) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.computed);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.downloaded);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.started);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_psnr, sizeof(double) * cfg->max_batch);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_psnr, sizeof(double) * cfg->max_batch, cudaHostAllocDefault);
  }
  // the reference event that places device timestamps on the host clock
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_ref);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_ref, s->h2d);
  if (e == cudaSuccess) e = cudaEventSynchronize(s->ev_ref);
  s->host_ref = now_s();
  if (e != cudaSuccess) {
    destroy_server(s);
    return ATDCT16_ECUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return ATDCT16_OK;
}

double atdct16_server_clock(void) { return now_s(); }

atdct16_status atdct16_server_submit(atdct16_server_t s, const atdct16_request* r, uint64_t* ticket) {
  return atdct16_server_submit_at(s, r, -1.0, ticket);
}

atdct16_status atdct16_server_submit_at(atdct16_server_t s, const atdct16_request* r, double arrival_s,
                                        uint64_t* ticket) {
  if (!s || !r || !ticket || !r->h_src || !r->h_dst || r->width <= 0 || r->height <= 0 || (r->width & 15) ||
      (r->height & 15) || r->src_pitch < r->width || r->dst_pitch < r->width || r->r < 0 || r->r > 256 ||
      r->reserved != 0)
    return ATDCT16_EINVAL;
  if (req_bytes(*r) > s->arena.size()) return ATDCT16_ENOMEM;  // could never be admitted
  if (s->sticky_error != ATDCT16_OK) return (atdct16_status)s->sticky_error;
  Req* rq = new (std::nothrow) Req();
  if (!rq) return ATDCT16_ENOMEM;
  rq->r = *r;
  rq->bytes = req_bytes(*r);
  rq->t_submit = now_s();
  rq->t_arrival = arrival_s >= 0.0 && arrival_s <= rq->t_submit ? arrival_s : rq->t_submit;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rq->id = s->next_id++;
    s->all[rq->id] = rq;
    s->incoming.push_back(rq);
    if (s->first_submit < 0) s->first_submit = rq->t_submit;
  }
  s->cv_submit.notify_one();
  *ticket = rq->id;
  return ATDCT16_OK;
}

atdct16_status atdct16_server_wait(atdct16_server_t s, uint64_t ticket, double* psnr, double* latency_s,
                                   int64_t timeout_us) {
  if (!s) return ATDCT16_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return ATDCT16_EINVAL;
  Req* rq = it->second;
  const auto pred = [&] { return rq->done; };
  if (timeout_us < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return ATDCT16_ETIMEOUT;
  if (psnr) *psnr = rq->psnr;
  if (latency_s) *latency_s = rq->t_done - rq->t_arrival;
  const int st = rq->status;
  s->all.erase(it);
  delete rq;
  return (atdct16_status)st;
}

atdct16_status atdct16_server_wait_timing(atdct16_server_t s, uint64_t ticket, double* psnr,
                                          atdct16_request_timing* timing, int64_t timeout_us) {
  if (!s) return ATDCT16_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return ATDCT16_EINVAL;
  Req* rq = it->second;
  const auto pred = [&] { return rq->done; };
  if (timeout_us < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return ATDCT16_ETIMEOUT;
  if (psnr) *psnr = rq->psnr;
  if (timing) *timing = rq->timing;
  const int st = rq->status;
  s->all.erase(it);
  delete rq;
  return (atdct16_status)st;
}

atdct16_status atdct16_server_stats(atdct16_server_t s, uint64_t* completed, uint64_t* launches, double* pixels,
                                    double* busy_s, size_t* arena_used) {
  if (!s) return ATDCT16_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (launches) *launches = s->launches;
  if (pixels) *pixels = s->pixels;
  if (busy_s) *busy_s = s->first_submit < 0 ? 0.0 : s->last_done - s->first_submit;
  if (arena_used) *arena_used = s->arena.used();
  return ATDCT16_OK;
}

atdct16_status atdct16_server_destroy(atdct16_server_t s) {
  if (!s) return ATDCT16_EINVAL;
  s->stop.store(true);
  s->cv_submit.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  destroy_server(s);
  return ATDCT16_OK;
}

}  // extern "C"

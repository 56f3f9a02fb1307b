// server.cu -- continuous-batching request server (host code).
//
// Requests (OU-ABC jobs and p-value jobs of any size) arrive at any time from
// any host thread.  A scheduler thread admits them in arrival order whenever a
// stream slot is free and the job's device footprint fits in the caller's
// arena, and enqueues the job's whole pipeline (simulation, selection,
// result copy) on that slot's stream.  Jobs on different slots run
// concurrently on the GPU, so a request that arrives while others are running
// starts as soon as a slot and memory free up instead of waiting for the
// queue to drain.  With one slot the server is the plain one-job-at-a-time
// form.  Small jobs go to their slot's high-priority stream, so that they
// start ahead of a large job's remaining CTAs.  Accepted samples stay in
// device memory until fetched or released.
//
// Nothing on the GPU waits for the host: completion is observed by polling
// CUDA events, and host waits have timeouts.
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace ppabc {
namespace {

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// First-fit allocator over the caller's device arena (offsets only; the
// arena is never touched from the host).
class Arena {
 public:
  void init(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    total_ = bytes;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        sizes_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto s = sizes_.find(off);
    if (s == sizes_.end()) return;
    size_t bytes = s->second;
    sizes_.erase(s);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      free_.erase(next);
    }
    auto it = free_.lower_bound(off);
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }
  size_t total() const { return total_; }

 private:
  std::map<size_t, size_t> free_;   // offset -> length
  std::map<size_t, size_t> sizes_;  // live allocations
  size_t total_ = 0, used_ = 0;
};

enum JobState { kQueued, kRunning, kDone, kFailed, kCancelled };

struct JobRec {
  ppabc_request req;
  JobState state = kQueued;
  int status = PPABC_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  size_t work_off = 0, keep_off = 0;  // arena blocks: scratch (freed at completion), results
  bool has_work = false, has_keep = false;
  size_t work_bytes = 0, keep_bytes = 0;
  int slot = -1;
  // results
  uint64_t n_acc = 0, count = 0;
  double eps = 0, p = 0, post[6] = {0, 0, 0, 0, 0, 0};
  uint64_t cap = 0;
};

// Pinned per-slot staging for the scalar results of the job on that slot.
struct SlotHost {
  uint64_t n_acc;
  double eps;
  double post[6];
  uint64_t count;
  double p;
  double lambda;
};
// launch_job copies (n_acc, eps, post) and (count, p) back in one piece each
static_assert(offsetof(SlotHost, eps) == 8 && offsetof(SlotHost, post) == 16 &&
                  offsetof(SlotHost, p) == offsetof(SlotHost, count) + 8,
              "the result fields are contiguous");

struct Slot {
  cudaStream_t stream = nullptr;     // lowest priority: large jobs
  cudaStream_t stream_hi = nullptr;  // highest priority: small jobs
  cudaEvent_t done = nullptr;
  SlotHost* host = nullptr;  // pinned
  uint64_t job = 0;
  bool busy = false;
};

}  // namespace
}  // namespace ppabc

using namespace ppabc;

struct ppabc_server {
  char* arena_base = nullptr;
  int device = 0;
  Arena arena;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;     // wakes the scheduler
  std::condition_variable done_cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, JobRec> jobs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  ppabc_server_stats stats{};
  char err[256] = "";

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device bytes a job needs while running (scratch) and until released
// (results).
void footprint(const ppabc_request& r, size_t* work, size_t* keep) {
  if (r.kind == PPABC_JOB_ABC) {
    *work = align256(sizeof(double) * r.n_samples) + align256(select_workspace_bytes(r.n_samples)) +
            256;
    *keep = align256(sizeof(uint32_t) * r.k) + align256(16 * r.k) + 3 * 256;
  } else {
    *work = 3 * 256;  // lambda, counts, p
    *keep = 0;
  }
}

int validate_request(const ppabc_request* r) {
  if (!r) return set_error(PPABC_EINVAL, "request is NULL");
  if (r->kind == PPABC_JOB_ABC) {
    OUConst P;
    int rc = make_ou_const(&r->model, r->y_obs, r->seed, r->substream, &P);
    if (rc) return rc;
    if (r->n_samples == 0 || r->n_samples > 0xFFFFFFFFull)
      return set_error(PPABC_EINVAL, "n_samples must be in [1, 2^32)");
    if (r->k == 0 || r->k > r->n_samples) return set_error(PPABC_EINVAL, "k must be in [1, n_samples]");
    return PPABC_OK;
  }
  if (r->kind == PPABC_JOB_PVALUE) {
    if (r->n_obs == 0) return set_error(PPABC_EINVAL, "n_obs must be >= 1");
    if (r->m_sets == 0 || r->m_sets > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "m_sets must be in [1, 2^32)");
    if (!(r->lambda >= 0.0) || r->lambda != r->lambda) return set_error(PPABC_EINVAL, "lambda must be >= 0");
    if (r->ybar_obs != r->ybar_obs) return set_error(PPABC_EINVAL, "ybar_obs is NaN");
    return PPABC_OK;
  }
  return set_error(PPABC_EINVAL, "unknown request kind %d", r->kind);
}

// Jobs of fewer path-steps than this (ABC: samples x EM steps; p-value: data
// sets x normals) run on their slot's high-priority stream: the block
// scheduler then starts their CTAs ahead of a large job's remaining ones,
// instead of after them, and the large job loses only the small one's
// short work.  (Measured in 10 s replays at 200 / 1000 / 2000 jobs/s: the
// p-value jobs' p99 0.35 / 0.94 / 1.81 -> 0.26 / 0.42 / 0.69 ms, the overall
// p99 at 2000/s 2.54 -> 2.17 ms; giving the large jobs priority instead
// helped neither.)
constexpr double kSmallJobPathSteps = 2e8;

// Enqueues job `id` on slot `si` (called with the lock held).
int launch_job(ppabc_server* S, uint64_t id, int si) {
  JobRec& J = S->jobs[id];
  Slot& sl = S->slots[si];
  const double work = J.req.kind == PPABC_JOB_ABC
                          ? static_cast<double>(J.req.n_samples) * static_cast<double>(J.req.model.n_steps)
                          : static_cast<double>(J.req.m_sets) * static_cast<double>(J.req.n_obs + 1);
  // a slot runs one job at a time, so its two streams never hold work at once
  cudaStream_t st = work < kSmallJobPathSteps ? sl.stream_hi : sl.stream;
  char* w = S->arena_base + J.work_off;
  cudaError_t e = cudaSuccess;
  if (J.req.kind == PPABC_JOB_ABC) {
    const ppabc_request& r = J.req;
    OUConst P;
    make_ou_const(&r.model, r.y_obs, r.seed, r.substream, &P);
    double* dist = reinterpret_cast<double*>(w);
    char* sel_ws = w + align256(sizeof(double) * r.n_samples);
    char* k = S->arena_base + J.keep_off;
    uint32_t* idx = reinterpret_cast<uint32_t*>(k);
    float* rec = reinterpret_cast<float*>(k + align256(sizeof(uint32_t) * r.k));
    char* tail = k + align256(sizeof(uint32_t) * r.k) + align256(16 * r.k);
    // the count, epsilon and moments side by side, as in SlotHost, so one
    // copy brings them back
    uint64_t* n_acc = reinterpret_cast<uint64_t*>(tail);
    double* eps = reinterpret_cast<double*>(tail + 8);
    double* post = reinterpret_cast<double*>(tail + 16);
    e = launch_em_ou(P, 0, static_cast<uint32_t>(r.n_samples), nullptr, nullptr, dist, st);
    if (e == cudaSuccess)
      e = launch_select(dist, static_cast<uint32_t>(r.n_samples), r.k, 0.0, P, 0, nullptr, idx, rec, r.k,
                        n_acc, eps, post, sel_ws, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sl.host->n_acc, tail, 64, cudaMemcpyDeviceToHost, st);
    J.cap = r.k;
  } else {
    const ppabc_request& r = J.req;
    double* lam = reinterpret_cast<double*>(w);
    uint64_t* counts = reinterpret_cast<uint64_t*>(w + 256);
    double* p = reinterpret_cast<double*>(w + 264);  // next to the count, as in SlotHost
    sl.host->lambda = r.lambda;
    e = cudaMemcpyAsync(lam, &sl.host->lambda, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_pvalue(lam, 1, r.n_obs, static_cast<uint32_t>(r.m_sets), 0, r.ybar_obs, r.seed, counts, p,
                        nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sl.host->count, counts, 16, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) {
    snprintf(S->err, sizeof(S->err), "job %llu launch: %s", (unsigned long long)id, cudaGetErrorString(e));
    return PPABC_ECUDA;
  }
  sl.busy = true;
  sl.job = id;
  J.slot = si;
  J.state = kRunning;
  J.t_admit = S->now();
  return PPABC_OK;
}

void free_work(ppabc_server* S, JobRec& J) {
  if (J.has_work) S->arena.release(J.work_off);
  J.has_work = false;
}

void free_keep(ppabc_server* S, JobRec& J) {
  if (J.has_keep) S->arena.release(J.keep_off);
  J.has_keep = false;
}

// Scheduler: retire finished slots, then admit queued jobs in order.
void scheduler(ppabc_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    bool changed = false;
    for (size_t si = 0; si < S->slots.size(); ++si) {
      Slot& sl = S->slots[si];
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      JobRec& J = S->jobs[sl.job];
      J.t_done = S->now();
      if (q == cudaSuccess) {
        // Only the fields this kind of job wrote; the staging area keeps the
        // previous job's values in the others.
        if (J.req.kind == PPABC_JOB_ABC) {
          J.n_acc = sl.host->n_acc;
          J.eps = sl.host->eps;
          memcpy(J.post, sl.host->post, sizeof(J.post));
        } else {
          J.count = sl.host->count;
          J.p = sl.host->p;
        }
        J.state = (J.state == kCancelled) ? kCancelled : kDone;
        J.status = (J.state == kCancelled) ? PPABC_ECANCELLED : PPABC_OK;
        S->stats.completed += 1;
      } else {
        J.state = kFailed;
        J.status = PPABC_ECUDA;
        S->stats.failed += 1;
      }
      free_work(S, J);
      if (J.state != kDone) free_keep(S, J);
      sl.busy = false;
      changed = true;
    }
    // FIFO admission: the head job waits for a slot and for its memory.
    while (!S->queue.empty()) {
      int free_slot = -1;
      for (size_t si = 0; si < S->slots.size(); ++si)
        if (!S->slots[si].busy) {
          free_slot = static_cast<int>(si);
          break;
        }
      if (free_slot < 0) break;
      const uint64_t id = S->queue.front();
      JobRec& J = S->jobs[id];
      if (J.state == kCancelled) {
        S->queue.pop_front();
        changed = true;
        continue;
      }
      size_t off_w = 0, off_k = 0;
      if (!S->arena.alloc(J.work_bytes, &off_w)) break;
      if (J.keep_bytes && !S->arena.alloc(J.keep_bytes, &off_k)) {
        S->arena.release(off_w);
        break;
      }
      J.work_off = off_w;
      J.has_work = true;
      J.keep_off = off_k;
      J.has_keep = J.keep_bytes > 0;
      S->queue.pop_front();
      if (launch_job(S, id, free_slot) != PPABC_OK) {
        J.state = kFailed;
        J.status = PPABC_ECUDA;
        J.t_done = S->now();
        free_work(S, J);
        free_keep(S, J);
        S->stats.failed += 1;
      } else {
        S->stats.admitted += 1;
      }
      changed = true;
    }
    if (S->arena.used() > S->stats.peak_arena_bytes) S->stats.peak_arena_bytes = S->arena.used();
    if (changed) S->done_cv.notify_all();
    bool any_busy = false;
    for (auto& sl : S->slots) any_busy |= sl.busy;
    // Busy: poll the completion events about every 2 us, with the lock
    // released meanwhile so that submits go through.  (A timed wait would
    // sleep at least the thread's timer slack, about 50 us on Linux, and that
    // would land in every job's latency.)  Idle: sleep until a submit wakes us.
    if (any_busy) {
      lock.unlock();
      const auto t_spin = std::chrono::steady_clock::now();
      while (std::chrono::steady_clock::now() - t_spin < std::chrono::microseconds(2)) std::this_thread::yield();
      lock.lock();
    } else {
      S->cv.wait_for(lock, std::chrono::milliseconds(50));
    }
  }
}

void fill_result(const JobRec& J, uint64_t id, ppabc_result* out) {
  memset(out, 0, sizeof(*out));
  out->job_id = id;
  out->kind = J.req.kind;
  out->status = J.status;
  out->t_submit = J.t_submit;
  out->t_admit = J.t_admit;
  out->t_done = J.t_done;
  out->n_acc = J.n_acc;
  out->eps = J.eps;
  memcpy(out->post, J.post, sizeof(J.post));
  out->count = J.count;
  out->p = J.p;
}

}  // namespace

extern "C" {

int ppabc_server_create(void* d_arena, size_t arena_bytes, uint32_t n_slots, ppabc_server** out) {
  if (!out) return set_error(PPABC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d_arena || arena_bytes < 4096) return set_error(PPABC_EINVAL, "arena must be >= 4096 bytes");
  if (reinterpret_cast<uintptr_t>(d_arena) & 255u) return set_error(PPABC_EINVAL, "arena must be 256-byte aligned");
  if (n_slots < 1 || n_slots > 64) return set_error(PPABC_EINVAL, "n_slots must be in [1, 64]");
  int rc = require_device();
  if (rc) return rc;
  ppabc_server* S = new (std::nothrow) ppabc_server();
  if (!S) return set_error(PPABC_ENOMEM, "host allocation failed");
  cudaGetDevice(&S->device);
  S->arena_base = static_cast<char*>(d_arena);
  S->arena.init(arena_bytes & ~static_cast<size_t>(255));
  S->slots.resize(n_slots);
  for (auto& sl : S->slots) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&sl.host), sizeof(SlotHost), cudaHostAllocDefault);
    if (e != cudaSuccess) {
      ppabc_server_destroy(S);
      return check_cuda(e, "server slot setup");
    }
  }
  S->t0 = std::chrono::steady_clock::now();
  S->worker = std::thread(scheduler, S);
  *out = S;
  return PPABC_OK;
}

int ppabc_server_submit(ppabc_server* S, const ppabc_request* r, uint64_t* job_id) {
  if (!S || !job_id) return set_error(PPABC_EINVAL, "server and job_id must be non-NULL");
  int rc = validate_request(r);
  if (rc) return rc;
  JobRec J;
  J.req = *r;
  footprint(*r, &J.work_bytes, &J.keep_bytes);
  if (align256(J.work_bytes) + align256(J.keep_bytes) > S->arena.total())
    return set_error(PPABC_ENOMEM, "job needs %zu bytes of device memory, the arena holds %zu",
                     align256(J.work_bytes) + align256(J.keep_bytes), S->arena.total());
  {
    std::lock_guard<std::mutex> lock(S->mu);
    const uint64_t id = S->next_id++;
    J.t_submit = S->now();
    S->jobs[id] = J;
    S->queue.push_back(id);
    S->stats.submitted += 1;
    *job_id = id;
  }
  S->cv.notify_one();
  return PPABC_OK;
}

int ppabc_server_poll(ppabc_server* S, uint64_t job_id, ppabc_result* out) {
  if (!S || !out) return set_error(PPABC_EINVAL, "server and out must be non-NULL");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(PPABC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
  const JobRec& J = it->second;
  if (J.state == kQueued || J.state == kRunning) return PPABC_PENDING;
  fill_result(J, job_id, out);
  return PPABC_OK;
}

int ppabc_server_wait(ppabc_server* S, uint64_t job_id, double timeout_s, ppabc_result* out) {
  if (!S || !out) return set_error(PPABC_EINVAL, "server and out must be non-NULL");
  std::unique_lock<std::mutex> lock(S->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return set_error(PPABC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
    if (it->second.state != kQueued && it->second.state != kRunning) {
      fill_result(it->second, job_id, out);
      return PPABC_OK;
    }
    if (S->done_cv.wait_until(lock, deadline) == std::cv_status::timeout)
      return set_error(PPABC_ETIMEOUT, "job %llu not finished after %.3f s", (unsigned long long)job_id,
                       timeout_s);
  }
}

int ppabc_server_fetch(ppabc_server* S, uint64_t job_id, uint32_t* h_idx, float* h_rec, uint64_t cap,
                       uint64_t* n_out) {
  if (!S) return set_error(PPABC_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(PPABC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
  JobRec& J = it->second;
  if (J.state != kDone) return J.state == kCancelled ? set_error(PPABC_ECANCELLED, "job cancelled")
                                                     : set_error(PPABC_PENDING, "job not finished");
  if (J.req.kind != PPABC_JOB_ABC || !J.has_keep) return set_error(PPABC_EINVAL, "no accepted samples held");
  const uint64_t n = J.n_acc < J.cap ? J.n_acc : J.cap;
  const uint64_t w = n < cap ? n : cap;
  const char* k = S->arena_base + J.keep_off;
  cudaError_t e = cudaSuccess;
  if (w && h_idx) e = cudaMemcpy(h_idx, k, sizeof(uint32_t) * w, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && w && h_rec)
    e = cudaMemcpy(h_rec, k + align256(sizeof(uint32_t) * J.cap), 16 * w, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return check_cuda(e, "fetch copy");
  if (n_out) *n_out = w;
  return PPABC_OK;
}

int ppabc_server_release(ppabc_server* S, uint64_t job_id) {
  if (!S) return set_error(PPABC_EINVAL, "server is NULL");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return set_error(PPABC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
    if (it->second.state == kQueued || it->second.state == kRunning)
      return set_error(PPABC_PENDING, "job not finished");
    free_keep(S, it->second);
    S->jobs.erase(it);
  }
  S->cv.notify_one();
  return PPABC_OK;
}

int ppabc_server_cancel(ppabc_server* S, uint64_t job_id) {
  if (!S) return set_error(PPABC_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(PPABC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
  JobRec& J = it->second;
  if (J.state == kQueued) {
    J.state = kCancelled;
    J.status = PPABC_ECANCELLED;
    J.t_done = S->now();
    S->stats.cancelled += 1;
    S->done_cv.notify_all();
    return PPABC_OK;
  }
  if (J.state == kRunning) {  // the GPU work finishes; its result is discarded
    J.state = kCancelled;
    S->stats.cancelled += 1;
    return PPABC_OK;
  }
  return set_error(PPABC_EINVAL, "job already finished");
}

int ppabc_server_get_stats(ppabc_server* S, ppabc_server_stats* out) {
  if (!S || !out) return set_error(PPABC_EINVAL, "server and out must be non-NULL");
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  out->queued = S->queue.size();
  out->arena_used_bytes = S->arena.used();
  uint64_t running = 0;
  for (auto& sl : S->slots) running += sl.busy ? 1 : 0;
  out->running = running;
  return PPABC_OK;
}

double ppabc_server_now(ppabc_server* S) { return S ? S->now() : 0.0; }

int ppabc_server_destroy(ppabc_server* S) {
  if (!S) return PPABC_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.stream_hi) cudaStreamDestroy(sl.stream_hi);
    if (sl.host) cudaFreeHost(sl.host);
  }
  delete S;
  return PPABC_OK;
}

}  // extern "C"

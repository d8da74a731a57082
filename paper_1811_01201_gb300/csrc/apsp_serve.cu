// Continuous-batching APSP server (C ABI apsp_serve_* in include/apsp.h).
//
// Requests arrive on host threads (apsp_serve_submit) and wait in a FIFO.
// A scheduler thread admits them while the sum of admitted device
// footprints stays within the HBM budget and the number of resident jobs
// within max_slots, then dispatches admitted work onto a pool of CUDA streams
// as soon as a stream is free:
//   * graphs of order <= 512 go together into persistent batched launches,
//     one per size class (n <= 128, <= 256, <= 512; every graph of the class
//     admitted since the last dispatch joins the next batch), so requests that
//     arrive while earlier batches run are picked up by the next one instead of
//     waiting for them to finish, and small ones do not wait for large ones;
//   * larger graphs run the single-graph blocked path on their own stream.
// Work on different streams overlaps on the device; the batched launches run on
// high-priority streams, so that they get SMs while a large solve runs. A host callback at the
// end of each dispatch stamps completion time and wakes the scheduler, which
// returns the memory to the budget and admits more work.
//
// Each result equals what apsp_fw with default options returns for the same
// graph: small graphs run with BS = 32 (the default block size for n <= 512)
// in fp32, which the 16-bit path reproduces bit for bit; large graphs use the
// default block size and the same 16-bit eligibility rule. A job submitted
// with explicit options (apsp_serve_submit_ex) that the batched kernel does not
// cover runs the single-graph path with them.
//
// Failure detection: a single-graph dispatch runs in a workspace of its own,
// whose fault word the phase kernels set when a bounded wait expires. The
// dispatch copies that word to host memory after its kernels, and the
// completion callback fails the job with APSP_ETIMEOUT if it is set, so one
// failing job never marks the jobs running beside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_internal.h"

namespace apsp {

using Clock = std::chrono::steady_clock;

static double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// Page-locked host buffers recycled by power-of-two size class.
class PinnedPool {
 public:
  ~PinnedPool() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
  }
  void* get(size_t bytes, size_t* cls_out) {
    size_t cls = 256;
    while (cls < bytes) cls <<= 1;
    *cls_out = cls;
    {
      std::lock_guard<std::mutex> g(m_);
      auto& v = free_[cls];
      if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        return p;
      }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, cls) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cls) {
    if (!p) return;
    std::lock_guard<std::mutex> g(m_);
    free_[cls].push_back(p);
  }

 private:
  std::mutex m_;
  std::map<size_t, std::vector<void*>> free_;
};

enum JobState { kQueued = 0, kAdmitted = 1, kRunning = 2, kDone = 3, kFailed = 4, kCancelled = 5 };

struct Job {
  uint64_t id = 0;
  int n = 0;
  int bs = 32;
  int dtype = APSP_DTYPE_F32;
  int flags = 0;      // APSP_FLAG_* of a job submitted with options (single-graph path only)
  bool small = true;  // runs in a batched launch
  bool integral = false;
  size_t footprint = 0;
  float* hW = nullptr;
  float* hD = nullptr;
  int32_t* hP = nullptr;
  size_t clsW = 0, clsD = 0, clsP = 0;
  float* dD = nullptr;
  int32_t* dP = nullptr;
  JobState state = kQueued;
  apsp_status status = APSP_OK;
  double t_submit = 0, t_done = 0;
};

struct Dispatch;

struct ServerImpl {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  std::vector<bool> stream_high;  // high-priority stream: small-graph batches
  bool has_high = false;
  PinnedPool pool;

  std::mutex m;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Job>> queue;            // submitted, not admitted
  std::vector<std::shared_ptr<Job>> admitted;        // admitted, not dispatched
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<Dispatch*> finished;                   // completed dispatches to retire
  uint64_t next_id = 1;
  bool stop = false;
  std::thread sched;

  uint64_t submitted = 0, completed = 0, rejected = 0, in_flight = 0;
  size_t hbm_in_use = 0, hbm_peak = 0;
  double t_first = 0, t_last = 0;
  std::vector<double> lat_ms;
};

struct Dispatch {
  ServerImpl* srv = nullptr;
  int stream_idx = 0;
  std::vector<std::shared_ptr<Job>> jobs;
  void* staging = nullptr;  // pinned: descriptor table of a batch, or the fault word of a single-graph solve
  size_t staging_cls = 0;
  apsp_status status = APSP_OK;
  bool check_fault = false;  // staging holds the solve's fault word, copied back after its kernels
};

static void CUDART_CB on_dispatch_done(void* arg) {
  // Runs on a CUDA driver thread: no CUDA calls here.
  Dispatch* d = static_cast<Dispatch*>(arg);
  ServerImpl* s = d->srv;
  const double t = now_s();
  if (d->status == APSP_OK && d->check_fault && *static_cast<volatile unsigned*>(d->staging) != 0u)
    d->status = APSP_ETIMEOUT;  // a bounded device wait of this solve expired: its D and P are not valid
  {
    std::lock_guard<std::mutex> g(s->m);
    for (auto& j : d->jobs) {
      j->t_done = t;
      j->state = (d->status == APSP_OK) ? kDone : kFailed;
      j->status = d->status;
    }
    s->finished.push_back(d);
  }
  s->cv_sched.notify_one();
  s->cv_done.notify_all();
}

// Size class of a small graph for batching: n <= 128, <= 256, <= 512.
static int small_class(int n) { return n <= 128 ? 0 : (n <= 256 ? 1 : 2); }

static size_t job_footprint(int n, bool small, int bs, int dtype) {
  const size_t nn = (size_t)n * n;
  size_t f = nn * (sizeof(float) + sizeof(int32_t));
  if (!small) f += fw_exec_workspace(n, bs, dtype, nullptr, nullptr);
  return f + 4096;
}

// Enqueue one dispatch (already holding a free stream). Called by the
// scheduler thread without the lock held.
static void run_dispatch(ServerImpl* s, Dispatch* d) {
  cudaStream_t st = s->streams[d->stream_idx];
  apsp_status status = APSP_OK;
  for (auto& j : d->jobs) {
    const size_t nn = (size_t)j->n * j->n;
    if (cudaMallocAsync(reinterpret_cast<void**>(&j->dD), nn * sizeof(float), st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&j->dP), nn * sizeof(int32_t), st) != cudaSuccess) {
      cudaGetLastError();
      status = APSP_ENOMEM;
      break;
    }
    if (cudaMemcpyAsync(j->dD, j->hW, nn * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
      status = APSP_ECUDA;
  }
  if (status == APSP_OK) {
    if (d->jobs.front()->small) {
      const int count = (int)d->jobs.size();
      BatchGraphDesc* tbl = static_cast<BatchGraphDesc*>(d->staging);
      int* order = reinterpret_cast<int*>(tbl + count);
      for (int g = 0; g < count; ++g) {
        const auto& j = d->jobs[g];
        tbl[g] = BatchGraphDesc{j->dD, j->dD, j->dP, j->n, default_ph3_rows(j->n)};
        order[g] = g;
      }
      std::stable_sort(order, order + count, [&](int a, int b) { return tbl[a].n > tbl[b].n; });
      status = batch_launch_async(tbl, count, st);
    } else {
      auto& j = d->jobs.front();
      // own workspace, so that this solve's fault word is read back for this job alone
      const size_t wsb = fw_exec_workspace(j->n, j->bs, j->dtype, j->dD, j->dP);
      void* ws = nullptr;
      if (cudaMallocAsync(&ws, wsb, st) != cudaSuccess) {
        cudaGetLastError();
        status = APSP_ENOMEM;
      } else {
        status = fw_exec(j->dD, j->dD, j->dP, j->n, j->bs, j->dtype, j->integral ? 1 : 0, j->flags, ws, wsb,
                         nullptr, st);
        if (status == APSP_OK) {
          *static_cast<unsigned*>(d->staging) = 0u;
          if (cudaMemcpyAsync(d->staging, static_cast<char*>(ws) + fw_fault_word_offset(), sizeof(unsigned),
                              cudaMemcpyDeviceToHost, st) != cudaSuccess)
            status = APSP_ECUDA;
          d->check_fault = status == APSP_OK;
        }
        cudaFreeAsync(ws, st);
      }
    }
  }
  for (auto& j : d->jobs) {
    const size_t nn = (size_t)j->n * j->n;
    if (status == APSP_OK) {
      if (cudaMemcpyAsync(j->hD, j->dD, nn * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(j->hP, j->dP, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        status = APSP_ECUDA;
    }
    if (j->dD) cudaFreeAsync(j->dD, st);
    if (j->dP) cudaFreeAsync(j->dP, st);
    j->dD = nullptr;
    j->dP = nullptr;
  }
  d->status = status;
  if (cudaLaunchHostFunc(st, on_dispatch_done, d) != cudaSuccess) {
    // the callback could not be queued: finish synchronously
    cudaGetLastError();
    cudaStreamSynchronize(st);
    d->status = APSP_ECUDA;
    on_dispatch_done(d);
  }
}

static void scheduler(ServerImpl* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->m);
  for (;;) {
    // retire finished dispatches: free their stream, return their memory
    for (Dispatch* d : s->finished) {
      s->stream_busy[d->stream_idx] = false;
      for (auto& j : d->jobs) {
        s->hbm_in_use -= j->footprint;
        --s->in_flight;
        if (j->state == kDone) {
          ++s->completed;
          s->lat_ms.push_back((j->t_done - j->t_submit) * 1e3);
          s->t_last = std::max(s->t_last, j->t_done);
        }
        s->pool.put(j->hW, j->clsW);
        j->hW = nullptr;
      }
      s->pool.put(d->staging, d->staging_cls);
      delete d;
    }
    s->finished.clear();
    if (s->stop && s->in_flight == 0) break;
    // admission: FIFO while slots and budget allow
    while (!s->stop && !s->queue.empty()) {
      auto& j = s->queue.front();
      if ((int)s->in_flight >= s->max_slots || s->hbm_in_use + j->footprint > s->budget) break;
      s->hbm_in_use += j->footprint;
      s->hbm_peak = std::max(s->hbm_peak, s->hbm_in_use);
      ++s->in_flight;
      j->state = kAdmitted;
      s->admitted.push_back(j);
      s->queue.pop_front();
    }
    // dispatch onto free streams: all admitted small graphs as one batch on a high-priority
    // stream, large graphs one each on the others (a single stream takes both)
    std::vector<Dispatch*> todo;
    for (size_t si = 0; si < s->streams.size() && !s->admitted.empty(); ++si) {
      if (s->stream_busy[si]) continue;
      const bool serves_small = s->stream_high[si] || !s->has_high;
      const bool serves_large = !s->stream_high[si];
      const bool have_small = std::any_of(s->admitted.begin(), s->admitted.end(),
                                          [](const std::shared_ptr<Job>& j) { return j->small; });
      const bool have_large = std::any_of(s->admitted.begin(), s->admitted.end(),
                                          [](const std::shared_ptr<Job>& j) { return !j->small; });
      const bool small_batch = serves_small && have_small;
      if (!small_batch && !(serves_large && have_large)) continue;
      Dispatch* d = new Dispatch();
      d->srv = s;
      d->stream_idx = (int)si;
      if (small_batch) {
        // one size class per batch, smallest first: every job of a batch completes with its
        // largest graph, so a small request does not wait for a 512-vertex one
        int cls = 3;
        for (auto& j : s->admitted)
          if (j->small) cls = std::min(cls, small_class(j->n));
        auto in_batch = [cls](const std::shared_ptr<Job>& j) { return j->small && small_class(j->n) == cls; };
        for (auto& j : s->admitted)
          if (in_batch(j)) d->jobs.push_back(j);
        s->admitted.erase(std::remove_if(s->admitted.begin(), s->admitted.end(), in_batch), s->admitted.end());
        const size_t need = d->jobs.size() * (sizeof(BatchGraphDesc) + sizeof(int));
        d->staging = s->pool.get(need, &d->staging_cls);
        if (!d->staging) {
          for (auto& j : d->jobs) { j->state = kAdmitted; s->admitted.push_back(j); }
          delete d;
          break;
        }
      } else {
        d->staging = s->pool.get(sizeof(unsigned), &d->staging_cls);  // the solve's fault word
        if (!d->staging) {
          delete d;
          break;
        }
        auto it = std::find_if(s->admitted.begin(), s->admitted.end(),
                               [](const std::shared_ptr<Job>& j) { return !j->small; });
        d->jobs.push_back(*it);
        s->admitted.erase(it);
      }
      for (auto& j : d->jobs) j->state = kRunning;
      s->stream_busy[si] = true;
      todo.push_back(d);
    }
    if (!todo.empty()) {
      lk.unlock();
      for (Dispatch* d : todo) run_dispatch(s, d);
      lk.lock();
      continue;
    }
    s->cv_sched.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace apsp

using namespace apsp;

struct apsp_server {
  ServerImpl impl;
};

extern "C" apsp_status apsp_serve_create(apsp_server** out, size_t hbm_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || hbm_budget_bytes < (1u << 20)) return APSP_EINVAL;
  *out = nullptr;
  apsp_server* srv = new apsp_server();
  ServerImpl& s = srv->impl;
  if (cudaGetDevice(&s.device) != cudaSuccess) {
    delete srv;
    return APSP_ECUDA;
  }
  s.budget = hbm_budget_bytes;
  s.max_slots = max_slots;
  // keep freed blocks in the stream-ordered pool up to the budget
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s.device) == cudaSuccess) {
    uint64_t thr = hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  // Half the streams (at least one, when there are two or more) run the batched launches of
  // small graphs at the device's highest stream priority: a batched CTA needs a whole SM, and
  // with the priority the block scheduler gives it the next SM that drains instead of another
  // CTA of a large solve, so small requests overlap a running large one instead of waiting.
  const int ns = std::min(max_slots, 16);
  int prio_low = 0, prio_high = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
    cudaGetLastError();
    prio_low = prio_high = 0;
  }
  const int n_high = ns >= 2 ? ns / 2 : 0;
  for (int i = 0; i < ns; ++i) {
    cudaStream_t st;
    const bool high = i < n_high;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, high ? prio_high : prio_low) != cudaSuccess) {
      for (cudaStream_t x : s.streams) cudaStreamDestroy(x);
      delete srv;
      return APSP_ECUDA;
    }
    s.streams.push_back(st);
    s.stream_busy.push_back(false);
    s.stream_high.push_back(high);
  }
  s.has_high = n_high > 0;
  s.sched = std::thread(scheduler, &s);
  *out = srv;
  return APSP_OK;
}

extern "C" apsp_status apsp_serve_submit_ex(apsp_server* srv, const float* W, int n, const apsp_options* opt,
                                            uint64_t* job_id) {
  if (!srv || !W || !job_id || n < 1 || n > 65536) return APSP_EINVAL;
  ServerImpl& s = srv->impl;
  int want_bs = 0, want_dtype = APSP_DTYPE_AUTO, flags = 0;
  if (opt) {
    want_bs = opt->bs;
    want_dtype = opt->dtype;
    flags = opt->flags;
    if ((want_bs != 0 && want_bs != 32 && want_bs != 64 && want_bs != 128) || want_dtype < APSP_DTYPE_AUTO ||
        want_dtype > APSP_DTYPE_U16X2 || (flags & ~APSP_FLAG_TEST_PANEL_TIMEOUT) != 0)
      return APSP_EINVAL;
  }
  const size_t nn = (size_t)n * n;
  // host-side validation and 16-bit eligibility (same rule as apsp_fw)
  bool frac = false, bad = false, absent = false;
  float mx = 0.f;
  for (int i = 0; i < n; ++i) {
    const float* row = W + (size_t)i * n;
    for (int j = 0; j < n; ++j) {
      const float v = row[j];
      if (j == i) continue;
      bad |= !(v >= 0.f);  // negative or NaN
      if (v < INFINITY) {
        frac |= v != std::floor(v);
        mx = v > mx ? v : mx;
      } else {
        absent = true;
      }
    }
  }
  const bool eligible = u16_eligible(!frac, !absent, mx, n);
  if (bad || (want_dtype == APSP_DTYPE_U16X2 && !eligible)) {
    std::lock_guard<std::mutex> g(s.m);
    ++s.rejected;
    return APSP_EINVAL;
  }
  auto j = std::make_shared<Job>();
  j->n = n;
  // the batched kernel covers fp32 (or equal 16-bit) results at BS = 32 without test flags
  j->small = n <= kBatchMaxN && (want_bs == 0 || want_bs == 32) && want_dtype != APSP_DTYPE_U16X2 && flags == 0;
  j->dtype = (!j->small && eligible && want_dtype != APSP_DTYPE_F32) ? APSP_DTYPE_U16X2 : APSP_DTYPE_F32;
  j->bs = j->small ? 32 : (want_bs ? want_bs : default_bs_for(n, j->dtype));
  j->flags = flags;
  j->integral = !frac;
  j->footprint = job_footprint(n, j->small, j->bs, j->dtype);
  if (j->footprint > s.budget) {
    std::lock_guard<std::mutex> g(s.m);
    ++s.rejected;
    return APSP_ENOMEM;
  }
  j->hW = static_cast<float*>(s.pool.get(nn * sizeof(float), &j->clsW));
  j->hD = static_cast<float*>(s.pool.get(nn * sizeof(float), &j->clsD));
  j->hP = static_cast<int32_t*>(s.pool.get(nn * sizeof(int32_t), &j->clsP));
  if (!j->hW || !j->hD || !j->hP) {
    s.pool.put(j->hW, j->clsW);
    s.pool.put(j->hD, j->clsD);
    s.pool.put(j->hP, j->clsP);
    return APSP_ENOMEM;
  }
  std::memcpy(j->hW, W, nn * sizeof(float));
  {
    std::lock_guard<std::mutex> g(s.m);
    if (s.stop) {
      s.pool.put(j->hW, j->clsW);
      s.pool.put(j->hD, j->clsD);
      s.pool.put(j->hP, j->clsP);
      return APSP_ECANCELLED;
    }
    j->id = s.next_id++;
    j->t_submit = now_s();
    if (s.submitted == 0) s.t_first = j->t_submit;
    ++s.submitted;
    s.jobs[j->id] = j;
    s.queue.push_back(j);
    *job_id = j->id;
  }
  s.cv_sched.notify_one();
  return APSP_OK;
}

extern "C" apsp_status apsp_serve_submit(apsp_server* srv, const float* W, int n, uint64_t* job_id) {
  return apsp_serve_submit_ex(srv, W, n, nullptr, job_id);
}

extern "C" apsp_status apsp_serve_poll(apsp_server* srv, uint64_t job_id, float* D, int32_t* P, int* bs_used,
                                       int timeout_ms) {
  if (!srv) return APSP_EINVAL;
  ServerImpl& s = srv->impl;
  std::unique_lock<std::mutex> lk(s.m);
  auto it = s.jobs.find(job_id);
  if (it == s.jobs.end()) return APSP_ENOTFOUND;
  std::shared_ptr<Job> j = it->second;
  auto ready = [&] { return j->state == kDone || j->state == kFailed || j->state == kCancelled; };
  if (!ready()) {
    if (timeout_ms == 0) return APSP_EBUSY;
    if (timeout_ms < 0) s.cv_done.wait(lk, ready);
    else if (!s.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return APSP_ETIMEOUT;
  }
  s.jobs.erase(job_id);
  lk.unlock();
  apsp_status st = j->state == kDone ? APSP_OK : (j->state == kCancelled ? APSP_ECANCELLED : j->status);
  const size_t nn = (size_t)j->n * j->n;
  if (st == APSP_OK) {
    if (D) std::memcpy(D, j->hD, nn * sizeof(float));
    if (P) std::memcpy(P, j->hP, nn * sizeof(int32_t));
    if (bs_used) *bs_used = j->bs;
  }
  s.pool.put(j->hD, j->clsD);
  s.pool.put(j->hP, j->clsP);
  j->hD = nullptr;
  j->hP = nullptr;
  return st;
}

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

extern "C" apsp_status apsp_serve_stats(apsp_server* srv, apsp_stats* out) {
  if (!srv || !out) return APSP_EINVAL;
  ServerImpl& s = srv->impl;
  std::lock_guard<std::mutex> g(s.m);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s.submitted;
  out->completed = s.completed;
  out->rejected = s.rejected;
  out->in_flight = s.in_flight;
  out->queued = s.queue.size();
  const double span = s.t_last - s.t_first;
  out->graphs_per_s = (span > 0 && s.completed) ? (double)s.completed / span : 0.0;
  out->p50_ms = percentile(s.lat_ms, 0.50);
  out->p99_ms = percentile(s.lat_ms, 0.99);
  double sum = 0, mx = 0;
  for (double x : s.lat_ms) { sum += x; mx = std::max(mx, x); }
  out->mean_ms = s.lat_ms.empty() ? 0.0 : sum / (double)s.lat_ms.size();
  out->max_ms = mx;
  out->hbm_in_use = s.hbm_in_use;
  out->hbm_peak = s.hbm_peak;
  return APSP_OK;
}

extern "C" apsp_status apsp_serve_destroy(apsp_server* srv) {
  if (!srv) return APSP_EINVAL;
  ServerImpl& s = srv->impl;
  {
    std::lock_guard<std::mutex> g(s.m);
    s.stop = true;
    for (auto& j : s.queue) {
      j->state = kCancelled;
      j->status = APSP_ECANCELLED;
      s.pool.put(j->hW, j->clsW);
      j->hW = nullptr;
    }
    s.queue.clear();
    // admitted-but-not-dispatched jobs still hold budget and slots: release them
    for (auto& j : s.admitted) {
      j->state = kCancelled;
      s.hbm_in_use -= j->footprint;
      --s.in_flight;
      s.pool.put(j->hW, j->clsW);
      j->hW = nullptr;
    }
    s.admitted.clear();
  }
  s.cv_sched.notify_all();
  s.cv_done.notify_all();
  if (s.sched.joinable()) s.sched.join();
  for (cudaStream_t st : s.streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  {
    std::lock_guard<std::mutex> g(s.m);
    for (auto& kv : s.jobs) {
      auto& j = kv.second;
      s.pool.put(j->hW, j->clsW);
      s.pool.put(j->hD, j->clsD);
      s.pool.put(j->hP, j->clsP);
    }
    s.jobs.clear();
  }
  delete srv;
  return APSP_OK;
}

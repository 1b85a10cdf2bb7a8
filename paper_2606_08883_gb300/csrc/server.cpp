// Request server: continuous batching of whole MRCM-OS / GMRES solves on one GPU.
//
// Memory: the caller's device arena is carved by a first-fit free list (256-byte granules); each
// admitted request holds one block (its workspace plus its K, boundary data, source and solution
// arrays) until it finishes.  Admission: the oldest queued request whose block fits, while fewer
// than max_inflight run; a request passed over more than 8 times stops the backfilling until it is
// admitted.  Execution: one host worker thread and one CUDA stream per slot; every request runs
// mrcm_setup, mrcm_factor_local and mrcm_gmres_solve on its stream, so requests overlap on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, size) with coalescing on free.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

enum State { QUEUED, RUNNING, FINISHED };

struct Request {
  uint64_t id = 0;
  mrcm_problem prob{};
  mrcm_params prm{};
  size_t n = 0, footprint = 0, block = 0, off = 0;
  std::vector<double> K, Ky, f, p, hist;
  std::vector<double> bc[6];
  int state = QUEUED;
  int skipped = 0;
  volatile int cancel = 0;
  mrcm_status status = MRCM_OK;
  mrcm_result res{};
  std::string err;
  Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct mrcm_server {
  char* arena_base = nullptr;
  std::unique_ptr<Arena> arena;
  int max_inflight = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_work;
  std::deque<Request*> queue;
  std::deque<Request*> ready;  // admitted, waiting for a worker
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> workers;
  std::thread scheduler;
  bool stopping = false;
  int running = 0;
  uint64_t next_id = 1;
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0;
  std::vector<double> latencies;
};

namespace {

void run_request(mrcm_server* S, Request* r, cudaStream_t st) {
  // every exit waits for the request's stream, so that no copy or kernel still touches its arena
  // block when the worker releases it (another request may be admitted to the same bytes)
  struct StreamIdleOnExit {
    cudaStream_t st;
    ~StreamIdleOnExit() { cudaStreamSynchronize(st); }
  } idle_on_exit{st};
  char* base = S->arena_base + r->off;
  const size_t n = r->n;
  const int nx = r->prob.n[0], ny = r->prob.n[1];
  const size_t len = (size_t)std::max(nx, ny);
  size_t o = align256(r->footprint);
  double* K = reinterpret_cast<double*>(base + o);
  o = align256(o + 8 * n);
  double* f = reinterpret_cast<double*>(base + o);
  o = align256(o + 8 * n);
  double* p = reinterpret_cast<double*>(base + o);
  o = align256(o + 8 * n);
  double* bcv = reinterpret_cast<double*>(base + o);
  o = align256(o + 8 * 4 * len);
  double* Ky = reinterpret_cast<double*>(base + o);  // only when the request has a tensor
  mrcm_problem dp = r->prob;
  auto set_err = [&](mrcm_status s, const char* what) {
    r->status = s;
    r->err = std::string(what);
  };
  cudaError_t e = cudaMemcpyAsync(K, r->K.data(), 8 * n, cudaMemcpyHostToDevice, st);
  dp.K = K;
  if (e == cudaSuccess && !r->Ky.empty()) e = cudaMemcpyAsync(Ky, r->Ky.data(), 8 * n, cudaMemcpyHostToDevice, st);
  dp.K_y = r->Ky.empty() ? nullptr : Ky;
  dp.K_z = nullptr;
  if (e == cudaSuccess && !r->f.empty()) e = cudaMemcpyAsync(f, r->f.data(), 8 * n, cudaMemcpyHostToDevice, st);
  dp.f = r->f.empty() ? nullptr : f;
  for (int s = 0; s < 6 && e == cudaSuccess; ++s) {
    if (!r->bc[s].empty() && s < 4) {
      e = cudaMemcpyAsync(bcv + s * len, r->bc[s].data(), 8 * r->bc[s].size(), cudaMemcpyHostToDevice, st);
      dp.bc_val[s] = bcv + s * len;
    } else {
      dp.bc_val[s] = nullptr;
    }
  }
  if (e != cudaSuccess) {
    set_err(MRCM_ERR_CUDA, cudaGetErrorString(e));
    return;
  }
  mrcm_handle h = nullptr;
  mrcm_status s = mrcm_setup(&dp, &r->prm, base, r->footprint, st, &h);
  if (s != MRCM_OK) {
    set_err(s, mrcm_last_error(nullptr));
    return;
  }
  h->cancel = &r->cancel;
  s = mrcm_factor_local(h, st);
  if (s == MRCM_OK) {
    e = cudaMemsetAsync(p, 0, 8 * n, st);
    r->hist.assign(4096, 0.0);
    r->res.history = r->hist.data();
    r->res.history_cap = (int32_t)r->hist.size();
    s = e == cudaSuccess ? mrcm_gmres_solve(h, nullptr, p, nullptr, nullptr, nullptr, &r->res, st) : MRCM_ERR_CUDA;
    r->hist.resize(std::max(0, r->res.history_len));
    if (s == MRCM_OK || s == MRCM_ERR_NOT_CONVERGED) {
      r->p.resize(n);
      e = cudaMemcpyAsync(r->p.data(), p, 8 * n, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = MRCM_ERR_CUDA;
    }
  }
  r->status = s;
  if (s != MRCM_OK) r->err = mrcm_last_error(h);
  cudaStreamSynchronize(st);
  mrcm_destroy(h);
}

void worker_loop(mrcm_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stopping || !S->ready.empty(); });
      if (S->ready.empty()) break;  // stopping and nothing admitted
      r = S->ready.front();
      S->ready.pop_front();
    }
    if (st == nullptr) {
      r->status = MRCM_ERR_CUDA;
      r->err = "could not create a stream";
    } else if (r->cancel) {
      r->status = MRCM_ERR_CANCELLED;
      r->err = "cancelled";
    } else {
      run_request(S, r, st);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->t_done = Clock::now();
      r->state = FINISHED;
      S->arena->release(r->off, r->block);
      S->running--;
      if (r->status == MRCM_OK || r->status == MRCM_ERR_NOT_CONVERGED) {
        S->n_completed++;
        S->latencies.push_back(ms_since(r->t_submit, r->t_done));
      } else {
        S->n_failed++;
      }
    }
    S->cv_sched.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

void scheduler_loop(mrcm_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_sched.wait(lk, [&] { return S->stopping || (!S->queue.empty() && S->running < S->max_inflight); });
    if (S->stopping) break;
    bool admitted = false;
    for (auto it = S->queue.begin(); it != S->queue.end() && S->running < S->max_inflight; ++it) {
      Request* r = *it;
      size_t off = 0;
      if (S->arena->alloc(r->block, &off)) {
        r->off = off;
        r->state = RUNNING;
        r->t_start = Clock::now();
        for (auto jt = S->queue.begin(); jt != it; ++jt) (*jt)->skipped++;
        S->queue.erase(it);
        S->ready.push_back(r);
        S->running++;
        admitted = true;
        break;
      }
      if (r->skipped > 8) break;  // do not backfill past a request that has waited too long
    }
    if (admitted) {
      S->cv_work.notify_one();
      continue;
    }
    // nothing fits now: wait for a completion (or a new request)
    S->cv_sched.wait(lk);
  }
}

}  // namespace

extern "C" {

mrcm_status mrcm_server_create(void* arena, size_t arena_bytes, int32_t max_inflight, mrcm_server_handle* out) {
  if (!out || !arena || arena_bytes == 0 || max_inflight < 1 || max_inflight > 64) return MRCM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return MRCM_ERR_INVALID_ARG;
  auto* S = new (std::nothrow) mrcm_server();
  if (!S) return MRCM_ERR_OOM;
  S->arena_base = static_cast<char*>(arena);
  S->arena.reset(new Arena(arena_bytes));
  S->max_inflight = max_inflight;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return MRCM_ERR_CUDA;
  }
  for (int i = 0; i < max_inflight; ++i) S->workers.emplace_back(worker_loop, S);
  S->scheduler = std::thread(scheduler_loop, S);
  *out = S;
  return MRCM_OK;
}

mrcm_status mrcm_submit(mrcm_server_handle S, const mrcm_problem* problem, const mrcm_params* params, uint64_t* ticket) {
  if (!S || !problem || !params || !ticket || !problem->K) return MRCM_ERR_INVALID_ARG;
  size_t fp = 0;
  mrcm_status s = mrcm_footprint(problem, params, &fp);
  if (s != MRCM_OK) return s;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return MRCM_ERR_OOM;
  r->prob = *problem;
  r->prm = *params;
  r->n = (size_t)problem->n[0] * problem->n[1] * problem->n[2];
  r->footprint = fp;
  const size_t len = (size_t)std::max(problem->n[0], problem->n[1]);
  r->block = align256(fp) + 3 * align256(8 * r->n) + align256(8 * 4 * len) + (problem->K_y ? align256(8 * r->n) : 0);
  if (r->block > S->arena->size()) return MRCM_ERR_OOM;
  r->K.assign(problem->K, problem->K + r->n);
  if (problem->K_y) r->Ky.assign(problem->K_y, problem->K_y + r->n);
  if (problem->f) r->f.assign(problem->f, problem->f + r->n);
  for (int side = 0; side < 4; ++side)
    if (problem->bc_val[side]) {
      const size_t cnt = side < 2 ? (size_t)problem->n[1] : (size_t)problem->n[0];
      r->bc[side].assign(problem->bc_val[side], problem->bc_val[side] + cnt);
    }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    *ticket = r->id;
    S->queue.push_back(r.get());
    S->reqs[r->id] = std::move(r);
    S->n_submitted++;
  }
  S->cv_sched.notify_all();
  return MRCM_OK;
}

mrcm_status mrcm_poll(mrcm_server_handle S, uint64_t ticket, double* p_out, mrcm_result* result, int32_t* done) {
  if (!S || !done) return MRCM_ERR_INVALID_ARG;
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MRCM_ERR_INVALID_ARG;
    if (it->second->state != FINISHED) {
      *done = 0;
      return MRCM_OK;
    }
    r = std::move(it->second);
    S->reqs.erase(it);
  }
  *done = 1;
  if (p_out && !r->p.empty()) std::memcpy(p_out, r->p.data(), 8 * r->p.size());
  if (result) {
    double* keep = result->history;
    const int32_t cap = result->history_cap;
    *result = r->res;
    result->history = keep;
    result->history_cap = cap;
    const int nh = std::min<int>(cap > 0 && keep ? cap : 0, (int)r->hist.size());
    for (int i = 0; i < nh; ++i) keep[i] = r->hist[i];
    result->history_len = nh;
    result->latency_ms = ms_since(r->t_submit, r->t_done);
    result->queue_ms = r->state == FINISHED && r->t_start.time_since_epoch().count() ? ms_since(r->t_submit, r->t_start) : 0.0;
    result->status = r->status;
  }
  if (r->status != MRCM_OK) mrcm::set_thread_error(r->err);
  return r->status;
}

mrcm_status mrcm_cancel(mrcm_server_handle S, uint64_t ticket) {
  if (!S) return MRCM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return MRCM_ERR_INVALID_ARG;
  Request* r = it->second.get();
  r->cancel = 1;
  if (r->state == QUEUED) {
    S->queue.erase(std::find(S->queue.begin(), S->queue.end(), r));
    r->state = FINISHED;
    r->status = MRCM_ERR_CANCELLED;
    r->t_done = Clock::now();
    S->n_failed++;
  }
  return MRCM_OK;
}

mrcm_status mrcm_server_stats(mrcm_server_handle S, int64_t* counts, double* latency_ms, size_t cap, size_t* len,
                              size_t* arena_peak) {
  if (!S) return MRCM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (counts) {
    counts[0] = S->n_submitted;
    counts[1] = (int64_t)S->queue.size();
    counts[2] = S->running;
    counts[3] = S->n_completed;
    counts[4] = S->n_failed;
  }
  if (len) *len = S->latencies.size();
  if (latency_ms) std::memcpy(latency_ms, S->latencies.data(), 8 * std::min(cap, S->latencies.size()));
  if (arena_peak) *arena_peak = S->arena->peak();
  return MRCM_OK;
}

void mrcm_server_destroy(mrcm_server_handle S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    for (Request* r : S->queue) r->cancel = 1;
    S->queue.clear();
  }
  S->cv_sched.notify_all();
  S->cv_work.notify_all();
  if (S->scheduler.joinable()) S->scheduler.join();
  for (auto& t : S->workers)
    if (t.joinable()) t.join();
  delete S;
}

}  // extern "C"

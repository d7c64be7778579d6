// Serving loop: continuous batching of RLOBPCG solves under an HBM budget.
//
// Requests (A on the host, m, n, k, options) join a FIFO queue. A request is admitted when its
// device footprint (plan workspace + a device copy of A) fits in what the budget has left and a
// worker slot is free; each worker owns a CUDA stream. A solve keeps its whole LOBPCG state in
// its plan's device buffers between iterations and releases them (stream-ordered) when it
// finishes, which admits the next request.
//
// Two modes. RLOBPCG_SERVE_STREAMS: each worker runs the whole solve (rlobpcg_solve) on its
// stream; admitted solves overlap on the GPU. RLOBPCG_SERVE_BATCHED: each worker runs its
// request's set-up and outputs on its stream, and the LOBPCG iterations of every admitted small
// solve run together in the batch engine (one thread, one stream, persistent kernels over all
// joined solves, replayed from a captured graph); solves join and leave between replays.
// Requests the batched kernels do not take (complex, block > 5, n > 512, locking, SVQB) run whole
// on their worker. In both modes a result does not depend on what else is running.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  const void* A = nullptr;
  int64_t m = 0, n = 0, lda = 0;
  int k = 0, dtype = 0;
  rlobpcg_opts opts{};
  size_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  bool claimed = false;  // a thread is in rlobpcg_server_wait for this ticket
  bool engine = false;   // its iterations run in the batch engine
  int rc = 0;
  char err[512] = "";  // the worker's last error message when rc != RLOBPCG_OK
  clock_t_::time_point t_arrive, t_start, t_done;
  std::vector<double> sigma, resid;
  std::vector<unsigned char> V;
  rlobpcg_info info{};
};

size_t elem_bytes(int dtype) { return dtype == RLOBPCG_C128 ? 16 : 8; }

}  // namespace

struct rlobpcg_server_s {
  int device = 0;
  int mode = RLOBPCG_SERVE_STREAMS;
  rl::BatchEngine* engine = nullptr;   // batched mode
  std::atomic<int64_t> batch_limit{RLOBPCG_SERVE_BATCH_LIMIT_DEFAULT};   // largest m n b the engine takes
  size_t budget = 0, in_use = 0, peak = 0;
  int max_active = 1, running = 0, peak_running = 0;
  bool stop = false;
  int64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, Request*> all;
  std::vector<double> latencies_ms;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;  // one per worker, created by rlobpcg_server_create
  int waiters = 0;                    // threads inside rlobpcg_server_wait
  clock_t_::time_point t_first{}, t_last{};
  bool any_done = false;
};

namespace {

// Does the batch engine take this request? Batched mode, a shape and options the batched kernels
// run, and m n b at most the server's limit (larger solves keep their own launches, where the Gram
// products run on the tensor cores).
bool routed_to_engine(const rlobpcg_server_s* s, int64_t m, int64_t n, int k, int dtype, const rlobpcg_opts& o) {
  const int b = o.block > 0 ? o.block : k;
  return s->engine && rl::batch_request_eligible(n, k, dtype, o) && m * n * (int64_t)b <= s->batch_limit;
}

// Device footprint of one request: the plan's workspace plus a device copy of A (plus the
// batched iterations' buffers when the batch engine takes it; its plan then has no split of A).
size_t request_bytes(int64_t m, int64_t n, int k, int dtype, rlobpcg_opts o, bool engine) {
  size_t extra = 0;
  if (engine) {
    o.gram_split = 0;
    extra = rl::batch_extra_bytes(m, n, o.block > 0 ? o.block : k);
  }
  const size_t ws = rlobpcg_plan_workspace_size(m, n, k, dtype, &o);
  if (ws == 0) return 0;
  return ws + extra + (((size_t)m * n * elem_bytes(dtype) + 255) & ~(size_t)255);
}

void worker_main(rlobpcg_server_s* s, cudaStream_t st) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || (!s->queue.empty() && s->queue.front()->bytes <= s->budget - s->in_use);
      });
      if (s->stop) break;
      if (s->queue.empty()) continue;
      r = s->queue.front();
      s->queue.pop_front();
      s->in_use += r->bytes;
      s->peak = std::max(s->peak, s->in_use);
      ++s->running;
      s->peak_running = std::max(s->peak_running, s->running);
      r->state = 1;
      r->t_start = clock_t_::now();
    }
    // the solve: plan (stream-ordered workspace), device copy of A, rlobpcg_solve, release
    const size_t esz = elem_bytes(r->dtype);
    rlobpcg_plan_t plan = nullptr;
    void* Ad = nullptr;
    const bool engine = r->engine;
    rlobpcg_opts po = r->opts;
    if (engine) po.gram_split = 0;   // the set-up's one Gram pass on the FP64 cores: no split of A
    int rc = rlobpcg_plan(&plan, r->m, r->n, r->k, r->dtype, &po, st);
    if (rc == RLOBPCG_OK) {
      if (cudaMallocAsync(&Ad, (size_t)r->m * r->n * esz, st) != cudaSuccess) {
        cudaGetLastError();
        rc = RLOBPCG_ERR_OOM;
      }
    }
    if (rc == RLOBPCG_OK) {
      if (cudaMemcpy2DAsync(Ad, r->n * esz, r->A, r->lda * esz, r->n * esz, r->m, cudaMemcpyHostToDevice, st) !=
          cudaSuccess) {
        cudaGetLastError();
        rc = RLOBPCG_ERR_CUDA;
      }
    }
    if (rc == RLOBPCG_OK) {
      if (engine) {
        // set-up here, iterations in the batch engine with every other admitted solve, outputs here
        rl::BatchSolve* h = nullptr;
        rc = rl::batch_solve_setup(plan, (const double*)Ad, r->n, &h);
        if (rc == RLOBPCG_OK) {
          rl::batch_solve_submit(s->engine, h);
          rl::batch_solve_wait(h);
          rc = rl::batch_solve_finish(h, r->sigma.data(), r->V.data(), nullptr, r->resid.data(), &r->info);
        }
      } else {
        rc = rlobpcg_solve(plan, Ad, r->n, -1.0, r->sigma.data(), r->V.data(), nullptr, r->resid.data(), &r->info);
      }
    }
    if (rc < 0) snprintf(r->err, sizeof(r->err), "%s", rlobpcg_last_error());
    if (Ad) cudaFreeAsync(Ad, st);
    rlobpcg_plan_destroy(plan);
    cudaStreamSynchronize(st);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->bytes;
      --s->running;
      r->rc = rc;
      r->state = 2;
      r->t_done = clock_t_::now();
      s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_arrive).count());
      if (!s->any_done || r->t_done > s->t_last) s->t_last = r->t_done;
      s->any_done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

using namespace rl;

extern "C" int rlobpcg_server_create(rlobpcg_server_t* out, size_t hbm_budget_bytes, int max_active, int device) {
  return rlobpcg_server_create_ex(out, hbm_budget_bytes, max_active, device, RLOBPCG_SERVE_STREAMS);
}

extern "C" int rlobpcg_server_create_ex(rlobpcg_server_t* out, size_t hbm_budget_bytes, int max_active, int device,
                                        int mode) {
  const int cap = mode == RLOBPCG_SERVE_BATCHED ? 256 : 64;
  if (!out || hbm_budget_bytes == 0 || max_active < 1 || max_active > cap ||
      (mode != RLOBPCG_SERVE_STREAMS && mode != RLOBPCG_SERVE_BATCHED))
    return RLOBPCG_ERR_INVALID_ARG;
  int ndev = 0;
  RL_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return RLOBPCG_ERR_INVALID_ARG;
  RL_CUDA(cudaSetDevice(device));
  // keep freed pool memory cached up to the budget so that admissions do not go back to the OS
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  auto* s = new rlobpcg_server_s();
  s->device = device;
  s->mode = mode;
  if (mode == RLOBPCG_SERVE_BATCHED) {
    const int rc = rl::batch_engine_create(device, &s->engine);
    if (rc != RLOBPCG_OK) {
      delete s;
      return rc;
    }
  }
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  // every worker's stream exists before any worker starts: a server either has all its slots or
  // is not created
  // batched mode: worker streams (set-ups, outputs) at the highest priority, above the engine's
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int prio = mode == RLOBPCG_SERVE_BATCHED ? greatest : 0;
  for (int i = 0; i < max_active; ++i) {
    cudaStream_t st = nullptr;
    const cudaError_t e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
      for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
      if (s->engine) rl::batch_engine_destroy(s->engine);
      delete s;
      return RLOBPCG_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s, s->streams[i]);
  *out = s;
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_server_submit(rlobpcg_server_t s, const void* A, int64_t m, int64_t n, int64_t lda, int k,
                                     int dtype, const rlobpcg_opts* opts, int64_t* ticket) {
  if (!s || !A || !ticket || lda < n || k < 1 || (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128))
    return RLOBPCG_ERR_INVALID_ARG;
  auto* r = new Request();
  if (opts) r->opts = *opts; else rlobpcg_default_opts(&r->opts);
  r->A = A; r->m = m; r->n = n; r->lda = lda; r->k = k; r->dtype = dtype;
  r->engine = routed_to_engine(s, m, n, k, dtype, r->opts);
  r->bytes = request_bytes(m, n, k, dtype, r->opts, r->engine);
  if (r->bytes == 0) {
    delete r;
    return RLOBPCG_ERR_INVALID_ARG;
  }
  if (r->bytes > s->budget) {
    delete r;
    set_last_error("request larger than the server's HBM budget", __FILE__, __LINE__);
    return RLOBPCG_ERR_OOM;
  }
  r->sigma.resize(k);
  r->resid.resize(k);
  r->V.resize((size_t)n * k * elem_bytes(dtype));
  r->t_arrive = clock_t_::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    if (s->all.empty()) s->t_first = r->t_arrive;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_server_poll(rlobpcg_server_t s, int64_t ticket) {
  if (!s) return RLOBPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return RLOBPCG_ERR_INVALID_ARG;
  return it->second->state;
}

extern "C" int rlobpcg_server_wait(rlobpcg_server_t s, int64_t ticket, double* sigma, void* V, double* resid,
                                   rlobpcg_info* info, double* latency_ms) {
  if (!s) return RLOBPCG_ERR_INVALID_ARG;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    // an unknown ticket, or one another thread is already waiting for
    if (it == s->all.end() || it->second->claimed) return RLOBPCG_ERR_INVALID_ARG;
    r = it->second;
    r->claimed = true;
    ++s->waiters;
    s->cv_done.wait(lk, [&] { return r->state == 2; });
    s->all.erase(ticket);   // look up again: the map may have rehashed while waiting
    --s->waiters;
    // rlobpcg_server_destroy may be waiting for the last waiter to leave; notified under the
    // lock, so that the server cannot be deleted before this thread is done with it
    s->cv_done.notify_all();
  }
  if (sigma) std::copy(r->sigma.begin(), r->sigma.end(), sigma);
  if (resid) std::copy(r->resid.begin(), r->resid.end(), resid);
  if (V) std::copy(r->V.begin(), r->V.end(), (unsigned char*)V);
  if (info) *info = r->info;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_arrive).count();
  const int rc = r->rc;
  if (rc < 0) rl::set_last_error_text(r->err);
  delete r;
  return rc;
}

extern "C" int rlobpcg_server_stats(rlobpcg_server_t s, int64_t* completed, double* p50_ms, double* p99_ms,
                                    double* solves_per_s, size_t* peak_bytes, int* peak_running) {
  if (!s) return RLOBPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> l = s->latencies_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const double x = q * (double)(l.size() - 1);
    const size_t i = (size_t)x;
    const double f = x - (double)i;
    return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
  };
  if (completed) *completed = (int64_t)l.size();
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (solves_per_s) {
    const double span = s->any_done ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    *solves_per_s = span > 0 ? (double)l.size() / span : 0.0;
  }
  if (peak_bytes) *peak_bytes = s->peak;
  if (peak_running) *peak_running = s->peak_running;
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_server_set_batch_limit(rlobpcg_server_t s, int64_t max_mnb) {
  if (!s || max_mnb < 0) return RLOBPCG_ERR_INVALID_ARG;
  s->batch_limit = max_mnb;
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_server_engine_stats(rlobpcg_server_t s, rlobpcg_engine_stats* out) {
  if (!s || !out) return RLOBPCG_ERR_INVALID_ARG;
  if (!s->engine) {
    *out = rlobpcg_engine_stats{};
    return RLOBPCG_OK;
  }
  rl::batch_engine_stats(s->engine, out);
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_server_destroy(rlobpcg_server_t s) {
  if (!s) return RLOBPCG_OK;
  {
    // requests not yet admitted are cancelled: done, with RLOBPCG_ERR_CANCELLED, so that a thread
    // waiting for one of them returns instead of waiting for a worker that will never run it
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    const auto now = clock_t_::now();
    for (Request* r : s->queue) {
      r->state = 2;
      r->rc = RLOBPCG_ERR_CANCELLED;
      r->t_done = now;
      snprintf(r->err, sizeof(r->err), "request cancelled by rlobpcg_server_destroy before it was admitted");
    }
    s->queue.clear();
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  // running solves finish and wake their waiters
  for (auto& t : s->workers) t.join();
  {
    // every waiter has left rlobpcg_server_wait before the server's memory goes away
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->waiters == 0; });
  }
  for (auto& kv : s->all) delete kv.second;
  if (s->engine) rl::batch_engine_destroy(s->engine);   // every batched solve has been waited for
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return RLOBPCG_OK;
}

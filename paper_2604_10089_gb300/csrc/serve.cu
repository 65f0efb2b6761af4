// Batched solves and a continuous-batching solve server.
//
// Each context owns its device state and (with own_stream) its own CUDA
// stream, so contexts are independent: workers (host threads) drive different
// contexts at the same time and their kernels overlap on the GPU.  Results do
// not depend on what else runs (per-context buffers, fixed reduction orders).
//
// lcp_batch_solve: one call solves a set of contexts with a pool of workers.
// lcp_server_*: a long-lived pool that takes solve requests as they arrive
// (continuous batching: a request starts as soon as a worker is free, while
// others are in flight), admits resident contexts against a device-memory
// budget and hands results back by ticket.  Every wait is bounded.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "common.cuh"

extern "C" int lcp_batch_solve(lcp_ctx** ctxs, int count, int method, double tol, double* const* x_dev,
                               lcp_stats* stats, int* statuses, int workers) {
  if (count < 0 || (count > 0 && (!ctxs || !statuses)) || workers < 1 || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN && method != LCP_BB_PGD) return LCP_ERR_INVALID_ARG;
  for (int i = 0; i < count; i++)
    if (!ctxs[i]) return LCP_ERR_INVALID_ARG;
  std::atomic<int> next(0);
  auto work = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) return;
      lcp_ctx* c = ctxs[i];
      if (cudaSetDevice(c->device) != cudaSuccess) {
        statuses[i] = LCP_ERR_CUDA;
        continue;
      }
      lcp_stats st{};
      double* x = (x_dev && x_dev[i]) ? x_dev[i] : c->tmp_n3;
      statuses[i] = lcp_solve_device(c, method, tol, nullptr, x, &st);
      if (stats) stats[i] = st;
    }
  };
  const int nt = workers < count ? workers : (count > 0 ? count : 1);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; t++) pool.emplace_back(work);
  for (auto& th : pool) th.join();
  int worst = LCP_OK;
  for (int i = 0; i < count; i++)
    if (statuses[i] != LCP_OK && worst == LCP_OK) worst = statuses[i];
  return worst;
}

namespace {
struct Request {
  uint64_t ticket;
  lcp_ctx* ctx;
  int method;
  double tol;
};
struct Result {
  int status = LCP_OK;
  lcp_stats st{};
  std::vector<double> x;
};
}  // namespace

struct lcp_server {
  std::mutex mu;
  std::condition_variable cv_q, cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Result> done;
  std::unordered_map<lcp_ctx*, size_t> admitted;   // context -> bytes counted against the budget
  std::unordered_set<lcp_ctx*> busy;               // queued or running
  size_t budget = 0, resident = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> threads;
};

static void server_worker(lcp_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request r;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_q.wait(lock, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop && s->queue.empty()) return;
      r = s->queue.front();
      s->queue.pop_front();
    }
    Result res;
    lcp_ctx* c = r.ctx;
    res.status = lcp_solve_device(c, r.method, r.tol, nullptr, c->tmp_n3, &res.st);
    res.x.resize(c->n);
    if (c->n > 0 && (res.status == LCP_OK || res.status == LCP_ERR_NOT_CONVERGED)) {
      if (cudaMemcpyAsync(res.x.data(), c->tmp_n3, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        res.status = LCP_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->done[r.ticket] = std::move(res);
      s->busy.erase(c);
    }
    s->cv_done.notify_all();
  }
}

extern "C" int lcp_server_create(int workers, size_t hbm_budget_bytes, lcp_server** out) {
  if (!out || workers < 1 || workers > 256) return LCP_ERR_INVALID_ARG;
  lcp_server* s = new (std::nothrow) lcp_server();
  if (!s) return LCP_ERR_OOM;
  s->budget = hbm_budget_bytes;
  cudaGetDevice(&s->device);
  for (int t = 0; t < workers; t++) s->threads.emplace_back(server_worker, s);
  *out = s;
  return LCP_OK;
}

extern "C" void lcp_server_destroy(lcp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_q.notify_all();
  for (auto& th : s->threads) th.join();
  delete s;
}

extern "C" int lcp_server_admit(lcp_server* s, lcp_ctx* ctx) {
  if (!s || !ctx) return LCP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->admitted.count(ctx)) return LCP_OK;
  const size_t need = ctx->bytes;
  if (s->resident + need > s->budget) return LCP_ERR_REJECTED;
  s->admitted[ctx] = need;
  s->resident += need;
  return LCP_OK;
}

extern "C" int lcp_server_release(lcp_server* s, lcp_ctx* ctx) {
  if (!s || !ctx) return LCP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->admitted.find(ctx);
  if (it == s->admitted.end()) return LCP_ERR_INVALID_ARG;
  if (s->busy.count(ctx)) return LCP_ERR_INVALID_ARG;
  s->resident -= it->second;
  s->admitted.erase(it);
  return LCP_OK;
}

extern "C" int lcp_server_submit(lcp_server* s, lcp_ctx* ctx, int method, double tol, uint64_t* ticket) {
  if (!s || !ctx || !ticket || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN && method != LCP_BB_PGD) return LCP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->admitted.count(ctx)) return LCP_ERR_REJECTED;
    if (s->busy.count(ctx)) return LCP_ERR_INVALID_ARG;
    *ticket = s->next_ticket++;
    s->busy.insert(ctx);
    s->queue.push_back(Request{*ticket, ctx, method, tol});
  }
  s->cv_q.notify_one();
  return LCP_OK;
}

extern "C" int lcp_server_poll(lcp_server* s, uint64_t ticket, double* x, int x_len, lcp_stats* st,
                               int timeout_us) {
  if (!s || timeout_us < 0) return LCP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  const bool ready = s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us),
                                         [&] { return s->done.count(ticket) > 0; });
  if (!ready) return LCP_ERR_TIMEOUT;
  Result r = std::move(s->done[ticket]);
  s->done.erase(ticket);
  lock.unlock();
  if (x) {
    if (x_len < (int)r.x.size()) return LCP_ERR_INVALID_ARG;
    for (size_t i = 0; i < r.x.size(); i++) x[i] = r.x[i];
  }
  if (st) *st = r.st;
  return r.status;
}

extern "C" int lcp_server_stats(lcp_server* s, size_t* resident_bytes, int* queued, int* in_flight) {
  if (!s) return LCP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (resident_bytes) *resident_bytes = s->resident;
  if (queued) *queued = (int)s->queue.size();
  if (in_flight) *in_flight = (int)s->busy.size() - (int)s->queue.size();
  return LCP_OK;
}

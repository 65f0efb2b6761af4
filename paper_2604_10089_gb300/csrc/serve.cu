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
  lcp_ctx* ctx;      // caller-owned context, or NULL for a server-owned simulation
  uint64_t sim;      // simulation id when ctx is NULL
  int method;
  double tol;
  double step_dt;    // > 0: advance the simulation by one time step after the solve
};
// A simulation whose context the server owns: created when its estimated
// device footprint fits the budget, kept resident across requests, destroyed
// on close.
struct Sim {
  lcp_config cfg{};
  int M = 0;
  std::vector<double> centers, axes;
  lcp_ctx* ctx = nullptr;
  size_t est = 0;          // estimated device footprint (lcp_footprint_estimate)
  size_t reserved = 0;     // bytes counted against the budget (0: not admitted)
  bool busy = false;       // a request is pending, queued or running
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
  std::deque<Request> queue;                       // admitted, waiting for a worker
  std::deque<Request> held;                        // simulations waiting for budget (FIFO)
  std::unordered_map<uint64_t, Sim> sims;
  uint64_t next_sim = 1;
  std::unordered_map<uint64_t, Result> done;
  std::unordered_map<lcp_ctx*, size_t> admitted;   // context -> bytes counted against the budget
  std::unordered_set<lcp_ctx*> busy;               // queued or running
  size_t budget = 0, resident = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> threads;
};

// Moves held simulation requests to the run queue, first come first served,
// while their estimated footprints fit the budget (caller holds the lock).
static void admit_held(lcp_server* s) {
  while (!s->held.empty()) {
    const Request& h = s->held.front();
    Sim& x = s->sims[h.sim];
    const size_t need = x.reserved ? 0 : x.est;
    if (s->resident + need > s->budget) break;
    x.reserved += need;
    s->resident += need;
    s->queue.push_back(h);
    s->held.pop_front();
  }
}

static void server_worker(lcp_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request r;
    Sim* sim = nullptr;
    lcp_ctx* c = nullptr;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_q.wait(lock, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop && s->queue.empty()) return;
      r = s->queue.front();
      s->queue.pop_front();
      if (r.ctx) {
        c = r.ctx;
      } else {
        sim = &s->sims[r.sim];   // stays valid: a busy simulation is never erased
        c = sim->ctx;
      }
    }
    Result res;
    if (!c) {   // first request of an admitted simulation: create its context
      lcp_ctx* nc = nullptr;
      res.status = lcp_setup(&sim->cfg, sim->M, sim->centers.data(), sim->axes.empty() ? nullptr : sim->axes.data(),
                             0, nullptr, &nc);
      if (res.status == LCP_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        sim->ctx = nc;
        c = nc;
      }
    }
    if (c) {
      res.status = lcp_solve_device(c, r.method, r.tol, nullptr, c->tmp_n3, &res.st);
      res.x.resize(c->n);
      if (c->n > 0 && (res.status == LCP_OK || res.status == LCP_ERR_NOT_CONVERGED)) {
        if (cudaMemcpyAsync(res.x.data(), c->tmp_n3, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
          res.status = LCP_ERR_CUDA;
      }
      if (sim && r.step_dt > 0.0 && res.status == LCP_OK) res.status = lcp_step(c, r.step_dt, nullptr, nullptr);
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (sim) {
        // a context can outgrow its estimate (more contacts than estimated):
        // the excess is counted from now on
        if (c && c->bytes > sim->reserved) {
          s->resident += c->bytes - sim->reserved;
          sim->reserved = c->bytes;
        }
        sim->busy = false;
      } else {
        s->busy.erase(c);
      }
      s->done[r.ticket] = std::move(res);
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
  cudaSetDevice(s->device);
  for (auto& kv : s->sims)
    if (kv.second.ctx) lcp_destroy(kv.second.ctx);
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
  admit_held(s);
  s->cv_q.notify_all();
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
    s->queue.push_back(Request{*ticket, ctx, 0, method, tol, 0.0});
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
  int busy = (int)s->busy.size();
  for (const auto& kv : s->sims) busy += kv.second.busy ? 1 : 0;
  const int waiting = (int)(s->queue.size() + s->held.size());
  if (queued) *queued = waiting;
  if (in_flight) *in_flight = busy - waiting;
  return LCP_OK;
}

// ---------------------------------------------------------------- simulations
extern "C" int lcp_server_open(lcp_server* s, const lcp_config* cfg, int n_bodies, const double* centers,
                               const double* axes, uint64_t* sim) {
  if (!s || !cfg || n_bodies < 1 || !centers || !sim) return LCP_ERR_INVALID_ARG;
  Sim x;
  x.cfg = *cfg;
  x.cfg.own_stream = 1;        // every simulation runs on its own stream
  x.cfg.cuda_stream = nullptr;
  x.M = n_bodies;
  x.centers.assign(centers, centers + 3 * (size_t)n_bodies);
  if (axes) x.axes.assign(axes, axes + 3 * (size_t)n_bodies);
  // contacts are not known before the context exists: six per body bounds the
  // packings of the workloads (contacts grow the estimate only slightly)
  const int st = lcp_footprint_estimate(&x.cfg, n_bodies, 6 * n_bodies, &x.est);
  if (st != LCP_OK) return st;
  std::lock_guard<std::mutex> lock(s->mu);
  *sim = s->next_sim++;
  s->sims.emplace(*sim, std::move(x));
  return LCP_OK;
}

extern "C" int lcp_server_request(lcp_server* s, uint64_t sim, int method, double tol, double step_dt,
                                  uint64_t* ticket) {
  if (!s || !ticket || !(tol >= 0.0) || !(step_dt >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN && method != LCP_BB_PGD) return LCP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end() || it->second.busy) return LCP_ERR_INVALID_ARG;
    Sim& x = it->second;
    if (!x.reserved && x.est > s->budget) return LCP_ERR_REJECTED;   // can never fit
    *ticket = s->next_ticket++;
    x.busy = true;
    const Request r{*ticket, nullptr, sim, method, tol, step_dt};
    if (x.reserved) {
      s->queue.push_back(r);
    } else {
      s->held.push_back(r);   // behind earlier held requests: first come, first admitted
      admit_held(s);
    }
  }
  s->cv_q.notify_all();
  return LCP_OK;
}

extern "C" int lcp_server_close(lcp_server* s, uint64_t sim) {
  if (!s) return LCP_ERR_INVALID_ARG;
  lcp_ctx* ctx = nullptr;
  size_t reserved = 0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end() || it->second.busy) return LCP_ERR_INVALID_ARG;
    ctx = it->second.ctx;
    reserved = it->second.reserved;
    s->sims.erase(it);
  }
  if (ctx) {
    cudaSetDevice(s->device);
    lcp_destroy(ctx);   // the memory is free before its budget is handed on
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->resident -= reserved;
    admit_held(s);
  }
  s->cv_q.notify_all();
  return LCP_OK;
}

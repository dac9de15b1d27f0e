// Request-serving engine for hx_solve (see hx27.h, "serving").  Not part of
// the paper's method: it runs many independent solves of [M + S] p = s
// (Eq. 3) concurrently on one GPU.
//
// Workers are host threads, each owning an hx_ctx and a non-blocking CUDA
// stream, so the kernels of different requests overlap on the device.  A
// single mutex guards the queue, the admission bookkeeping, the model cache
// and the results; solves run outside it.
//
// Admission order (hx_server_config.order): first come, first served, or the
// smallest request (grid points x RHS) first, where a request that has waited
// max_wait_s or longer goes ahead of the rest, oldest first.  The selected
// request (the "head") starts when a worker is free and
//     estimate(head) + sum over other workers of their committed bytes
//                    + bytes of resident models <= budget.
// A worker's committed bytes are the estimate of the request it runs, or of
// the workspace it keeps resident between requests.  When the head does not
// fit, idle workers drop their resident workspaces and unreferenced models
// are evicted (least recently used first) before it waits again.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

#include "hx_context.h"
#include "hx_internal.h"
#include "hx_trace.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Pending {
  int64_t ticket;
  hx_request req;                 // pointers to caller buffers (v_host, wavefield_host)
  std::vector<hx_source> src;     // copied sources
  hx_solve_opts opts;             // copied options
  double est;                     // admission estimate (bytes)
  Clock::time_point t_submit;
  std::shared_ptr<int> cancel;    // the solve's cancel flag (hx_server_cancel)
};

struct Model {
  float* v = nullptr;             // device copy
  size_t bytes = 0;
  int nx = 0, ny = 0, nz = 0;
  int refs = 0;                   // requests using it now
  Clock::time_point last_use;
};

struct Worker {
  hx_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  void* wf = nullptr;             // device wavefield buffer (complex128)
  size_t wf_bytes = 0;
  double committed = 0;           // bytes counted against the budget
  bool busy = false;
  bool drop_cache = false;        // asked to release its resident workspace
  std::thread th;
};

// Device bytes of one request: the solver workspace (Krylov vectors, FP64
// residual, multigrid levels) and the device wavefield, per point * RHS,
// plus per-point level velocities and a fixed margin.
double estimate_bytes(const hx_grid& g, int nrhs, int mode) {
  const double N = (double)g.nx * g.ny * g.nz;
  const double per = mode == HX_SOLVE_FP64 ? 10 * 16 + 16 + 16 + 3 * 16 * 0.15 : 10 * 8 + 16 + 16 + 3 * 8 * 0.15;
  return N * nrhs * per + N * 4 * 0.2 + 64.0 * (1 << 20);
}

}  // namespace

struct hx_server {
  int device = 0;
  double budget = 0;
  int order = 0;                     // 0: first come, first served; 1: smallest first
  double max_wait_s = 0;             // order 1: waits this long or longer go first (0: never)
  std::vector<double> table;
  int n_g = 0;
  double d_inv_g = 0;

  std::mutex mu;
  std::condition_variable cv_work;   // workers: queue / memory changed
  std::condition_variable cv_done;   // waiters: a request completed
  std::deque<Pending> queue;
  std::vector<Worker> workers;
  std::map<std::tuple<uint64_t, int, int, int>, Model> models;   // (id, nx, ny, nz)
  double model_bytes = 0;
  std::map<int64_t, hx_request_result> results;
  std::set<int64_t> outstanding;     // submitted and not yet waited for
  std::map<int64_t, std::shared_ptr<int>> running_flags;   // cancel flags of running requests
  int64_t next_ticket = 0;
  bool stop = false;

  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0;
  double point_rhs = 0, peak_committed = 0;
  int running = 0, max_running = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;

  // the request admission considers next (queue not empty)
  std::deque<Pending>::iterator select_head() {
    if (order == 0) return queue.begin();
    const auto now = Clock::now();
    if (max_wait_s > 0 && std::chrono::duration<double>(now - queue.front().t_submit).count() >= max_wait_s)
      return queue.begin();                      // the queue is in submission order
    auto work = [](const Pending& p) {
      return (double)p.req.grid.nx * p.req.grid.ny * p.req.grid.nz * p.req.nrhs;
    };
    auto best = queue.begin();
    for (auto it = queue.begin(); it != queue.end(); ++it)
      if (work(*it) < work(*best)) best = it;    // ties: the earlier submission
    return best;
  }

  double committed_except(int w) const {
    double c = model_bytes;
    for (size_t i = 0; i < workers.size(); ++i)
      if ((int)i != w) c += workers[i].committed;
    return c;
  }
  // evict unreferenced models (LRU) until `need` bytes fit next to the rest
  void evict_models(double need, int w) {
    while (committed_except(w) + need > budget) {
      auto victim = models.end();
      for (auto it = models.begin(); it != models.end(); ++it)
        if (it->second.refs == 0 && (victim == models.end() || it->second.last_use < victim->second.last_use))
          victim = it;
      if (victim == models.end()) return;
      cudaFree(victim->second.v);
      model_bytes -= (double)victim->second.bytes;
      models.erase(victim);
    }
  }
  void worker_main(int w);
};

namespace {
std::tuple<uint64_t, int, int, int> model_key(const hx_request& r) {
  return std::make_tuple(r.model_id, r.grid.nx, r.grid.ny, r.grid.nz);
}
double model_size(const hx_grid& g) { return 4.0 * g.nx * g.ny * g.nz; }

void release_workspace(Worker& W) {
  W.ctx->solvers.clear();
  W.ctx->solver_lru.clear();
  if (W.wf) cudaFree(W.wf);
  W.wf = nullptr;
  W.wf_bytes = 0;
  W.committed = 0;
}
}  // namespace

void hx_server::worker_main(int w) {
  Worker& W = workers[w];
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // ---- admission of the selected request
    double need = 0;
    std::deque<Pending>::iterator sel;
    for (;;) {
      if (W.drop_cache) {
        release_workspace(W);
        W.drop_cache = false;
        cv_work.notify_all();
      }
      if (queue.empty()) {
        if (stop) return;
        cv_work.wait(lk);
        continue;
      }
      sel = select_head();
      const Pending& head = *sel;
      need = head.est + (models.count(model_key(head.req)) ? 0.0 : model_size(head.req.grid));
      if (committed_except(w) + need <= budget) break;
      evict_models(need, w);
      if (committed_except(w) + need <= budget) break;
      if (W.committed > 0) {                      // this worker is idle: give its cache back
        release_workspace(W);
        continue;
      }
      for (auto& o : workers)
        if (&o != &W && !o.busy && o.committed > 0) o.drop_cache = true;
      cv_work.notify_all();
      cv_work.wait(lk);
    }
    Pending p = std::move(*sel);
    queue.erase(sel);
    running_flags[p.ticket] = p.cancel;
    W.busy = true;
    W.committed = p.est;
    const auto t_start = Clock::now();
    ++running;
    max_running = std::max(max_running, running);
    // ---- the model's device copy (uploaded once per id and grid size)
    Model& m = models[model_key(p.req)];
    int status = HX_OK;
    if (!m.v) {
      m.bytes = (size_t)model_size(p.req.grid);
      m.nx = p.req.grid.nx;
      m.ny = p.req.grid.ny;
      m.nz = p.req.grid.nz;
      cudaError_t e = cudaMalloc(&m.v, m.bytes);
      if (e == cudaSuccess) e = cudaMemcpyAsync(m.v, p.req.v_host, m.bytes, cudaMemcpyHostToDevice, W.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(W.stream);
      if (e != cudaSuccess) {
        if (m.v) cudaFree(m.v);
        models.erase(model_key(p.req));
        status = e == cudaErrorMemoryAllocation ? HX_ERR_OOM : HX_ERR_CUDA;
      } else {
        model_bytes += (double)m.bytes;
      }
    }
    double tot = 0;
    for (auto& o : workers) tot += o.committed;
    peak_committed = std::max(peak_committed, tot + model_bytes);
    const float* vdev = status == HX_OK ? m.v : nullptr;
    if (vdev) ++m.refs;
    lk.unlock();

    // ---- the solve, outside the lock
    hx_solve_report rep;
    std::memset(&rep, 0, sizeof(rep));
    const hx_grid& g = p.req.grid;
    const size_t wfb = (size_t)p.req.nrhs * g.nx * g.ny * g.nz * 16;
    if (status == HX_OK && W.wf_bytes < wfb) {
      if (W.wf) cudaFree(W.wf);
      W.wf = nullptr;
      W.wf_bytes = 0;
      if (cudaMalloc(&W.wf, wfb) == cudaSuccess) W.wf_bytes = wfb;
      else status = HX_ERR_OOM;
    }
    if (status == HX_OK) {
      hx::TraceRange trace_req("served request");
      status = hx_solve(W.ctx, &g, vdev, p.src.data(), (int)p.src.size(), p.req.nrhs, W.wf, &p.opts, &rep,
                        W.stream);
      rep.status = status;
      if (status == HX_OK || status == HX_ERR_NOT_CONVERGED || status == HX_ERR_CANCELLED) {
        cudaError_t e = cudaMemcpyAsync(p.req.wavefield_host, W.wf, wfb, cudaMemcpyDeviceToHost, W.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(W.stream);
        if (e != cudaSuccess) status = HX_ERR_CUDA;
      }
    }
    const auto t_end = Clock::now();

    // ---- bookkeeping
    lk.lock();
    running_flags.erase(p.ticket);
    if (status == HX_ERR_CANCELLED) ++cancelled;
    if (vdev) {
      auto it = models.find(model_key(p.req));
      if (it != models.end()) {
        --it->second.refs;
        it->second.last_use = t_end;
      }
    }
    hx_request_result r;
    std::memset(&r, 0, sizeof(r));
    r.status = status;
    r.report = rep;
    r.queue_ms = ms_between(p.t_submit, t_start);
    r.run_ms = ms_between(t_start, t_end);
    r.latency_ms = ms_between(p.t_submit, t_end);
    r.worker = w;
    results[p.ticket] = r;
    if (status == HX_OK) {
      ++completed;
      lat_ms.push_back(r.latency_ms);
      point_rhs += (double)g.nx * g.ny * g.nz * p.req.nrhs;
    } else {
      ++failed;
    }
    t_last = t_end;
    --running;
    W.busy = false;
    W.committed = W.wf ? p.est : 0.0;             // the workspace stays resident
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

int hx_server_create(hx_server** out, const hx_server_config* cfg) {
  if (!out) return HX_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->slots < 1 || cfg->slots > 64 || !cfg->table || cfg->n_g < 2 || !(cfg->d_inv_g > 0) ||
      cfg->order < 0 || cfg->order > 1 || !(cfg->max_wait_s >= 0))
    return HX_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return HX_ERR_CUDA;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return HX_ERR_CUDA;
  auto* srv = new (std::nothrow) hx_server();
  if (!srv) return HX_ERR_OOM;
  srv->device = cfg->device;
  srv->table.assign(cfg->table, cfg->table + 7 * (size_t)cfg->n_g);
  srv->n_g = cfg->n_g;
  srv->d_inv_g = cfg->d_inv_g;
  srv->order = cfg->order;
  srv->max_wait_s = cfg->max_wait_s;
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
    delete srv;
    return HX_ERR_CUDA;
  }
  srv->budget = cfg->mem_budget > 0 ? cfg->mem_budget : 0.85 * (double)freeb;
  srv->workers.resize(cfg->slots);
  int st = HX_OK;
  for (auto& W : srv->workers) {
    if ((st = hx_ctx_create(&W.ctx, cfg->device)) != HX_OK) break;
    if ((st = hx_set_table(W.ctx, srv->table.data(), srv->n_g, srv->d_inv_g)) != HX_OK) break;
    W.ctx->max_solvers = 1;                     // one resident workspace per worker
    if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess) {
      st = HX_ERR_CUDA;
      break;
    }
  }
  if (st != HX_OK) {
    for (auto& W : srv->workers) {
      if (W.stream) cudaStreamDestroy(W.stream);
      if (W.ctx) hx_ctx_destroy(W.ctx);
    }
    delete srv;
    return st;
  }
  for (int w = 0; w < cfg->slots; ++w) srv->workers[w].th = std::thread(&hx_server::worker_main, srv, w);
  *out = srv;
  return HX_OK;
}

int hx_server_submit(hx_server* srv, const hx_request* req, int64_t* ticket) {
  if (!srv || !req || !ticket) return HX_ERR_ARG;
  *ticket = -1;
  if (hx::check_grid(nullptr, &req->grid) != HX_OK) return HX_ERR_ARG;
  if (!req->v_host || !req->wavefield_host || !req->src || req->nsrc < 1 || req->nrhs < 1 ||
      req->nrhs > 65535)
    return HX_ERR_ARG;
  for (int k = 0; k < req->nsrc; ++k) {
    const hx_source& q = req->src[k];
    if (q.ix < 0 || q.ix >= req->grid.nx || q.iy < 0 || q.iy >= req->grid.ny || q.iz < 0 ||
        q.iz >= req->grid.nz || q.rhs < 0 || q.rhs >= req->nrhs)
      return HX_ERR_ARG;
  }
  Pending p;
  p.req = *req;
  p.src.assign(req->src, req->src + req->nsrc);
  p.req.src = nullptr;
  if (req->opts) p.opts = *req->opts;
  else hx_solve_default_opts(&p.opts);
  p.opts.autotune = 0;                          // results must not depend on timing
  p.cancel = std::make_shared<int>(0);
  p.opts.cancel = p.cancel.get();
  p.est = estimate_bytes(req->grid, req->nrhs, p.opts.mode);
  if (p.est + model_size(req->grid) > srv->budget) return HX_ERR_OOM;
  p.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return HX_ERR_STATE;
  p.ticket = srv->next_ticket++;
  *ticket = p.ticket;
  srv->outstanding.insert(p.ticket);
  if (!srv->have_first) {
    srv->have_first = true;
    srv->t_first = p.t_submit;
  }
  ++srv->submitted;
  srv->queue.push_back(std::move(p));
  srv->cv_work.notify_all();
  return HX_OK;
}

int hx_server_wait(hx_server* srv, int64_t ticket, double timeout_s, hx_request_result* res) {
  if (!srv) return HX_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (!srv->outstanding.count(ticket)) return HX_ERR_ARG;
  auto ready = [&] { return srv->results.count(ticket) > 0; };
  if (timeout_s < 0) {
    srv->cv_done.wait(lk, ready);
  } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return HX_ERR_TIMEOUT;
  }
  const hx_request_result r = srv->results[ticket];
  srv->results.erase(ticket);
  srv->outstanding.erase(ticket);
  if (res) *res = r;
  return r.status;
}

int hx_server_get_stats(hx_server* srv, hx_server_stats* st, int reset) {
  if (!srv || !st) return HX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->failed = srv->failed;
  std::vector<double> l = srv->lat_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const size_t i = (size_t)std::min<double>((double)l.size() - 1, std::ceil(q * l.size()) - 1);
    return l[i];
  };
  st->p50_ms = pct(0.50);
  st->p99_ms = pct(0.99);
  st->max_ms = l.empty() ? 0.0 : l.back();
  st->point_rhs = srv->point_rhs;
  st->busy_s = srv->have_first && srv->completed ? ms_between(srv->t_first, srv->t_last) / 1e3 : 0.0;
  st->peak_committed = srv->peak_committed;
  st->max_concurrent = srv->max_running;
  st->cancelled = srv->cancelled;
  if (reset) {
    srv->submitted = srv->completed = srv->failed = srv->cancelled = 0;
    srv->lat_ms.clear();
    srv->point_rhs = 0;
    srv->peak_committed = 0;
    srv->max_running = srv->running;
    srv->have_first = false;
  }
  return HX_OK;
}

int hx_server_cancel(hx_server* srv, int64_t ticket) {
  if (!srv) return HX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (!srv->outstanding.count(ticket)) return HX_ERR_ARG;
  if (srv->results.count(ticket)) return HX_ERR_STATE;
  auto run = srv->running_flags.find(ticket);
  if (run != srv->running_flags.end()) {
    __atomic_store_n(run->second.get(), 1, __ATOMIC_RELAXED);   // seen at the next check
    return HX_OK;
  }
  for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
    if (it->ticket != ticket) continue;
    hx_request_result r;
    std::memset(&r, 0, sizeof(r));
    r.status = HX_ERR_CANCELLED;
    r.report.status = HX_ERR_CANCELLED;
    r.queue_ms = r.latency_ms = ms_between(it->t_submit, Clock::now());
    r.worker = -1;
    srv->queue.erase(it);
    srv->results[ticket] = r;
    ++srv->failed;
    ++srv->cancelled;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();                  // the next request may be admitted now
    return HX_OK;
  }
  return HX_ERR_STATE;
}

void hx_server_destroy(hx_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  for (auto& W : srv->workers)
    if (W.th.joinable()) W.th.join();
  cudaSetDevice(srv->device);
  for (auto& W : srv->workers) {
    if (W.wf) cudaFree(W.wf);
    if (W.stream) cudaStreamDestroy(W.stream);
    if (W.ctx) hx_ctx_destroy(W.ctx);
  }
  for (auto& kv : srv->models)
    if (kv.second.v) cudaFree(kv.second.v);
  delete srv;
}

}  // extern "C"

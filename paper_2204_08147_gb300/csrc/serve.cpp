// Request loop of the C ABI: continuous admission of estimator requests by device
// footprint, each admitted request running on its own CUDA stream so that requests
// arriving while others run overlap with them on the GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "rdm_api_internal.h"

namespace rdm {

struct Request {
  uint64_t id = 0;
  std::vector<double> jx, jy, jz, hz, gx, betas;
  rdm_model model{};
  HostModel hm;
  int n_v = 0, k = 0;
  uint64_t seed = 0;
  rdm_opts opts{};
  rdm_result* out = nullptr;
  size_t footprint = 0;
  bool packable = false;  // runs its first pass in a packed launch with other requests
  rdm_status status = RDM_OK;
  bool done = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::string error;
};

struct ServeState {
  rdm_ctx* ctx = nullptr;  // the owning context (its autotuner serves the packed launches)
  int device = 0;
  size_t budget = 0, used = 0;
  int max_inflight = 1, inflight = 0;
  int busy_workers = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1;
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First request in arrival order whose footprint fits the free budget.
static std::shared_ptr<Request> take_admissible(ServeState& S) {
  for (auto it = S.queue.begin(); it != S.queue.end(); ++it)
    if (S.used + (*it)->footprint <= S.budget) {
      auto r = *it;
      S.queue.erase(it);
      return r;
    }
  return nullptr;
}

static rdm_status run_request(ServeState& S, Request& r, cudaStream_t st) {
  if (cudaSetDevice(S.device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return RDM_ECUDA;
  }
  rdm_ham ham;
  ham.ctx = nullptr;
  ham.model = r.hm;
  TermImage img;
  make_term_image(r.hm, &img);
  char* mem = nullptr;
  const size_t off = (img.bytes.size() + 255) / 256 * 256;
  if (cudaMallocAsync(reinterpret_cast<void**>(&mem), off + r.footprint, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("request %llu: device allocation of %zu bytes failed", (unsigned long long)r.id,
              off + r.footprint);
    return RDM_ENOMEM;
  }
  bind_terms(img, mem, &ham);
  rdm_status s = RDM_OK;
  if (cudaMemcpyAsync(mem, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    s = RDM_ECUDA;
  if (s == RDM_OK)
    s = estimate_impl(&ham, st, mem + off, r.footprint, r.betas.data(), (int)r.betas.size(), r.n_v,
                      r.k, r.seed, &r.opts, r.out, nullptr);
  else
    set_error("request %llu: term upload failed", (unsigned long long)r.id);
  cudaFreeAsync(mem, st);
  cudaStreamSynchronize(st);
  return s;
}

// A batch of packable requests: their first passes share one packed launch
// (estimate_batch_impl); each request's result is the same as when it runs alone.
static rdm_status run_batch(ServeState& S, std::vector<std::shared_ptr<Request>>& rs, cudaStream_t st,
                            std::vector<rdm_status>& status) {
  if (cudaSetDevice(S.device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return RDM_ECUDA;
  }
  const int n = (int)rs.size();
  std::vector<rdm_ham> hams(n);
  std::vector<TermImage> imgs(n);
  std::vector<rdm_batch_item> items(n);
  std::vector<size_t> avail(n), need(n);
  size_t terms = 0;
  for (int i = 0; i < n; ++i) {
    hams[i].ctx = nullptr;
    hams[i].model = rs[i]->hm;
    make_term_image(rs[i]->hm, &imgs[i]);
    terms += (imgs[i].bytes.size() + 255) / 256 * 256;
    items[i] = rdm_batch_item{&hams[i], rs[i]->betas.data(), (int)rs[i]->betas.size(), rs[i]->n_v, rs[i]->k,
                              rs[i]->seed, rs[i]->opts, rs[i]->out, RDM_OK};
    avail[i] = rs[i]->footprint;
  }
  const size_t ws = batch_workspace_bytes(items.data(), n, avail.data(), need.data());
  if (ws == 0) return RDM_EINVAL;
  char* mem = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&mem), terms + ws, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("batch of %d requests: device allocation of %zu bytes failed", n, terms + ws);
    return RDM_ENOMEM;
  }
  size_t off = 0;
  rdm_status s = RDM_OK;
  for (int i = 0; i < n && s == RDM_OK; ++i) {
    bind_terms(imgs[i], mem + off, &hams[i]);
    if (cudaMemcpyAsync(mem + off, imgs[i].bytes.data(), imgs[i].bytes.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      set_error("batch: term upload failed");
      s = RDM_ECUDA;
    }
    off += (imgs[i].bytes.size() + 255) / 256 * 256;
  }
  if (s == RDM_OK) s = estimate_batch_impl(S.ctx, st, mem + terms, ws, items.data(), n, need.data(), nullptr);
  for (int i = 0; i < n; ++i) status[i] = s == RDM_OK || items[i].status != RDM_OK ? items[i].status : s;
  cudaFreeAsync(mem, st);
  cudaStreamSynchronize(st);  // the term images are pageable host memory
  return s;
}

constexpr int kServeMaxBatch = 64;

static void worker_loop(ServeState* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Request>> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        for (auto& q : S->queue)
          if (S->used + q->footprint <= S->budget) return true;
        return false;
      });
      if (S->stop) break;
      std::shared_ptr<Request> r = take_admissible(*S);
      if (!r) continue;
      // A packable request takes along every other queued packable request that fits
      // the budget now (continuous batching: whatever arrived while others ran).
      batch.push_back(r);
      S->used += r->footprint;
      // share what is queued with the other idle workers: at most a 1/(idle workers)
      // part of the queued packable requests per batch
      int queued = 0;
      for (auto& q : S->queue) queued += q->packable ? 1 : 0;
      const int idle = std::max(1, S->max_inflight - S->busy_workers);
      const int cap = std::min(kServeMaxBatch, 1 + (queued + idle - 1) / idle);
      if (r->packable)
        for (auto it = S->queue.begin(); it != S->queue.end() && (int)batch.size() < cap;) {
          if ((*it)->packable && S->used + (*it)->footprint <= S->budget) {
            S->used += (*it)->footprint;
            batch.push_back(*it);
            it = S->queue.erase(it);
          } else {
            ++it;
          }
        }
      const double t = now_s();
      for (auto& q : batch) q->t_admit = t;
      S->inflight += (int)batch.size();
      S->busy_workers++;
    }
    std::vector<rdm_status> status(batch.size(), RDM_OK);
    if (batch[0]->packable) {
      run_batch(*S, batch, st, status);
    } else {
      status[0] = run_request(*S, *batch[0], st);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const double t = now_s();
      for (size_t i = 0; i < batch.size(); ++i) {
        Request& r = *batch[i];
        r.status = status[i];
        if (status[i] != RDM_OK) r.error = rdm_last_error();
        r.t_done = t;
        r.done = true;
        S->used -= r.footprint;
        S->inflight--;
      }
      S->busy_workers--;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

}  // namespace rdm

rdm_ctx::rdm_ctx() = default;
rdm_ctx::~rdm_ctx() = default;

using namespace rdm;

extern "C" rdm_status rdm_serve_start(rdm_ctx* ctx, size_t budget, int max_inflight) {
  if (!ctx || budget == 0 || max_inflight < 1 || max_inflight > 64) {
    set_error("rdm_serve_start: need ctx, budget > 0 and 1 <= max_inflight <= 64");
    return RDM_EINVAL;
  }
  if (ctx->serve) {
    set_error("rdm_serve_start: already serving");
    return RDM_EINVAL;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("rdm_serve_start: cudaSetDevice failed");
    return RDM_ECUDA;
  }
  // Keep freed request memory in the stream-ordered pool between requests.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
    uint64_t thr = budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  auto S = std::make_unique<ServeState>();
  S->ctx = ctx;
  S->device = ctx->device;
  S->budget = budget;
  S->max_inflight = max_inflight;
  ServeState* raw = S.get();
  ctx->serve = std::move(S);
  for (int i = 0; i < max_inflight; ++i) raw->workers.emplace_back(worker_loop, raw);
  return RDM_OK;
}

extern "C" rdm_status rdm_serve_stop(rdm_ctx* ctx) {
  if (!ctx) {
    set_error("rdm_serve_stop: ctx is NULL");
    return RDM_EINVAL;
  }
  if (!ctx->serve) return RDM_OK;
  ServeState* S = ctx->serve.get();
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // Let queued and running requests finish first.
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->inflight == 0; });
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  ctx->serve.reset();
  return RDM_OK;
}

extern "C" rdm_status rdm_submit(rdm_ctx* ctx, const rdm_model* model, const double* betas,
                                 int n_beta, int n_v, int k, uint64_t seed, const rdm_opts* opts,
                                 rdm_result* out, uint64_t* ticket) {
  if (!ctx || !ctx->serve || !ticket) {
    set_error("rdm_submit: context is not serving (call rdm_serve_start) or ticket is NULL");
    return RDM_EINVAL;
  }
  auto r = std::make_shared<Request>();
  if (!model || model->n_sites < 1 || model->n_sites > 30) {
    set_error("rdm_submit: invalid model");
    return RDM_EINVAL;
  }
  const int n = model->n_sites;
  auto copy = [&](const double* src, std::vector<double>& dst, size_t cnt) -> const double* {
    if (!src) return nullptr;
    dst.assign(src, src + cnt);
    return dst.data();
  };
  r->model = *model;
  r->model.jx = copy(model->jx, r->jx, (size_t)n * n);
  r->model.jy = copy(model->jy, r->jy, (size_t)n * n);
  r->model.jz = copy(model->jz, r->jz, (size_t)n * n);
  r->model.hz = copy(model->hz, r->hz, n);
  r->model.gx = copy(model->gx, r->gx, n);
  rdm_status st = compile_model(&r->model, &r->hm);
  if (st != RDM_OK) return st;
  if (ctx->bath_order) order_bath_bits(&r->hm);  // the same bath order rdm_build_hamiltonian picks
  rdm_ham probe;
  probe.model = r->hm;
  if (n_beta < 1 || !betas) {
    set_error("rdm_submit: need n_beta >= 1 and betas");
    return RDM_EINVAL;
  }
  st = check_estimate_args(&probe, betas, n_beta, opts, out);
  if (st != RDM_OK) return st;
  r->betas.assign(betas, betas + n_beta);
  r->n_v = n_v;
  r->k = k;
  r->seed = seed;
  r->opts = *opts;
  r->out = out;
  ServeState* S = ctx->serve.get();
  // Footprint: all betas in one pass-2 sweep if that takes at most a quarter of
  // the budget, else halve the sweep until it does (results do not depend on it).
  int nbc = n_beta;
  const double bmax = *std::max_element(betas, betas + n_beta);
  size_t fp = estimate_footprint(r->hm, n_beta, n_v, k, opts->precision, opts->vec_dist, opts->passes, nbc,
                                 opts->recurrence, bmax);
  while (nbc > 1 && fp > S->budget / 4) {
    nbc = (nbc + 1) / 2;
    fp = estimate_footprint(r->hm, n_beta, n_v, k, opts->precision, opts->vec_dist, opts->passes, nbc,
                            opts->recurrence, bmax);
  }
  if (fp == 0) return RDM_EINVAL;  // make_plan set the error
  // Small requests keep their Krylov basis and join packed launches (rdm_estimate_batch)
  // when that takes at most a quarter of the budget.
  if (opts->passes != RDM_PASSES_RECOMPUTE) {
    const size_t fs = packed_store_footprint(r->hm, n_beta, n_v, k, opts, bmax);
    if (fs > 0 && fs <= S->budget / 4) {
      fp = fs;
      r->packable = true;
    }
  }
  if (fp > S->budget) {
    set_error("rdm_submit: request needs %zu bytes, serving budget is %zu", fp, S->budget);
    return RDM_ENOMEM;
  }
  r->footprint = fp;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->queue.push_back(r);
  }
  S->cv_work.notify_all();
  *ticket = r->id;
  return RDM_OK;
}

static rdm_status report(Request& r, rdm_status* status_out) {
  if (status_out) *status_out = r.status;
  if (r.status != RDM_OK) set_error("%s", r.error.c_str());
  return RDM_OK;
}

extern "C" rdm_status rdm_poll(rdm_ctx* ctx, uint64_t ticket, rdm_status* status_out) {
  return rdm_wait(ctx, ticket, 0, status_out);
}

extern "C" rdm_status rdm_wait(rdm_ctx* ctx, uint64_t ticket, int timeout_ms,
                               rdm_status* status_out) {
  if (!ctx || !ctx->serve) {
    set_error("rdm_wait: context is not serving");
    return RDM_EINVAL;
  }
  ServeState* S = ctx->serve.get();
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return RDM_ENOTFOUND;
  }
  auto r = it->second;
  if (!r->done) {
    if (timeout_ms == 0) return RDM_EBUSY;
    if (timeout_ms < 0)
      S->cv_done.wait(lk, [&] { return r->done; });
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
      return RDM_ETIMEOUT;
  }
  return report(*r, status_out);
}

extern "C" rdm_status rdm_request_times(rdm_ctx* ctx, uint64_t ticket, double* latency_s,
                                        double* queued_s) {
  if (!ctx || !ctx->serve) {
    set_error("rdm_request_times: context is not serving");
    return RDM_EINVAL;
  }
  ServeState* S = ctx->serve.get();
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return RDM_ENOTFOUND;
  }
  if (!it->second->done) return RDM_EBUSY;
  if (latency_s) *latency_s = it->second->t_done - it->second->t_submit;
  if (queued_s) *queued_s = it->second->t_admit - it->second->t_submit;
  return RDM_OK;
}

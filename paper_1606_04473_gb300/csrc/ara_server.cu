// Request server: many risk queries (portfolios of layers over a resident pool of ELTs, each on
// a slice of a resident YET) served concurrently on one GPU.  This is the single-GPU form of the
// paper's many tenants sharing GPUs (Section V-D): the ELTs stay resident across requests,
// requests are admitted first-come first-served whenever a worker is free and their estimated
// device memory fits the budget (continuous admission as earlier requests finish and release
// memory), and admitted requests run on separate streams so their transfers and kernels
// overlap on the device.  Every request's computation is the deterministic single-request path,
// so its results do not depend on what else is running.

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

struct Request {
  int64_t ticket = 0;
  std::vector<int32_t> layer_off, layer_elts;
  std::vector<double> occ_ret, occ_lim, agg_ret, agg_lim, rps, levels;
  int64_t t0 = 0, t1 = 0;
  int32_t want_mean = 0, want_adjoint = 0, flags = 0, tenant = 0;
  double adjoint_level = 0.99;
  int64_t mem = 0;
  // results
  ara_status status = ARA_OK;
  std::vector<double> pml, tvar, mean, grad_layer;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace ara

using namespace ara;

struct ara_server {
  Portfolio* pool = nullptr;
  const int64_t* d_off = nullptr;
  const int32_t* d_ids = nullptr;
  int64_t n_trials = 0, n_events = 0;
  int64_t budget = 0, in_use = 0, peak_in_use = 0;
  int32_t max_concurrent = 0, running = 0, peak_running = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<int64_t, std::shared_ptr<Request>> by_ticket;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_ticket = 1;
};

namespace {

// Device memory a request may hold at once (upper estimate).
int64_t estimate_bytes(const Portfolio& pool, const Request& r) {
  const int64_t nl = (int64_t)r.layer_off.size() - 1, n = r.t1 - r.t0, C = pool.catalogue;
  int64_t b = nl * (8 * C + 4 * (pool.bm_words + pool.cbits_stride)) + 4096 * nl;   // layer set
  b += nl * n * 9;                                                                  // YLT + regimes
  b += 8192 * (int64_t)(r.rps.size() + r.levels.size() + 2) * nl + (1 << 20);       // selection
  if (r.flags & ARA_RUN_BATCHED) {
    int64_t bound = 0;
    for (int32_t j : r.layer_elts) bound += pool.rec_off[j + 1] - pool.rec_off[j];
    b += 12 * C + 8 * bound;
  }
  if (r.want_adjoint) {
    int64_t recs = 0;
    for (int32_t j : r.layer_elts) recs += pool.rec_off[j + 1] - pool.rec_off[j];
    b += 14 * C + 4 * pool.bm_words + 16 * recs + 64 * (int64_t)r.layer_elts.size() + 64 * nl;
  }
  return b;
}

void run_request(ara_server& S, Request& r, cudaStream_t s) {
  const int32_t nl = (int32_t)r.layer_off.size() - 1;
  const int64_t n = r.t1 - r.t0;
  ara_portfolio* ls = nullptr;
  double* ylt = nullptr;
  uint8_t* reg = nullptr;
  ara_status st = ara_create_layer_set(static_cast<ara_portfolio*>(S.pool), nl, r.layer_off.data(),
                                       r.layer_elts.data(), r.occ_ret.data(), r.occ_lim.data(),
                                       r.agg_ret.data(), r.agg_lim.data(), s, &ls);
  if (st == ARA_OK && cudaMallocAsync((void**)&ylt, 8 * (size_t)nl * n, s) != cudaSuccess) st = ARA_ENOMEM;
  if (st == ARA_OK && r.want_adjoint &&
      cudaMallocAsync((void**)&reg, (size_t)nl * n, s) != cudaSuccess)
    st = ARA_ENOMEM;
  if (st == ARA_OK)
    st = ara_run_ylt(ls, n, S.d_off + r.t0, S.n_events, S.d_ids, nullptr, 0, nullptr, ylt, reg,
                     r.flags, s);
  if (st == ARA_OK && (!r.rps.empty() || !r.levels.empty() || r.want_mean)) {
    r.pml.assign((size_t)nl * r.rps.size(), 0.0);
    r.tvar.assign((size_t)nl * r.levels.size(), 0.0);
    r.mean.assign(r.want_mean ? (size_t)nl : 0, 0.0);
    st = risk_metrics_device(ylt, n, nl, (int32_t)r.rps.size(), r.rps.data(), (int32_t)r.levels.size(),
                             r.levels.data(), r.pml.data(), r.tvar.data(),
                             r.want_mean ? r.mean.data() : nullptr, s);
  }
  if (st == ARA_OK && r.want_adjoint) {
    int64_t K = 0, M = 0;
    for (int32_t j : r.layer_elts) {
      ++K;
      M += S.pool->rec_off[j + 1] - S.pool->rec_off[j];
    }
    double *ge = nullptr, *gl = nullptr, *gx = nullptr;
    if (cudaMallocAsync((void**)&ge, 8 * (size_t)std::max<int64_t>(4 * K, 1), s) != cudaSuccess ||
        cudaMallocAsync((void**)&gl, 8 * (size_t)(8 * nl), s) != cudaSuccess ||
        cudaMallocAsync((void**)&gx, 8 * (size_t)std::max<int64_t>(2 * M, 1), s) != cudaSuccess) {
      st = ARA_ENOMEM;
    } else {
      st = ara_adjoint(ls, n, S.d_off + r.t0, S.n_events, S.d_ids, 0, nullptr, ylt, reg,
                       r.adjoint_level, ge, gl, gx, nullptr, s);
      if (st == ARA_OK) {
        r.grad_layer.assign((size_t)8 * nl, 0.0);
        if (cudaMemcpyAsync(r.grad_layer.data(), gl, 8 * (size_t)(8 * nl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          st = ARA_ECUDA;
      }
    }
    if (ge) cudaFreeAsync(ge, s);
    if (gl) cudaFreeAsync(gl, s);
    if (gx) cudaFreeAsync(gx, s);
  }
  if (st == ARA_OK) st = ara_check(ls, s);
  if (ylt) cudaFreeAsync(ylt, s);
  if (reg) cudaFreeAsync(reg, s);
  if (ls) ara_destroy_portfolio(ls);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
  r.status = st;
}

void worker_main(ara_server* S) {
  DeviceGuard g(S->pool->device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop && S->pending.empty()) return true;
        if (S->pending.empty()) return false;
        // first come, first served: the head of the queue is admitted when it fits, or when
        // nothing else is running (a request larger than the budget still runs, alone)
        const int64_t need = S->pending.front()->mem;
        return S->running == 0 || S->in_use + need <= S->budget;
      });
      if (S->pending.empty()) break;
      r = S->pending.front();
      S->pending.pop_front();
      S->in_use += r->mem;
      S->running += 1;
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->peak_running = std::max(S->peak_running, S->running);
    }
    r->t_start = now_s();
    if (s) run_request(*S, *r, s);
    else r->status = ARA_ECUDA;
    r->t_done = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= r->mem;
      S->running -= 1;
      r->done = true;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

ara_status ara_server_create(ara_portfolio* pool, int64_t n_trials, const int64_t* d_off,
                             int64_t n_events, const int32_t* d_ids, int32_t max_concurrent,
                             int64_t memory_budget, ara_server** out) {
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  if (!pool || pool->borrowed_elts || n_trials < 1 || n_events < 0 || !d_off ||
      (n_events > 0 && !d_ids) || max_concurrent < 1 || max_concurrent > 64)
    return ARA_EINVAL;
  ara_server* S = new (std::nothrow) ara_server();
  if (!S) return ARA_ENOMEM;
  S->pool = pool;
  S->d_off = d_off;
  S->d_ids = d_ids;
  S->n_trials = n_trials;
  S->n_events = n_events;
  S->max_concurrent = max_concurrent;
  if (memory_budget <= 0) {
    DeviceGuard g(pool->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete S;
      return ARA_ECUDA;
    }
    memory_budget = (int64_t)(0.8 * (double)free_b);
  }
  S->budget = memory_budget;
  for (int i = 0; i < max_concurrent; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return ARA_OK;
}

ara_status ara_server_submit(ara_server* S, const ara_query* q, int64_t* ticket) {
  if (!S || !q || !ticket) return ARA_EINVAL;
  const Portfolio& pool = *S->pool;
  if (q->n_layers < 1 || !q->layer_elt_offsets || q->trial_begin < 0 ||
      q->trial_end <= q->trial_begin || q->trial_end > S->n_trials)
    return ARA_EINVAL;
  if (q->n_rp < 0 || q->n_tvar < 0 || (q->n_rp > 0 && !q->return_periods) ||
      (q->n_tvar > 0 && !q->tvar_levels))
    return ARA_EINVAL;
  const int32_t nl = q->n_layers;
  auto r = std::make_shared<Request>();
  r->layer_off.assign(q->layer_elt_offsets, q->layer_elt_offsets + nl + 1);
  if (r->layer_off[0] != 0) return ARA_EINVAL;
  for (int32_t l = 0; l < nl; ++l)
    if (r->layer_off[l + 1] < r->layer_off[l]) return ARA_EINVAL;
  if (r->layer_off[nl] > 0 && !q->layer_elt_ids) return ARA_EINVAL;
  r->layer_elts.assign(q->layer_elt_ids, q->layer_elt_ids + r->layer_off[nl]);
  for (int32_t j : r->layer_elts)
    if (j < 0 || j >= pool.n_elts) return ARA_EINVAL;
  if (!q->occ_ret || !q->occ_lim || !q->agg_ret || !q->agg_lim) return ARA_EINVAL;
  r->occ_ret.assign(q->occ_ret, q->occ_ret + nl);
  r->occ_lim.assign(q->occ_lim, q->occ_lim + nl);
  r->agg_ret.assign(q->agg_ret, q->agg_ret + nl);
  r->agg_lim.assign(q->agg_lim, q->agg_lim + nl);
  r->rps.assign(q->return_periods, q->return_periods + q->n_rp);
  r->levels.assign(q->tvar_levels, q->tvar_levels + q->n_tvar);
  r->t0 = q->trial_begin;
  r->t1 = q->trial_end;
  r->want_mean = q->want_mean;
  r->want_adjoint = q->want_adjoint;
  r->adjoint_level = q->adjoint_level;
  r->flags = q->flags;
  r->tenant = q->tenant;
  if (validate_metrics(r->t1 - r->t0, (int32_t)r->rps.size(), r->rps.data(), (int32_t)r->levels.size(),
                       r->levels.data()) != ARA_OK)
    return ARA_EINVAL;
  if (r->want_adjoint && tail_count_snap(r->t1 - r->t0, r->adjoint_level) < 1) return ARA_EINVAL;
  if (r->flags & ~(ARA_RUN_BATCHED | ARA_RUN_LDG | ARA_RUN_NO_FILTER)) return ARA_EINVAL;
  r->mem = estimate_bytes(pool, *r);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return ARA_EBUSY;
    r->ticket = S->next_ticket++;
    S->by_ticket[r->ticket] = r;
    S->pending.push_back(r);
  }
  *ticket = r->ticket;
  S->cv_work.notify_one();
  return ARA_OK;
}

ara_status ara_server_wait(ara_server* S, int64_t ticket, double* h_pml, double* h_tvar,
                           double* h_mean, double* h_grad_layer, double* h_times) {
  if (!S) return ARA_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return ARA_EINVAL;
    r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    S->by_ticket.erase(ticket);
  }
  if (r->status == ARA_OK) {
    if (h_pml) std::copy(r->pml.begin(), r->pml.end(), h_pml);
    if (h_tvar) std::copy(r->tvar.begin(), r->tvar.end(), h_tvar);
    if (h_mean) std::copy(r->mean.begin(), r->mean.end(), h_mean);
    if (h_grad_layer) std::copy(r->grad_layer.begin(), r->grad_layer.end(), h_grad_layer);
  }
  if (h_times) {
    h_times[0] = r->t_start - r->t_submit;   // queued
    h_times[1] = r->t_done - r->t_start;     // running
    h_times[2] = r->t_done - r->t_submit;    // latency
  }
  return r->status;
}

ara_status ara_server_stats(ara_server* S, int32_t* queued_or_running, int32_t* peak_running,
                            int64_t* peak_bytes, int64_t* budget) {
  if (!S) return ARA_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (queued_or_running) *queued_or_running = (int32_t)S->pending.size() + S->running;
  if (peak_running) *peak_running = S->peak_running;
  if (peak_bytes) *peak_bytes = S->peak_in_use;
  if (budget) *budget = S->budget;
  return ARA_OK;
}

void ara_server_destroy(ara_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"

// Request server: many risk queries (portfolios of layers over a resident pool of ELTs, each on
// a slice of a resident YET) served concurrently on one GPU.  This is the single-GPU form of the
// paper's many tenants sharing GPUs (Section V-D): the ELTs stay resident across requests, and
// requests are admitted whenever a worker is free and their estimated device memory fits, both
// under the server's budget and within the device memory free at that moment (continuous
// admission as earlier requests finish and release memory).  A free worker takes the oldest
// queued request (or, when that one does not fit, a later one that does, a bounded number of
// times) and merges into it up to three more queued requests whose trial slices overlap the
// group's: their layers run in one batched pass over the union of the slices, each trial
// walking only the table entries of the requests that cover it, so overlapping requests share
// the reading of the YET.  Admitted groups run on separate streams, so their transfers and
// kernels overlap on the device.  Every request's arithmetic is exact or deterministic (integer
// trial sums, an exact selection, integer adjoint counts), so its results do not depend on what
// else is running or on the group it ran in.

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
  int64_t table_bound = 0;   // upper bound of its batched table: 8 B per record of its layers' ELTs
  int32_t passed = 0;     // times a later request was admitted ahead of this one
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
  // merging: at most max_merge requests per pass; a queued request joins a group when its
  // slice's overlap with the group's slice is at least min_overlap of their union
  int32_t max_merge = 4;
  double min_overlap = 0.6;
  int32_t window = 32;        // queued requests examined for a group or to pass a blocked head
  int32_t max_passed = 4;     // a blocked head is passed at most this many times
  // A group's event-major table is kept near L2 size: merged passes whose table far exceeds it
  // were measured slower than their requests run one after the other.  Bounded by 8 bytes per
  // record of every layer's ELTs (an upper bound of the table's entries).
  int64_t max_table_bytes = 192ll << 20;
  int64_t n_passes = 0, n_merged = 0, n_head_passed = 0;
  // Event-major index of the resident YET (ara_server_set_adjoint_index), or null: adjoint
  // requests whose slice covers at least half of the index blocks it touches read it instead of
  // the YET (the indexed pass reads those blocks whole).
  ara_yet_index* yx = nullptr;
  int64_t n_indexed = 0;
  // The YET passes (batched or single-layer streams, adjoint histograms) of different workers
  // run one after the other on the device: each waits for the previous one's completion event.
  // Concurrent passes each hold a large table in L2 and slow each other down; everything else
  // (folds, selections, host work) still overlaps.
  std::mutex pass_mu;
  cudaEvent_t pass_done = nullptr;
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
  {   // batched table (every request may run in a merged batched pass)
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

// Queue one YET pass on `s` behind the previous pass of any worker.
template <typename F>
ara_status chained_pass(ara_server& S, cudaStream_t s, F&& launch) {
  std::lock_guard<std::mutex> lk(S.pass_mu);
  if (S.pass_done && cudaStreamWaitEvent(s, S.pass_done, 0) != cudaSuccess) return ARA_ECUDA;
  const ara_status st = launch();
  if (S.pass_done && cudaEventRecord(S.pass_done, s) != cudaSuccess && st == ARA_OK) return ARA_ECUDA;
  return st;
}

// The metrics and the adjoint of one request whose YLT (and regimes) are computed: its layers are
// the layer set's layers [slot0, slot0 + nl), its trials [r.t0, r.t1) of the resident YET.
ara_status finish_request(ara_server& S, Request& r, ara_portfolio* ls, int32_t slot0, double* ylt,
                          uint8_t* reg, cudaStream_t s) {
  const int32_t nl = (int32_t)r.layer_off.size() - 1;
  const int64_t n = r.t1 - r.t0;
  ara_status st = ARA_OK;
  if (!r.rps.empty() || !r.levels.empty() || r.want_mean) {
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
    std::vector<int32_t> sel(nl);
    for (int32_t i = 0; i < nl; ++i) sel[i] = slot0 + i;
    double *ge = nullptr, *gl = nullptr, *gx = nullptr;
    if (dmalloc_async((void**)&ge, 8 * (size_t)std::max<int64_t>(4 * K, 1), s) != cudaSuccess ||
        dmalloc_async((void**)&gl, 8 * (size_t)(8 * nl), s) != cudaSuccess ||
        dmalloc_async((void**)&gx, 8 * (size_t)std::max<int64_t>(2 * M, 1), s) != cudaSuccess) {
      st = ARA_ENOMEM;
    } else {
      bool indexed = false;
      if (S.yx) {
        const int64_t B = S.yx->block;
        const int64_t span = ((r.t1 - 1) / B - r.t0 / B + 1) * B;
        indexed = 2 * n >= span;
      }
      st = chained_pass(S, s, [&] {
        if (indexed)
          return ara_adjoint_indexed(ls, S.yx, r.t0, n, nl, sel.data(), ylt, reg, r.adjoint_level,
                                     ge, gl, gx, nullptr, s);
        return ara_adjoint(ls, n, S.d_off + r.t0, S.n_events, S.d_ids, nl, sel.data(), ylt, reg,
                           r.adjoint_level, ge, gl, gx, nullptr, s);
      });
      if (indexed) {
        std::lock_guard<std::mutex> lk(S.mu);
        ++S.n_indexed;
      }
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
  return st;
}

void mark_done(ara_server& S, Request& r, ara_status st) {
  r.status = st;
  r.t_done = now_s();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    r.done = true;
  }
  S.cv_done.notify_all();
}

// One request on its own: its own layer set and the ordinary path (ARA_RUN_BATCHED or the
// single-layer stream, as the query asks).
void run_request(ara_server& S, Request& r, cudaStream_t s) {
  const int32_t nl = (int32_t)r.layer_off.size() - 1;
  const int64_t n = r.t1 - r.t0;
  ara_portfolio* ls = nullptr;
  double* ylt = nullptr;
  uint8_t* reg = nullptr;
  ara_status st = ara_create_layer_set(static_cast<ara_portfolio*>(S.pool), nl, r.layer_off.data(),
                                       r.layer_elts.data(), r.occ_ret.data(), r.occ_lim.data(),
                                       r.agg_ret.data(), r.agg_lim.data(), s, &ls);
  if (st == ARA_OK && dmalloc_async((void**)&ylt, 8 * (size_t)nl * n, s) != cudaSuccess) st = ARA_ENOMEM;
  if (st == ARA_OK && r.want_adjoint &&
      dmalloc_async((void**)&reg, (size_t)nl * n, s) != cudaSuccess)
    st = ARA_ENOMEM;
  if (st == ARA_OK)
    st = chained_pass(S, s, [&] {
      return ara_run_ylt(ls, n, S.d_off + r.t0, S.n_events, S.d_ids, nullptr, 0, nullptr, ylt, reg,
                         r.flags, s);
    });
  if (st == ARA_OK) st = finish_request(S, r, ls, 0, ylt, reg, s);
  if (st == ARA_OK) st = ara_check(ls, s);
  if (ylt) cudaFreeAsync(ylt, s);
  if (reg) cudaFreeAsync(reg, s);
  if (ls) ara_destroy_portfolio(ls);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
  mark_done(S, r, st);
}

// Several requests in one pass: one layer set holding every request's layers (request k's at the
// slots [first[k], first[k + 1])), one batched pass over the union of their trial slices, then
// each request's metrics and adjoint from its own YLT.  Each request is marked done as soon as
// its own results are in.
void run_group(ara_server& S, std::vector<std::shared_ptr<Request>>& g, cudaStream_t s) {
  const int nr = (int)g.size();
  GroupArgs ga;
  ga.n_req = nr;
  std::vector<int32_t> loff{0}, lel;
  std::vector<double> oR, oL, aR, aL;
  int64_t u0 = g[0]->t0, u1 = g[0]->t1;
  for (int k = 0; k < nr; ++k) {
    const Request& r = *g[k];
    const int32_t nl = (int32_t)r.layer_off.size() - 1;
    for (int32_t l = 0; l < nl; ++l) loff.push_back(loff.back() + r.layer_off[l + 1] - r.layer_off[l]);
    lel.insert(lel.end(), r.layer_elts.begin(), r.layer_elts.end());
    oR.insert(oR.end(), r.occ_ret.begin(), r.occ_ret.end());
    oL.insert(oL.end(), r.occ_lim.begin(), r.occ_lim.end());
    aR.insert(aR.end(), r.agg_ret.begin(), r.agg_ret.end());
    aL.insert(aL.end(), r.agg_lim.begin(), r.agg_lim.end());
    ga.slot_first[k + 1] = ga.slot_first[k] + nl;
    u0 = std::min(u0, r.t0);
    u1 = std::max(u1, r.t1);
  }
  ara_portfolio* ls = nullptr;
  ara_status st = ara_create_layer_set(static_cast<ara_portfolio*>(S.pool), ga.slot_first[nr],
                                       loff.data(), lel.data(), oR.data(), oL.data(), aR.data(),
                                       aL.data(), s, &ls);
  ga.n_trials = u1 - u0;
  ga.offsets = S.d_off + u0;
  ga.n_events = S.n_events;
  ga.ids = S.d_ids;
  for (int k = 0; k < nr && st == ARA_OK; ++k) {
    const Request& r = *g[k];
    const int64_t nl = (int64_t)r.layer_off.size() - 1, n = r.t1 - r.t0;
    ga.t0[k] = r.t0 - u0;
    ga.t1[k] = r.t1 - u0;
    if (dmalloc_async((void**)&ga.ylt[k], 8 * (size_t)(nl * n), s) != cudaSuccess ||
        (r.want_adjoint && dmalloc_async((void**)&ga.reg[k], (size_t)(nl * n), s) != cudaSuccess))
      st = ARA_ENOMEM;
  }
  if (st == ARA_OK)
    st = chained_pass(S, s, [&] { return run_batched_group_async(*static_cast<Portfolio*>(ls), ga, s); });
  if (st == ARA_OK) st = ara_check(ls, s);
  for (int k = 0; k < nr; ++k) {
    ara_status sk = st;
    if (sk == ARA_OK) sk = finish_request(S, *g[k], ls, ga.slot_first[k], ga.ylt[k], ga.reg[k], s);
    if (sk == ARA_OK && cudaStreamSynchronize(s) != cudaSuccess) sk = ARA_ECUDA;
    mark_done(S, *g[k], sk);
  }
  for (int k = 0; k < nr; ++k) {
    if (ga.ylt[k]) cudaFreeAsync(ga.ylt[k], s);
    if (ga.reg[k]) cudaFreeAsync(ga.reg[k], s);
  }
  if (ls) ara_destroy_portfolio(ls);
  cudaStreamSynchronize(s);
}

// Device memory that admission may still hand out: the budget left, and no more than the device
// has free now plus what the library's memory pool holds idle (reusable by the requests), less
// what admitted requests may still allocate.
int64_t admissible_bytes(ara_server& S) {
  int64_t avail = S.budget - S.in_use;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
    avail = std::min(avail, (int64_t)(0.95 * (double)free_b) + pool_idle_bytes(S.pool->device) - S.in_use);
  return avail;
}

int64_t overlap(int64_t a0, int64_t a1, int64_t b0, int64_t b1) {
  return std::max<int64_t>(0, std::min(a1, b1) - std::max(a0, b0));
}

// Choose the next group under the lock: the oldest request if it fits (or if nothing runs), else
// the first of the next `window` requests that fits, unless the oldest has already been passed
// max_passed times; then up to max_merge - 1 more requests of the window whose slices overlap the
// group's by at least min_overlap of the union, best overlap first, while the memory fits.
// Returns an empty group when nothing can be admitted now.
std::vector<std::shared_ptr<Request>> pick_group(ara_server& S) {
  std::vector<std::shared_ptr<Request>> g;
  if (S.pending.empty()) return g;
  // the oldest request runs even when it does not fit if nothing else runs (alone); every other
  // request, and every request merged into a group, must fit
  const int64_t avail = admissible_bytes(S);
  size_t lead = 0;
  if (S.pending[0]->mem > avail && S.running > 0) {
    if (S.pending[0]->passed >= S.max_passed) return g;
    lead = SIZE_MAX;
    for (size_t i = 1; i < S.pending.size() && i < (size_t)S.window; ++i)
      if (S.pending[i]->mem <= avail) { lead = i; break; }
    if (lead == SIZE_MAX) return g;
    S.pending[0]->passed += 1;
    S.n_head_passed += 1;
  }
  g.push_back(S.pending[lead]);
  S.pending.erase(S.pending.begin() + (long)lead);
  int64_t mem = g[0]->mem;
  int64_t table = g[0]->table_bound;
  int32_t slots = (int32_t)g[0]->layer_off.size() - 1;
  int64_t u0 = g[0]->t0, u1 = g[0]->t1;
  while ((int)g.size() < std::min(S.max_merge, (int)BT_MAX_REQ)) {
    size_t best = SIZE_MAX;
    double best_ov = 0.0;
    for (size_t i = 0; i < S.pending.size() && i < (size_t)S.window; ++i) {
      const Request& c = *S.pending[i];
      const int32_t nl = (int32_t)c.layer_off.size() - 1;
      if (slots + nl > 255 || mem + c.mem > avail || table + c.table_bound > S.max_table_bytes)
        continue;
      const int64_t ov = overlap(u0, u1, c.t0, c.t1);
      const double frac = (double)ov / (double)(std::max(u1, c.t1) - std::min(u0, c.t0));
      if (ov > 0 && frac >= S.min_overlap && frac > best_ov) { best = i; best_ov = frac; }
    }
    if (best == SIZE_MAX) break;
    std::shared_ptr<Request> c = S.pending[best];
    S.pending.erase(S.pending.begin() + (long)best);
    mem += c->mem;
    table += c->table_bound;
    slots += (int32_t)c->layer_off.size() - 1;
    u0 = std::min(u0, c->t0);
    u1 = std::max(u1, c->t1);
    g.push_back(c);
  }
  return g;
}

void worker_main(ara_server* S) {
  DeviceGuard dg(S->pool->device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  while (true) {
    std::vector<std::shared_ptr<Request>> g;
    int64_t mem = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop && S->pending.empty()) return true;
        g = pick_group(*S);
        return !g.empty();
      });
      if (g.empty()) break;
      for (auto& r : g) mem += r->mem;
      S->in_use += mem;
      S->running += (int32_t)g.size();
      S->n_passes += 1;
      if (g.size() > 1) S->n_merged += (int64_t)g.size();
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->peak_running = std::max(S->peak_running, S->running);
    }
    const double t = now_s();
    for (auto& r : g) r->t_start = t;
    if (!s) {
      for (auto& r : g) mark_done(*S, *r, ARA_ECUDA);
    } else if (g.size() == 1) {
      run_request(*S, *g[0], s);
    } else {
      run_group(*S, g, s);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= mem;
      S->running -= (int32_t)g.size();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (s) cudaStreamDestroy(s);
}

// Warm-up at creation: two small requests with every output (metrics and adjoint) run alone,
// batched, and merged, so that the first real requests pay no one-time costs (kernel loading,
// the stream-ordered allocator's first reservations).
ara_status warm_up(ara_server& S) {
  if (S.pool->n_elts < 1) return ARA_OK;
  cudaStream_t s = nullptr;
  ARA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  std::vector<std::shared_ptr<Request>> rs;
  ara_status st = ARA_OK;
  const int64_t n = std::min<int64_t>(S.n_trials, 256);
  for (int k = 0; k < 3; ++k) {
    auto r = std::make_shared<Request>();
    r->layer_off = {0, 1};
    r->layer_elts = {std::min(k, S.pool->n_elts - 1)};
    r->occ_ret = {0.0};
    r->occ_lim = {1e300};
    r->agg_ret = {0.0};
    r->agg_lim = {1e300};
    r->rps = {1.0};
    r->levels = {0.5};
    r->want_mean = 1;
    r->want_adjoint = tail_count_snap(n, 0.5) >= 1 ? 1 : 0;
    r->adjoint_level = 0.5;
    r->t0 = 0;
    r->t1 = n;
    r->flags = k == 0 ? 0 : ARA_RUN_BATCHED;
    rs.push_back(r);
  }
  run_request(S, *rs[0], s);
  run_request(S, *rs[1], s);
  std::vector<std::shared_ptr<Request>> g{rs[1], rs[2]};
  run_group(S, g, s);
  for (auto& r : rs)
    if (r->status != ARA_OK && st == ARA_OK) st = r->status;
  cudaStreamDestroy(s);
  return st;
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
  {
    DeviceGuard g(pool->device);
    if (cudaEventCreateWithFlags(&S->pass_done, cudaEventDisableTiming) != cudaSuccess) {
      delete S;
      return ARA_ECUDA;
    }
    const ara_status st = warm_up(*S);
    if (st != ARA_OK) {
      cudaEventDestroy(S->pass_done);
      delete S;
      return st;
    }
  }
  for (int i = 0; i < max_concurrent; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return ARA_OK;
}

}  // extern "C"

namespace {
// Validate a query and copy it into a request (no ticket, not queued).
ara_status make_request(ara_server* S, const ara_query* q, std::shared_ptr<Request>& out) {
  if (!S || !q) return ARA_EINVAL;
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
  for (int32_t j : r->layer_elts) r->table_bound += 8 * (pool.rec_off[j + 1] - pool.rec_off[j]);
  out = r;
  return ARA_OK;
}
}  // namespace

extern "C" {

ara_status ara_server_estimate_bytes(ara_server* S, const ara_query* q, int64_t* bytes) {
  if (!bytes) return ARA_EINVAL;
  std::shared_ptr<Request> r;
  const ara_status st = make_request(S, q, r);
  if (st != ARA_OK) return st;
  *bytes = r->mem;
  return ARA_OK;
}

ara_status ara_server_submit(ara_server* S, const ara_query* q, int64_t* ticket) {
  if (!ticket) return ARA_EINVAL;
  std::shared_ptr<Request> r;
  const ara_status st = make_request(S, q, r);
  if (st != ARA_OK) return st;
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

ara_status ara_server_set_merging(ara_server* S, int32_t max_requests_per_pass, double min_overlap) {
  if (!S || max_requests_per_pass < 1 || max_requests_per_pass > BT_MAX_REQ || !(min_overlap > 0.0) ||
      min_overlap > 1.0)
    return ARA_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_merge = max_requests_per_pass;
  S->min_overlap = min_overlap;
  return ARA_OK;
}

ara_status ara_server_set_adjoint_index(ara_server* S, int32_t on) {
  if (!S) return ARA_EINVAL;
  // Held throughout: no worker can take a request (nor read S->yx) while the index changes.
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->pending.empty() || S->running > 0) return ARA_EBUSY;
  DeviceGuard g(S->pool->device);
  if (!on) {
    ara_yet_index_destroy(S->yx);
    S->yx = nullptr;
    return ARA_OK;
  }
  if (S->yx) return ARA_OK;
  ara_yet_index* yx = nullptr;
  const ara_status st = ara_yet_index_create(static_cast<ara_portfolio*>(S->pool), S->n_trials,
                                             S->d_off, S->n_events, S->d_ids, nullptr, &yx);
  if (st != ARA_OK) return st;
  S->yx = yx;
  return ARA_OK;
}

ara_status ara_server_counters(ara_server* S, int64_t* passes, int64_t* merged_requests,
                               int64_t* head_passed, int64_t* indexed_adjoints) {
  if (!S) return ARA_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (passes) *passes = S->n_passes;
  if (merged_requests) *merged_requests = S->n_merged;
  if (head_passed) *head_passed = S->n_head_passed;
  if (indexed_adjoints) *indexed_adjoints = S->n_indexed;
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
  {
    DeviceGuard g(S->pool->device);
    if (S->pass_done) cudaEventDestroy(S->pass_done);
  }
  ara_yet_index_destroy(S->yx);
  delete S;
}

}  // extern "C"

// C ABI of libara: argument validation, portfolio lifecycle, dispatch of the YLT path
// (Algorithm 1 around Algorithm 3), the host-input pipeline (Algorithm 2's transfer
// overlapped with Algorithm 3's kernels), data-error reporting and timing.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

std::atomic<int64_t> g_launches{0};

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("ARA_DEBUG"))
    fprintf(stderr, "libara: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}

// ------------------------------------------------------------------------------------------
// Timing: event pairs per kernel class, recorded on the launching stream.
// ------------------------------------------------------------------------------------------
namespace {
struct TimedLaunch {
  cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimedLaunch> g_pending[ARA_K_COUNT];
std::vector<cudaEvent_t> g_event_pool;
double g_total_ms[ARA_K_COUNT];
int64_t g_count[ARA_K_COUNT];
thread_local cudaEvent_t t_open[ARA_K_COUNT];

cudaEvent_t get_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

ara_status drain(int k) {
  for (auto& tl : g_pending[k]) {
    float ms = 0.f;
    if (cudaEventSynchronize(tl.b) != cudaSuccess) return ARA_ECUDA;
    if (cudaEventElapsedTime(&ms, tl.a, tl.b) != cudaSuccess) return ARA_ECUDA;
    g_total_ms[k] += ms;
    g_count[k] += 1;
    g_event_pool.push_back(tl.a);
    g_event_pool.push_back(tl.b);
  }
  g_pending[k].clear();
  return ARA_OK;
}
}  // namespace

void timing_begin(int k, cudaStream_t s) {
  if (!g_timing) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t e = get_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) t_open[k] = e; else t_open[k] = nullptr;
}

void timing_end(int k, cudaStream_t s) {
  if (!g_timing || !t_open[k]) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t e = get_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) g_pending[k].push_back({t_open[k], e});
  t_open[k] = nullptr;
  if (g_pending[k].size() > 4096) drain(k);
}

void timing_add_host(int k, double ms) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_timing) return;
  g_total_ms[k] += ms;
  g_count[k] += 1;
}

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices];
}  // namespace

static cudaMemPool_t library_pool(int dev) {
  if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t mp = nullptr;
    if (cudaMemPoolCreate(&mp, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;   // keep freed memory until ara_release_memory
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = mp;
  }
  return g_pools[dev];
}

cudaError_t dmalloc_async(void** ptr, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t mp = library_pool(dev);
  if (!mp) return cudaMallocAsync(ptr, bytes, s);
  return cudaMallocFromPoolAsync(ptr, bytes, mp, s);
}

int64_t pool_idle_bytes(int dev) {
  if (dev < 0 || dev >= kMaxPoolDevices) return 0;
  cudaMemPool_t mp;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    mp = g_pools[dev];
  }
  if (!mp) return 0;
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(mp, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(mp, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
    return 0;
  return reserved > used ? (int64_t)(reserved - used) : 0;
}

bool timing_suspend() {
  std::lock_guard<std::mutex> lk(g_tmu);
  const bool was = g_timing;
  g_timing = false;
  return was;
}

void timing_resume(bool was_on) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_timing = was_on;
}

// ------------------------------------------------------------------------------------------
// Validation helpers
// ------------------------------------------------------------------------------------------
static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }
static bool limit_ok(double v) { return !std::isnan(v) && v >= 0.0; }  // +inf allowed

// Round a non-negative double to the nearest integer as a saturated unsigned 128-bit value.
static void to_u128(double v, uint64_t& lo, uint64_t& hi) {
  const double two64 = 18446744073709551616.0;
  if (!(v < 170141183460469231731687303715884105728.0)) {  // >= 2^127 or inf: saturate
    lo = ~0ull;
    hi = 0x7fffffffffffffffull;
    return;
  }
  v = std::nearbyint(v);
  hi = (uint64_t)std::floor(v / two64);
  lo = (uint64_t)(v - (double)hi * two64);
}

// Fixed-point scale of a layer: o(e) <= B, where B bounds the occurrence loss through the
// monotonicity of every clamp: s(e) <= sum_j C(max_loss_j; R_j, L_j), o(e) <= C(that; OccR, OccL).
static void layer_scale(Portfolio& pf, LayerConst& lc) {
  double sum = 0.0;
  for (int k = lc.elt_begin; k < lc.elt_end; ++k) {
    const int j = pf.layer_elts[k];
    double a = pf.elt_max_loss[j] - pf.elt_ret[j];
    a = a < 0.0 ? 0.0 : (a > pf.elt_lim[j] ? pf.elt_lim[j] : a);
    sum += a;
  }
  double b = sum - lc.occ_ret;
  b = b < 0.0 ? 0.0 : (b > lc.occ_lim ? lc.occ_lim : b);
  b = b * (1.0 + 1e-9) + 1e-300;  // margin for the device's own rounding of the same sums
  int ex = 0;
  std::frexp(b, &ex);             // b < 2^ex
  int fb = 55 - ex;               // q = o * 2^fb < 2^55 (8 bits free for a layer slot)
  fb = std::max(-1000, std::min(1000, fb));
  lc.frac_bits = fb;
  lc.scale = std::ldexp(1.0, fb);
  lc.inv_scale = std::ldexp(1.0, -fb);
  to_u128(lc.agg_ret * lc.scale, lc.agg_ret_lo, lc.agg_ret_hi);
  to_u128(lc.agg_lim * lc.scale, lc.agg_lim_lo, lc.agg_lim_hi);
}

static void free_portfolio(ara_portfolio* p) {
  if (!p) return;
  if (p->borrowed_elts) {
    // a layer set: its own buffers came from the stream-ordered allocator; the ELT tables
    // belong to the pool
    void* own[] = {p->d_layer_elts, p->d_layers, p->d_q, p->d_bits, p->d_cbits, p->d_err};
    for (void* q : own)
      if (q) cudaFreeAsync(q, p->owner_stream);
    void* staged[] = {p->d_stage_ids[0], p->d_stage_ids[1], p->d_stage_off[0], p->d_stage_off[1],
                      p->d_ylt_full};
    for (void* q : staged)
      if (q) cudaFree(q);
  } else {
    void* ptrs[] = {p->d_rec_off, p->d_rec_ids, p->d_rec_orig, p->d_rec_loss, p->d_rec_loss32,
                    p->d_elt_ret, p->d_elt_lim, p->d_tile_rec, p->d_layer_elts, p->d_layers, p->d_dense, p->d_q,
                    p->d_bits, p->d_cbits, p->d_err, p->d_stage_ids[0], p->d_stage_ids[1],
                    p->d_stage_off[0], p->d_stage_off[1], p->d_ylt_full};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  if (p->d_res) cudaFree(p->d_res);
  if (p->h_res) cudaFreeHost(p->h_res);
  void* alt[] = {p->d_q_alt, p->d_bits_alt, p->d_cbits_alt};
  for (void* q : alt)
    if (q) cudaFree(q);
  if (p->d_sel_scratch) cudaFree(p->d_sel_scratch);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
    if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
  }
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  delete p;
}

template <typename T>
static ara_status upload(T** dst, const T* src, size_t n) {
  if (n == 0) return ARA_OK;
  ARA_TRY(cudaMalloc((void**)dst, n * sizeof(T)));
  ARA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return ARA_OK;
}

}  // namespace ara

using namespace ara;

extern "C" {

const char* ara_status_string(ara_status s) {
  switch (s) {
    case ARA_OK: return "ok";
    case ARA_EINVAL: return "invalid argument";
    case ARA_ENOMEM: return "out of memory";
    case ARA_ECUDA: return "CUDA error";
    case ARA_ETIMEOUT: return "device wait timed out";
    case ARA_EBUSY: return "busy";
    case ARA_EDATA: return "device-side data check failed";
    case ARA_ERANGE: return "request exceeds a fixed capacity";
    default: return "unknown status";
  }
}

int64_t ara_launch_count(void) { return g_launches.load(); }

int32_t ara_stream_shapes(int32_t* warps, int32_t* stages, int32_t max) {
  const int32_t n = n_bulk_shapes();
  for (int32_t i = 0; i < n && i < max; ++i) bulk_shape(i, warps + i, stages + i);
  return n;
}

ara_status ara_debug_set(int32_t key, int64_t value) {
  switch (key) {
    case ARA_DBG_WAIT_LIMIT_NS:
      if (value < 1000) return ARA_EINVAL;
      set_wait_limit_ns((uint64_t)value);
      return ARA_OK;
    case ARA_DBG_STARVE_COPIES:
      if (value < 0 || value > 4096 || (value & 15)) return ARA_EINVAL;
      set_debug_extra_tx((uint32_t)value);
      return ARA_OK;
    case ARA_DBG_SKIP_BARRIER_ARRIVAL:
      if (value != 0 && value != 1) return ARA_EINVAL;
      set_debug_skip_arrival((int32_t)value);
      return ARA_OK;
    case ARA_DBG_ADJOINT_PER_LAYER:
      if (value != 0 && value != 1) return ARA_EINVAL;
      set_adjoint_per_layer((int32_t)value);
      return ARA_OK;
    default:
      return ARA_EINVAL;
  }
}

ara_status ara_set_stream_shape(int32_t index) {
  if (index < 0 || index >= n_bulk_shapes()) return ARA_EINVAL;
  set_bulk_shape(index);
  return ARA_OK;
}

ara_status ara_release_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  ara_status st = ARA_OK;
  for (int d = 0; d < kMaxPoolDevices; ++d)
    if (g_pools[d] && cudaMemPoolTrimTo(g_pools[d], 0) != cudaSuccess) st = ARA_ECUDA;
  return st;
}

void ara_timing_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_timing = on != 0;
}

void ara_timing_reset(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  for (int k = 0; k < ARA_K_COUNT; ++k) {
    drain(k);
    g_total_ms[k] = 0.0;
    g_count[k] = 0;
  }
}

ara_status ara_timing_read(int32_t k, double* total_ms, int64_t* launches) {
  if (k < 0 || k >= ARA_K_COUNT || !total_ms || !launches) return ARA_EINVAL;
  std::lock_guard<std::mutex> lk(g_tmu);
  ara_status st = drain(k);
  *total_ms = g_total_ms[k];
  *launches = g_count[k];
  return st;
}

ara_status ara_create_portfolio(int64_t C, int32_t n_elts, const int64_t* rec_off,
                                const int32_t* rec_ids, const double* rec_loss,
                                const double* elt_ret, const double* elt_lim, int32_t n_layers,
                                const int32_t* layer_off, const int32_t* layer_elts,
                                const double* occ_ret, const double* occ_lim,
                                const double* agg_ret, const double* agg_lim, int32_t flags,
                                ara_portfolio** out) {
  // ---- validation (host only; nothing is allocated before it passes) ----
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  if (C < 1 || C > 2147483647LL || n_elts < 0 || n_layers < 0) return ARA_EINVAL;
  if (flags & ~(ARA_LOSSES_F32 | ARA_DENSE_TABLES)) return ARA_EINVAL;
  if (!rec_off) return ARA_EINVAL;
  if (n_elts > 0 && (!elt_ret || !elt_lim)) return ARA_EINVAL;
  if (n_layers > 0 && (!layer_off || !occ_ret || !occ_lim || !agg_ret || !agg_lim))
    return ARA_EINVAL;
  if (rec_off[0] != 0) return ARA_EINVAL;
  for (int32_t j = 0; j < n_elts; ++j)
    if (rec_off[j + 1] < rec_off[j]) return ARA_EINVAL;
  const int64_t n_rec = rec_off[n_elts];
  if (n_rec > 0 && (!rec_ids || !rec_loss)) return ARA_EINVAL;
  const bool f32 = (flags & ARA_LOSSES_F32) != 0;
  for (int64_t r = 0; r < n_rec; ++r) {
    if (rec_ids[r] < 0 || rec_ids[r] >= C) return ARA_EINVAL;
    if (!finite_nonneg(rec_loss[r])) return ARA_EINVAL;
    if (f32 && (double)(float)rec_loss[r] != rec_loss[r]) return ARA_EINVAL;
  }
  for (int32_t j = 0; j < n_elts; ++j)
    if (!finite_nonneg(elt_ret[j]) || !limit_ok(elt_lim[j])) return ARA_EINVAL;
  if (n_layers > 0) {
    if (layer_off[0] != 0) return ARA_EINVAL;
    for (int32_t l = 0; l < n_layers; ++l) {
      if (layer_off[l + 1] < layer_off[l]) return ARA_EINVAL;
      if (!finite_nonneg(occ_ret[l]) || !limit_ok(occ_lim[l]) || !finite_nonneg(agg_ret[l]) ||
          !limit_ok(agg_lim[l]))
        return ARA_EINVAL;
    }
    if (layer_off[n_layers] > 0 && !layer_elts) return ARA_EINVAL;
    for (int32_t k = 0; k < layer_off[n_layers]; ++k)
      if (layer_elts[k] < 0 || layer_elts[k] >= n_elts) return ARA_EINVAL;
  }
  // records sorted by event ID within each ELT; duplicates rejected
  std::vector<int32_t> ids_sorted((size_t)n_rec);
  std::vector<int32_t> orig_pos((size_t)n_rec);
  std::vector<double> loss_sorted((size_t)n_rec);
  std::vector<double> max_loss((size_t)n_elts, 0.0);
  {
    std::vector<int64_t> idx;
    for (int32_t j = 0; j < n_elts; ++j) {
      const int64_t a = rec_off[j], b = rec_off[j + 1];
      idx.resize((size_t)(b - a));
      std::iota(idx.begin(), idx.end(), a);
      std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return rec_ids[x] < rec_ids[y]; });
      for (int64_t i = 0; i < b - a; ++i) {
        ids_sorted[(size_t)(a + i)] = rec_ids[idx[(size_t)i]];
        orig_pos[(size_t)(a + i)] = (int32_t)(idx[(size_t)i] - a);
        loss_sorted[(size_t)(a + i)] = rec_loss[idx[(size_t)i]];
        max_loss[(size_t)j] = std::max(max_loss[(size_t)j], rec_loss[idx[(size_t)i]]);
        if (i > 0 && ids_sorted[(size_t)(a + i)] == ids_sorted[(size_t)(a + i - 1)]) return ARA_EINVAL;
      }
    }
  }
  // ---- build ----
  ara_portfolio* p = new (std::nothrow) ara_portfolio();
  if (!p) return ARA_ENOMEM;
  auto fail = [&](ara_status st) {
    free_portfolio(p);
    return st;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(ARA_ECUDA);
  if (cudaDeviceGetAttribute(&p->n_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    return fail(ARA_ECUDA);
  if (cudaDeviceGetAttribute(&p->max_smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                             p->device) != cudaSuccess)
    return fail(ARA_ECUDA);
  p->catalogue = C;
  p->n_elts = n_elts;
  p->n_layers = n_layers;
  p->flags = flags;
  p->n_records = n_rec;
  p->rec_off.assign(rec_off, rec_off + n_elts + 1);
  if (n_elts > 0) {
    p->elt_ret.assign(elt_ret, elt_ret + n_elts);
    p->elt_lim.assign(elt_lim, elt_lim + n_elts);
  }
  p->elt_max_loss = max_loss;
  p->layer_off.assign(1, 0);
  if (n_layers > 0) p->layer_off.assign(layer_off, layer_off + n_layers + 1);
  if (n_layers > 0 && layer_off[n_layers] > 0)
    p->layer_elts.assign(layer_elts, layer_elts + layer_off[n_layers]);
  p->layers.resize((size_t)n_layers);
  for (int32_t l = 0; l < n_layers; ++l) {
    LayerConst& lc = p->layers[(size_t)l];
    memset(&lc, 0, sizeof(lc));
    lc.occ_ret = occ_ret[l];
    lc.occ_lim = occ_lim[l];
    lc.agg_ret = agg_ret[l];
    lc.agg_lim = agg_lim[l];
    lc.elt_begin = layer_off[l];
    lc.elt_end = layer_off[l + 1];
    layer_scale(*p, lc);
  }
  ara_status st;
  if ((st = upload(&p->d_rec_off, rec_off, (size_t)n_elts + 1)) != ARA_OK) return fail(st);
  if ((st = upload(&p->d_rec_ids, ids_sorted.data(), (size_t)n_rec)) != ARA_OK) return fail(st);
  if ((st = upload(&p->d_rec_orig, orig_pos.data(), (size_t)n_rec)) != ARA_OK) return fail(st);
  if (f32) {
    std::vector<float> l32(loss_sorted.begin(), loss_sorted.end());
    if ((st = upload(&p->d_rec_loss32, l32.data(), (size_t)n_rec)) != ARA_OK) return fail(st);
  } else if ((st = upload(&p->d_rec_loss, loss_sorted.data(), (size_t)n_rec)) != ARA_OK) {
    return fail(st);
  }
  {   // per ELT, the first record of every fold tile (records are sorted by event ID)
    p->n_tiles = (C + FOLD_TILE - 1) / FOLD_TILE;
    const int64_t nt1 = p->n_tiles + 1;
    std::vector<int64_t> tile_rec((size_t)std::max<int64_t>(1, (int64_t)n_elts * nt1));
    for (int32_t j = 0; j < n_elts; ++j) {
      int64_t r = rec_off[j];
      for (int64_t t = 0; t < nt1; ++t) {
        while (r < rec_off[j + 1] && (int64_t)ids_sorted[(size_t)r] < t * FOLD_TILE) ++r;
        tile_rec[(size_t)(j * nt1 + t)] = r;
      }
    }
    if ((st = upload(&p->d_tile_rec, tile_rec.data(), tile_rec.size())) != ARA_OK) return fail(st);
  }
  if ((st = upload(&p->d_elt_ret, elt_ret, (size_t)n_elts)) != ARA_OK) return fail(st);
  if ((st = upload(&p->d_elt_lim, elt_lim, (size_t)n_elts)) != ARA_OK) return fail(st);
  if ((st = upload(&p->d_layer_elts, p->layer_elts.data(), p->layer_elts.size())) != ARA_OK)
    return fail(st);
  if ((st = upload(&p->d_layers, p->layers.data(), p->layers.size())) != ARA_OK) return fail(st);
  p->bm_words = ((C + 31) / 32 + 3) / 4 * 4;
  p->cbits_stride = (((C + 1) / 2 + 31) / 32 + 3) / 4 * 4;   // coarsest needed: 1 bit per 2 events
  if (n_layers > 0) {
    if (cudaMalloc(&p->d_q, sizeof(uint64_t) * (size_t)n_layers * C) != cudaSuccess) return fail(ARA_ENOMEM);
    if (cudaMalloc(&p->d_bits, 4 * (size_t)n_layers * p->bm_words) != cudaSuccess) return fail(ARA_ENOMEM);
    if (cudaMemset(p->d_bits, 0, 4 * (size_t)n_layers * p->bm_words) != cudaSuccess) return fail(ARA_ECUDA);
    if (cudaMalloc(&p->d_cbits, 4 * (size_t)n_layers * p->cbits_stride) != cudaSuccess) return fail(ARA_ENOMEM);
  }
  if (cudaMalloc(&p->d_err, sizeof(uint32_t)) != cudaSuccess) return fail(ARA_ENOMEM);
  if (cudaMemset(p->d_err, 0, sizeof(uint32_t)) != cudaSuccess) return fail(ARA_ECUDA);
  if (flags & ARA_DENSE_TABLES) {
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    if (cudaMalloc(&p->d_dense, esz * (size_t)std::max(n_elts, 1) * C) != cudaSuccess) return fail(ARA_ENOMEM);
    if ((st = build_dense(*p, 0)) != ARA_OK) return fail(st);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(ARA_ECUDA);
  *out = p;
  return ARA_OK;
}

void ara_destroy_portfolio(ara_portfolio* pf) {
  if (!pf) return;
  DeviceGuard g(pf->device);
  if (pf->borrowed_elts) cudaStreamSynchronize(pf->owner_stream);
  else cudaDeviceSynchronize();
  free_portfolio(pf);
}

static ara_status validate_layers(const Portfolio& pool, int32_t n_layers, const int32_t* layer_off,
                                  const int32_t* layer_elts, const double* occ_ret,
                                  const double* occ_lim, const double* agg_ret,
                                  const double* agg_lim) {
  if (n_layers < 1 || !layer_off || !occ_ret || !occ_lim || !agg_ret || !agg_lim) return ARA_EINVAL;
  if (layer_off[0] != 0) return ARA_EINVAL;
  for (int32_t l = 0; l < n_layers; ++l) {
    if (layer_off[l + 1] < layer_off[l]) return ARA_EINVAL;
    if (!finite_nonneg(occ_ret[l]) || !limit_ok(occ_lim[l]) || !finite_nonneg(agg_ret[l]) ||
        !limit_ok(agg_lim[l]))
      return ARA_EINVAL;
  }
  if (layer_off[n_layers] > 0 && !layer_elts) return ARA_EINVAL;
  for (int32_t k = 0; k < layer_off[n_layers]; ++k)
    if (layer_elts[k] < 0 || layer_elts[k] >= pool.n_elts) return ARA_EINVAL;
  return ARA_OK;
}

ara_status ara_create_layer_set(ara_portfolio* pool, int32_t n_layers, const int32_t* layer_off,
                                const int32_t* layer_elts, const double* occ_ret,
                                const double* occ_lim, const double* agg_ret, const double* agg_lim,
                                void* stream, ara_portfolio** out) {
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  if (!pool || pool->borrowed_elts) return ARA_EINVAL;
  ara_status st = validate_layers(*pool, n_layers, layer_off, layer_elts, occ_ret, occ_lim, agg_ret, agg_lim);
  if (st != ARA_OK) return st;
  ara_portfolio* p = new (std::nothrow) ara_portfolio();
  if (!p) return ARA_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  p->borrowed_elts = true;
  p->owner_stream = s;
  p->device = pool->device;
  p->n_sms = pool->n_sms;
  p->max_smem_block = pool->max_smem_block;
  p->catalogue = pool->catalogue;
  p->n_elts = pool->n_elts;
  p->n_layers = n_layers;
  p->flags = pool->flags;
  p->n_records = pool->n_records;
  p->rec_off = pool->rec_off;
  p->elt_ret = pool->elt_ret;
  p->elt_lim = pool->elt_lim;
  p->elt_max_loss = pool->elt_max_loss;
  p->d_rec_off = pool->d_rec_off;
  p->d_rec_ids = pool->d_rec_ids;
  p->d_rec_orig = pool->d_rec_orig;
  p->d_rec_loss = pool->d_rec_loss;
  p->d_rec_loss32 = pool->d_rec_loss32;
  p->d_elt_ret = pool->d_elt_ret;
  p->d_elt_lim = pool->d_elt_lim;
  p->n_tiles = pool->n_tiles;
  p->d_tile_rec = pool->d_tile_rec;
  p->d_dense = pool->d_dense;
  p->layer_off.assign(layer_off, layer_off + n_layers + 1);
  p->layer_elts.assign(layer_elts, layer_elts + layer_off[n_layers]);
  p->layers.resize((size_t)n_layers);
  for (int32_t l = 0; l < n_layers; ++l) {
    LayerConst& lc = p->layers[(size_t)l];
    memset(&lc, 0, sizeof(lc));
    lc.occ_ret = occ_ret[l];
    lc.occ_lim = occ_lim[l];
    lc.agg_ret = agg_ret[l];
    lc.agg_lim = agg_lim[l];
    lc.elt_begin = layer_off[l];
    lc.elt_end = layer_off[l + 1];
    layer_scale(*p, lc);
  }
  DeviceGuard g(p->device);
  const int64_t C = p->catalogue;
  p->bm_words = pool->bm_words;
  p->cbits_stride = pool->cbits_stride;
  auto fail = [&](ara_status e) {
    free_portfolio(p);
    return e;
  };
  auto amalloc = [&](void** ptr, size_t n) { return dmalloc_async(ptr, std::max<size_t>(n, 8), s) == cudaSuccess; };
  if (!amalloc((void**)&p->d_layer_elts, 4 * p->layer_elts.size()) ||
      !amalloc((void**)&p->d_layers, sizeof(LayerConst) * (size_t)n_layers) ||
      !amalloc((void**)&p->d_q, 8 * (size_t)n_layers * C) ||
      !amalloc((void**)&p->d_bits, 4 * (size_t)n_layers * p->bm_words) ||
      !amalloc((void**)&p->d_cbits, 4 * (size_t)n_layers * p->cbits_stride) ||
      !amalloc((void**)&p->d_err, 4))
    return fail(ARA_ENOMEM);
  if ((!p->layer_elts.empty() &&
       cudaMemcpyAsync(p->d_layer_elts, p->layer_elts.data(), 4 * p->layer_elts.size(),
                       cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(p->d_layers, p->layers.data(), sizeof(LayerConst) * (size_t)n_layers,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(p->d_bits, 0, 4 * (size_t)n_layers * p->bm_words, s) != cudaSuccess ||
      cudaMemsetAsync(p->d_err, 0, 4, s) != cudaSuccess)
    return fail(ARA_ECUDA);
  *out = p;
  return ARA_OK;
}

static ara_status check_selection(const Portfolio& pf, int32_t n_sel, const int32_t* sel,
                                  std::vector<int32_t>& out) {
  out.clear();
  if (n_sel == 0 && sel == nullptr) {
    for (int32_t l = 0; l < pf.n_layers; ++l) out.push_back(l);
    return ARA_OK;
  }
  if (n_sel < 0 || !sel) return ARA_EINVAL;
  for (int32_t i = 0; i < n_sel; ++i) {
    if (sel[i] < 0 || sel[i] >= pf.n_layers) return ARA_EINVAL;
    out.push_back(sel[i]);
  }
  return ARA_OK;
}

static ara_status check_flags(const Portfolio& pf, int32_t flags) {
  if (flags & ~(ARA_RUN_PER_ELT | ARA_RUN_NO_FILTER | ARA_RUN_F64_SUM | ARA_RUN_LDG |
                ARA_RUN_HOST_DIRECT | ARA_RUN_BATCHED | ARA_RUN_OEP | ARA_RUN_PREPARED | ARA_RUN_SLOT1))
    return ARA_EINVAL;
  // a prepared fold slot serves the folded paths run from device memory
  if ((flags & (ARA_RUN_PREPARED | ARA_RUN_SLOT1)) &&
      (flags & (ARA_RUN_PER_ELT | ARA_RUN_BATCHED | ARA_RUN_HOST_DIRECT)))
    return ARA_EINVAL;
  if ((flags & ARA_RUN_SLOT1) && !(flags & ARA_RUN_PREPARED)) return ARA_EINVAL;
  if ((flags & ARA_RUN_OEP) && (flags & ~(ARA_RUN_OEP | ARA_RUN_PREPARED | ARA_RUN_SLOT1)))
    return ARA_EINVAL;   // default path only
  if ((flags & ARA_RUN_BATCHED) &&
      (flags & (ARA_RUN_PER_ELT | ARA_RUN_NO_FILTER | ARA_RUN_F64_SUM | ARA_RUN_LDG | ARA_RUN_HOST_DIRECT)))
    return ARA_EINVAL;
  if ((flags & ARA_RUN_PER_ELT) &&
      (flags & (ARA_RUN_NO_FILTER | ARA_RUN_F64_SUM | ARA_RUN_LDG | ARA_RUN_HOST_DIRECT)))
    return ARA_EINVAL;
  if ((flags & ARA_RUN_PER_ELT) && !pf.d_dense) return ARA_EINVAL;
  return ARA_OK;
}

ara_status ara_prepare_ylt(ara_portfolio* pf, int32_t n_sel, const int32_t* layer_sel, int32_t slot,
                           int32_t flags, void* stream) {
  if (!pf || slot < 0 || slot > 1) return ARA_EINVAL;
  std::vector<int32_t> sel;
  ara_status st = check_selection(*pf, n_sel, layer_sel, sel);
  if (st != ARA_OK) return st;
  if (flags & (ARA_RUN_PREPARED | ARA_RUN_SLOT1 | ARA_RUN_PER_ELT | ARA_RUN_BATCHED | ARA_RUN_HOST_DIRECT))
    return ARA_EINVAL;
  if ((st = check_flags(*pf, flags)) != ARA_OK) return st;
  if (sel.empty()) return ARA_OK;
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (slot == 1 && !pf->d_q_alt) {   // the second workspace, allocated on first use
    const size_t nl = (size_t)std::max(pf->n_layers, 1), C = (size_t)pf->catalogue;
    ARA_TRY(cudaStreamSynchronize(s));
    if (cudaMalloc(&pf->d_q_alt, sizeof(uint64_t) * nl * C) != cudaSuccess ||
        cudaMalloc(&pf->d_bits_alt, sizeof(uint32_t) * nl * (size_t)pf->bm_words) != cudaSuccess ||
        cudaMalloc(&pf->d_cbits_alt, sizeof(uint32_t) * nl * (size_t)pf->cbits_stride) != cudaSuccess) {
      cudaGetLastError();
      if (pf->d_q_alt) cudaFree(pf->d_q_alt);
      if (pf->d_bits_alt) cudaFree(pf->d_bits_alt);
      if (pf->d_cbits_alt) cudaFree(pf->d_cbits_alt);
      pf->d_q_alt = nullptr;
      pf->d_bits_alt = nullptr;
      pf->d_cbits_alt = nullptr;
      return ARA_ENOMEM;
    }
  }
  if ((st = launch_fold(*pf, (int32_t)sel.size(), sel.data(), flags, s, slot)) != ARA_OK) return st;
  return launch_coarsen(*pf, (int32_t)sel.size(), sel.data(), flags, s, slot);
}

ara_status ara_run_ylt(ara_portfolio* pf, int64_t n_trials, const int64_t* d_offsets,
                       int64_t n_events, const int32_t* d_ids, const float* d_timestamps,
                       int32_t n_sel, const int32_t* layer_sel, double* d_ylt, uint8_t* d_regimes,
                       int32_t flags, void* stream) {
  (void)d_timestamps;
  if (!pf || n_trials < 0 || n_events < 0 || n_trials > ((int64_t)1 << 40)) return ARA_EINVAL;
  std::vector<int32_t> sel;
  ara_status st = check_selection(*pf, n_sel, layer_sel, sel);
  if (st != ARA_OK) return st;
  if ((st = check_flags(*pf, flags)) != ARA_OK) return st;
  if (flags & ARA_RUN_HOST_DIRECT) return ARA_EINVAL;
  if (sel.empty() || n_trials == 0) return ARA_OK;
  if (!d_offsets || !d_ylt || (n_events > 0 && !d_ids)) return ARA_EINVAL;
  if (((uintptr_t)d_ids & 3) || ((uintptr_t)d_offsets & 7) || ((uintptr_t)d_ylt & 7)) return ARA_EINVAL;
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool prepared = (flags & ARA_RUN_PREPARED) != 0;
  const int slot = (flags & ARA_RUN_SLOT1) ? 1 : 0;
  if (slot == 1 && !pf->d_q_alt) return ARA_EINVAL;   // slot 1 never prepared
  if (!prepared && !(flags & (ARA_RUN_PER_ELT | ARA_RUN_BATCHED))) {
    if ((st = launch_fold(*pf, (int32_t)sel.size(), sel.data(), flags, s)) != ARA_OK) return st;
  }
  YltArgs a{};
  a.slot = slot;
  a.prepared = prepared;
  a.n_trials = n_trials;
  a.offsets = d_offsets;
  a.id_base = 0;
  a.n_events = n_events;
  a.ids = d_ids ? d_ids : reinterpret_cast<const int32_t*>(d_offsets);
  a.n_sel = (int32_t)sel.size();
  a.sel = sel.data();
  a.ylt = d_ylt;
  a.regimes = d_regimes;
  a.row_stride = n_trials;
  a.flags = flags;
  if (flags & ARA_RUN_BATCHED) return run_batched_async(*pf, a, s);
  return launch_ylt(*pf, a, s);
}

ara_status ara_check(ara_portfolio* pf, void* stream) {
  if (!pf) return ARA_EINVAL;
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t err = 0;
  ARA_TRY(cudaMemcpyAsync(&err, pf->d_err, sizeof(err), cudaMemcpyDeviceToHost, s));
  ARA_TRY(cudaStreamSynchronize(s));
  if (err) {
    ARA_TRY(cudaMemsetAsync(pf->d_err, 0, sizeof(uint32_t), s));
    ARA_TRY(cudaStreamSynchronize(s));
    return (err & DERR_TIMEOUT) ? ARA_ETIMEOUT : ARA_EDATA;
  }
  return ARA_OK;
}

static ara_status ensure_stage(Portfolio& pf, int64_t events, int64_t trials, int64_t ylt_elems) {
  if (!pf.copy_stream) {
    ARA_TRY(cudaStreamCreateWithFlags(&pf.copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      ARA_TRY(cudaEventCreateWithFlags(&pf.ev_copied[i], cudaEventDisableTiming));
      ARA_TRY(cudaEventCreateWithFlags(&pf.ev_done[i], cudaEventDisableTiming));
    }
  }
  if (events > pf.stage_events) {
    for (int i = 0; i < 2; ++i) {
      if (pf.d_stage_ids[i]) cudaFree(pf.d_stage_ids[i]);
      pf.d_stage_ids[i] = nullptr;
      ARA_TRY(cudaMalloc(&pf.d_stage_ids[i], sizeof(int32_t) * (size_t)std::max<int64_t>(events, 4)));
    }
    pf.stage_events = events;
  }
  if (trials > pf.stage_trials) {
    for (int i = 0; i < 2; ++i) {
      if (pf.d_stage_off[i]) cudaFree(pf.d_stage_off[i]);
      pf.d_stage_off[i] = nullptr;
      ARA_TRY(cudaMalloc(&pf.d_stage_off[i], sizeof(int64_t) * (size_t)(trials + 1)));
    }
    pf.stage_trials = trials;
  }
  if (ylt_elems > pf.ylt_full_elems) {
    if (pf.d_ylt_full) cudaFree(pf.d_ylt_full);
    pf.d_ylt_full = nullptr;
    ARA_TRY(cudaMalloc(&pf.d_ylt_full, sizeof(double) * (size_t)ylt_elems));
    pf.ylt_full_elems = ylt_elems;
  }
  return ARA_OK;
}

ara_status ara_run_ylt_host(ara_portfolio* pf, int64_t n_trials, const int64_t* h_off,
                            const int32_t* h_ids, int32_t n_sel, const int32_t* layer_sel,
                            double* h_ylt, int32_t n_rp, const double* rps, int32_t n_tvar,
                            const double* levels, double* h_pml, double* h_tvar, double* h_mean,
                            int32_t flags, void* stream) {
  if (!pf || n_trials < 0 || !h_off) return ARA_EINVAL;
  std::vector<int32_t> sel;
  ara_status st = check_selection(*pf, n_sel, layer_sel, sel);
  if (st != ARA_OK) return st;
  if ((st = check_flags(*pf, flags)) != ARA_OK) return st;
  if (n_rp < 0 || n_tvar < 0) return ARA_EINVAL;
  const bool metrics = n_rp + n_tvar > 0 || h_mean != nullptr;
  if (metrics && (sel.empty() || (n_rp > 0 && !h_pml) || (n_tvar > 0 && !h_tvar) ||
                  validate_metrics(n_trials, n_rp, rps, n_tvar, levels) != ARA_OK))
    return ARA_EINVAL;
  if (flags & (ARA_RUN_BATCHED | ARA_RUN_PREPARED | ARA_RUN_SLOT1)) return ARA_EINVAL;
  if (h_off[0] != 0) return ARA_EINVAL;
  // Host check that the offsets never decrease (no early exit, so the scan vectorises), timed
  // under ARA_K_HOST_CHECK.
  auto offsets_decrease = [&]() {
    const auto c0 = std::chrono::steady_clock::now();
    bool decreasing = false;
    for (int64_t t = 0; t < n_trials; ++t) decreasing |= h_off[t + 1] < h_off[t];
    timing_add_host(ARA_K_HOST_CHECK,
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c0).count());
    return decreasing;
  };
  const bool direct = (flags & ARA_RUN_HOST_DIRECT) != 0;
  if (!direct && offsets_decrease()) return ARA_EINVAL;   // the chunk cuts rely on the order
  const int64_t n_events = h_off[n_trials];
  if (n_events < 0) return ARA_EINVAL;
  if (sel.empty() || n_trials == 0) return direct && offsets_decrease() ? ARA_EINVAL : ARA_OK;
  if (n_events > 0 && !h_ids) return ARA_EINVAL;
  if (!h_ylt && !metrics) return ARA_EINVAL;
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (direct) {
    // The device reads the host arrays in place: they must be mapped into its address space.
    void* d_off_v = nullptr;
    void* d_ids_v = nullptr;
    if (cudaHostGetDevicePointer(&d_off_v, (void*)h_off, 0) != cudaSuccess ||
        (n_events > 0 && cudaHostGetDevicePointer(&d_ids_v, (void*)h_ids, 0) != cudaSuccess)) {
      cudaGetLastError();
      return ARA_EINVAL;
    }
    if ((st = ensure_stage(*pf, 0, 0, (int64_t)sel.size() * n_trials)) != ARA_OK) return st;
    const int32_t f = (flags & ~ARA_RUN_HOST_DIRECT) | ARA_RUN_LDG;  // plain loads of host memory
    if (!(f & ARA_RUN_PER_ELT)) {
      if ((st = launch_fold(*pf, (int32_t)sel.size(), sel.data(), f, s)) != ARA_OK) return st;
    }
    YltArgs a{};
    a.n_trials = n_trials;
    a.offsets = (const int64_t*)d_off_v;
    a.id_base = 0;
    a.n_events = n_events;
    a.ids = n_events > 0 ? (const int32_t*)d_ids_v : (const int32_t*)d_off_v;
    a.n_sel = (int32_t)sel.size();
    a.sel = sel.data();
    a.ylt = pf->d_ylt_full;
    a.regimes = nullptr;
    a.row_stride = n_trials;
    a.flags = f;
    if ((st = launch_ylt(*pf, a, s)) != ARA_OK) return st;
    // The offsets are checked while the kernels run: they bound every offset they read, so
    // decreasing offsets only make them record a data error, which ara_check clears.
    if (offsets_decrease()) {
      ara_check(pf, stream);
      return ARA_EINVAL;
    }
  } else {
  // chunk boundaries: at most CH_EVENTS events and CH_TRIALS trials per chunk
  const int64_t CH_EVENTS = (int64_t)1 << 24, CH_TRIALS = (int64_t)1 << 20;
  std::vector<int64_t> cut{0};
  int64_t max_ev = 0, max_tr = 0;
  for (int64_t t = 0; t < n_trials;) {
    // the last t1 in (t, t + CH_TRIALS] whose offset is within CH_EVENTS of h_off[t] (at least
    // t + 1: a trial longer than CH_EVENTS is a chunk of its own), by binary search
    const int64_t lim = std::min(n_trials, t + CH_TRIALS);
    const int64_t* up = std::upper_bound(h_off + t + 1, h_off + lim + 1, h_off[t] + CH_EVENTS);
    const int64_t t1 = std::max<int64_t>(t + 1, (int64_t)(up - h_off) - 1);
    max_ev = std::max(max_ev, h_off[t1] - h_off[t]);
    max_tr = std::max(max_tr, t1 - t);
    cut.push_back(t1);
    t = t1;
  }
  if ((st = ensure_stage(*pf, max_ev, max_tr, (int64_t)sel.size() * n_trials)) != ARA_OK) return st;
  if (!(flags & ARA_RUN_PER_ELT)) {
    if ((st = launch_fold(*pf, (int32_t)sel.size(), sel.data(), flags, s)) != ARA_OK) return st;
  }
  // The copy stream must not overwrite a staging buffer that work queued earlier on `s` reads.
  ARA_TRY(cudaEventRecord(pf->ev_done[0], s));
  ARA_TRY(cudaEventRecord(pf->ev_done[1], s));
  for (size_t c = 0; c + 1 < cut.size(); ++c) {
    const int b = (int)(c & 1);
    const int64_t t0 = cut[c], t1 = cut[c + 1], nt = t1 - t0;
    const int64_t e0 = h_off[t0], ne = h_off[t1] - e0;
    ARA_TRY(cudaStreamWaitEvent(pf->copy_stream, pf->ev_done[b], 0));
    timing_begin(ARA_K_TRANSFER, pf->copy_stream);
    if (ne > 0)
      ARA_TRY(cudaMemcpyAsync(pf->d_stage_ids[b], h_ids + e0, sizeof(int32_t) * (size_t)ne,
                              cudaMemcpyHostToDevice, pf->copy_stream));
    ARA_TRY(cudaMemcpyAsync(pf->d_stage_off[b], h_off + t0, sizeof(int64_t) * (size_t)(nt + 1),
                            cudaMemcpyHostToDevice, pf->copy_stream));
    timing_end(ARA_K_TRANSFER, pf->copy_stream);
    ARA_TRY(cudaEventRecord(pf->ev_copied[b], pf->copy_stream));
    ARA_TRY(cudaStreamWaitEvent(s, pf->ev_copied[b], 0));
    YltArgs a{};
    a.n_trials = nt;
    a.offsets = pf->d_stage_off[b];
    a.id_base = e0;
    a.n_events = ne;
    a.ids = pf->d_stage_ids[b];
    a.n_sel = (int32_t)sel.size();
    a.sel = sel.data();
    a.ylt = pf->d_ylt_full + t0;
    a.regimes = nullptr;
    a.row_stride = n_trials;
    a.flags = flags;
    if ((st = launch_ylt(*pf, a, s)) != ARA_OK) return st;
    ARA_TRY(cudaEventRecord(pf->ev_done[b], s));
  }
  }  // staged copies
  // Results.  The YLT goes back on the copy stream while the selection runs on `s`; the metrics,
  // the selection's status and the device error word come back in one small copy into pinned
  // memory; then one wait for both streams.
  const int32_t nsel = (int32_t)sel.size();
  if (h_ylt) {
    ARA_TRY(cudaEventRecord(pf->ev_done[0], s));
    ARA_TRY(cudaStreamWaitEvent(pf->copy_stream, pf->ev_done[0], 0));
    timing_begin(ARA_K_TRANSFER, pf->copy_stream);
    ARA_TRY(cudaMemcpyAsync(h_ylt, pf->d_ylt_full, sizeof(double) * (size_t)nsel * (size_t)n_trials,
                            cudaMemcpyDeviceToHost, pf->copy_stream));
    timing_end(ARA_K_TRANSFER, pf->copy_stream);
  }
  const int64_t n_pml = (int64_t)nsel * n_rp, n_tv = (int64_t)nsel * n_tvar;
  const int64_t n_mean = h_mean ? nsel : 0;
  const int64_t res_elems = n_pml + n_tv + n_mean + 1;   // + one slot: status and error words
  if (res_elems > pf->res_elems) {
    if (pf->d_res) cudaFree(pf->d_res);
    if (pf->h_res) cudaFreeHost(pf->h_res);
    pf->d_res = nullptr;
    pf->h_res = nullptr;
    pf->res_elems = 0;
    ARA_TRY(cudaMalloc((void**)&pf->d_res, sizeof(double) * (size_t)res_elems));
    ARA_TRY(cudaMallocHost((void**)&pf->h_res, sizeof(double) * (size_t)res_elems));
    pf->res_elems = res_elems;
  }
  uint32_t* d_words = reinterpret_cast<uint32_t*>(pf->d_res + n_pml + n_tv + n_mean);
  ARA_TRY(cudaMemsetAsync(d_words, 0, 2 * sizeof(uint32_t), s));
  if (metrics) {
    // the selection's scratch is kept with the portfolio, so repeated calls allocate nothing
    auto queue = [&](size_t* need) {
      return risk_metrics_queue(pf->d_ylt_full, n_trials, nsel, n_rp, rps, n_tvar, levels,
                                n_rp > 0 ? pf->d_res : nullptr, n_tvar > 0 ? pf->d_res + n_pml : nullptr,
                                h_mean ? pf->d_res + n_pml + n_tv : nullptr, d_words,
                                pf->d_sel_scratch, pf->sel_scratch_bytes, need, s);
    };
    size_t need = 0;
    st = queue(&need);
    if (st == ARA_ERANGE && need > pf->sel_scratch_bytes) {
      ARA_TRY(cudaStreamSynchronize(s));
      if (pf->d_sel_scratch) cudaFree(pf->d_sel_scratch);
      pf->d_sel_scratch = nullptr;
      pf->sel_scratch_bytes = 0;
      ARA_TRY(cudaMalloc(&pf->d_sel_scratch, need));
      pf->sel_scratch_bytes = need;
      st = queue(&need);
    }
    if (st != ARA_OK) {
      cudaStreamSynchronize(pf->copy_stream);
      cudaStreamSynchronize(s);
      return st;
    }
  }
  ARA_TRY(cudaMemcpyAsync(d_words + 1, pf->d_err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  ARA_TRY(cudaMemcpyAsync(pf->h_res, pf->d_res, sizeof(double) * (size_t)res_elems,
                          cudaMemcpyDeviceToHost, s));
  ARA_TRY(cudaStreamSynchronize(s));
  ARA_TRY(cudaStreamSynchronize(pf->copy_stream));
  const uint32_t* h_words = reinterpret_cast<const uint32_t*>(pf->h_res + n_pml + n_tv + n_mean);
  const uint32_t sel_status = h_words[0], err = h_words[1];
  if (err) {   // as ara_check: report and clear the device error word
    ARA_TRY(cudaMemsetAsync(pf->d_err, 0, sizeof(uint32_t), s));
    ARA_TRY(cudaStreamSynchronize(s));
    return (err & DERR_TIMEOUT) ? ARA_ETIMEOUT : ARA_EDATA;
  }
  if (sel_status & ARA_DEVICE_TIMEOUT) return ARA_ETIMEOUT;
  if (n_pml) std::copy(pf->h_res, pf->h_res + n_pml, h_pml);
  if (n_tv) std::copy(pf->h_res + n_pml, pf->h_res + n_pml + n_tv, h_tvar);
  if (n_mean) std::copy(pf->h_res + n_pml + n_tv, pf->h_res + n_pml + n_tv + n_mean, h_mean);
  return ARA_OK;
}

}  // extern "C"

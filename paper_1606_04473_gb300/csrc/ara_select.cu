// PML and TVaR (Section IV-A names both as metrics derived from the YLT) as empirical order
// statistics: PML(RP) is the ceil(N/RP)-th largest year loss, TVaR(p) the mean of the
// ceil(N(1-p)) largest.  Both come from an exact radix select on order-preserving 64-bit keys
// of the FP64 year losses (8 passes of 8 bits), followed by one pass summing the tail above
// the selected key.  Every block of a pass adds its shared-memory histogram into the pass's
// global histogram; the last block to finish (ticket counter, no waiting) advances the
// selection state.  Results are bit-exact copies of YLT entries (PML) and a deterministic
// FP64 sum (TVaR).

#include <cmath>
#include <mutex>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

constexpr int SEL_BITS = 8;
constexpr int SEL_BINS = 1 << SEL_BITS;
constexpr int SEL_PASSES = 64 / SEL_BITS;
constexpr int SEL_MAX_T = 16;
constexpr int SEL_THREADS = 256;

struct SelTargets {
  int32_t n_t;                 // targets per layer
  int32_t n_rp;                // targets [0, n_rp) are PML ranks, the rest TVaR counts
  int64_t rank[SEL_MAX_T];     // 1-based rank from the top
};

struct SelState {
  uint64_t prefix;             // key bits fixed so far
  int64_t k;                   // rank still to find among keys matching the prefix
};

// Scratch layout (one allocation, zero-filled before the first pass):
//   hist   [SEL_PASSES][n_layers][n_t][SEL_BINS]  uint32
//   ticket [SEL_PASSES + 1][n_layers]             uint32
//   state  [n_layers][n_t]                        SelState
//   psum   [n_layers][n_t][blocks]                double
//   pcnt   [n_layers][n_t][blocks]                int64
//   out    [n_layers][n_t]                        double
//   gt, eq [n_layers][n_t]                        int64: #{key > selected}, #{key == selected}
//   pmean  [n_layers][blocks]                     double (block partial sums of the whole row)
//   mean   [n_layers]                             double
struct SelScratch {
  uint32_t* hist;
  uint32_t* ticket;
  SelState* state;
  double* psum;
  int64_t* pcnt;
  double* out;
  unsigned long long* gt;
  unsigned long long* eq;
  double* pmean;
  double* mean;
};

size_t select_scratch_bytes(int32_t n_layers, int32_t n_t, int32_t blocks) {
  size_t b = 0;
  auto take = [&](size_t n) { b = (b + 255) / 256 * 256 + n; };
  take(sizeof(uint32_t) * SEL_PASSES * n_layers * n_t * SEL_BINS);
  take(sizeof(uint32_t) * (SEL_PASSES + 1) * n_layers);
  take(sizeof(SelState) * n_layers * n_t);
  take(sizeof(double) * n_layers * n_t * blocks);
  take(sizeof(int64_t) * n_layers * n_t * blocks);
  take(sizeof(double) * n_layers * n_t);
  take(sizeof(int64_t) * n_layers * n_t);
  take(sizeof(int64_t) * n_layers * n_t);
  take(sizeof(double) * n_layers * blocks);
  take(sizeof(double) * n_layers);
  return (b + 255) / 256 * 256;
}

static SelScratch carve(void* base, int32_t n_layers, int32_t n_t, int32_t blocks) {
  size_t b = 0;
  char* p = (char*)base;
  auto take = [&](size_t n) {
    b = (b + 255) / 256 * 256;
    void* r = p + b;
    b += n;
    return r;
  };
  SelScratch s;
  s.hist = (uint32_t*)take(sizeof(uint32_t) * SEL_PASSES * n_layers * n_t * SEL_BINS);
  s.ticket = (uint32_t*)take(sizeof(uint32_t) * (SEL_PASSES + 1) * n_layers);
  s.state = (SelState*)take(sizeof(SelState) * n_layers * n_t);
  s.psum = (double*)take(sizeof(double) * n_layers * n_t * blocks);
  s.pcnt = (int64_t*)take(sizeof(int64_t) * n_layers * n_t * blocks);
  s.out = (double*)take(sizeof(double) * n_layers * n_t);
  s.gt = (unsigned long long*)take(sizeof(int64_t) * n_layers * n_t);
  s.eq = (unsigned long long*)take(sizeof(int64_t) * n_layers * n_t);
  s.pmean = (double*)take(sizeof(double) * n_layers * blocks);
  s.mean = (double*)take(sizeof(double) * n_layers);
  return s;
}

// Order-preserving map of an IEEE double to an unsigned 64-bit key (total order).
__device__ __forceinline__ uint64_t key_of(double y) {
  const uint64_t b = (uint64_t)__double_as_longlong(y);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double value_of(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Elements are visited in sweeps: in sweep j, thread x of block b reads the SEL_VPT elements
// base + x + v * SEL_THREADS (v < SEL_VPT) with base = (j * gridDim.x + b) * SEL_THREADS * SEL_VPT,
// all loads of a sweep issued together.  The loop bound is uniform across each warp, so
// warp-collective operations see every lane.
constexpr int SEL_VPT = 8;
constexpr int SEL_SWEEP = SEL_THREADS * SEL_VPT;

__device__ __forceinline__ void load_sweep(const double* __restrict__ row, int64_t n, int64_t base,
                                           double (&y)[SEL_VPT], bool (&ok)[SEL_VPT]) {
#pragma unroll
  for (int v = 0; v < SEL_VPT; ++v) {
    const int64_t i = base + threadIdx.x + v * SEL_THREADS;
    ok[v] = i < n;
    y[v] = ok[v] ? __ldcg(row + i) : 0.0;
  }
}

// One radix pass: the digit histogram of the keys that match each target's prefix.  Targets
// whose prefixes are equal share one histogram (in pass 0 all of them do), counted once and
// stored under the group's first target.  Equal digits within a warp are added with one
// shared-memory atomic (lanes grouped by __match_any_sync).
__global__ void __launch_bounds__(SEL_THREADS)
k_select_pass(const double* __restrict__ ylt, int64_t n, SelTargets tg, SelScratch sc, int pass) {
  __shared__ uint32_t h[SEL_MAX_T * SEL_BINS];
  __shared__ uint64_t gpre[SEL_MAX_T];      // prefix of each group
  __shared__ int32_t gldr[SEL_MAX_T];       // first target of each group
  __shared__ int32_t tgrp[SEL_MAX_T];       // group of each target
  __shared__ int32_t ngrp;
  __shared__ bool last;
  const int layer = blockIdx.y, nt = tg.n_t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    int ng = 0;
    for (int t = 0; t < nt; ++t) {
      const uint64_t pr = pass == 0 ? 0ull : sc.state[layer * nt + t].prefix;
      int g = 0;
      while (g < ng && gpre[g] != pr) ++g;
      if (g == ng) {
        gpre[g] = pr;
        gldr[g] = t;
        ++ng;
      }
      tgrp[t] = g;
    }
    ngrp = ng;
  }
  __syncthreads();
  const int ng = ngrp;
  for (int i = threadIdx.x; i < ng * SEL_BINS; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int shift = 64 - SEL_BITS * (pass + 1);
  const double* row = ylt + (int64_t)layer * n;
  for (int64_t base = (int64_t)blockIdx.x * SEL_SWEEP; base < n; base += (int64_t)gridDim.x * SEL_SWEEP) {
    double y[SEL_VPT];
    bool ok[SEL_VPT];
    load_sweep(row, n, base, y, ok);
#pragma unroll
    for (int v = 0; v < SEL_VPT; ++v) {
      const uint64_t key = key_of(y[v]);
      const uint32_t d = (uint32_t)(key >> shift) & (SEL_BINS - 1);
      for (int g = 0; g < ng; ++g) {
        const bool m = ok[v] && (pass == 0 || (key >> (shift + SEL_BITS)) == (gpre[g] >> (shift + SEL_BITS)));
        if (!__any_sync(0xffffffffu, m)) continue;
        const uint32_t peers = __match_any_sync(0xffffffffu, m ? d : 0xffffffffu);
        if (m && lane == __ffs(peers) - 1) atomicAdd(&h[g * SEL_BINS + d], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  uint32_t* gh = sc.hist + ((int64_t)pass * gridDim.y + layer) * nt * SEL_BINS;
  for (int i = threadIdx.x; i < ng * SEL_BINS; i += blockDim.x)
    if (h[i]) atomicAdd(&gh[gldr[i / SEL_BINS] * SEL_BINS + (i % SEL_BINS)], h[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(&sc.ticket[pass * gridDim.y + layer], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Last block: pick the digit of every target from its group's histogram, scanning bins from
  // the top (one warp per target).
  for (int t = warp; t < nt; t += blockDim.x / 32) {
    SelState st = pass == 0 ? SelState{0ull, tg.rank[t]} : sc.state[layer * nt + t];
    const uint32_t* th = gh + gldr[tgrp[t]] * SEL_BINS;
    // lane l owns bins [SEL_BINS - 8(l+1), SEL_BINS - 8l) (descending order overall)
    uint32_t c[SEL_BINS / 32];
    uint32_t mine = 0;
#pragma unroll
    for (int u = 0; u < SEL_BINS / 32; ++u) {
      c[u] = __ldcg(&th[SEL_BINS - 1 - (lane * (SEL_BINS / 32) + u)]);
      mine += c[u];
    }
    uint32_t incl = mine;  // inclusive prefix over lanes (from the top bins down)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - mine;
    const bool here = (int64_t)excl < st.k && st.k <= (int64_t)incl;
    if (here) {
      int64_t before = excl;
      int u = 0;
      for (; u < SEL_BINS / 32; ++u) {
        if (before + c[u] >= st.k) break;
        before += c[u];
      }
      const uint32_t bin = SEL_BINS - 1 - (lane * (SEL_BINS / 32) + u);
      st.k -= before;
      st.prefix |= (uint64_t)bin << shift;
      sc.state[layer * nt + t] = st;
    }
  }
}

// Tail pass: for every target, the selected key and the counts of keys above / equal to it;
// for TVaR targets the sum of the values strictly above it; optionally the row sum (mean).
// Each element is read once; every thread keeps its own partial sums in a fixed order, warps
// and blocks combine them in a fixed order, and the last block adds the block partials in
// block order, so the result is deterministic.
__global__ void __launch_bounds__(SEL_THREADS)
k_select_tail(const double* __restrict__ ylt, int64_t n, SelTargets tg, SelScratch sc, int want_mean) {
  __shared__ double ssum[SEL_THREADS / 32][SEL_MAX_T + 1];
  __shared__ uint64_t thr[SEL_MAX_T];
  __shared__ bool last;
  const int layer = blockIdx.y, nt = tg.n_t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < nt) thr[threadIdx.x] = sc.state[layer * nt + threadIdx.x].prefix;
  __syncthreads();
  const double* row = ylt + (int64_t)layer * n;
  double s[SEL_MAX_T + 1];
  uint32_t cg[SEL_MAX_T], ce[SEL_MAX_T];
#pragma unroll
  for (int t = 0; t <= SEL_MAX_T; ++t) s[t] = 0.0;
#pragma unroll
  for (int t = 0; t < SEL_MAX_T; ++t) cg[t] = ce[t] = 0;
  for (int64_t base = (int64_t)blockIdx.x * SEL_SWEEP; base < n; base += (int64_t)gridDim.x * SEL_SWEEP) {
    double y[SEL_VPT];
    bool ok[SEL_VPT];
    load_sweep(row, n, base, y, ok);
#pragma unroll
    for (int v = 0; v < SEL_VPT; ++v) {
      if (!ok[v]) continue;
      const uint64_t k = key_of(y[v]);
      if (want_mean) s[SEL_MAX_T] = __dadd_rn(s[SEL_MAX_T], y[v]);
#pragma unroll
      for (int t = 0; t < SEL_MAX_T; ++t) {
        if (t >= nt) break;
        const uint64_t th = thr[t];
        if (k > th) {
          ++cg[t];
          if (t >= tg.n_rp) s[t] = __dadd_rn(s[t], y[v]);
        } else if (k == th) {
          ++ce[t];
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t <= SEL_MAX_T; ++t) {
    if (t < SEL_MAX_T && t >= nt) continue;
    if (t == SEL_MAX_T && !want_mean) continue;
    double a = s[t];
    unsigned long long g = t < SEL_MAX_T ? cg[t] : 0, e = t < SEL_MAX_T ? ce[t] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, o));
      g += __shfl_down_sync(0xffffffffu, g, o);
      e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if (lane == 0) {
      ssum[warp][t < SEL_MAX_T ? t : nt] = a;
      if (t < SEL_MAX_T) {
        if (g) atomicAdd(&sc.gt[layer * nt + t], g);
        if (e) atomicAdd(&sc.eq[layer * nt + t], e);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x <= nt && (threadIdx.x >= tg.n_rp || threadIdx.x == nt)) {
    const int t = threadIdx.x;
    if (t < nt || want_mean) {
      double a = 0.0;
      for (int w = 0; w < SEL_THREADS / 32; ++w) a = __dadd_rn(a, ssum[w][t]);
      if (t < nt) sc.psum[((int64_t)layer * nt + t) * gridDim.x + blockIdx.x] = a;
      else sc.pmean[(int64_t)layer * gridDim.x + blockIdx.x] = a;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(&sc.ticket[SEL_PASSES * gridDim.y + layer], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < nt) {
    const int t = threadIdx.x;
    const double v = value_of(thr[t]);
    double r = v;
    if (t >= tg.n_rp) {
      double a = 0.0;
      const int64_t base = ((int64_t)layer * nt + t) * gridDim.x;
      for (unsigned b = 0; b < gridDim.x; ++b) a = __dadd_rn(a, __ldcg(&sc.psum[base + b]));
      const int64_t m = tg.rank[t];
      const int64_t c = (int64_t)__ldcg(&sc.gt[layer * nt + t]);
      r = (a + (double)(m - c) * v) / (double)m;
    }
    sc.out[layer * nt + t] = r;
  } else if (threadIdx.x == nt && want_mean) {
    double a = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) a = __dadd_rn(a, __ldcg(&sc.pmean[(int64_t)layer * gridDim.x + b]));
    sc.mean[layer] = a / (double)n;
  }
}

// ceil(x), taking x within 1e-9 (relative) of an integer as that integer.
static int64_t ceil_snap(double x) {
  const double r = std::nearbyint(x);
  if (std::fabs(x - r) <= 1e-9 * std::fmax(1.0, std::fabs(x))) return (int64_t)r;
  return (int64_t)std::ceil(x);
}

ara_status select_targets(int64_t n, int32_t n_rp, const double* rps, int32_t n_tvar,
                          const double* levels, SelTargets& tg) {
  if (n < 1 || n_rp < 0 || n_tvar < 0 || n_rp + n_tvar > SEL_MAX_T) return ARA_EINVAL;
  if ((n_rp > 0 && !rps) || (n_tvar > 0 && !levels)) return ARA_EINVAL;
  tg.n_t = n_rp + n_tvar;
  tg.n_rp = n_rp;
  for (int i = 0; i < n_rp; ++i) {
    if (!(rps[i] >= 1.0) || !std::isfinite(rps[i])) return ARA_EINVAL;
    const int64_t k = ceil_snap((double)n / rps[i]);
    if (k < 1 || k > n) return ARA_EINVAL;
    tg.rank[i] = k;
  }
  for (int i = 0; i < n_tvar; ++i) {
    if (!(levels[i] >= 0.0 && levels[i] < 1.0)) return ARA_EINVAL;
    const int64_t m = ceil_snap((double)n * (1.0 - levels[i]));
    if (m < 1 || m > n) return ARA_EINVAL;
    tg.rank[n_rp + i] = m;
  }
  return ARA_OK;
}

int64_t tail_count_snap(int64_t n, double p) {
  if (!(p >= 0.0 && p < 1.0) || n < 1) return -1;
  const int64_t m = ceil_snap((double)n * (1.0 - p));
  return (m >= 1 && m <= n) ? m : -1;
}

ara_status validate_metrics(int64_t n, int32_t n_rp, const double* rps, int32_t n_tvar,
                            const double* levels) {
  SelTargets tg;
  return select_targets(n, n_rp, rps, n_tvar, levels, tg);
}

int32_t select_blocks(int64_t n, int n_sms, int32_t n_layers) {
  int64_t b = (n + SEL_SWEEP - 1) / SEL_SWEEP;
  const int64_t cap = std::max<int64_t>(1, 2 * (int64_t)n_sms / std::max(1, n_layers) + 1);
  return (int32_t)std::max<int64_t>(1, std::min(b, cap));
}

// Launch the whole selection into `scratch` (zero-filled here); results land in scratch.out.
ara_status launch_select(const double* d_ylt, int64_t n, int32_t n_layers, const SelTargets& tg,
                         void* scratch, size_t scratch_bytes, int32_t blocks, int want_mean,
                         cudaStream_t s, SelScratch* out) {
  SelScratch sc = carve(scratch, n_layers, tg.n_t, blocks);
  ARA_TRY(cudaMemsetAsync(scratch, 0, scratch_bytes, s));
  {
    LaunchScope ls(ARA_K_SELECT, s, tg.n_t > 0 ? SEL_PASSES + 1 : 1);
    dim3 grid(blocks, n_layers);
    if (tg.n_t > 0)
      for (int p = 0; p < SEL_PASSES; ++p) k_select_pass<<<grid, SEL_THREADS, 0, s>>>(d_ylt, n, tg, sc, p);
    k_select_tail<<<grid, SEL_THREADS, 0, s>>>(d_ylt, n, tg, sc, want_mean);
    ARA_TRY(cudaGetLastError());
  }
  *out = sc;
  return ARA_OK;
}

}  // namespace ara

using namespace ara;

namespace ara {

ara_status select_one_rank(const double* d_ylt, int64_t n, int32_t n_layers, int64_t m, int n_sms,
                           cudaStream_t s, SelectResult* out) {
  SelTargets tg;
  tg.n_t = 1;
  tg.n_rp = 0;
  tg.rank[0] = m;
  const int32_t blocks = select_blocks(n, n_sms, n_layers);
  const size_t bytes = select_scratch_bytes(n_layers, 1, blocks);
  void* scratch = nullptr;
  ARA_TRY(cudaMallocAsync(&scratch, bytes, s));
  SelScratch sc;
  ara_status st = launch_select(d_ylt, n, n_layers, tg, scratch, bytes, blocks, 0, s, &sc);
  if (st != ARA_OK) {
    cudaFreeAsync(scratch, s);
    return st;
  }
  out->scratch = scratch;
  out->thr_key = &sc.state[0].prefix;
  out->thr_stride = sizeof(SelState) / sizeof(uint64_t);
  out->gt = sc.gt;
  out->eq = sc.eq;
  return ARA_OK;
}

void free_select_result(SelectResult& r, cudaStream_t s) {
  if (r.scratch) cudaFreeAsync(r.scratch, s);
  r.scratch = nullptr;
}

ara_status risk_metrics_device(const double* d_ylt, int64_t n_trials, int32_t n_layers,
                               int32_t n_rp, const double* rps, int32_t n_tvar,
                               const double* levels, double* h_pml, double* h_tvar,
                               double* h_mean, cudaStream_t s) {
  SelTargets tg;
  if (!d_ylt || n_layers < 1) return ARA_EINVAL;
  if ((n_rp > 0 && !h_pml) || (n_tvar > 0 && !h_tvar)) return ARA_EINVAL;
  if ((uintptr_t)d_ylt & 7) return ARA_EINVAL;
  ara_status st = select_targets(n_trials, n_rp, rps, n_tvar, levels, tg);
  if (st != ARA_OK) return st;
  if (tg.n_t == 0 && !h_mean) return ARA_EINVAL;
  int dev = 0, sms = 0;
  ARA_TRY(cudaGetDevice(&dev));
  ARA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int32_t blocks = select_blocks(n_trials, sms, n_layers);
  const size_t bytes = select_scratch_bytes(n_layers, tg.n_t, blocks);
  void* scratch = nullptr;
  ARA_TRY(cudaMallocAsync(&scratch, bytes, s));
  SelScratch sc;
  st = launch_select(d_ylt, n_trials, n_layers, tg, scratch, bytes, blocks, h_mean != nullptr, s, &sc);
  std::vector<double> out((size_t)n_layers * tg.n_t);
  if (st == ARA_OK) {
    cudaError_t e = cudaMemcpyAsync(out.data(), sc.out, sizeof(double) * out.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_mean)
      e = cudaMemcpyAsync(h_mean, sc.mean, sizeof(double) * n_layers, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = ARA_ECUDA;
  }
  cudaFreeAsync(scratch, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
  if (st != ARA_OK) return st;
  for (int32_t l = 0; l < n_layers; ++l) {
    for (int i = 0; i < n_rp; ++i) h_pml[(size_t)l * n_rp + i] = out[(size_t)l * tg.n_t + i];
    for (int i = 0; i < n_tvar; ++i) h_tvar[(size_t)l * n_tvar + i] = out[(size_t)l * tg.n_t + n_rp + i];
  }
  return ARA_OK;
}

}  // namespace ara

extern "C" ara_status ara_risk_metrics(const double* d_ylt, int64_t n_trials, int32_t n_layers,
                                       int32_t n_rp, const double* rps, int32_t n_tvar,
                                       const double* levels, double* h_pml, double* h_tvar,
                                       double* h_mean, void* stream) {
  return risk_metrics_device(d_ylt, n_trials, n_layers, n_rp, rps, n_tvar, levels, h_pml, h_tvar,
                             h_mean, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant: the selection scratch lives in a fixed device array of this
// library.  Host code cannot use the array's name as a device address, so its address is
// looked up once per device (with that device current) and cached.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_select_scratch[ARA_STATIC_SELECT_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_scratch[kMaxDevices];
}  // namespace

static ara_status static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return ARA_ECUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
    if (e != cudaSuccess || !p) {
      note_cuda_error(e, "cudaGetSymbolAddress(g_select_scratch)", __FILE__, __LINE__);
      return ARA_ECUDA;
    }
    g_static_scratch[dev] = p;
  }
  *out = g_static_scratch[dev];
  return ARA_OK;
}

extern "C" ara_status ara_risk_metrics_static(const double* d_ylt, int64_t n_trials,
                                              int32_t n_layers, int32_t n_rp, const double* rps,
                                              int32_t n_tvar, const double* levels, double* h_pml,
                                              double* h_tvar, double* h_mean, void* stream) {
  SelTargets tg;
  if (!d_ylt || n_layers < 1) return ARA_EINVAL;
  if ((n_rp > 0 && !h_pml) || (n_tvar > 0 && !h_tvar)) return ARA_EINVAL;
  if ((uintptr_t)d_ylt & 7) return ARA_EINVAL;
  ara_status st = select_targets(n_trials, n_rp, rps, n_tvar, levels, tg);
  if (st != ARA_OK) return st;
  if (tg.n_t == 0 && !h_mean) return ARA_EINVAL;
  int dev = 0, sms = 0;
  ARA_TRY(cudaGetDevice(&dev));
  ARA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // Fewer blocks shrink the per-block partials; if even one block does not fit, refuse.
  int32_t blocks = select_blocks(n_trials, sms, n_layers);
  while (blocks > 1 && select_scratch_bytes(n_layers, tg.n_t, blocks) > ARA_STATIC_SELECT_BYTES)
    blocks = blocks / 2;
  const size_t bytes = select_scratch_bytes(n_layers, tg.n_t, blocks);
  if (bytes > ARA_STATIC_SELECT_BYTES) return ARA_ERANGE;
  void* scratch = nullptr;
  if ((st = static_scratch(dev, &scratch)) != ARA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SelScratch sc;
  // launch_select clears the used part of the scratch before its first kernel
  if ((st = launch_select(d_ylt, n_trials, n_layers, tg, scratch, bytes, blocks, h_mean != nullptr,
                          s, &sc)) != ARA_OK)
    return st;
  const size_t row = sizeof(double) * (size_t)tg.n_t;
  if (n_rp > 0)
    ARA_TRY(cudaMemcpy2DAsync(h_pml, sizeof(double) * n_rp, sc.out, row, sizeof(double) * n_rp,
                              (size_t)n_layers, cudaMemcpyDeviceToHost, s));
  if (n_tvar > 0)
    ARA_TRY(cudaMemcpy2DAsync(h_tvar, sizeof(double) * n_tvar, sc.out + n_rp, row,
                              sizeof(double) * n_tvar, (size_t)n_layers, cudaMemcpyDeviceToHost, s));
  if (h_mean)
    ARA_TRY(cudaMemcpyAsync(h_mean, sc.mean, sizeof(double) * n_layers, cudaMemcpyDeviceToHost, s));
  ARA_TRY(cudaStreamSynchronize(s));
  return ARA_OK;
}

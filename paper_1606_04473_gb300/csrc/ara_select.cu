// PML and TVaR (Section IV-A names both as metrics derived from the YLT) as empirical order
// statistics: PML(RP) is the ceil(N/RP)-th largest year loss, TVaR(p) the mean of the
// ceil(N(1-p)) largest.  Both come from an exact radix select on order-preserving 64-bit keys
// of the FP64 year losses (up to 8 passes of 8 bits), followed by one pass summing the tail
// above the selected key.  One cooperative launch runs every pass: each block adds its
// shared-memory digit histogram into the pass's global histogram, the layer's blocks meet at a
// grid barrier (a bounded wait), and every block then reads the histogram and advances the
// selection itself.
// Results are bit-exact copies of YLT entries (PML) and deterministic FP64 sums (TVaR, mean):
// fixed per-thread order, fixed warp and block trees, block partials combined in a fixed order.

#include <cmath>
#include <mutex>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

constexpr int SEL_BITS = 8;
constexpr int SEL_BINS = 1 << SEL_BITS;
constexpr int SEL_PASSES = 64 / SEL_BITS;
constexpr int SEL_MAX_T = 16;
constexpr int SEL_THREADS = 1024;

struct SelTargets {
  int32_t n_t;                 // targets per layer
  int32_t n_rp;                // targets [0, n_rp) are PML ranks, the rest TVaR counts
  int64_t rank[SEL_MAX_T];     // 1-based rank from the top
};

struct SelState {
  uint64_t prefix;             // written at the end: the selected key
  int64_t k;                   // rank still to find among keys matching the prefix
};

// Scratch layout (one allocation, zero-filled before the launch):
//   hist   [n_layers][SEL_PASSES][n_t][SEL_BINS]  uint32
//   bar    [n_layers]                             uint32 grid-barrier counter of the layer
//   err    [1]                                    uint32: a grid barrier timed out
//   state  [n_layers][n_t]                        SelState
//   psum   [n_layers][n_t][blocks]                double   block partial: sum of y > key
//   pgt    [n_layers][n_t][blocks]                uint64   block partial: #{y > key}
//   peq    [n_layers][n_t][blocks]                uint64   block partial: #{y == key}
//   out    [n_layers][n_t]                        double   PML / TVaR
//   gt, eq [n_layers][n_t]                        uint64   totals
//   pmean  [n_layers][blocks]                     double   block partial of the row sum
//   mean   [n_layers]                             double
struct SelScratch {
  uint32_t* hist;
  uint32_t* bar;
  uint32_t* err;
  SelState* state;
  double* psum;
  unsigned long long* pgt;
  unsigned long long* peq;
  double* out;
  unsigned long long* gt;
  unsigned long long* eq;
  double* pmean;
  double* mean;
  uint32_t* ext_err;     // optional (nullptr): also gets DERR_TIMEOUT when a barrier times out
  // optional caller outputs, written directly (nullptr: results stay in out / mean only)
  double* user_pml;      // [n_layers][n_rp]
  double* user_tvar;     // [n_layers][n_t - n_rp]
  double* user_mean;     // [n_layers]
};

template <typename F>
static size_t layout(int32_t n_layers, int32_t n_t, int32_t blocks, F&& take) {
  const size_t lt = (size_t)n_layers * n_t, ltb = lt * blocks;
  size_t b = 0;
  auto t = [&](size_t n) { b = (b + 255) / 256 * 256; take(b); b += n; };
  t(sizeof(uint32_t) * SEL_PASSES * lt * SEL_BINS);
  t(sizeof(uint32_t) * n_layers);
  t(sizeof(uint32_t));
  t(sizeof(SelState) * lt);
  t(sizeof(double) * ltb);
  t(sizeof(uint64_t) * ltb);
  t(sizeof(uint64_t) * ltb);
  t(sizeof(double) * lt);
  t(sizeof(uint64_t) * lt);
  t(sizeof(uint64_t) * lt);
  t(sizeof(double) * (size_t)n_layers * blocks);
  t(sizeof(double) * n_layers);
  return (b + 255) / 256 * 256;
}

size_t select_scratch_bytes(int32_t n_layers, int32_t n_t, int32_t blocks) {
  return layout(n_layers, n_t, blocks, [](size_t) {});
}

static SelScratch carve(void* base, int32_t n_layers, int32_t n_t, int32_t blocks) {
  size_t off[12];
  int i = 0;
  layout(n_layers, n_t, blocks, [&](size_t o) { off[i++] = o; });
  char* p = (char*)base;
  SelScratch s;
  s.hist = (uint32_t*)(p + off[0]);
  s.bar = (uint32_t*)(p + off[1]);
  s.err = (uint32_t*)(p + off[2]);
  s.state = (SelState*)(p + off[3]);
  s.psum = (double*)(p + off[4]);
  s.pgt = (unsigned long long*)(p + off[5]);
  s.peq = (unsigned long long*)(p + off[6]);
  s.out = (double*)(p + off[7]);
  s.gt = (unsigned long long*)(p + off[8]);
  s.eq = (unsigned long long*)(p + off[9]);
  s.pmean = (double*)(p + off[10]);
  s.mean = (double*)(p + off[11]);
  s.ext_err = nullptr;
  s.user_pml = s.user_tvar = s.user_mean = nullptr;
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

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t sel_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch: every block adds one to *bar, then waits until it
// reaches `target` (the number of blocks times the barrier's ordinal).  The wait is bounded by
// limit_ns; on timeout the block sets *err (and DERR_TIMEOUT in *ext_err) and the whole block
// returns false.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t target, uint64_t limit_ns,
                                             uint32_t* err, uint32_t* ext_err, int skip_arrival,
                                             int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (!skip_arrival) atomicAdd(bar, 1u);
    int ok = 1;
    if (ld_acquire_gpu(bar) < target) {
      const uint64_t t0 = sel_globaltimer();
      while (ld_acquire_gpu(bar) < target) {
        if (sel_globaltimer() - t0 > limit_ns) {
          ok = 0;
          atomicOr(err, 1u);
          if (ext_err) atomicOr(ext_err, DERR_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

constexpr int SEL_WARPS = SEL_THREADS / 32;
// Values of a block's slice kept in shared memory across the passes (when the slice fits).
constexpr int SEL_SMEM_VALUES = 24000;

// Sub-histograms per block: S = SEL_SUBH / ng copies of each group's histogram, warp w adding
// into copy w mod S, so warps whose keys share a digit (in the first passes, nearly all) do not
// contend for one shared-memory word.
constexpr int SEL_SUBH = 32;

// The whole selection of the layers [l0, l0 + gridDim.y): up to 8 radix passes and the tail pass.
// Block b of a layer owns the contiguous slice [b n / B, (b + 1) n / B) of the layer's row;
// when it fits, the slice is read once into shared memory and every pass reads it there.
//
// Pass: the digit histogram of the keys that match each target's prefix.  Targets whose
// prefixes are equal share one histogram (in pass 0 all of them do), counted once and stored
// under the group's first target.  Equal digits within a warp are added with one
// shared-memory atomic (lanes grouped by __match_any_sync).  After the grid barrier every
// block picks each target's digit from the global histogram (one warp per target, bins
// scanned from the top) and keeps the selection state in shared memory.  The counts of the
// bins above the chosen one add up, over the passes, to #{key > selected key}; the chosen
// bin's count in the last pass is #{key == selected key}.  The passes stop early once every
// target's chosen bin holds a single key (distinct values near the targets, the usual case);
// one scan of the slice then finds those keys.
//
// Tail (TVaR targets and the row sum only): the sum of the values above the selected key.
// Every thread sums its own values in index order, warps and blocks combine with fixed trees,
// and after a last grid barrier block 0 of each layer combines the block partials in a fixed
// order: the sums are deterministic.
__global__ void __launch_bounds__(SEL_THREADS, 1)
k_select(const double* __restrict__ ylt, int64_t n, int32_t l0, SelTargets tg, SelScratch sc,
         int want_mean, uint64_t limit_ns, int64_t smem_values, int skip_arrival) {
  extern __shared__ double vals[];
  __shared__ uint32_t h[SEL_SUBH * SEL_BINS];
  __shared__ uint64_t pre[SEL_MAX_T];
  __shared__ int64_t kk[SEL_MAX_T];
  __shared__ unsigned long long cgt[SEL_MAX_T], ceq[SEL_MAX_T];
  __shared__ uint64_t gpre[SEL_MAX_T];      // prefix of each group
  __shared__ int32_t gldr[SEL_MAX_T];       // first target of each group
  __shared__ int32_t tgrp[SEL_MAX_T];       // group of each target
  __shared__ int32_t ngrp;
  __shared__ int bar_ok;
  __shared__ double wsum[SEL_WARPS];
  const int layer = l0 + blockIdx.y, nt = tg.n_t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // The blocks of a layer depend only on one another: each layer has its own barrier counter.
  const uint32_t nblk = gridDim.x;
  uint32_t* bar = sc.bar + layer;
  const int64_t i0 = (int64_t)blockIdx.x * n / gridDim.x;
  const int64_t cnt = ((int64_t)blockIdx.x + 1) * n / gridDim.x - i0;
  const double* src = ylt + (int64_t)layer * n + i0;
  const bool resident = cnt <= smem_values;   // smem_values: doubles of dynamic shared memory
  if (resident) {
    constexpr int U = 8;   // independent loads in flight per thread
    for (int64_t j = 0; j < cnt; j += (int64_t)U * SEL_THREADS) {
      double y[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = j + u * SEL_THREADS + threadIdx.x;
        y[u] = i < cnt ? __ldcg(src + i) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = j + u * SEL_THREADS + threadIdx.x;
        if (i < cnt) vals[i] = y[u];
      }
    }
  }
  if (threadIdx.x < nt) {
    pre[threadIdx.x] = 0ull;
    kk[threadIdx.x] = tg.rank[threadIdx.x];
    cgt[threadIdx.x] = 0ull;
    ceq[threadIdx.x] = 0ull;
  }
  __syncthreads();
  auto value = [&](int64_t i) -> double { return resident ? vals[i] : __ldcg(src + i); };

  const int passes = nt > 0 ? SEL_PASSES : 0;
  int done = passes;            // passes run
  for (int pass = 0; pass < passes; ++pass) {
    if (threadIdx.x == 0) {
      int ng = 0;
      for (int t = 0; t < nt; ++t) {
        int g = 0;
        while (g < ng && gpre[g] != pre[t]) ++g;
        if (g == ng) {
          gpre[g] = pre[t];
          gldr[g] = t;
          ++ng;
        }
        tgrp[t] = g;
      }
      ngrp = ng;
    }
    __syncthreads();
    const int ng = ngrp;
    int S = SEL_SUBH / ng;                 // sub-histograms per group (a power of two)
    S = 1 << (31 - __clz(S));
    for (int i = threadIdx.x; i < ng * S * SEL_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int shift = 64 - SEL_BITS * (pass + 1);
    uint32_t* hw = h + (warp & (S - 1)) * SEL_BINS;   // this warp's copy (group g: + g S BINS)
    for (int64_t j = 0; j < cnt; j += SEL_THREADS) {   // bound uniform over the block
      const int64_t i = j + threadIdx.x;
      const bool ok = i < cnt;
      const uint64_t key = key_of(ok ? value(i) : 0.0);
      const uint32_t d = (uint32_t)(key >> shift) & (SEL_BINS - 1);
      for (int g = 0; g < ng; ++g) {
        const bool m = ok && (pass == 0 || (key >> (shift + SEL_BITS)) == (gpre[g] >> (shift + SEL_BITS)));
        if (!__any_sync(0xffffffffu, m)) continue;
        const uint32_t peers = __match_any_sync(0xffffffffu, m ? d : 0xffffffffu);
        if (m && lane == __ffs(peers) - 1) atomicAdd(&hw[g * S * SEL_BINS + d], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    uint32_t* gh = sc.hist + ((int64_t)layer * SEL_PASSES + pass) * nt * SEL_BINS;
    for (int i = threadIdx.x; i < ng * SEL_BINS; i += blockDim.x) {
      const int g = i / SEL_BINS, d = i % SEL_BINS;
      uint32_t c = 0;
      for (int k = 0; k < S; ++k) c += h[(g * S + k) * SEL_BINS + d];
      if (c) atomicAdd(&gh[gldr[g] * SEL_BINS + d], c);
    }
    if (!grid_barrier(bar, (uint32_t)(pass + 1) * nblk, limit_ns, sc.err, sc.ext_err, skip_arrival, &bar_ok)) return;
    for (int t = warp; t < nt; t += SEL_WARPS) {
      const int64_t k = kk[t];
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
      if ((int64_t)excl < k && k <= (int64_t)incl) {
        int64_t before = excl;
        int u = 0;
        for (; u < SEL_BINS / 32; ++u) {
          if (before + c[u] >= k) break;
          before += c[u];
        }
        const uint32_t bin = SEL_BINS - 1 - (lane * (SEL_BINS / 32) + u);
        kk[t] = k - before;
        pre[t] |= (uint64_t)bin << shift;
        cgt[t] += (unsigned long long)before;           // keys above, with this prefix
        ceq[t] = c[u];                                  // keys with the new prefix
      }
    }
    __syncthreads();
    // When every target's prefix matches exactly one key, that key is the selected one and
    // the remaining passes would change no count: stop.  Every block of the layer read the
    // same histogram, so all of them stop after the same pass.
    bool unique = true;
    for (int t = 0; t < nt; ++t) unique = unique && ceq[t] == 1ull;
    if (unique) {
      done = pass + 1;
      break;
    }
  }
  // Key bits fixed by the passes run: [sh, 64).  Keys above the selected key are the keys whose
  // fixed bits are above its prefix (after a full selection sh = 0, the plain comparison).
  const int sh = done > 0 ? 64 - SEL_BITS * done : 0;
  auto above = [&](uint64_t key, uint64_t prefix) -> bool {
    return sh == 0 ? key > prefix : (key >> sh) > (prefix >> sh);
  };
  if (sh > 0) {   // stopped early: the one key under each target's prefix is its selected key
    for (int64_t i = threadIdx.x; i < cnt; i += SEL_THREADS) {
      const uint64_t key = key_of(value(i));
      for (int t = 0; t < nt; ++t)
        if ((key >> sh) == (pre[t] >> sh)) sc.state[(int64_t)layer * nt + t].prefix = key;
    }
  }

  // ---- tail pass: sums above the selected key (TVaR targets) and the row sum ----
  for (int t = tg.n_rp; t <= nt; ++t) {
    if (t == nt && !want_mean) break;
    const uint64_t thr = t < nt ? pre[t] : 0ull;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < cnt; i += SEL_THREADS) {
      const double y = value(i);
      if (t == nt || above(key_of(y), thr)) a = __dadd_rn(a, y);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, o));
    if (lane == 0) wsum[warp] = a;
    __syncthreads();
    if (warp == 0) {   // the warps' sums, combined by a fixed tree
      double s = wsum[lane];
#pragma unroll
      for (int o = 16; o; o >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
      if (lane == 0) {
        if (t < nt) sc.psum[((int64_t)layer * nt + t) * gridDim.x + blockIdx.x] = s;
        else sc.pmean[(int64_t)layer * gridDim.x + blockIdx.x] = s;
      }
    }
    __syncthreads();
  }
  if (!grid_barrier(bar, (uint32_t)(done + 1) * nblk, limit_ns, sc.err, sc.ext_err, skip_arrival, &bar_ok)) return;
  if (blockIdx.x != 0) return;
  // Block 0 of the layer: one warp per target (and one for the mean) combines the block
  // partials: lane l adds blocks l, l + 32, ... in order, then a fixed shuffle tree.
  const unsigned B = gridDim.x;
  for (int t = warp; t <= nt; t += SEL_WARPS) {
    if (t == nt && !want_mean) continue;
    double a = 0.0;
    if (t == nt) {
      for (unsigned b = lane; b < B; b += 32) a = __dadd_rn(a, __ldcg(&sc.pmean[(int64_t)layer * B + b]));
    } else if (t >= tg.n_rp) {
      const int64_t base = ((int64_t)layer * nt + t) * B;
      for (unsigned b = lane; b < B; b += 32) a = __dadd_rn(a, __ldcg(&sc.psum[base + b]));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, o));
    if (lane != 0) continue;
    if (t == nt) {
      sc.mean[layer] = a / (double)n;
      if (sc.user_mean) sc.user_mean[layer] = a / (double)n;
      continue;
    }
    const uint64_t key = sh > 0 ? __ldcg(&sc.state[(int64_t)layer * nt + t].prefix) : pre[t];
    const double v = value_of(key);
    double r = v;
    if (t >= tg.n_rp) {
      const int64_t m = tg.rank[t];
      r = (a + (double)(m - (int64_t)cgt[t]) * v) / (double)m;
    }
    sc.out[layer * nt + t] = r;
    if (t < tg.n_rp) {
      if (sc.user_pml) sc.user_pml[(int64_t)layer * tg.n_rp + t] = r;
    } else if (sc.user_tvar) {
      sc.user_tvar[(int64_t)layer * (nt - tg.n_rp) + (t - tg.n_rp)] = r;
    }
    sc.gt[layer * nt + t] = cgt[t];
    sc.eq[layer * nt + t] = ceq[t];
    sc.state[layer * nt + t] = SelState{key, kk[t]};
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

constexpr int SEL_DYN_SMEM = SEL_SMEM_VALUES * (int)sizeof(double);

// Co-resident blocks of k_select on this device (cached per device); 0 on failure.
static int select_resident_blocks() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[dev]) {
    int per_sm = 0, sms = 0;
    if (cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_DYN_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_select, SEL_THREADS, SEL_DYN_SMEM) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return 0;
    cached[dev] = per_sm * sms;
  }
  return cached[dev];
}

// Blocks per layer: one per SM for a single layer, fewer per layer when several share a
// launch, and never more than one per SEL_THREADS values.
int32_t select_blocks(int64_t n, int n_sms, int32_t n_layers) {
  const int64_t b = (n + SEL_THREADS - 1) / SEL_THREADS;
  const int64_t cap = std::max<int64_t>(1, (int64_t)n_sms / std::max(1, n_layers));
  return (int32_t)std::max<int64_t>(1, std::min(b, cap));
}

// Launch the whole selection into `scratch` (zero-filled here); results land in scratch.out.
// Layers are split into cooperative launches whose blocks are all co-resident.
ara_status launch_select(const double* d_ylt, int64_t n, int32_t n_layers, const SelTargets& tg,
                         void* scratch, size_t scratch_bytes, int32_t blocks, int want_mean,
                         cudaStream_t s, SelScratch* out, uint32_t* ext_err = nullptr,
                         double* user_pml = nullptr, double* user_tvar = nullptr,
                         double* user_mean = nullptr) {
  SelScratch sc = carve(scratch, n_layers, tg.n_t, blocks);
  sc.ext_err = ext_err;
  sc.user_pml = user_pml;
  sc.user_tvar = user_tvar;
  sc.user_mean = user_mean;
  ARA_TRY(cudaMemsetAsync(scratch, 0, scratch_bytes, s));
  const int resident = select_resident_blocks();
  if (resident < blocks) return ARA_ECUDA;
  const int32_t per_launch = std::max(1, resident / blocks);
  const uint64_t limit = wait_limit_ns();
  const int64_t slice = (n + blocks - 1) / blocks;
  const int dyn = slice <= SEL_SMEM_VALUES ? (int)(slice * sizeof(double)) : 0;
  for (int32_t l0 = 0; l0 < n_layers; l0 += per_launch) {
    const int32_t nl = std::min(per_launch, n_layers - l0);
    LaunchScope ls(ARA_K_SELECT, s);
    int64_t nn = n;
    int32_t ll0 = l0;
    SelTargets t2 = tg;
    SelScratch s2 = sc;
    int wm = want_mean;
    uint64_t lim = limit;
    int64_t cap = dyn / (int)sizeof(double);
    int skip = debug_skip_arrival();
    void* args[] = {(void*)&d_ylt, &nn, &ll0, &t2, &s2, &wm, &lim, &cap, &skip};
    ARA_TRY(cudaLaunchCooperativeKernel((const void*)k_select, dim3(blocks, nl), dim3(SEL_THREADS),
                                        args, (size_t)dyn, s));
  }
  *out = sc;
  return ARA_OK;
}

}  // namespace ara

using namespace ara;

namespace ara {

ara_status select_one_rank(const double* d_ylt, int64_t n, int32_t n_layers, int64_t m, int n_sms,
                           cudaStream_t s, SelectResult* out, uint32_t* err) {
  SelTargets tg;
  tg.n_t = 1;
  tg.n_rp = 0;
  tg.rank[0] = m;
  const int32_t blocks = select_blocks(n, n_sms, n_layers);
  const size_t bytes = select_scratch_bytes(n_layers, 1, blocks);
  void* scratch = nullptr;
  ARA_TRY(dmalloc_async(&scratch, bytes, s));
  SelScratch sc;
  ara_status st = launch_select(d_ylt, n, n_layers, tg, scratch, bytes, blocks, 0, s, &sc, err);
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
  ARA_TRY(dmalloc_async(&scratch, bytes, s));
  SelScratch sc;
  st = launch_select(d_ylt, n_trials, n_layers, tg, scratch, bytes, blocks, h_mean != nullptr, s, &sc);
  std::vector<double> out((size_t)n_layers * tg.n_t);
  uint32_t timed_out = 0;
  if (st == ARA_OK) {
    cudaError_t e = cudaMemcpyAsync(out.data(), sc.out, sizeof(double) * out.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_mean)
      e = cudaMemcpyAsync(h_mean, sc.mean, sizeof(double) * n_layers, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&timed_out, sc.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = ARA_ECUDA;
  }
  cudaFreeAsync(scratch, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
  if (st != ARA_OK) return st;
  if (timed_out) return ARA_ETIMEOUT;
  for (int32_t l = 0; l < n_layers; ++l) {
    for (int i = 0; i < n_rp; ++i) h_pml[(size_t)l * n_rp + i] = out[(size_t)l * tg.n_t + i];
    for (int i = 0; i < n_tvar; ++i) h_tvar[(size_t)l * n_tvar + i] = out[(size_t)l * tg.n_t + n_rp + i];
  }
  return ARA_OK;
}

}  // namespace ara

namespace ara {
// ara_risk_metrics_async with caller-owned scratch (the host pipeline keeps one per portfolio):
// ARA_ERANGE with *need set when scratch_bytes is too small, nothing queued.
ara_status risk_metrics_queue(const double* d_ylt, int64_t n_trials, int32_t n_layers, int32_t n_rp,
                              const double* rps, int32_t n_tvar, const double* levels,
                              double* d_pml, double* d_tvar, double* d_mean, uint32_t* d_status,
                              void* scratch, size_t scratch_bytes, size_t* need, cudaStream_t s) {
  SelTargets tg;
  if (!d_ylt || n_layers < 1 || !d_status || !need) return ARA_EINVAL;
  if ((n_rp > 0 && !d_pml) || (n_tvar > 0 && !d_tvar)) return ARA_EINVAL;
  if ((uintptr_t)d_ylt & 7) return ARA_EINVAL;
  ara_status st = select_targets(n_trials, n_rp, rps, n_tvar, levels, tg);
  if (st != ARA_OK) return st;
  if (tg.n_t == 0 && !d_mean) return ARA_EINVAL;
  int dev = 0, sms = 0;
  ARA_TRY(cudaGetDevice(&dev));
  ARA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int32_t blocks = select_blocks(n_trials, sms, n_layers);
  *need = select_scratch_bytes(n_layers, tg.n_t, blocks);
  if (!scratch || scratch_bytes < *need) return ARA_ERANGE;
  SelScratch sc;
  ARA_TRY(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
  return launch_select(d_ylt, n_trials, n_layers, tg, scratch, *need, blocks, d_mean != nullptr, s,
                       &sc, d_status, n_rp > 0 ? d_pml : nullptr, n_tvar > 0 ? d_tvar : nullptr,
                       d_mean);
}
}  // namespace ara

extern "C" ara_status ara_risk_metrics_async(const double* d_ylt, int64_t n_trials,
                                             int32_t n_layers, int32_t n_rp, const double* rps,
                                             int32_t n_tvar, const double* levels, double* d_pml,
                                             double* d_tvar, double* d_mean, uint32_t* d_status,
                                             void* stream) {
  SelTargets tg;
  if (!d_ylt || n_layers < 1 || !d_status) return ARA_EINVAL;
  if ((n_rp > 0 && !d_pml) || (n_tvar > 0 && !d_tvar)) return ARA_EINVAL;
  if ((uintptr_t)d_ylt & 7) return ARA_EINVAL;
  ara_status st = select_targets(n_trials, n_rp, rps, n_tvar, levels, tg);
  if (st != ARA_OK) return st;
  if (tg.n_t == 0 && !d_mean) return ARA_EINVAL;
  static_assert(ARA_DEVICE_TIMEOUT == DERR_TIMEOUT, "device timeout flag");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  ARA_TRY(cudaGetDevice(&dev));
  ARA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int32_t blocks = select_blocks(n_trials, sms, n_layers);
  const size_t bytes = select_scratch_bytes(n_layers, tg.n_t, blocks);
  void* scratch = nullptr;
  if (dmalloc_async(&scratch, bytes, s) != cudaSuccess) return ARA_ENOMEM;
  ara_status r = ARA_OK;
  SelScratch sc;
  if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s) != cudaSuccess) r = ARA_ECUDA;
  if (r == ARA_OK)   // the kernel writes the results straight into d_pml / d_tvar / d_mean
    r = launch_select(d_ylt, n_trials, n_layers, tg, scratch, bytes, blocks, d_mean != nullptr, s,
                      &sc, d_status, n_rp > 0 ? d_pml : nullptr, n_tvar > 0 ? d_tvar : nullptr,
                      d_mean);
  cudaFreeAsync(scratch, s);
  return r;
}

extern "C" ara_status ara_risk_metrics(const double* d_ylt, int64_t n_trials, int32_t n_layers,
                                       int32_t n_rp, const double* rps, int32_t n_tvar,
                                       const double* levels, double* h_pml, double* h_tvar,
                                       double* h_mean, void* stream) {
  return risk_metrics_device(d_ylt, n_trials, n_layers, n_rp, rps, n_tvar, levels, h_pml, h_tvar,
                             h_mean, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant: the selection scratch lives in a fixed device array of this
// library.  Host code cannot use the array's name as a device address, so every call looks the
// address up on the current device (with that device current).  The lookup is a cheap host
// query; not caching it keeps the address right after anything that tears down and recreates
// the device's primary context (cudaDeviceReset), which reloads the module elsewhere.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_select_scratch[ARA_STATIC_SELECT_BYTES];

static ara_status static_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
  if (e != cudaSuccess || !p) {
    note_cuda_error(e, "cudaGetSymbolAddress(g_select_scratch)", __FILE__, __LINE__);
    return ARA_ECUDA;
  }
  *out = p;
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
  if ((st = static_scratch(&scratch)) != ARA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SelScratch sc;
  // launch_select clears the used part of the scratch before its first kernel
  if ((st = launch_select(d_ylt, n_trials, n_layers, tg, scratch, bytes, blocks, h_mean != nullptr,
                          s, &sc)) != ARA_OK)
    return st;
  // Keep the first failing copy's status, but always wait for the stream before returning, so
  // that no copy queued here can land in the caller's buffers after the call has returned.
  cudaError_t e = cudaSuccess;
  const size_t row = sizeof(double) * (size_t)tg.n_t;
  if (e == cudaSuccess && n_rp > 0)
    e = cudaMemcpy2DAsync(h_pml, sizeof(double) * n_rp, sc.out, row, sizeof(double) * n_rp,
                          (size_t)n_layers, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && n_tvar > 0)
    e = cudaMemcpy2DAsync(h_tvar, sizeof(double) * n_tvar, sc.out + n_rp, row,
                          sizeof(double) * n_tvar, (size_t)n_layers, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && h_mean)
    e = cudaMemcpyAsync(h_mean, sc.mean, sizeof(double) * n_layers, cudaMemcpyDeviceToHost, s);
  uint32_t timed_out = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&timed_out, sc.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) note_cuda_error(e, "static risk metrics: result copy", __FILE__, __LINE__);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess && es != cudaSuccess) {
    note_cuda_error(es, "cudaStreamSynchronize", __FILE__, __LINE__);
    e = es;
  }
  if (e != cudaSuccess) return ARA_ECUDA;
  return timed_out ? ARA_ETIMEOUT : ARA_OK;
}

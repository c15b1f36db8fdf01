// YLT kernels: the per-layer fold of per-ELT and occurrence terms, and the YET stream.
//
// Section IV-B (Algorithm 3): for every trial, for every event, for every ELT of the layer,
// look the event up, apply the ELT terms, combine across the ELTs, apply the occurrence terms,
// add to the trial's aggregate loss; then apply the aggregate terms.  Occurrence terms act on
// each occurrence independently of the trial, so the occurrence loss o(e) is a function of
// the event alone.  The folded path computes o(e) once per catalogue event and layer
// (k_fold), then streams the YET with one table gather per occurrence whose o(e) is non-zero
// (k_ylt_folded).  k_ylt_per_elt keeps the literal per-occurrence, per-ELT lookups.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <optional>

#include "ara_device.cuh"

namespace ara {

constexpr int FOLD_THREADS = 128;
constexpr int YLT_THREADS = 1024;
constexpr int MAX_SEL = 256;

struct SelList {
  int32_t n;
  int32_t idx[MAX_SEL];
};



// ------------------------------------------------------------------------------------------
// Fold: o(e) = C(sum_j C(x_j(e); R_j, L_j); OccR, OccL) for every catalogue event e of one
// tile, for the layer sel.idx[blockIdx.y].  The ELT sum runs in the layer's ELT order, the
// order of the FP64 reference.  Output: the fixed point q(e) = round(o(e) * 2^frac_bits) (or the
// FP64 bits of o(e) when f64_table), and the hit bitmap (bit e set iff the stored value is
// non-zero).
// ------------------------------------------------------------------------------------------
struct FoldOut {
  uint64_t* q;          // table, or nullptr
  uint32_t* bits;       // hit bitmap
  uint8_t* regime;      // occurrence-clamp regime per event (0 / 1 / 2), or nullptr
  int64_t q_stride, bits_stride, regime_stride;   // per output slot
  int by_slot;          // outputs indexed by blockIdx.y (else by layer index)
  int f64_table;        // store the FP64 bits of o(e) instead of fixed point
  int bits_from_regime; // bitmap bit = (regime != 0) instead of (stored value != 0)
  int nonzero_only;     // store only the non-zero table entries (readers consult the bitmap)
};

constexpr int FOLD_GROUP = 32;     // ELTs whose record ranges are searched together
constexpr int FOLD_REC = 512;      // records staged in shared memory per window
// Occupancy: FOLD_THREADS threads and about 28 KB of static shared memory per block give 7
// blocks per SM (the launch bounds keep the registers within that), so the 977 tiles of a
// 2 M-event catalogue run in one wave on 152 SMs.

template <typename LossT>
__global__ void __launch_bounds__(FOLD_THREADS, 7)
k_fold(int64_t catalogue, const int64_t* __restrict__ tile_rec, int64_t n_tiles,
       const int32_t* __restrict__ rec_ids,
       const LossT* __restrict__ rec_loss, const double* __restrict__ elt_ret,
       const double* __restrict__ elt_lim, const int32_t* __restrict__ layer_elts,
       const LayerConst* __restrict__ layers, SelList sel, FoldOut out) {
  static_assert(FOLD_TILE % FOLD_THREADS == 0 && FOLD_TILE <= 65536, "tile layout");
  __shared__ double s[FOLD_TILE];
  __shared__ double rx[FOLD_REC];            // staged records after the ELT terms
  __shared__ uint16_t rev[FOLD_REC];         // their events, relative to the tile
  __shared__ uint16_t touched[FOLD_TILE];    // events whose sum became non-zero, in that order
  __shared__ uint8_t reg[FOLD_TILE];
  __shared__ int64_t lo[FOLD_GROUP];
  __shared__ double eR[FOLD_GROUP], eL[FOLD_GROUP];
  __shared__ int32_t cnt_off[FOLD_GROUP + 1];
  __shared__ int32_t n_list;
  const int layer = sel.idx[blockIdx.y];
  const int64_t slot = out.by_slot ? blockIdx.y : layer;
  const LayerConst lc = layers[layer];
  const int64_t t0 = (int64_t)blockIdx.x * FOLD_TILE;
  const int64_t t1 = min(t0 + (int64_t)FOLD_TILE, catalogue);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool want_regime = out.regime != nullptr || out.bits_from_regime;
#pragma unroll
  for (int i = threadIdx.x; i < FOLD_TILE; i += FOLD_THREADS) s[i] = 0.0;
  if (want_regime)
    for (int i = threadIdx.x; i < FOLD_TILE; i += FOLD_THREADS) reg[i] = 0;
  int n_touched = 0;   // kept by warp 0
  if (threadIdx.x == 0) n_list = 0;
  // The layer's ELTs in order, in groups of up to FOLD_GROUP: warp 0 reads the group's record
  // ranges within this tile from the portfolio's tile index.  The group's records, taken ELT
  // after ELT, are then handled in windows of FOLD_REC (an ELT may straddle two windows): all
  // threads stage a window's records with their ELT terms applied (one record per thread, so
  // that the FP64 instructions run on full warps), then warp 0 adds them into the tile in that
  // order, which keeps every event's FP64 sum in the layer's ELT order (IDs are unique within an
  // ELT, so the lanes never collide within one ELT).
  for (int k0 = lc.elt_begin; k0 < lc.elt_end; k0 += FOLD_GROUP) {
    const int G = min(FOLD_GROUP, lc.elt_end - k0);
    if (warp == 0) {
      int32_t c = 0;
      if (lane < G) {
        const int j = layer_elts[k0 + lane];
        const int64_t* tr = tile_rec + (int64_t)j * (n_tiles + 1) + blockIdx.x;
        const int64_t a = tr[0];
        lo[lane] = a;
        c = (int32_t)(tr[1] - a);
        eR[lane] = elt_ret[j];
        eL[lane] = elt_lim[j];
      }
      int32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
      }
      cnt_off[lane + 1] = incl;
      if (lane == 0) cnt_off[0] = 0;
    }
    __syncthreads();
    const int32_t total = cnt_off[G];
    if (total == 0) {   // no window: every thread reads total before warp 0 rewrites the ranges
      __syncthreads();
      continue;
    }
    for (int32_t w0 = 0; w0 < total; w0 += FOLD_REC) {
      // Between two windows of a group: warp 0 is done adding the previous window before it
      // is restaged.  (Before a group's first window, the group's barrier above does this.)
      if (w0 > 0) __syncthreads();
      const int32_t wn = min(FOLD_REC, total - w0);
      for (int i = threadIdx.x; i < wn; i += FOLD_THREADS) {
        const int32_t x = w0 + i;
        int g = 0;   // the group ELT of record x: the last g < G with cnt_off[g] <= x
#pragma unroll
        for (int step = FOLD_GROUP / 2; step > 0; step >>= 1)
          if (g + step < G && cnt_off[g + step] <= x) g += step;
        const int64_t r = lo[g] + (x - cnt_off[g]);
        rev[i] = (uint16_t)(rec_ids[r] - t0);
        rx[i] = clamp_terms_bits(to_f64(rec_loss[r]), eR[g], eL[g]);
      }
      __syncthreads();
      if (warp == 0) {
        const int32_t w1 = w0 + wn;
        for (int g = 0; g < G; ++g) {
          const int32_t a = max(cnt_off[g], w0) - w0, b1 = min(cnt_off[g + 1], w1) - w0;
          for (int i = a + lane; i - lane < b1; i += 32) {
            bool first = false;
            int e = 0;
            if (i < b1) {
              e = rev[i];
              const double old = s[e], x = rx[i];
              s[e] = __dadd_rn(old, x);
              // Sums only grow (the ELT terms give x >= 0), so an event turns non-zero exactly
              // once: when a zero sum meets a non-zero x (tested on the bits, off the add's path).
              first = ((uint64_t)__double_as_longlong(old) << 1) == 0ull &&
                      ((uint64_t)__double_as_longlong(x) << 1) != 0ull;
            }
            const unsigned m = __ballot_sync(FULL, first);
            if (first) touched[n_touched + __popc(m & ((1u << lane) - 1u))] = (uint16_t)e;
            n_touched += __popc(m);
          }
          __syncwarp();
        }
        if (lane == 0) n_list = n_touched;
      }
    }
    // No barrier here: the next group's barrier keeps the other warps' staging away from the
    // records warp 0 is still adding, and warp 0 rewrites the ranges only after its adds.
  }
  __syncthreads();
  const int n_nz = n_list;
  uint64_t* sq = reinterpret_cast<uint64_t*>(s);  // in place: untouched entries are +0.0 == 0
  for (int p = threadIdx.x; p < n_nz; p += FOLD_THREADS) {
    const int i = touched[p];
    const double sv = s[i];
    const double o = clamp_terms(sv, lc.occ_ret, lc.occ_lim);
    if (want_regime) {
      const double ex = __dsub_rn(sv, lc.occ_ret);
      reg[i] = (ex > 0.0 && ex < lc.occ_lim) ? 1 : (ex > lc.occ_lim ? 2 : 0);
    }
    sq[i] = out.f64_table ? (uint64_t)__double_as_longlong(o) : __double2ull_rn(__dmul_rn(o, lc.scale));
  }
  __syncthreads();
  uint64_t* qo = out.q ? out.q + slot * out.q_stride : nullptr;
  uint32_t* bo = out.bits + slot * out.bits_stride;
  uint8_t* ro = out.regime ? out.regime + slot * out.regime_stride : nullptr;
#pragma unroll 4
  for (int i = threadIdx.x; i < FOLD_TILE; i += FOLD_THREADS) {
    const int64_t e = t0 + i;
    const bool in = e < t1;
    const uint64_t q = in ? sq[i] : 0ull;
    const uint8_t r = (in && want_regime) ? reg[i] : 0;
    if (in && qo && (q != 0ull || !out.nonzero_only)) qo[e] = q;
    if (in && ro) ro[e] = r;
    const unsigned b = __ballot_sync(FULL, out.bits_from_regime ? r != 0 : q != 0ull);
    if (lane == 0) {
      const int64_t w = (t0 + (i & ~31)) >> 5;
      if (w < out.bits_stride) bo[w] = b;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Stream helpers
// ------------------------------------------------------------------------------------------
// Coarse hit bitmap word cw, interleaved: coarse bit i is the OR of bit i of the exact words
// [cw << shift, (cw + 1) << shift), i.e. of the hit bits of the 2^shift events e with
// e >> (5 + shift) == cw and e mod 32 == i.  A lookup therefore reads word e >> (5 + shift)
// and tests bit e mod 32, the same bit position as in the exact bitmap.
__device__ __forceinline__ uint32_t coarsen_word(const uint32_t* __restrict__ src, int64_t cw,
                                                 int shift, int64_t n_words) {
  const int64_t w0 = cw << shift;
  const int64_t w1 = min(w0 + ((int64_t)1 << shift), n_words);
  uint32_t out = 0;
  for (int64_t w = w0; w < w1; ++w) out |= src[w];
  return out;
}

struct StreamParams {
  int64_t n_trials;
  const int64_t* offsets;
  int64_t id_base;
  int64_t n_events;
  const int32_t* ids;
  int32_t mis;             // (address of ids >> 2) & 3: element index of the 16-byte frame
  int32_t shift;           // bitmap coarsening
  int64_t catalogue;
  const uint64_t* q;       // this layer's table
  const uint32_t* bits;    // this layer's exact bitmap
  int64_t bm_words;
  int64_t smem_words;
  const LayerConst* layer;
  double* ylt;             // this layer's YLT row
  uint8_t* regimes;        // this layer's regime row or nullptr
  uint32_t* err;
  uint64_t wait_limit_ns;  // bound of every mbarrier wait
  uint32_t debug_extra_tx; // test hook: bytes announced but never copied (0 in normal use)
  uint32_t word_bytes;     // 4 (bytes per bitmap word), passed at run time for the address IMAD
};

// One event ID: range check, hit filter, gather, accumulate.
template <bool FILTER, typename Acc>
__device__ __forceinline__ void consume(int e, bool valid, const StreamParams& p,
                                        const uint32_t* bm, const uint64_t* __restrict__ q,
                                        Acc& acc, bool& bad) {
  if (!valid) return;
  if ((unsigned)e >= (unsigned)p.catalogue) { bad = true; return; }
  if (FILTER) {
    if (!((bm[(uint32_t)e >> (p.shift + 5)] >> (e & 31)) & 1u)) return;
  }
  AccOps<Acc>::add(acc, __ldg(q + e));
}

// ------------------------------------------------------------------------------------------
// Folded YET stream.  A warp owns groups of 32 consecutive trials; for each trial the warp
// reads the trial's event IDs with coalesced 16-byte streaming loads (scalar loads for the
// unaligned head and tail), tests each ID against the layer's hit bitmap held in shared
// memory, gathers q(e) from the L2-resident table only on hits, and sums exactly.  Lane k
// keeps trial k's sum; the aggregate terms of all 32 trials run at once at the end.
// ------------------------------------------------------------------------------------------
template <bool FILTER, typename Acc, int U>
__global__ void __launch_bounds__(YLT_THREADS, 1) k_ylt_folded(StreamParams p) {
  extern __shared__ uint32_t bm[];
  if (FILTER) {
    for (int64_t cw = threadIdx.x; cw < p.smem_words; cw += blockDim.x)
      bm[cw] = coarsen_word(p.bits, cw, p.shift, p.bm_words);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const LayerConst lc = *p.layer;
  const uint64_t* __restrict__ q = p.q;
  const int4* __restrict__ base4 = reinterpret_cast<const int4*>(p.ids - p.mis);
  const int64_t n_groups = (p.n_trials + 31) >> 5;
  bool bad_id = false, bad_off = false;

  for (int64_t g = warp; g < n_groups; g += nwarps) {
    const int64_t t0 = g << 5;
    const int nt = (int)min((int64_t)32, p.n_trials - t0);
    const int64_t my_off = (lane <= nt) ? __ldg(p.offsets + t0 + lane) - p.id_base : 0;
    const int64_t last_off = (nt == 32) ? __ldg(p.offsets + t0 + 32) - p.id_base : 0;
    Acc mine = AccOps<Acc>::zero();
    for (int k = 0; k < nt; ++k) {
      int64_t beg = __shfl_sync(FULL, my_off, k);
      int64_t end = (k + 1 < 32) ? __shfl_sync(FULL, my_off, k + 1) : last_off;
      if (!(0 <= beg && beg <= end && end <= p.n_events)) { bad_off = true; beg = end = 0; }
      Acc acc = AccOps<Acc>::zero();
      const int64_t pb = beg + p.mis, pe = end + p.mis;
      const int64_t vb = (pb + 3) >> 2, ve = pe >> 2;
      {  // scalar edges: the unaligned head and tail (all of a trial with no full vector)
        int64_t pos = -1;
        if (vb >= ve) {
          if (lane < pe - pb) pos = pb + lane;
        } else {
          const int nh = (int)(4 * vb - pb), ntl = (int)(pe - 4 * ve);
          if (lane < nh) pos = pb + lane;
          else if (lane >= 4 && lane < 4 + ntl) pos = 4 * ve + (lane - 4);
        }
        const int e = pos >= 0 ? __ldg(p.ids + (pos - p.mis)) : 0;
        consume<FILTER>(e, pos >= 0, p, bm, q, acc, bad_id);
      }
      for (int64_t v = vb + lane; v < ve; v += 32 * U) {
        int4 x[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          ok[u] = v + 32 * u < ve;
          x[u] = ok[u] ? __ldcs(base4 + v + 32 * u) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          consume<FILTER>(x[u].x, ok[u], p, bm, q, acc, bad_id);
          consume<FILTER>(x[u].y, ok[u], p, bm, q, acc, bad_id);
          consume<FILTER>(x[u].z, ok[u], p, bm, q, acc, bad_id);
          consume<FILTER>(x[u].w, ok[u], p, bm, q, acc, bad_id);
        }
      }
      acc = AccOps<Acc>::warp_sum(acc);
      if (lane == k) mine = acc;
    }
    if (lane < nt) {
      uint8_t reg;
      const double y = AccOps<Acc>::finish(mine, lc, reg);
      p.ylt[t0 + lane] = y;
      if (p.regimes) p.regimes[t0 + lane] = reg;
    }
  }
  if (bad_id) atomicOr(p.err, DERR_EVENT_RANGE);
  if (bad_off) atomicOr(p.err, DERR_OFFSETS);
}

// ------------------------------------------------------------------------------------------
// Bulk-staged YET stream (the default).  Warp w of the grid owns the contiguous trials
// [w N / W, (w+1) N / W) and therefore one contiguous range of event IDs.  It streams that range
// through its own ring of BK_STAGES shared-memory stages of BK_CHUNK_IDS IDs, each filled by one
// cp.async.bulk (TMA bulk copy, L2 evict-first) that completes on the stage's mbarrier; lane 0
// refills a stage as soon as the warp has read it, so BK_STAGES - 1 chunks are in flight while
// one is processed, across trial boundaries.  The unaligned head and tail of the range (< 4 IDs
// each) use plain loads.  Positions are attributed to trials by a segmented walk over the
// trial offsets (prefetched 32 at a time), with the per-lane partial sums reduced at each trial
// end (three redux.sync limb sums); lane k of a group collects trial k's sum and the aggregate
// terms of 32 trials run at once.
// Every mbarrier wait is bounded: on timeout the warp records DERR_TIMEOUT, waits (bounded) for
// its own copies still in flight, and returns.
// ------------------------------------------------------------------------------------------
template <int WARPS, int STAGES, int CHUNK> struct BulkShape {
  static constexpr int ring_bytes = WARPS * STAGES * CHUNK * 4;
  static constexpr int bar_bytes = WARPS * STAGES * 8;
};

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)),
      "l"(pol) : "memory");
}
// Test a phase of an mbarrier; while it is incomplete the thread is suspended (not spinning)
// until the phase completes or about hint_ns nanoseconds pass.  False if it is still incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns) : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for a phase of an mbarrier for at most about limit_ns nanoseconds; false on timeout.
// Each try suspends the warp for up to kWaitHintNs, so a warp whose copy is still in flight
// leaves its issue slots to the others instead of spinning.
constexpr uint32_t kWaitHintNs = 20000;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t hint = limit_ns < kWaitHintNs ? (uint32_t)limit_ns : kWaitHintNs;
  if (mbar_try_wait(bar, parity, hint)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity, hint)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Coarse hit bitmap of a layer, built once per run when the exact one does not fit in shared
// memory, in the interleaved layout of coarsen_word.
__global__ void k_coarsen(const uint32_t* __restrict__ exact, int64_t n_exact, int shift,
                          uint32_t* __restrict__ coarse, int64_t n_coarse) {
  for (int64_t cw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cw < n_coarse;
       cw += (int64_t)gridDim.x * blockDim.x)
    coarse[cw] = coarsen_word(exact, cw, shift, n_exact);
}

// Table value of one event for the bulk stream.  The event index is clamped into the catalogue
// for addressing (an out-of-range ID is caught by the caller's running maximum, which makes the
// whole run a data error).  The hit bit is bit (e mod 32) of shared-memory word
// e >> (5 + shift) (a funnel shift takes its count mod 32, so no mask is needed); the word's
// byte address floor(e * 2^(32 - 5 - shift) / 2^32) * 4 + base is formed with a high multiply
// and a multiply-add whose factors are run-time parameters, which keeps it on the FMA pipe
// (the integer ALU pipe is this kernel's busiest).  The gather is predicated, with its 64-bit
// address formed by one wide multiply-add, and cached in L2 only (.cg): random table entries are
// almost never reused from L1.
struct BitmapAddr {
  uint32_t base;   // shared-memory address of word 0
  uint32_t mul;    // 2^(32 - 5 - shift)
  uint32_t four;   // 4, bytes per word
};

template <bool FILTER>
__device__ __forceinline__ uint64_t bulk_value(int e, uint32_t cat1, const BitmapAddr& ba,
                                               const uint64_t* __restrict__ q) {
  const uint32_t ce = min((uint32_t)e, cat1);
  uint32_t hit = 1u;
  if (FILTER) {
    uint32_t word;
    asm("{\n\t.reg .u32 w, a;\n\tmul.hi.u32 w, %1, %2;\n\tmad.lo.u32 a, w, %3, %4;\n\t"
        "ld.shared.u32 %0, [a];\n\t}"
        : "=r"(word) : "r"(ce), "r"(ba.mul), "r"(ba.four), "r"(ba.base));
    hit = __funnelshift_r(word, 0u, ce) & 1u;
  }
  uint64_t v = 0;
  asm("{\n\t.reg .pred p;\n\t.reg .u64 a;\n\tsetp.ne.u32 p, %2, 0;\n\t"
      "mad.wide.u32 a, %3, 8, %1;\n\t@p ld.global.cg.u64 %0, [a];\n\t}"
      : "+l"(v) : "l"(q), "r"(hit), "r"(ce));
  return v;
}

// State of one warp's walk over its trials (all fields warp-uniform except acc/res, which are
// per-lane partial sums).  Positions and trial numbers are relative to the warp's range.
template <typename Acc>
struct Walk {
  int32_t k;        // current trial, relative to t_lo
  int32_t nk;       // number of trials of the warp
  int32_t end;      // relative end position of trial k
  int32_t span;     // E1 - E0
  int32_t gbase;    // first trial of the current group of 32
  int32_t bbase;    // trial whose end is in lane 0 of nxt
  int32_t nxt;      // lane i: relative end of trial bbase + i
  bool bad;
  typename LaneOps<Acc>::T acc;   // this lane's partial of trial k
  Acc res;                        // lane (t - gbase): the sum of trial t of the current group
};

template <typename Acc>
__device__ __forceinline__ void walk_load_ends(Walk<Acc>& w, const StreamParams& p, int64_t t_lo,
                                               int64_t base_abs, int lane) {
  const int64_t t = t_lo + w.bbase + 1 + lane;       // trial end index into offsets
  int32_t v = w.span;
  if (w.bbase + 1 + lane <= w.nk) {
    const int64_t rel = __ldg(p.offsets + t) - base_abs;
    v = (rel < 0 || rel > w.span) ? -1 : (int32_t)rel;
  }
  w.nxt = v;
}

// Finish trial k: reduce the lanes' partial sums, park the sum in lane (k - gbase), flush a
// full group of 32 (aggregate terms for all of them at once), move to trial k + 1.
template <typename Acc>
__device__ __forceinline__ void walk_finish(Walk<Acc>& w, const StreamParams& p, const LayerConst& lc,
                                         int64_t t_lo, int64_t base_abs, int lane) {
  const Acc r = LaneOps<Acc>::reduce(w.acc);
  if (lane == w.k - w.gbase) w.res = r;
  w.acc = LaneOps<Acc>::zero();
  const int32_t prev = w.end;
  ++w.k;
  if (w.k - w.gbase == 32 || w.k == w.nk) {
    if (w.gbase + lane < w.k) {
      uint8_t reg;
      const double y = AccOps<Acc>::finish(w.res, lc, reg);
      p.ylt[t_lo + w.gbase + lane] = y;
      if (p.regimes) p.regimes[t_lo + w.gbase + lane] = reg;
    }
    w.res = AccOps<Acc>::zero();
    w.gbase = w.k;
  }
  if (w.k < w.nk) {
    if (w.k - w.bbase == 32) {
      w.bbase = w.k;
      walk_load_ends(w, p, t_lo, base_abs, lane);
    }
    w.end = __shfl_sync(FULL, w.nxt, w.k - w.bbase);
    if (w.end < prev) {          // out of [0, span] (-1) or decreasing: bad offsets
      w.bad = true;
      w.end = w.span;
    }
  }
}

// Slow path: attribute values at relative positions pos[i] (< 0: none) of the window
// [rb, re) to trials, finishing every trial that ends inside the window.
template <typename Acc, int K>
__device__ __forceinline__ void walk_window(Walk<Acc>& w, const StreamParams& p, const LayerConst& lc,
                                            int64_t t_lo, int64_t base_abs, int lane, int32_t rb,
                                            int32_t re, const int32_t (&pos)[K],
                                            const uint64_t (&val)[K]) {
  int32_t done = rb;
  while (true) {
    while (w.k < w.nk && w.end <= done) walk_finish(w, p, lc, t_lo, base_abs, lane);
    if (w.k >= w.nk) return;
    const int32_t seg = min(w.end, re);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (pos[i] >= done && pos[i] < seg) LaneOps<Acc>::add(w.acc, val[i]);
    done = seg;
    if (done >= re) return;
  }
}

template <bool FILTER, typename Acc, int BK_WARPS, int BK_STAGES, int BK_CHUNK_IDS>
__global__ void __launch_bounds__(BK_WARPS * 32, 1) k_ylt_bulk(StreamParams p) {
  constexpr int NV = BK_CHUNK_IDS / 32;               // values per lane per chunk
  constexpr int NQ = BK_CHUNK_IDS / 128;              // 16-byte loads per lane per chunk
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int64_t bm_bytes = FILTER ? ((p.smem_words * 4 + 127) / 128) * 128 : 0;
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* ring = reinterpret_cast<int32_t*>(smem_raw + bm_bytes) + wid * BK_STAGES * BK_CHUNK_IDS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + bm_bytes +
                                               BulkShape<BK_WARPS, BK_STAGES, BK_CHUNK_IDS>::ring_bytes) +
                   wid * BK_STAGES;
  if (lane == 0)
    for (int s = 0; s < BK_STAGES; ++s) mbar_init(&bars[s], 1);
  if (FILTER) {  // the layer's (coarse) hit bitmap, 16 bytes per thread per step
    const uint4* src = reinterpret_cast<const uint4*>(p.bits);
    uint4* dst = reinterpret_cast<uint4*>(bm);
    const int64_t n16 = (p.smem_words + 3) / 4;   // source padded to whole 16-byte words
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  if (lane == 0) fence_mbar_init();
  __syncthreads();

  const int64_t W = (int64_t)gridDim.x * BK_WARPS;
  const int64_t gw = (int64_t)blockIdx.x * BK_WARPS + wid;
  const int64_t t_lo = gw * p.n_trials / W, t_hi = (gw + 1) * p.n_trials / W;
  if (t_lo >= t_hi) return;
  const LayerConst lc = *p.layer;
  const uint64_t* __restrict__ q = p.q;
  const uint32_t cat = (uint32_t)p.catalogue;
  BitmapAddr ba;
  ba.base = smem_u32(bm);
  ba.mul = 1u << (32 - 5 - p.shift);   // shift <= 26: the coarse bitmap always has >= 2 words
  ba.four = p.word_bytes;

  const int64_t E0 = __ldg(p.offsets + t_lo) - p.id_base;
  const int64_t E1 = __ldg(p.offsets + t_hi) - p.id_base;
  // A warp's range stays below 2^31 - 512 events: relative positions fit in int32, and no lane
  // holds 2^26 or more values of one trial, the bound the warp reduction of the split partials
  // relies on.
  constexpr int64_t kMaxWarpSpan = ((int64_t)1 << 31) - 512;
  if (!(0 <= E0 && E0 <= E1 && E1 <= p.n_events && E1 - E0 < kMaxWarpSpan)) {
    if (lane == 0) atomicOr(p.err, DERR_OFFSETS);
    return;
  }
  const int64_t base_abs = E0 + p.id_base;          // absolute offset of relative position 0
  Walk<Acc> w;
  w.k = 0;
  w.nk = (int32_t)(t_hi - t_lo);
  w.span = (int32_t)(E1 - E0);
  w.gbase = 0;
  w.bbase = 0;
  w.bad = false;
  w.acc = LaneOps<Acc>::zero();
  w.res = AccOps<Acc>::zero();
  walk_load_ends(w, p, t_lo, base_abs, lane);
  w.end = __shfl_sync(FULL, w.nxt, 0);
  if (w.end < 0) { w.bad = true; w.end = w.span; }
  uint32_t emax = 0;                 // largest event ID seen (as unsigned): >= catalogue is an error
  const uint32_t cat1 = cat - 1u;
  auto val_of = [&](int e, bool valid) -> uint64_t {
    if (!valid) return 0ull;
    emax = max(emax, (uint32_t)e);
    return bulk_value<FILTER>(e, cat1, ba, q);
  };

  // Frame: element i at frame position i + mis; 16-byte vectors at frame multiples of 4.
  const int32_t mis_head = (int32_t)((4 - ((E0 + p.mis) & 3)) & 3);
  const int32_t head = min(mis_head, w.span);
  const int32_t n_body = ((w.span - head) >> 2) << 2;
  const int32_t tail0 = head + n_body;
  // head and tail (< 4 IDs each): scalar loads, slow path
  if (head > 0) {
    int32_t pos[1] = {lane < head ? lane : -1};
    uint64_t val[1] = {val_of(lane < head ? __ldg(p.ids + E0 + lane) : 0, lane < head)};
    walk_window<Acc, 1>(w, p, lc, t_lo, base_abs, lane, 0, head, pos, val);
  }
  const int32_t n_chunks = (n_body + BK_CHUNK_IDS - 1) / BK_CHUNK_IDS;
  const int32_t* gbase = p.ids + E0 + head;          // 16-byte aligned
  const uint64_t pol = l2_evict_first_policy();
  if (lane == 0)
    for (int32_t ch = 0; ch < min(BK_STAGES, n_chunks); ++ch) {
      const int32_t n = min(BK_CHUNK_IDS, n_body - ch * BK_CHUNK_IDS);
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[ch], (uint32_t)n * 4 + p.debug_extra_tx);
      bulk_g2s(ring + ch * BK_CHUNK_IDS, gbase + ch * BK_CHUNK_IDS, (uint32_t)n * 4, &bars[ch], pol);
    }
  __syncwarp();
  int32_t timed_out_at = -1;
  int s = 0;                 // stage of chunk ch (ch mod BK_STAGES) and its mbarrier phase parity
  uint32_t phase = 0;
  for (int32_t ch = 0; ch < n_chunks; ++ch) {
    const bool ok = mbar_wait_bounded(&bars[s], phase, p.wait_limit_ns);
    if (__any_sync(FULL, !ok)) { timed_out_at = ch; break; }
    const int32_t rb = head + ch * BK_CHUNK_IDS;
    const int32_t n = min(BK_CHUNK_IDS, n_body - ch * BK_CHUNK_IDS);
    // lane l holds chunk slots 128u + 4l .. 128u + 4l + 3 for u < NQ (conflict-free 16-byte loads)
    int4 ids4[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u)
      ids4[u] = reinterpret_cast<const int4*>(ring + s * BK_CHUNK_IDS)[32 * u + lane];
    __syncwarp();
    if (lane == 0 && ch + BK_STAGES < n_chunks) {
      const int32_t c2 = ch + BK_STAGES;
      const int32_t n2 = min(BK_CHUNK_IDS, n_body - c2 * BK_CHUNK_IDS);
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[s], (uint32_t)n2 * 4 + p.debug_extra_tx);
      bulk_g2s(ring + s * BK_CHUNK_IDS, gbase + c2 * BK_CHUNK_IDS, (uint32_t)n2 * 4, &bars[s], pol);
    }
    uint64_t v[NV];
    if (n == BK_CHUNK_IDS) {        // full chunk: every slot is a real event
#pragma unroll
      for (int u = 0; u < NQ; ++u) {
        emax = __vimax3_u32(emax, (uint32_t)ids4[u].x, (uint32_t)ids4[u].y);
        emax = __vimax3_u32(emax, (uint32_t)ids4[u].z, (uint32_t)ids4[u].w);
        v[4 * u + 0] = bulk_value<FILTER>(ids4[u].x, cat1, ba, q);
        v[4 * u + 1] = bulk_value<FILTER>(ids4[u].y, cat1, ba, q);
        v[4 * u + 2] = bulk_value<FILTER>(ids4[u].z, cat1, ba, q);
        v[4 * u + 3] = bulk_value<FILTER>(ids4[u].w, cat1, ba, q);
      }
    } else {
#pragma unroll
      for (int u = 0; u < NQ; ++u) {
        const int sl = 128 * u + 4 * lane;
        v[4 * u + 0] = val_of(ids4[u].x, sl + 0 < n);
        v[4 * u + 1] = val_of(ids4[u].y, sl + 1 < n);
        v[4 * u + 2] = val_of(ids4[u].z, sl + 2 < n);
        v[4 * u + 3] = val_of(ids4[u].w, sl + 3 < n);
      }
    }
    while (w.k < w.nk && w.end <= rb) walk_finish(w, p, lc, t_lo, base_abs, lane);
    if (w.k < w.nk && w.end >= rb + n) {
      // fast path: the whole chunk belongs to the current trial
      LaneOps<Acc>::add_all(w.acc, v);
    } else {
      // A trial ends inside the chunk, at relative slot r (0 < r < n).  Lane l's values sit in
      // runs of four consecutive slots 128u + 4l + j, so the end splits run u at
      // js = clamp(r - 128u - 4l, 0, 4): values j < js finish the current trial, the others
      // start the next one.  More than one end in the chunk takes the general walk.
      int32_t done = rb;
      if (w.k < w.nk) {
        const int32_t r = w.end - rb;
        int32_t js[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) js[u] = min(max(r - 128 * u - 4 * lane, 0), 4);
#pragma unroll
        for (int u = 0; u < NQ; ++u)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < js[u]) LaneOps<Acc>::add(w.acc, v[4 * u + j]);
        walk_finish(w, p, lc, t_lo, base_abs, lane);
        done = rb + r;
        if (w.k < w.nk && w.end >= rb + n) {
#pragma unroll
          for (int u = 0; u < NQ; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (j >= js[u]) LaneOps<Acc>::add(w.acc, v[4 * u + j]);
          done = rb + n;
        }
      }
      if (done < rb + n) {
        int32_t pos[NV];
#pragma unroll
        for (int u = 0; u < NQ; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i) pos[4 * u + i] = rb + 128 * u + 4 * lane + i;
        walk_window<Acc, NV>(w, p, lc, t_lo, base_abs, lane, done, rb + n, pos, v);
      }
    }
    if (++s == BK_STAGES) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (timed_out_at >= 0) {
    // chunks timed_out_at .. timed_out_at + BK_STAGES - 1 may still be in flight: wait for
    // them (bounded) before leaving; the range is abandoned.
    for (int32_t ch = timed_out_at; ch < min(timed_out_at + BK_STAGES, n_chunks); ++ch)
      mbar_wait_bounded(&bars[ch % BK_STAGES], (uint32_t)((ch / BK_STAGES) & 1), p.wait_limit_ns);
    if (lane == 0) atomicOr(p.err, DERR_TIMEOUT);
    return;
  }
  if (tail0 < w.span) {
    const int32_t nt = w.span - tail0;
    int32_t pos[1] = {lane < nt ? tail0 + lane : -1};
    uint64_t val[1] = {val_of(lane < nt ? __ldg(p.ids + E0 + tail0 + lane) : 0, lane < nt)};
    walk_window<Acc, 1>(w, p, lc, t_lo, base_abs, lane, tail0, w.span, pos, val);
  }
  while (w.k < w.nk) walk_finish(w, p, lc, t_lo, base_abs, lane);
  if (emax >= cat) atomicOr(p.err, DERR_EVENT_RANGE);
  if (lane == 0 && w.bad) atomicOr(p.err, DERR_OFFSETS);
}

// ------------------------------------------------------------------------------------------
// Literal Algorithm 3: for every occurrence, every ELT of the layer is looked up in its
// direct-access table.  Lanes are split into segments of W (a power of two >= the ELT count,
// capped at 32); segment s handles one event, lane j of the segment the layer's j-th ELT.
// The segment then sums the per-ELT results in the layer's ELT order (shuffles), applies the
// occurrence terms, and adds the same fixed point q as the folded path, so both paths give
// identical YLTs.
// ------------------------------------------------------------------------------------------
template <typename LossT>
__global__ void __launch_bounds__(256)
k_ylt_per_elt(StreamParams p, const LossT* __restrict__ dense, const int32_t* __restrict__ layer_elts,
              const double* __restrict__ elt_ret, const double* __restrict__ elt_lim) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const LayerConst lc = *p.layer;
  const int n_le = lc.elt_end - lc.elt_begin;
  int W = 1;
  while (W < n_le && W < 32) W <<= 1;
  const int E = 32 / W;                       // events per warp step
  const int seg = lane / W, jl = lane % W;
  const int n_chunks = (n_le + 31) / 32;      // ELT chunks when n_le > 32 (then W = 32, E = 1)
  const int64_t n_groups = (p.n_trials + 31) >> 5;
  bool bad_id = false, bad_off = false;
  for (int64_t g = warp; g < n_groups; g += nwarps) {
    const int64_t t0 = g << 5;
    const int nt = (int)min((int64_t)32, p.n_trials - t0);
    const int64_t my_off = (lane <= nt) ? __ldg(p.offsets + t0 + lane) - p.id_base : 0;
    const int64_t last_off = (nt == 32) ? __ldg(p.offsets + t0 + 32) - p.id_base : 0;
    U128 mine = U128{0ull, 0ull};
    for (int k = 0; k < nt; ++k) {
      int64_t beg = __shfl_sync(FULL, my_off, k);
      int64_t end = (k + 1 < 32) ? __shfl_sync(FULL, my_off, k + 1) : last_off;
      if (!(0 <= beg && beg <= end && end <= p.n_events)) { bad_off = true; beg = end = 0; }
      U128 acc = U128{0ull, 0ull};
      for (int64_t base = beg; base < end; base += E) {
        const int64_t pos = base + seg;
        const bool have = pos < end;
        int e = have ? __ldg(p.ids + pos) : 0;
        const bool in_range = (unsigned)e < (unsigned)p.catalogue;
        if (have && !in_range) bad_id = true;
        const bool use = have && in_range;
        double s = 0.0;
        for (int c = 0; c < n_chunks; ++c) {
          const int jj = c * 32 + jl;
          double a = 0.0;
          if (use && jl < W && jj < n_le) {
            const int j = layer_elts[lc.elt_begin + jj];
            const double x = (double)dense[(int64_t)j * p.catalogue + e];
            if (x != 0.0) a = clamp_terms(x, elt_ret[j], elt_lim[j]);  // absent: C(0) = 0
          }
          const int lim = min(32, n_le - c * 32);
          for (int m = 0; m < min(lim, W); ++m) {
            const double am = __shfl_sync(FULL, a, seg * W + m);
            if (am != 0.0) s = __dadd_rn(s, am);
          }
        }
        if (use && jl == 0 && s != 0.0) {
          const double o = clamp_terms(s, lc.occ_ret, lc.occ_lim);
          add_u64(acc, __double2ull_rn(__dmul_rn(o, lc.scale)));
        }
      }
      acc = AccOps<U128>::warp_sum(acc);
      if (lane == k) mine = acc;
    }
    if (lane < nt) {
      uint8_t reg;
      const double y = AccOps<U128>::finish(mine, lc, reg);
      p.ylt[t0 + lane] = y;
      if (p.regimes) p.regimes[t0 + lane] = reg;
    }
  }
  if (bad_id) atomicOr(p.err, DERR_EVENT_RANGE);
  if (bad_off) atomicOr(p.err, DERR_OFFSETS);
}

// Dense direct-access tables from the records: table[j][e] = loss (zero-filled beforehand).
template <typename LossT>
__global__ void k_scatter_dense(int32_t n_elts, int64_t catalogue, const int64_t* __restrict__ rec_off,
                                const int32_t* __restrict__ rec_ids, const LossT* __restrict__ rec_loss,
                                LossT* __restrict__ dense) {
  const int j = blockIdx.y;
  for (int64_t r = rec_off[j] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rec_off[j + 1];
       r += (int64_t)gridDim.x * blockDim.x)
    dense[(int64_t)j * catalogue + rec_ids[r]] = rec_loss[r];
}

// ------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------
// 32-bit words of the interleaved hit bitmap with one bit per 2^shift catalogue events.
static int64_t coarse_words(int64_t catalogue, int shift) {
  const int64_t exact = (catalogue + 31) / 32;
  return (exact + ((int64_t)1 << shift) - 1) >> shift;
}

static int bitmap_shift(int64_t catalogue, int64_t max_bytes) {
  int s = 0;
  while (coarse_words(catalogue, s) * 4 > max_bytes) ++s;
  return s;
}

static ara_status set_smem(const void* fn, int bytes) {
  ARA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return ARA_OK;
}

ara_status build_dense(Portfolio& pf, cudaStream_t s) {
  if (pf.n_elts == 0) return ARA_OK;
  const size_t esz = pf.d_rec_loss32 ? sizeof(float) : sizeof(double);
  ARA_TRY(cudaMemsetAsync(pf.d_dense, 0, esz * (size_t)pf.n_elts * pf.catalogue, s));
  dim3 grid(64, pf.n_elts);
  LaunchScope ls(ARA_K_FOLD, s);
  if (pf.d_rec_loss32)
    k_scatter_dense<float><<<grid, 256, 0, s>>>(pf.n_elts, pf.catalogue, pf.d_rec_off, pf.d_rec_ids,
                                                pf.d_rec_loss32, (float*)pf.d_dense);
  else
    k_scatter_dense<double><<<grid, 256, 0, s>>>(pf.n_elts, pf.catalogue, pf.d_rec_off, pf.d_rec_ids,
                                                 pf.d_rec_loss, (double*)pf.d_dense);
  ARA_TRY(cudaGetLastError());
  return ARA_OK;
}

ara_status launch_fold_to(Portfolio& pf, int32_t n_sel, const int32_t* sel_host,
                          const FoldOutHost& o, cudaStream_t s, bool counted) {
  FoldOut out;
  out.q = o.q;
  out.bits = o.bits;
  out.regime = o.regime;
  out.q_stride = o.q_stride;
  out.bits_stride = o.bits_stride;
  out.regime_stride = o.regime_stride;
  out.by_slot = o.by_slot;
  out.f64_table = o.f64_table;
  out.bits_from_regime = o.bits_from_regime;
  out.nonzero_only = o.nonzero_only;
  for (int32_t b = 0; b < n_sel; b += MAX_SEL) {
    SelList sl;
    sl.n = min(MAX_SEL, n_sel - b);
    for (int i = 0; i < sl.n; ++i) sl.idx[i] = sel_host[b + i];
    FoldOut ob = out;
    if (ob.by_slot) {  // slots continue across batches of MAX_SEL layers
      if (ob.q) ob.q += (int64_t)b * ob.q_stride;
      ob.bits += (int64_t)b * ob.bits_stride;
      if (ob.regime) ob.regime += (int64_t)b * ob.regime_stride;
    }
    dim3 grid((unsigned)((pf.catalogue + FOLD_TILE - 1) / FOLD_TILE), sl.n);
    std::optional<LaunchScope> ls;
    if (counted) ls.emplace(ARA_K_FOLD, s);
    if (pf.d_rec_loss32)
      k_fold<float><<<grid, FOLD_THREADS, 0, s>>>(pf.catalogue, pf.d_tile_rec, pf.n_tiles, pf.d_rec_ids,
                                                  pf.d_rec_loss32, pf.d_elt_ret, pf.d_elt_lim,
                                                  pf.d_layer_elts, pf.d_layers, sl, ob);
    else
      k_fold<double><<<grid, FOLD_THREADS, 0, s>>>(pf.catalogue, pf.d_tile_rec, pf.n_tiles, pf.d_rec_ids,
                                                   pf.d_rec_loss, pf.d_elt_ret, pf.d_elt_lim,
                                                   pf.d_layer_elts, pf.d_layers, sl, ob);
    ARA_TRY(cudaGetLastError());
  }
  return ARA_OK;
}

ara_status launch_fold(Portfolio& pf, int32_t n_sel, const int32_t* sel_host, int32_t flags,
                       cudaStream_t s, int slot) {
  const FoldSlot ws = fold_slot(pf, slot);
  if (!ws.q || !ws.bits) return ARA_EINVAL;
  FoldOutHost o{};
  o.q = ws.q;
  o.bits = ws.bits;
  o.q_stride = pf.catalogue;
  o.bits_stride = pf.bm_words;
  o.f64_table = (flags & ARA_RUN_F64_SUM) ? 1 : 0;
  return launch_fold_to(pf, n_sel, sel_host, o, s);
}

template <bool FILTER, typename Acc>
static ara_status launch_folded_one(Portfolio& pf, StreamParams& sp, cudaStream_t s) {
  constexpr int U = 2;
  const auto fn = k_ylt_folded<FILTER, Acc, U>;
  const int smem = FILTER ? (int)(sp.smem_words * 4) : 0;
  if (smem > 48 * 1024) {
    ara_status st = set_smem((const void*)fn, smem);
    if (st != ARA_OK) return st;
  }
  LaunchScope ls(ARA_K_YLT, s);
  fn<<<pf.n_sms, YLT_THREADS, smem, s>>>(sp);
  ARA_TRY(cudaGetLastError());
  return ARA_OK;
}

// Compiled shapes of the bulk kernel (warps per block, ring stages, IDs per stage); the active
// one is chosen with ara_set_stream_shape.  The default, 28 warps, measured fastest at paper
// scale: it leaves each thread up to 72 registers (32 warps: 64), which costs fewer extra
// instructions, while keeping enough warps to hide the gathers' latency.
static const int kBulkShapes[][3] = {{28, 2, 256}, {32, 2, 256}, {24, 4, 256}, {24, 2, 512},
                                     {16, 3, 512}, {16, 4, 256}};
static std::atomic<int> g_bulk_shape{0};
static std::atomic<uint64_t> g_wait_limit_ns{1000000000ull};
static std::atomic<uint32_t> g_debug_extra_tx{0};

void set_wait_limit_ns(uint64_t ns) { g_wait_limit_ns.store(ns); }
uint64_t wait_limit_ns() { return g_wait_limit_ns.load(); }
static std::atomic<int32_t> g_skip_arrival{0};
void set_debug_skip_arrival(int32_t on) { g_skip_arrival.store(on); }
int32_t debug_skip_arrival() { return g_skip_arrival.load(); }
void set_debug_extra_tx(uint32_t b) { g_debug_extra_tx.store(b); }

template <bool FILTER, typename Acc, int WARPS, int STAGES, int CHUNK>
static ara_status launch_bulk_shape(Portfolio& pf, StreamParams& sp, cudaStream_t s) {
  const auto fn = k_ylt_bulk<FILTER, Acc, WARPS, STAGES, CHUNK>;
  const int64_t bm_bytes = FILTER ? ((sp.smem_words * 4 + 127) / 128) * 128 : 0;
  using Sh = BulkShape<WARPS, STAGES, CHUNK>;
  const int smem = (int)(bm_bytes + Sh::ring_bytes + Sh::bar_bytes);
  ara_status st = set_smem((const void*)fn, smem);
  if (st != ARA_OK) return st;
  LaunchScope ls(ARA_K_YLT, s);
  fn<<<pf.n_sms, WARPS * 32, smem, s>>>(sp);
  ARA_TRY(cudaGetLastError());
  return ARA_OK;
}

template <bool FILTER, typename Acc>
static ara_status launch_bulk_one(Portfolio& pf, StreamParams& sp, cudaStream_t s) {
  switch (g_bulk_shape.load()) {
    case 1: return launch_bulk_shape<FILTER, Acc, 32, 2, 256>(pf, sp, s);
    case 2: return launch_bulk_shape<FILTER, Acc, 24, 4, 256>(pf, sp, s);
    case 3: return launch_bulk_shape<FILTER, Acc, 24, 2, 512>(pf, sp, s);
    case 4: return launch_bulk_shape<FILTER, Acc, 16, 3, 512>(pf, sp, s);
    case 5: return launch_bulk_shape<FILTER, Acc, 16, 4, 256>(pf, sp, s);
    default: return launch_bulk_shape<FILTER, Acc, 28, 2, 256>(pf, sp, s);
  }
}

static int bulk_ring_bytes() {
  const int* sh = kBulkShapes[g_bulk_shape.load()];
  return sh[0] * sh[1] * (sh[2] * 4 + 8);
}

int32_t n_bulk_shapes() { return (int32_t)(sizeof(kBulkShapes) / sizeof(kBulkShapes[0])); }
void set_bulk_shape(int32_t i) { g_bulk_shape.store(i); }
void bulk_shape(int32_t i, int32_t* warps, int32_t* stages) {
  *warps = kBulkShapes[i][0];
  *stages = kBulkShapes[i][1] * 10000 + kBulkShapes[i][2];   // stages * 10000 + chunk IDs
}

// Shift of the hit bitmap the stream kernel of these run flags keeps in shared memory: what the
// block may use beyond the staging ring (the register-staged kernel has no ring).
static int run_bitmap_shift(const Portfolio& pf, int32_t flags) {
  const bool ldg = (flags & ARA_RUN_LDG) != 0;
  const int64_t max_smem_bitmap =
      ldg ? 200 * 1024 : (int64_t)pf.max_smem_block - bulk_ring_bytes() - 128;
  return bitmap_shift(pf.catalogue, max_smem_bitmap);
}

ara_status launch_coarsen(Portfolio& pf, int32_t n_sel, const int32_t* sel_host, int32_t flags,
                          cudaStream_t s, int slot) {
  const bool ldg = (flags & ARA_RUN_LDG) != 0, per_elt = (flags & ARA_RUN_PER_ELT) != 0;
  const bool nof = (flags & ARA_RUN_NO_FILTER) != 0;
  const int shift = run_bitmap_shift(pf, flags);
  if (ldg || per_elt || nof || shift == 0) return ARA_OK;   // no coarse bitmap is read
  if (shift > 26) return ARA_EINVAL;
  const FoldSlot ws = fold_slot(pf, slot);
  if (!ws.bits || !ws.cbits) return ARA_EINVAL;
  const int64_t cwords_pad = (coarse_words(pf.catalogue, shift) + 3) / 4 * 4;
  if (cwords_pad > pf.cbits_stride) return ARA_EINVAL;
  for (int32_t i = 0; i < n_sel; ++i) {
    const int layer = sel_host[i];
    LaunchScope ls(ARA_K_FOLD, s);
    k_coarsen<<<(unsigned)std::min<int64_t>((cwords_pad + 255) / 256, 4096), 256, 0, s>>>(
        ws.bits + (int64_t)layer * pf.bm_words, pf.bm_words, shift,
        ws.cbits + (int64_t)layer * pf.cbits_stride, cwords_pad);
    ARA_TRY(cudaGetLastError());
  }
  return ARA_OK;
}

ara_status launch_ylt(Portfolio& pf, const YltArgs& a, cudaStream_t s) {
  const bool ldg = (a.flags & ARA_RUN_LDG) != 0;
  const FoldSlot ws = fold_slot(pf, a.slot);
  if (!ws.q || !ws.bits) return ARA_EINVAL;
  StreamParams sp{};
  sp.n_trials = a.n_trials;
  sp.offsets = a.offsets;
  sp.id_base = a.id_base;
  sp.n_events = a.n_events;
  sp.ids = a.ids;
  sp.mis = (int32_t)(((uintptr_t)a.ids >> 2) & 3);
  sp.catalogue = pf.catalogue;
  sp.shift = run_bitmap_shift(pf, a.flags);
  if (sp.shift > 26) return ARA_EINVAL;   // the bulk lookup's multiplier is 2^(27 - shift)
  sp.smem_words = coarse_words(pf.catalogue, sp.shift);
  sp.bm_words = pf.bm_words;
  sp.err = pf.d_err;
  // the bulk kernel copies a ready bitmap: exact when it fits, else the coarse one (built here,
  // or by ara_prepare_ylt for a prepared run)
  if (!a.prepared) {
    const ara_status st0 = launch_coarsen(pf, a.n_sel, a.sel, a.flags, s, a.slot);
    if (st0 != ARA_OK) return st0;
  }
  sp.wait_limit_ns = g_wait_limit_ns.load();
  sp.debug_extra_tx = g_debug_extra_tx.load();
  sp.word_bytes = 4;
  const bool per_elt = (a.flags & ARA_RUN_PER_ELT) != 0;
  const bool nof = (a.flags & ARA_RUN_NO_FILTER) != 0;
  const bool f64 = (a.flags & ARA_RUN_F64_SUM) != 0;
  for (int32_t i = 0; i < a.n_sel; ++i) {
    const int layer = a.sel[i];
    sp.q = ws.q + (int64_t)layer * pf.catalogue;
    sp.bits = ws.bits + (int64_t)layer * pf.bm_words;
    sp.layer = pf.d_layers + layer;
    if (!ldg && !per_elt && !nof && sp.shift > 0) sp.bits = ws.cbits + (int64_t)layer * pf.cbits_stride;
    sp.ylt = a.ylt + (int64_t)i * a.row_stride;
    sp.regimes = a.regimes ? a.regimes + (int64_t)i * a.row_stride : nullptr;
    if (a.n_trials == 0) continue;
    ara_status st;
    if (per_elt) {
      LaunchScope ls(ARA_K_YLT, s);
      const int grid = pf.n_sms * 8;
      if (pf.d_rec_loss32)
        k_ylt_per_elt<float><<<grid, 256, 0, s>>>(sp, (const float*)pf.d_dense, pf.d_layer_elts,
                                                  pf.d_elt_ret, pf.d_elt_lim);
      else
        k_ylt_per_elt<double><<<grid, 256, 0, s>>>(sp, (const double*)pf.d_dense, pf.d_layer_elts,
                                                   pf.d_elt_ret, pf.d_elt_lim);
      ARA_TRY(cudaGetLastError());
      st = ARA_OK;
    } else if (ldg) {
      if (f64) st = nof ? launch_folded_one<false, double>(pf, sp, s) : launch_folded_one<true, double>(pf, sp, s);
      else st = nof ? launch_folded_one<false, U128>(pf, sp, s) : launch_folded_one<true, U128>(pf, sp, s);
    } else if (a.flags & ARA_RUN_OEP) {
      st = launch_bulk_one<true, OepMax>(pf, sp, s);
    } else {
      if (f64) st = nof ? launch_bulk_one<false, double>(pf, sp, s) : launch_bulk_one<true, double>(pf, sp, s);
      else st = nof ? launch_bulk_one<false, U128>(pf, sp, s) : launch_bulk_one<true, U128>(pf, sp, s);
    }
    if (st != ARA_OK) return st;
  }
  return ARA_OK;
}

}  // namespace ara

// Batched portfolio: every selected layer of a portfolio in one pass over the YET (the program
// and layer loops of Algorithm 1 folded into one launch).
//
// Preparation, per run (all on the stream, captured in the plan's CUDA graph):
//   1. q_i(e) = round(C(sum_j C(x_j(e); R_j, L_j); OccR_i, OccL_i) * 2^f_i) and the hit bitmap
//      of every selected layer i, in one launch of the single-layer fold kernel (slot i of the
//      fold workspace; only the non-zero q are stored).  The batched and the single-layer paths
//      thus share the folded table bit for bit.
//   2. per-event counts of non-zero q, read from the bitmaps, and their exclusive scan -> CSR
//      row pointers.
//   3. event-major CSR rows: for event e, its (layer slot, q) pairs in layer order, packed as
//      slot << 56 | q (q < 2^55); q is read only where the bitmap bit is set.  The event's row
//      descriptor holds its first entry and, per request of a merged serving pass (slots are
//      grouped by request), the number of its entries in one byte each (a row has at most 255
//      entries, one per slot), so that a trial covered by some of the requests walks only
//      their part of the row.
// Stream (persistent, atomic trial queue for uneven trial lengths): a warp takes trials from the
// queue; for every 32 occurrences it joins their events' CSR rows into one list, walks it 32
// entries at a time and adds each q to the warp's per-layer accumulator in shared memory (exact
// 128-bit: 64-bit atomic add with carry); at the end of a trial its lanes apply every layer's
// aggregate terms to the exact sums and write the YLT entries.  Integer sums make the result independent of the order of the additions and
// bitwise equal to the single-layer path.

#include <algorithm>
#include <vector>

#include "ara_device.cuh"

namespace ara {

constexpr int BT_MAX_LAYERS = 255;          // slot fits in 8 bits (255 = no slot)
constexpr int BT_SCAN_BLOCK = 1024;

struct BtLayers {
  int32_t n_sel;
  int32_t layer[BT_MAX_LAYERS];
};

// ------------------------------------------------------------------------------------------
// 2. per-event counts and their exclusive scan (two levels: block sums, then their scan)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[BT_SCAN_BLOCK / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// count of event e: the number of selected layers whose bitmap has bit e set (the 32 lanes of a
// warp read the same word of each bitmap)
__device__ __forceinline__ uint32_t bt_count(const uint32_t* __restrict__ bits, int64_t bits_stride,
                                             int32_t n_sel, int64_t e) {
  const uint32_t* b = bits + (e >> 5);
  const int sh = (int)(e & 31);
  uint32_t c = 0;
#pragma unroll 8
  for (int i = 0; i < n_sel; ++i) c += (__ldg(b + (int64_t)i * bits_stride) >> sh) & 1u;
  return c;
}

__global__ void __launch_bounds__(BT_SCAN_BLOCK)
k_bt_scan_blocks(const uint32_t* __restrict__ bits, int64_t bits_stride, int32_t n_sel, int64_t n,
                 uint32_t* __restrict__ ptr, uint32_t* __restrict__ block_sums) {
  const int64_t e = (int64_t)blockIdx.x * BT_SCAN_BLOCK + threadIdx.x;
  const uint32_t v = e < n ? bt_count(bits, bits_stride, n_sel, e) : 0u;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(v, &tot);
  if (e < n) ptr[e] = ex;
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the block sums (loops for many blocks)
__global__ void __launch_bounds__(BT_SCAN_BLOCK)
k_bt_scan_sums(uint32_t* __restrict__ block_sums, int64_t n_blocks, uint32_t* __restrict__ total) {
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < n_blocks; b0 += BT_SCAN_BLOCK) {
    const int64_t b = b0 + threadIdx.x;
    const uint32_t v = b < n_blocks ? block_sums[b] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, &tot);
    if (b < n_blocks) block_sums[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_bt_scan_add(uint32_t* __restrict__ ptr, int64_t n, const uint32_t* __restrict__ block_sums,
                              const uint32_t* __restrict__ total) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) ptr[e] += block_sums[e / BT_SCAN_BLOCK];
  if (e == n) ptr[n] = *total;
}

// Row pointers of an event-major table: ptr[e] = number of set bits of event e over all
// n_sel bitmaps before e (exclusive scan), ptr[n] = total; block_sums holds ceil(n / 1024)
// words of scratch, total one word.
ara_status launch_event_scan(const uint32_t* bits, int64_t bits_stride, int32_t n_sel, int64_t n,
                             uint32_t* ptr, uint32_t* block_sums, uint32_t* total, cudaStream_t s) {
  const int64_t n_blocks = (n + BT_SCAN_BLOCK - 1) / BT_SCAN_BLOCK;
  k_bt_scan_blocks<<<(unsigned)n_blocks, BT_SCAN_BLOCK, 0, s>>>(bits, bits_stride, n_sel, n, ptr,
                                                              block_sums);
  k_bt_scan_sums<<<1, BT_SCAN_BLOCK, 0, s>>>(block_sums, n_blocks, total);
  k_bt_scan_add<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(ptr, n, block_sums, total);
  ARA_TRY(cudaGetLastError());
  return ARA_OK;
}

// ------------------------------------------------------------------------------------------
// 3. CSR rows: one thread per event, layers in slot order (deterministic layout), and the
//    event's row descriptor (first entry | length << 32)
// ------------------------------------------------------------------------------------------
// Request boundaries of a merged pass, in slots: request r owns [first[r], first[r + 1]); unused
// requests start at BT_MAX_LAYERS + 1 (past every slot).
struct BtReqSlots {
  int32_t first[BT_MAX_REQ + 1];
};

__device__ __forceinline__ uint32_t bt_req_of_slot(const BtReqSlots& rs, int i) {
  return (uint32_t)(i >= rs.first[1]) + (uint32_t)(i >= rs.first[2]) + (uint32_t)(i >= rs.first[3]);
}

__global__ void __launch_bounds__(256)
k_bt_fill(int32_t n_sel, const uint64_t* __restrict__ q, const uint32_t* __restrict__ bits,
          int64_t bits_stride, int64_t catalogue, const uint32_t* __restrict__ ptr,
          uint64_t* __restrict__ entries, uint64_t* __restrict__ rows, BtReqSlots rs) {
  constexpr int U = 8;   // slots per step: their bitmap words and table entries load together
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= catalogue) return;
  const uint32_t pos0 = ptr[e];
  uint32_t pos = pos0;
  const uint32_t end = ptr[e + 1];
  uint32_t lens = 0;   // entries of request r in byte r (one 8-byte descriptor per occurrence)
  const uint32_t* b = bits + (e >> 5);
  const int sh = (int)(e & 31);
  for (int i0 = 0; i0 < n_sel && pos < end; i0 += U) {
    bool hit[U];
    uint64_t v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      hit[u] = i0 + u < n_sel && ((__ldg(b + (int64_t)(i0 + u) * bits_stride) >> sh) & 1u);
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = hit[u] ? __ldg(q + (int64_t)(i0 + u) * catalogue + e) : 0ull;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (hit[u]) {
        if (pos < end) {
          entries[pos] = ((uint64_t)(i0 + u) << 56) | v[u];
          lens += 1u << (8 * bt_req_of_slot(rs, i0 + u));
        }
        ++pos;
      }
  }
  rows[e] = (uint64_t)pos0 | ((uint64_t)lens << 32);
}

// ------------------------------------------------------------------------------------------
// Stream
// ------------------------------------------------------------------------------------------
struct BtStream {
  int64_t n_trials;
  const int64_t* offsets;
  int64_t n_events;
  const int32_t* ids;
  uint32_t catalogue;
  const uint64_t* rows;        // [catalogue]: first entry | length << 32
  const uint64_t* entries;
  int32_t n_sel;
  const LayerConst* layers;    // device, indexed by layer id
  BtLayers sel;                // slot -> layer id
  // Requests of the pass (one outside serving): request r owns the slots [rs.first[r],
  // rs.first[r + 1]) and the trials [t0[r], t1[r]); row i of its YLT (its slot first + i) is
  // ylt[r] + i * (t1[r] - t0[r]), indexed by t - t0[r]; regimes likewise (or nullptr).
  int32_t n_req;
  BtReqSlots rs;
  int64_t t0[BT_MAX_REQ], t1[BT_MAX_REQ];
  double* ylt[BT_MAX_REQ];
  uint8_t* regimes[BT_MAX_REQ];
  unsigned long long* queue;   // trial counter (zeroed before the launch)
  int32_t trials_per_grab;
  int32_t copies;              // accumulator copies per warp: 1, 2 or 4
  uint32_t* err;
};

// Non-returning 64-bit shared-memory add.  A segment of at most BT_SEG occurrences adds at most
// one value below 2^55 per occurrence to a slot's word (a row holds each slot once), so the word
// cannot wrap: BT_SEG * 2^55 <= 2^64.
constexpr int BT_SEG = 512;
__device__ __forceinline__ void smem_red_u64(unsigned long long* a, uint64_t q) {
  asm volatile("red.shared.add.u64 [%0], %1;" :: "r"((uint32_t)__cvta_generic_to_shared(a)), "l"(q) : "memory");
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_bt_stream(BtStream p) {
  // [WARPS][copies + 2][n_sel]: per copy the 64-bit sums of the current segment, then the
  // trial's exact 128-bit totals (low and high words) of the finished segments
  extern __shared__ __align__(16) unsigned long long bt_acc[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = p.n_sel;
  // Each group of 32 / copies lanes has its own copy of the warp's accumulators, so that lanes
  // of different groups never add to the same word; the copies are summed exactly at the end of
  // a trial.
  const int nc = p.copies;
  unsigned long long* const acc0 = bt_acc + (int64_t)wid * (nc + 2) * ns;
  unsigned long long* const lo = acc0 + (int64_t)(lane / (32 / nc)) * ns;
  unsigned long long* const tot = acc0 + (int64_t)nc * ns;   // [2][n_sel]
  for (int i = lane; i < (nc + 2) * ns; i += 32) acc0[i] = 0ull;
  __syncwarp();
  bool bad_id = false, bad_off = false;
  while (true) {
    unsigned long long t0 = 0;
    if (lane == 0) t0 = atomicAdd(p.queue, (unsigned long long)p.trials_per_grab);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    if (t0 >= (unsigned long long)p.n_trials) break;
    const int64_t t1 = min((int64_t)t0 + p.trials_per_grab, p.n_trials);
    for (int64_t t = (int64_t)t0; t < t1; ++t) {
      // The requests covering trial t (warp-uniform): each occurrence walks the part of its row
      // from the first to the last of them, [fa, la]; a request inside that range that does not
      // cover t (at most the two middle ones of four, always adjacent) owns the slots
      // [skip_lo, skip_hi), whose entries are skipped.
      uint32_t amask = 0;
      for (int r = 0; r < p.n_req; ++r)
        if (t >= p.t0[r] && t < p.t1[r]) amask |= 1u << r;
      if (amask == 0) continue;
      const int fa = __ffs(amask) - 1, la = 31 - __clz(amask);
      const uint32_t sh_lo = 8u * (uint32_t)fa, sh_hi = 8u * (uint32_t)la;
      const uint32_t inner = ((2u << la) - (1u << fa)) & ~amask;   // uncovered, between fa and la
      const uint32_t skip_lo = inner ? (uint32_t)p.rs.first[__ffs(inner) - 1] : 0u;
      const uint32_t skip_n =
          inner ? (uint32_t)p.rs.first[32 - __clz(inner)] - skip_lo : 0u;
      int64_t beg = __ldg(p.offsets + t), end = __ldg(p.offsets + t + 1);
      if (!(0 <= beg && beg <= end && end <= p.n_events)) { bad_off = true; beg = end = 0; }
      // 32 occurrences at a time.  Their rows are laid end to end (a warp scan of the lengths)
      // and the warp walks the joined list 32 entries per step: every lane has an entry, and
      // the lanes of one row read consecutive words.  The lane owning item x is the first lane
      // whose inclusive length sum exceeds x (a 5-step search over the lanes' sums).
      // Software pipeline over the rounds: the row descriptors of round k + 1 and the event IDs
      // of round k + 2 are in flight while round k's entries are walked.
      auto load_id = [&](int64_t i) -> int64_t {   // -1 past the trial's end
        return i < end ? (int64_t)(uint32_t)__ldcs(p.ids + i) : (int64_t)-1;
      };
      auto load_row = [&](int64_t e) -> uint64_t {
        if (e < 0) return 0ull;
        if (e >= (int64_t)p.catalogue) { bad_id = true; return 0ull; }
        return __ldg(p.rows + e);
      };
      uint64_t ri_cur = load_row(load_id(beg + lane));
      int64_t e_nxt = load_id(beg + 32 + lane);
      // Adds the segment sums of every copy into the trial's totals and clears them.
      auto flush = [&]() {
        __syncwarp();
        for (int i = lane; i < ns; i += 32) {
          U128 S{tot[i], tot[ns + i]};
          for (int c = 0; c < nc; ++c) {
            add_u64(S, acc0[(int64_t)c * ns + i]);
            acc0[(int64_t)c * ns + i] = 0ull;
          }
          tot[i] = S.lo;
          tot[ns + i] = S.hi;
        }
        __syncwarp();
      };
      int rounds = 0;
      for (int64_t i0 = beg; i0 < end; i0 += 32) {
        const uint64_t ri_nxt = load_row(e_nxt);
        e_nxt = load_id(i0 + 64 + lane);
        // byte r of lens * 0x01010101 is the number of entries of requests 0..r (< 256)
        const uint32_t incl_b = (uint32_t)(ri_cur >> 32) * 0x01010101u;
        const uint32_t skip_b = ((incl_b << 8) >> sh_lo) & 0xffu;   // entries before request fa
        const uint32_t rb = (uint32_t)ri_cur + skip_b;
        const uint32_t len = ((incl_b >> sh_hi) & 0xffu) - skip_b;
        ri_cur = ri_nxt;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t base = rb - (incl - len);   // entry of item x (in this lane's row): base + x
        for (uint32_t w0 = 0; w0 < total; w0 += 32) {
          const uint32_t x = w0 + (uint32_t)lane;
          int own = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, incl, own + step - 1);
            if (v <= x) own += step;
          }
          const uint32_t b = __shfl_sync(0xffffffffu, base, own);
          if (x < total) {
            const uint64_t v = __ldg(p.entries + (uint32_t)(b + x));
            const int s = (int)(v >> 56);
            if ((uint32_t)s - skip_lo >= skip_n) smem_red_u64(&lo[s], v & ((1ull << 56) - 1));
          }
        }
        if (++rounds == BT_SEG / 32) {
          flush();
          rounds = 0;
        }
      }
      __syncwarp();
      // aggregate terms of every layer on the exact sums; reset the accumulators
      for (int i = lane; i < ns; i += 32) {
        U128 S{tot[i], tot[ns + i]};
        tot[i] = 0ull;
        tot[ns + i] = 0ull;
        for (int c = 0; c < nc; ++c) {
          add_u64(S, acc0[(int64_t)c * ns + i]);
          acc0[(int64_t)c * ns + i] = 0ull;
        }
        const uint32_t r = bt_req_of_slot(p.rs, i);
        if (!((amask >> r) & 1u)) continue;
        const LayerConst lc = p.layers[p.sel.layer[i]];
        uint8_t reg;
        const double y = AccOps<U128>::finish(S, lc, reg);
        const int64_t at = (int64_t)(i - p.rs.first[r]) * (p.t1[r] - p.t0[r]) + (t - p.t0[r]);
        p.ylt[r][at] = y;
        if (p.regimes[r]) p.regimes[r][at] = reg;
      }
      __syncwarp();
    }
  }
  if (bad_id) atomicOr(p.err, DERR_EVENT_RANGE);
  if (bad_off) atomicOr(p.err, DERR_OFFSETS);
}

}  // namespace ara

// ------------------------------------------------------------------------------------------
// Host: plan = scratch + autotuned schedule + CUDA graph of the whole run
// ------------------------------------------------------------------------------------------
using namespace ara;

struct ara_plan {
  Portfolio* pf = nullptr;
  int64_t n_trials = 0, n_events = 0;
  const int64_t* d_off = nullptr;
  const int32_t* d_ids = nullptr;
  std::vector<int32_t> sel;
  double* d_ylt = nullptr;
  uint8_t* d_reg = nullptr;
  // requests of a merged serving pass (one request otherwise: all trials, d_ylt / d_reg)
  int32_t n_req = 1;
  BtReqSlots rs{{0, BT_MAX_LAYERS + 1, BT_MAX_LAYERS + 1, BT_MAX_LAYERS + 1, BT_MAX_LAYERS + 1}};
  int64_t req_t0[BT_MAX_REQ] = {0, 0, 0, 0}, req_t1[BT_MAX_REQ] = {0, 0, 0, 0};
  double* req_ylt[BT_MAX_REQ] = {nullptr, nullptr, nullptr, nullptr};
  uint8_t* req_reg[BT_MAX_REQ] = {nullptr, nullptr, nullptr, nullptr};
  uint32_t* d_ptr = nullptr;
  uint64_t* d_rows = nullptr;
  uint32_t* d_bsum = nullptr;
  uint32_t* d_total = nullptr;
  uint64_t* d_entries = nullptr;
  unsigned long long* d_queue = nullptr;
  int64_t n_blocks = 0;
  int warps = 16, ctas_per_sm = 2, tpg = 2, copies = 2;
  double tuned_ms = 0.0;
  int n_kernels = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// The plan as one request: every selected layer over every trial, into d_ylt / d_reg.
void single_request(ara_plan& P) {
  P.n_req = 1;
  P.req_t0[0] = 0;
  P.req_t1[0] = P.n_trials;
  P.req_ylt[0] = P.d_ylt;
  P.req_reg[0] = P.d_reg;
}

ara_status bt_prep(ara_plan& P, cudaStream_t s, bool fill, int* n_kernels) {
  Portfolio& pf = *P.pf;
  const int n_sel = (int)P.sel.size();
  const int64_t C = pf.catalogue;
  FoldOutHost fo;
  fo.q = pf.d_q;                 // slot i at d_q + i * C (workspace of the single-layer runs)
  fo.bits = pf.d_bits;
  fo.q_stride = C;
  fo.bits_stride = pf.bm_words;
  fo.by_slot = 1;
  fo.nonzero_only = 1;
  ara_status st = launch_fold_to(pf, n_sel, P.sel.data(), fo, s, false);
  if (st != ARA_OK) return st;
  k_bt_scan_blocks<<<(unsigned)P.n_blocks, BT_SCAN_BLOCK, 0, s>>>(pf.d_bits, pf.bm_words, n_sel, C,
                                                                  P.d_ptr, P.d_bsum);
  k_bt_scan_sums<<<1, BT_SCAN_BLOCK, 0, s>>>(P.d_bsum, P.n_blocks, P.d_total);
  k_bt_scan_add<<<(unsigned)((C + 1 + 255) / 256), 256, 0, s>>>(P.d_ptr, C, P.d_bsum, P.d_total);
  int k = 4;
  if (fill) {
    k_bt_fill<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(n_sel, pf.d_q, pf.d_bits, pf.bm_words, C,
                                                          P.d_ptr, P.d_entries, P.d_rows, P.rs);
    ++k;
  }
  ARA_TRY(cudaGetLastError());
  if (n_kernels) *n_kernels = k;
  return ARA_OK;
}

template <int W>
ara_status bt_launch_w(ara_plan& P, const BtStream& bs, cudaStream_t s) {
  const int smem = W * (P.copies + 2) * (int)P.sel.size() * 8;
  const auto fn = k_bt_stream<W>;
  if (smem > 48 * 1024)
    ARA_TRY(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  fn<<<P.pf->n_sms * P.ctas_per_sm, W * 32, smem, s>>>(bs);
  ARA_TRY(cudaGetLastError());
  return ARA_OK;
}

ara_status bt_stream(ara_plan& P, cudaStream_t s) {
  BtStream bs{};
  bs.n_trials = P.n_trials;
  bs.offsets = P.d_off;
  bs.n_events = P.n_events;
  bs.ids = P.d_ids;
  bs.catalogue = (uint32_t)P.pf->catalogue;
  bs.rows = P.d_rows;
  bs.entries = P.d_entries;
  bs.n_sel = (int32_t)P.sel.size();
  bs.layers = P.pf->d_layers;
  bs.sel.n_sel = bs.n_sel;
  for (int i = 0; i < bs.n_sel; ++i) bs.sel.layer[i] = P.sel[i];
  bs.n_req = P.n_req;
  bs.rs = P.rs;
  for (int r = 0; r < BT_MAX_REQ; ++r) {
    bs.t0[r] = P.req_t0[r];
    bs.t1[r] = P.req_t1[r];
    bs.ylt[r] = P.req_ylt[r];
    bs.regimes[r] = P.req_reg[r];
  }
  if (!bs.ylt[0]) return ARA_EINVAL;
  bs.queue = P.d_queue;
  bs.trials_per_grab = P.tpg;
  bs.copies = P.copies;
  bs.err = P.pf->d_err;
  ARA_TRY(cudaMemsetAsync(P.d_queue, 0, sizeof(unsigned long long), s));
  switch (P.warps) {
    case 8: return bt_launch_w<8>(P, bs, s);
    case 32: return bt_launch_w<32>(P, bs, s);
    default: return bt_launch_w<16>(P, bs, s);
  }
}

void bt_free(ara_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  void* ptrs[] = {P->d_ptr, P->d_rows, P->d_bsum, P->d_total, P->d_entries, P->d_queue};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete P;
}

}  // namespace

namespace ara {
namespace {
ara_status run_plan_async(ara_plan& P, cudaStream_t s);
}  // namespace

// The batched path as one asynchronous call (no graph, default schedule): scratch comes from the
// stream-ordered allocator, the table is sized by a host-known bound (every non-zero entry of
// layer i is an event of one of its ELTs), and nothing waits on the host.
ara_status run_batched_async(Portfolio& pf, const YltArgs& a, cudaStream_t s) {
  ara_plan P;
  P.pf = &pf;
  P.n_trials = a.n_trials;
  P.n_events = a.n_events;
  P.d_off = a.offsets;
  P.d_ids = a.ids;
  P.sel.assign(a.sel, a.sel + a.n_sel);
  P.d_ylt = a.ylt;
  P.d_reg = a.regimes;
  if (a.id_base != 0 || a.row_stride != a.n_trials) return ARA_EINVAL;
  single_request(P);
  return run_plan_async(P, s);
}

// Several requests in one pass (serving): every layer of the portfolio, request r owning the
// slots [slot_first[r], slot_first[r + 1]) and the trials [t0[r], t1[r]) of the union range.
ara_status run_batched_group_async(Portfolio& pf, const GroupArgs& g, cudaStream_t s) {
  if (g.n_req < 1 || g.n_req > BT_MAX_REQ || g.n_trials < 1 || !g.offsets) return ARA_EINVAL;
  if (g.slot_first[0] != 0 || g.slot_first[g.n_req] != pf.n_layers) return ARA_EINVAL;
  ara_plan P;
  P.pf = &pf;
  P.n_trials = g.n_trials;
  P.n_events = g.n_events;
  P.d_off = g.offsets;
  P.d_ids = g.ids;
  for (int32_t l = 0; l < pf.n_layers; ++l) P.sel.push_back(l);
  P.n_req = g.n_req;
  for (int r = 0; r < BT_MAX_REQ; ++r) {
    P.rs.first[r + 1] = r < g.n_req ? g.slot_first[r + 1] : BT_MAX_LAYERS + 1;
    if (r >= g.n_req) continue;
    if (g.slot_first[r + 1] <= g.slot_first[r] || g.t0[r] < 0 || g.t1[r] <= g.t0[r] ||
        g.t1[r] > g.n_trials || !g.ylt[r])
      return ARA_EINVAL;
    P.req_t0[r] = g.t0[r];
    P.req_t1[r] = g.t1[r];
    P.req_ylt[r] = g.ylt[r];
    P.req_reg[r] = g.reg[r];
  }
  P.rs.first[0] = 0;
  return run_plan_async(P, s);
}

namespace {
ara_status run_plan_async(ara_plan& P, cudaStream_t s) {
  Portfolio& pf = *P.pf;
  if ((int)P.sel.size() > BT_MAX_LAYERS || (int)P.sel.size() > pf.n_layers ||
      (int64_t)P.sel.size() * pf.catalogue >= ((int64_t)1 << 32))
    return ARA_ERANGE;
  int64_t bound = 0;
  for (int32_t l : P.sel) {
    const LayerConst& lc = pf.layers[l];
    for (int k = lc.elt_begin; k < lc.elt_end; ++k) {
      const int j = pf.layer_elts[k];
      bound += pf.rec_off[j + 1] - pf.rec_off[j];
    }
  }
  const int64_t C = pf.catalogue;
  P.n_blocks = (C + BT_SCAN_BLOCK - 1) / BT_SCAN_BLOCK;
  size_t off = 0;
  auto take = [&](size_t n) { size_t o = (off + 255) / 256 * 256; off = o + n; return o; };
  const size_t o_ptr = take(4 * (size_t)(C + 1)), o_rows = take(8 * (size_t)C);
  const size_t o_bsum = take(4 * (size_t)P.n_blocks), o_tot = take(4), o_q = take(8);
  const size_t o_ent = take(8 * (size_t)std::max<int64_t>(bound, 1));
  char* buf = nullptr;
  ARA_TRY(dmalloc_async((void**)&buf, off, s));
  P.d_ptr = (uint32_t*)(buf + o_ptr);
  P.d_rows = (uint64_t*)(buf + o_rows);
  P.d_bsum = (uint32_t*)(buf + o_bsum);
  P.d_total = (uint32_t*)(buf + o_tot);
  P.d_queue = (unsigned long long*)(buf + o_q);
  P.d_entries = (uint64_t*)(buf + o_ent);
  ara_status st = ARA_OK;
  {
    LaunchScope ls(ARA_K_BATCHED, s, 6);
    st = bt_prep(P, s, true, nullptr);
    if (st == ARA_OK) st = bt_stream(P, s);
  }
  cudaFreeAsync(buf, s);
  P.d_ptr = P.d_bsum = P.d_total = nullptr;
  P.d_rows = nullptr;
  P.d_entries = nullptr;
  P.d_queue = nullptr;
  return st;
}
}  // namespace
}  // namespace ara

extern "C" {

ara_status ara_plan_batched(ara_portfolio* pf_, int64_t n_trials, const int64_t* d_off,
                            int64_t n_events, const int32_t* d_ids, int32_t n_sel_in,
                            const int32_t* layer_sel, double* d_ylt, uint8_t* d_reg, int32_t flags,
                            void* stream, ara_plan** out) {
  Portfolio* pf = static_cast<Portfolio*>(pf_);
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  if (!pf || n_trials < 1 || n_events < 0 || !d_off || !d_ylt || (n_events > 0 && !d_ids))
    return ARA_EINVAL;
  if (flags & ~ARA_PLAN_AUTOTUNE) return ARA_EINVAL;
  if (((uintptr_t)d_ids & 3) || ((uintptr_t)d_off & 7) || ((uintptr_t)d_ylt & 7)) return ARA_EINVAL;
  if (pf->catalogue > 0xffffffffll) return ARA_ERANGE;
  ara_plan* P = new (std::nothrow) ara_plan();
  if (!P) return ARA_ENOMEM;
  P->pf = pf;
  P->n_trials = n_trials;
  P->n_events = n_events;
  P->d_off = d_off;
  P->d_ids = d_ids ? d_ids : reinterpret_cast<const int32_t*>(d_off);
  P->d_ylt = d_ylt;
  P->d_reg = d_reg;
  single_request(*P);
  if (n_sel_in == 0 && layer_sel == nullptr) {
    for (int32_t l = 0; l < pf->n_layers; ++l) P->sel.push_back(l);
  } else {
    if (n_sel_in < 0 || !layer_sel) { bt_free(P); return ARA_EINVAL; }
    for (int32_t i = 0; i < n_sel_in; ++i) {
      if (layer_sel[i] < 0 || layer_sel[i] >= pf->n_layers) { bt_free(P); return ARA_EINVAL; }
      P->sel.push_back(layer_sel[i]);
    }
  }
  if (P->sel.empty()) { bt_free(P); return ARA_EINVAL; }
  if ((int)P->sel.size() > BT_MAX_LAYERS || (int)P->sel.size() > pf->n_layers ||
      (int64_t)P->sel.size() * pf->catalogue >= ((int64_t)1 << 32)) {   // 32-bit row pointers
    bt_free(P);
    return ARA_ERANGE;
  }
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t C = pf->catalogue;
  P->n_blocks = (C + BT_SCAN_BLOCK - 1) / BT_SCAN_BLOCK;
  auto fail = [&](ara_status st) {
    cudaStreamSynchronize(s);
    bt_free(P);
    return st;
  };
  if (cudaMalloc(&P->d_ptr, 4 * (size_t)(C + 1)) != cudaSuccess ||
      cudaMalloc(&P->d_rows, 8 * (size_t)std::max<int64_t>(C, 1)) != cudaSuccess ||
      cudaMalloc(&P->d_bsum, 4 * (size_t)P->n_blocks) != cudaSuccess ||
      cudaMalloc(&P->d_total, 4) != cudaSuccess ||
      cudaMalloc(&P->d_queue, sizeof(unsigned long long)) != cudaSuccess)
    return fail(ARA_ENOMEM);
  // size the table once: the counts depend on the portfolio only
  ara_status st = bt_prep(*P, s, false, nullptr);
  if (st != ARA_OK) return fail(st);
  uint32_t total = 0;
  if (cudaMemcpyAsync(&total, P->d_total, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(ARA_ECUDA);
  if (cudaMalloc(&P->d_entries, 8 * (size_t)std::max<uint32_t>(total, 1)) != cudaSuccess)
    return fail(ARA_ENOMEM);
  if ((st = bt_prep(*P, s, true, nullptr)) != ARA_OK) return fail(st);
  // schedule: the fastest of the candidates on these inputs, or a fixed default
  if (flags & ARA_PLAN_AUTOTUNE) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return fail(ARA_ECUDA);
    const int cand_w[] = {8, 16, 32};
    const int cand_c[] = {1, 2, 4};
    const int cand_t[] = {1, 4};
    const int cand_k[] = {1, 2, 4};
    float best = 1e30f;
    int bw = P->warps, bc = P->ctas_per_sm, bt = P->tpg, bk = P->copies;
    for (int w : cand_w)
      for (int c : cand_c)
        for (int t : cand_t)
          for (int k : cand_k) {
          const int64_t smem = (int64_t)w * (k + 2) * (int64_t)P->sel.size() * 8;
          if (smem * c > (int64_t)pf->max_smem_block || w * 32 * c > 2048) continue;
          P->warps = w;
          P->ctas_per_sm = c;
          P->tpg = t;
          P->copies = k;
          float ms = 0.f, tot = 0.f;
          for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a, s);
            if ((st = bt_stream(*P, s)) != ARA_OK) {
              cudaEventDestroy(a);
              cudaEventDestroy(b);
              return fail(st);
            }
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) return fail(ARA_ECUDA);
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) tot += ms;
          }
          if (tot / 2 < best) { best = tot / 2; bw = w; bc = c; bt = t; bk = k; }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P->warps = bw;
    P->ctas_per_sm = bc;
    P->tpg = bt;
    P->copies = bk;
    P->tuned_ms = best;
  }
  // capture the whole run into a graph on a private stream
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(ARA_ECUDA);
  const bool timing_was = timing_suspend();
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  int nk = 0;
  if (ok) ok = bt_prep(*P, cs, true, &nk) == ARA_OK;
  if (ok) ok = bt_stream(*P, cs) == ARA_OK;
  cudaGraph_t graph = nullptr;
  const bool ended = cudaStreamEndCapture(cs, &graph) == cudaSuccess;
  timing_resume(timing_was);
  cudaStreamDestroy(cs);
  if (!ok || !ended || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(ARA_ECUDA);
  }
  P->graph = graph;
  P->n_kernels = nk + 1;
  if (cudaGraphInstantiate(&P->exec, graph, 0) != cudaSuccess) return fail(ARA_ECUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ARA_ECUDA);
  *out = P;
  return ARA_OK;
}

ara_status ara_run_ylt_requests(ara_portfolio* pf_, int64_t n_trials, const int64_t* d_off,
                                int64_t n_events, const int32_t* d_ids, int32_t n_req,
                                const int32_t* req_layer_first, const int64_t* req_trial_begin,
                                const int64_t* req_trial_end, double* const* d_ylt,
                                uint8_t* const* d_regimes, void* stream) {
  Portfolio* pf = static_cast<Portfolio*>(pf_);
  if (!pf || n_trials < 1 || n_events < 0 || !d_off || (n_events > 0 && !d_ids)) return ARA_EINVAL;
  if (n_req < 1 || !req_layer_first || !req_trial_begin || !req_trial_end || !d_ylt) return ARA_EINVAL;
  if (n_req > BT_MAX_REQ || pf->n_layers > BT_MAX_LAYERS) return ARA_ERANGE;
  if (((uintptr_t)d_ids & 3) || ((uintptr_t)d_off & 7)) return ARA_EINVAL;
  if (pf->catalogue > 0xffffffffll) return ARA_ERANGE;
  GroupArgs g;
  g.n_trials = n_trials;
  g.offsets = d_off;
  g.n_events = n_events;
  g.ids = d_ids ? d_ids : reinterpret_cast<const int32_t*>(d_off);
  g.n_req = n_req;
  if (req_layer_first[0] != 0 || req_layer_first[n_req] != pf->n_layers) return ARA_EINVAL;
  for (int32_t r = 0; r < n_req; ++r) {
    if (req_layer_first[r + 1] <= req_layer_first[r]) return ARA_EINVAL;
    if (req_trial_begin[r] < 0 || req_trial_end[r] <= req_trial_begin[r] || req_trial_end[r] > n_trials)
      return ARA_EINVAL;
    if (!d_ylt[r] || ((uintptr_t)d_ylt[r] & 7)) return ARA_EINVAL;
    g.slot_first[r] = req_layer_first[r];
    g.t0[r] = req_trial_begin[r];
    g.t1[r] = req_trial_end[r];
    g.ylt[r] = d_ylt[r];
    g.reg[r] = d_regimes ? d_regimes[r] : nullptr;
  }
  g.slot_first[n_req] = req_layer_first[n_req];
  DeviceGuard dg(pf->device);
  return run_batched_group_async(*pf, g, (cudaStream_t)stream);
}

ara_status ara_plan_launch(ara_plan* P, void* stream) {
  if (!P || !P->exec) return ARA_EINVAL;
  DeviceGuard g(P->pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  LaunchScope ls(ARA_K_BATCHED, s, P->n_kernels);
  ARA_TRY(cudaGraphLaunch(P->exec, s));
  return ARA_OK;
}

ara_status ara_plan_info(ara_plan* P, int32_t* warps, int32_t* bpsm, int32_t* tpg, double* ms,
                         int32_t* copies) {
  if (!P) return ARA_EINVAL;
  if (warps) *warps = P->warps;
  if (bpsm) *bpsm = P->ctas_per_sm;
  if (tpg) *tpg = P->tpg;
  if (ms) *ms = P->tuned_ms;
  if (copies) *copies = P->copies;
  return ARA_OK;
}

ara_status ara_plan_table(ara_plan* P, const uint64_t** d_rows, int64_t* n_entries) {
  if (!P || !P->d_rows || !P->d_total) return ARA_EINVAL;
  DeviceGuard g(P->pf->device);
  if (d_rows) *d_rows = P->d_rows;
  if (n_entries) {
    uint32_t total = 0;
    ARA_TRY(cudaDeviceSynchronize());
    ARA_TRY(cudaMemcpy(&total, P->d_total, 4, cudaMemcpyDeviceToHost));
    *n_entries = total;
  }
  return ARA_OK;
}

void ara_plan_destroy(ara_plan* P) {
  if (!P) return;
  DeviceGuard g(P->pf->device);
  cudaDeviceSynchronize();
  bt_free(P);
}

}  // extern "C"

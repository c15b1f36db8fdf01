// Adjoint of the YLT path: sensitivities of each layer's mean year loss and TVaR to every
// retention and limit (per-ELT terms I, layer terms T of Section IV-B) and to every ELT loss.
//
// With J = sum_t w_t y_t and the clamp C(x; R, L) = min(max(x - R, 0), L) (slope 1 in x and -1
// in R when 0 < x - R < L, slope 1 in L when x - R > L, 0 at the kinks):
//   g_t  = [aggregate clamp interior for trial t]        (recorded by the forward as regime 1)
//   c(e) = sum_t w_t g_t cnt_t(e)                          (weighted event histogram)
//   dJ/dAggR = -sum_t w_t g_t            dJ/dAggL = sum_t w_t [regime_t == 2]
//   dJ/dOccR = -sum_e c(e) [r_o(e)==1]   dJ/dOccL = sum_e c(e) [r_o(e)==2]
//   dJ/dx_j(e) = c(e) [r_o(e)==1][r_j(e)==1]
//   dJ/dR_j  = -sum_e c(e) [r_o(e)==1][r_j(e)==1]   dJ/dL_j = sum_e c(e) [r_o(e)==1][r_j(e)==2]
// Mean: w_t = 1/N.  TVaR_p: w_t = 1/m above the m-th largest year loss v, and f/m on the
// trials equal to v, f = (m - #{y > v}) / #{y == v} (ties share the boundary weight).
// Every sum is kept as an exact integer count (histograms and counters of trials/events);
// the only roundings are the final divisions by N and m and the products by f.

#include <algorithm>
#include <atomic>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

constexpr unsigned FULLM = 0xffffffffu;

static std::atomic<int32_t> g_adjoint_per_layer{0};
void set_adjoint_per_layer(int32_t on) { g_adjoint_per_layer.store(on); }
int32_t adjoint_per_layer() { return g_adjoint_per_layer.load(); }
constexpr int ADJ_MAX_SLOTS = 256;

struct AdjCounts {          // per layer
  unsigned long long occ[2][3];   // [regime 1 / 2][mean, gt, eq] sums of histogram counts
  unsigned long long agg[2][3];   // [regime 1 / 2][mean, gt, eq] trial counts
};
struct SlotCounts {          // per ELT slot
  unsigned long long rl[2][3];    // [R (interior) / L (above)][mean, gt, eq]
};

__device__ __forceinline__ uint64_t adj_key(double y) {
  const uint64_t b = (uint64_t)__double_as_longlong(y);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <typename T>
__device__ __forceinline__ T warp_sum_int(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULLM, v, o);
  return v;
}

// Block-wide sum of K unsigned 64-bit counters into global counters (one atomic per counter).
template <int K>
__device__ __forceinline__ void block_add(unsigned long long (&v)[K], unsigned long long* out) {
  __shared__ unsigned long long part[32][K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum_int(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) part[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < K) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w][threadIdx.x];
    if (s) atomicAdd(&out[threadIdx.x], s);
  }
}

// ------------------------------------------------------------------------------------------
// Histogram of the events of interior trials, restricted to events whose occurrence clamp is
// not in its zero regime (hit bitmap in shared memory).  One warp per trial; trials outside the
// aggregate interior are skipped without reading their events.
// ------------------------------------------------------------------------------------------
struct AdjHistParams {
  int64_t n_trials;
  const int64_t* offsets;
  int64_t n_events;
  const int32_t* ids;
  int64_t catalogue;
  const uint8_t* regimes;     // this layer's recorded aggregate regimes [n_trials]
  const double* ylt;          // this layer's YLT [n_trials]
  const uint64_t* thr_key;    // device: key of the m-th largest year loss
  const uint32_t* bits;       // exact bitmap of r_o(e) != 0
  int64_t bm_words, smem_words;
  int32_t shift;
  uint32_t* h_mean;
  uint32_t* h_gt;
  uint32_t* h_eq;
  uint32_t* err;
  AdjCounts* acc;             // this layer's trial counts (agg) are added here
};

// Coarse regime bitmap word cw, interleaved: bit i is the OR of bit i of the exact words
// [cw << shift, (cw + 1) << shift), so event e is tested at bit (e mod 32) of word
// e >> (5 + shift).
__device__ __forceinline__ uint32_t adj_coarsen(const uint32_t* __restrict__ src, int64_t cw,
                                                int shift, int64_t n_words) {
  const int64_t w0 = cw << shift;
  const int64_t w1 = min(w0 + ((int64_t)1 << shift), n_words);
  uint32_t out = 0;
  for (int64_t w = w0; w < w1; ++w) out |= src[w];
  return out;
}

// Hint that bytes [a, b) of the ID array will be read soon: one bulk prefetch into L2 of the
// 16-byte-aligned part of the range that lies inside the array (a hint; nothing is loaded into
// registers or shared memory).
__device__ __forceinline__ void prefetch_ids_l2(const int32_t* ids, int64_t n_events, int64_t b0,
                                                int64_t b1) {
  const uintptr_t base = (uintptr_t)ids, lo = base + 4 * (uintptr_t)max(b0, (int64_t)0);
  const uintptr_t hi = base + 4 * (uintptr_t)min(b1, n_events);
  const uintptr_t a = (lo + 15) & ~(uintptr_t)15, e = hi & ~(uintptr_t)15;
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

__global__ void __launch_bounds__(1024, 1) k_adj_hist(AdjHistParams p) {
  extern __shared__ uint32_t bm[];
  // per warp: trial counts [regime 1 / 2][all, above, equal to the threshold]
  __shared__ unsigned int tcnt[32][6];
  for (int64_t cw = threadIdx.x; cw < p.smem_words; cw += blockDim.x)
    bm[cw] = adj_coarsen(p.bits, cw, p.shift, p.bm_words);
  if (threadIdx.x < 32 * 6) tcnt[threadIdx.x / 6][threadIdx.x % 6] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t thr = *p.thr_key;
  const int shift5 = p.shift + 5;
  bool bad_id = false, bad_off = false;
  // Trials are dealt one at a time, round-robin over every warp of the grid, so each warp gets
  // n_trials / warps of them (a 32-trial unit left most warps idle or doubly loaded).  The
  // class and range of the warp's next 32 trials are loaded at once, one trial per lane, so the
  // chain regime -> year loss -> offsets is paid once per 32 trials; while a trial is processed,
  // the IDs of the warp's next interior trial are fetched into L2.
  for (int64_t tb = warp; tb < p.n_trials; tb += 32 * nwarps) {
    const int64_t tl = tb + (int64_t)lane * nwarps;
    int cls = 0;
    int64_t mb = 0, me = 0;
    const uint8_t rg = tl < p.n_trials ? p.regimes[tl] : 0;
    bool above = false, equal = false;
    if (rg != 0) {
      const uint64_t key = adj_key(p.ylt[tl]);
      above = key > thr;
      equal = key == thr;
    }
    if (rg == 1) {
      cls = above ? 2 : (equal ? 3 : 1);
      mb = __ldg(p.offsets + tl);
      me = __ldg(p.offsets + tl + 1);
    }
    {   // the batch's trial counts, by regime and position against the threshold
      const unsigned c0 = __popc(__ballot_sync(FULLM, rg == 1));
      const unsigned c1 = __popc(__ballot_sync(FULLM, rg == 1 && above));
      const unsigned c2 = __popc(__ballot_sync(FULLM, rg == 1 && equal));
      const unsigned c3 = __popc(__ballot_sync(FULLM, rg == 2));
      const unsigned c4 = __popc(__ballot_sync(FULLM, rg == 2 && above));
      const unsigned c5 = __popc(__ballot_sync(FULLM, rg == 2 && equal));
      if (lane == 0) {
        unsigned int* tc = tcnt[threadIdx.x >> 5];
        tc[0] += c0; tc[1] += c1; tc[2] += c2; tc[3] += c3; tc[4] += c4; tc[5] += c5;
      }
    }
    unsigned todo = __ballot_sync(FULLM, cls != 0);
    while (todo) {
      const int k = __ffs(todo) - 1;
      todo &= todo - 1;
      const int c = __shfl_sync(FULLM, cls, k);
      const int64_t beg = __shfl_sync(FULLM, mb, k), end = __shfl_sync(FULLM, me, k);
      if (todo) {   // the next interior trial of this batch
        const int kn = __ffs(todo) - 1;
        const int64_t nb = __shfl_sync(FULLM, mb, kn), ne = __shfl_sync(FULLM, me, kn);
        if (lane == 0 && 0 <= nb && nb <= ne && ne <= p.n_events)
          prefetch_ids_l2(p.ids, p.n_events, nb, ne);
      }
      if (!(0 <= beg && beg <= end && end <= p.n_events)) { bad_off = true; continue; }
      // the trial's second histogram (above / equal to the threshold), uniform over the warp
      uint32_t* const hx = c == 2 ? p.h_gt : (c == 3 ? p.h_eq : nullptr);
      // segments of at most 2^30 IDs keep the per-ID offsets in 32 bits
      for (int64_t sb = beg; sb < end; sb += ((int64_t)1 << 30)) {
        const int32_t* const idp = p.ids + sb;
        const int32_t n = (int32_t)min(end - sb, (int64_t)1 << 30);
        // sixteen independent streaming loads per lane in flight, then the filtered atomics; the
        // range, ID and bitmap tests are predicates, not branches
        for (int32_t o = 0; o < n; o += 512) {
          int ev[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int32_t j = o + 32 * u + lane;
            ev[u] = j < n ? __ldcs(idp + j) : 0;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int32_t j = o + 32 * u + lane;
            const uint32_t e = (uint32_t)ev[u];
            const bool in = j < n, ok = e < (uint32_t)p.catalogue;
            bad_id |= in && !ok;
            const uint32_t w = (in && ok) ? bm[e >> shift5] : 0u;
            if ((w >> (e & 31)) & 1u) {
              atomicAdd(p.h_mean + e, 1u);
              if (hx) atomicAdd(hx + e, 1u);
            }
          }
        }
      }
    }
  }
  if (bad_id) atomicOr(p.err, DERR_EVENT_RANGE);
  if (bad_off) atomicOr(p.err, DERR_OFFSETS);
  __syncthreads();
  if (threadIdx.x < 6) {
    unsigned long long sum = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += tcnt[w][threadIdx.x];
    if (sum) atomicAdd(&p.acc->agg[0][0] + threadIdx.x, sum);
  }
}

// Sums over catalogue events of the histograms, split by occurrence regime.
__global__ void __launch_bounds__(256) k_adj_events(int64_t catalogue, const uint8_t* __restrict__ reg,
                                                    const uint32_t* __restrict__ hm,
                                                    const uint32_t* __restrict__ hg,
                                                    const uint32_t* __restrict__ he,
                                                    AdjCounts* __restrict__ acc) {
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < catalogue;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t r = reg[e];
    if (r == 0) continue;
    const int o = (r == 1) ? 0 : 3;
    v[o + 0] += hm[e];
    v[o + 1] += hg[e];
    v[o + 2] += he[e];
  }
  block_add<6>(v, &acc->occ[0][0]);
}

// Per ELT record: its loss gradient for both objectives, and per ELT slot the counts of the
// retention (interior) and limit (above) derivatives.
struct AdjRecParams {
  const int64_t* rec_off;
  const int32_t* rec_ids;
  const float* loss32;
  const double* loss64;
  const int32_t* rec_orig;     // original position of each (sorted) record within its ELT
  const double* elt_ret;
  const double* elt_lim;
  const uint8_t* reg;
  const uint32_t* hm;
  const uint32_t* hg;
  const uint32_t* he;
  const unsigned long long* sel_gt;   // #{y > v} of this layer
  const unsigned long long* sel_eq;   // #{y == v}
  int64_t n_trials, m;
  double* grad_loss_mean;      // [M] objective 0
  double* grad_loss_tvar;      // [M] objective 1
  SlotCounts* slots;           // [n_slots of this layer]
  int32_t n_slots;
  int32_t elt[ADJ_MAX_SLOTS];
  int64_t base[ADJ_MAX_SLOTS];
};

__global__ void __launch_bounds__(256) k_adj_records(AdjRecParams p) {
  const int k = blockIdx.y;
  const int j = p.elt[k];
  const double R = p.elt_ret[j], L = p.elt_lim[j];
  const double invN = 1.0 / (double)p.n_trials, invM = 1.0 / (double)p.m;
  const unsigned long long cg = *p.sel_gt, ce = *p.sel_eq;
  const double f = ce ? (double)(p.m - (int64_t)cg) / (double)ce : 0.0;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t r = p.rec_off[j] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < p.rec_off[j + 1];
       r += (int64_t)gridDim.x * blockDim.x) {
    const int e = p.rec_ids[r];
    const double x = p.loss32 ? (double)p.loss32[r] : p.loss64[r];
    const double ex = __dsub_rn(x, R);
    const int rj = (ex > 0.0 && ex < L) ? 1 : (ex > L ? 2 : 0);
    double gm = 0.0, gt = 0.0;
    if (p.reg[e] == 1 && rj != 0) {
      const uint32_t a = p.hm[e], b = p.hg[e], c = p.he[e];
      const int o = (rj == 1) ? 0 : 3;
      v[o + 0] += a;
      v[o + 1] += b;
      v[o + 2] += c;
      if (rj == 1) {
        gm = (double)a * invN;
        gt = ((double)b + f * (double)c) * invM;
      }
    }
    const int64_t pos = p.base[k] + p.rec_orig[r];
    p.grad_loss_mean[pos] = gm;
    p.grad_loss_tvar[pos] = gt;
  }
  block_add<6>(v, &p.slots[k].rl[0][0]);
}

// Per trial: counts of interior / saturated aggregate regimes, overall and in TVaR's top set.
// Final per-layer gradients from the integer counts.
__global__ void k_adj_finish(const AdjCounts* __restrict__ acc, const SlotCounts* __restrict__ slots,
                             int32_t n_slots, const unsigned long long* sel_gt,
                             const unsigned long long* sel_eq, int64_t n, int64_t m,
                             double* grad_layer_mean, double* grad_layer_tvar,
                             double* grad_elt_mean, double* grad_elt_tvar) {
  const double invN = 1.0 / (double)n, invM = 1.0 / (double)m;
  const unsigned long long cg = *sel_gt, ce = *sel_eq;
  const double f = ce ? (double)(m - (int64_t)cg) / (double)ce : 0.0;
  auto mean_of = [&](const unsigned long long (&c)[3]) { return (double)c[0] * invN; };
  auto tvar_of = [&](const unsigned long long (&c)[3]) {
    return ((double)c[1] + f * (double)c[2]) * invM;
  };
  if (threadIdx.x == 0) {
    grad_layer_mean[0] = -mean_of(acc->occ[0]);
    grad_layer_mean[1] = mean_of(acc->occ[1]);
    grad_layer_mean[2] = -mean_of(acc->agg[0]);
    grad_layer_mean[3] = mean_of(acc->agg[1]);
    grad_layer_tvar[0] = -tvar_of(acc->occ[0]);
    grad_layer_tvar[1] = tvar_of(acc->occ[1]);
    grad_layer_tvar[2] = -tvar_of(acc->agg[0]);
    grad_layer_tvar[3] = tvar_of(acc->agg[1]);
  }
  for (int k = threadIdx.x; k < n_slots; k += blockDim.x) {
    grad_elt_mean[2 * k + 0] = -mean_of(slots[k].rl[0]);
    grad_elt_mean[2 * k + 1] = mean_of(slots[k].rl[1]);
    grad_elt_tvar[2 * k + 0] = -tvar_of(slots[k].rl[0]);
    grad_elt_tvar[2 * k + 1] = tvar_of(slots[k].rl[1]);
  }
}

// Weighted accumulation of one layer's gradients into the portfolio's parameter layout:
// out += w0 * objective-0 gradient + w1 * objective-1 gradient.
struct AdjScatterParams {
  double w0, w1;
  int32_t layer, n_slots;
  const double* gl0;   // [4] layer gradients, objective 0
  const double* gl1;
  const double* ge0;   // [n_slots][2] ELT-slot gradients
  const double* ge1;
  const double* gx0;   // [records of the layer's slots] loss gradients
  const double* gx1;
  const int64_t* rec_off;
  const int32_t* rec_orig;
  double* g_elt_ret;   // [n_elts]
  double* g_elt_lim;
  double* g_layer;     // [n_layers][4]
  double* g_loss;      // [n_records], creation order
  int32_t elt[ADJ_MAX_SLOTS];
  int64_t base[ADJ_MAX_SLOTS];
};

__global__ void __launch_bounds__(256) k_adj_scatter(AdjScatterParams p) {
  const int k = blockIdx.y;
  const int j = p.elt[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&p.g_elt_ret[j], p.w0 * p.ge0[2 * k] + p.w1 * p.ge1[2 * k]);
    atomicAdd(&p.g_elt_lim[j], p.w0 * p.ge0[2 * k + 1] + p.w1 * p.ge1[2 * k + 1]);
    if (k == 0)
      for (int c = 0; c < 4; ++c) p.g_layer[4 * p.layer + c] += p.w0 * p.gl0[c] + p.w1 * p.gl1[c];
  }
  const int64_t r0 = p.rec_off[j], n = p.rec_off[j + 1] - r0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = p.rec_orig[r0 + i];        // creation-order position within the ELT
    const int64_t src = p.base[k] + o;
    const double g = p.w0 * p.gx0[src] + p.w1 * p.gx1[src];
    if (g != 0.0) atomicAdd(&p.g_loss[r0 + o], g);
  }
}

// ------------------------------------------------------------------------------------------
// Several layers in one pass over the YET.  Event-major rows list, for every catalogue event, the
// selected layers (slots, ascending) whose occurrence regime for the event is not 0, and the
// histograms are kept per row entry, so no count is made for an event of regime 0.  A trial is
// read once if any slot has it in the aggregate interior, and each of its occurrences adds to
// the entries of exactly those slots.  The counts equal those of the per-layer passes.
// ------------------------------------------------------------------------------------------
constexpr int ADJB_WARPS = 32;
constexpr int ADJB_MAX_SEL = 255;   // slots fit in one byte

// Row descriptor and the slot of every entry.  The descriptor holds the first entry (bits 0-31),
// the length (bits 32-39) and the slots of the first three entries (bits 40-47, 48-55, 56-63),
// so that most rows (1.4 entries on average on the adjoint workload) need no entry loads in the
// histogram pass.  Entries at or beyond cap are not written (cap bounds the allocation; a larger
// table is reported as a data error).
__global__ void __launch_bounds__(256)
k_adjb_fill(int32_t n_sel, const uint32_t* __restrict__ bits, int64_t bits_stride, int64_t C,
            const uint32_t* __restrict__ ptr, uint32_t cap, uint8_t* __restrict__ ent,
            uint64_t* __restrict__ rows, uint32_t* __restrict__ err) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= C) return;
  uint32_t pos = ptr[e];
  uint32_t end = ptr[e + 1];
  if (end > cap) {
    atomicOr(err, DERR_EVENT_RANGE);
    end = cap;
    pos = min(pos, cap);
  }
  uint64_t desc = (uint64_t)pos | ((uint64_t)(end - pos) << 32);
  const uint32_t* b = bits + (e >> 5);
  const int sh = (int)(e & 31);
  int k = 0;
  for (int i = 0; i < n_sel && pos < end; ++i)
    if ((__ldg(b + (int64_t)i * bits_stride) >> sh) & 1u) {
      ent[pos++] = (uint8_t)i;
      if (k < 3) desc |= (uint64_t)i << (40 + 8 * k);
      ++k;
    }
  rows[e] = desc;
}

// Class of every (trial, slot), trial-major [n_trials][n_sel]: 0 outside the slot's aggregate
// interior; 1 interior, below TVaR's threshold value v; 2 above v; 3 equal to v.  Also each
// slot's trial counts by aggregate regime and position against v (AdjCounts.agg).
__global__ void __launch_bounds__(256)
k_adjb_class(int64_t n_trials, int32_t n_sel, const uint8_t* __restrict__ regimes,
             const double* __restrict__ ylt, const uint64_t* __restrict__ thr_key,
             int64_t thr_stride, uint8_t* __restrict__ cls, AdjCounts* __restrict__ acc) {
  const int i = blockIdx.y;
  const uint64_t thr = thr_key[(int64_t)i * thr_stride];
  const uint8_t* rg_row = regimes + (int64_t)i * n_trials;
  const double* y_row = ylt + (int64_t)i * n_trials;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_trials;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t rg = rg_row[t];
    uint8_t c = 0;
    if (rg != 0) {
      const uint64_t key = adj_key(y_row[t]);
      const bool above = key > thr, equal = key == thr;
      const int o = rg == 1 ? 0 : 3;
      v[o] += 1;
      v[o + 1] += above ? 1 : 0;
      v[o + 2] += equal ? 1 : 0;
      if (rg == 1) c = above ? 2 : (equal ? 3 : 1);
    }
    cls[t * n_sel + i] = c;
  }
  block_add<6>(v, &acc[i].agg[0][0]);
}

struct AdjbHistParams {
  int64_t n_trials;
  const int64_t* offsets;
  int64_t n_events;
  const int32_t* ids;
  int64_t catalogue;
  int32_t n_sel;
  uint32_t cap;               // entries allocated
  const uint8_t* cls;         // [n_trials][n_sel]
  const uint64_t* rows;       // [catalogue]
  const uint8_t* ent;         // [cap]
  uint32_t* h_mean;           // [cap] each
  uint32_t* h_gt;
  uint32_t* h_eq;
  uint32_t* err;
};

// One warp per trial, dealt round-robin over the grid.  The trial's class row goes to the warp's
// shared memory; a trial interior for no slot is skipped without reading its events.  Eight IDs
// per lane are loaded at once, then their row descriptors, then the row entries are walked.
__global__ void __launch_bounds__(ADJB_WARPS * 32) k_adjb_hist(AdjbHistParams p) {
  __shared__ uint8_t cls_s[ADJB_WARPS][ADJB_MAX_SEL + 1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint8_t* const cs = cls_s[wl];
  const uint32_t cat = (uint32_t)p.catalogue;
  bool bad_id = false, bad_off = false;
  for (int64_t t = warp; t < p.n_trials; t += nwarps) {
    unsigned any = 0;
    for (int i = lane; i < p.n_sel; i += 32) {
      const uint8_t c = p.cls[t * p.n_sel + i];
      cs[i] = c;
      any |= c;
    }
    __syncwarp();
    if (!__any_sync(FULLM, any != 0)) continue;
    const int64_t beg = __ldg(p.offsets + t), end = __ldg(p.offsets + t + 1);
    if (!(0 <= beg && beg <= end && end <= p.n_events)) {
      bad_off = true;
      continue;
    }
    for (int64_t o = beg; o < end; o += 32 * 8) {
      int ev[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = o + 32 * u + lane;
        ev[u] = j < end ? __ldcs(p.ids + j) : -1;
      }
      uint64_t rw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = o + 32 * u + lane;
        const bool in = j < end, ok = (uint32_t)ev[u] < cat;
        bad_id |= in && !ok;
        rw[u] = (in && ok) ? __ldg(p.rows + (uint32_t)ev[u]) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t first = (uint32_t)rw[u], len = (uint32_t)(rw[u] >> 32) & 0xffu;
        for (uint32_t k = 0; k < len; ++k) {
          const uint32_t x = first + k;
          if (x >= p.cap) break;
          const uint32_t sl = k < 3 ? (uint32_t)(rw[u] >> (40 + 8 * k)) & 0xffu : p.ent[x];
          const uint8_t c = cs[sl];
          if (c) {
            atomicAdd(p.h_mean + x, 1u);
            if (c == 2) atomicAdd(p.h_gt + x, 1u);
            else if (c == 3) atomicAdd(p.h_eq + x, 1u);
          }
        }
      }
    }
    __syncwarp();
  }
  if (bad_id) atomicOr(p.err, DERR_EVENT_RANGE);
  if (bad_off) atomicOr(p.err, DERR_OFFSETS);
}

// The same histograms from an event-major index of the YET (YetIndex).  Per group of up to 16
// selected layers (slots [q0, q0 + nq)), each trial's classes are packed into one word, 2 bits
// per slot: bit 0 the aggregate interior (class != 0), bit 1 at or above TVaR's threshold value
// (class 2 or 3).  A trial equal to the threshold value for some slot of the group (class 3, a
// handful of trials) instead has its slot-0 field set to 0b10, which no class gives; its
// occurrences take an exact path that reads the classes from the byte table.  One launch per
// block of trials: every CTA holds the block's class words in shared memory (the padding offset
// YX_PAD reads a zero word), and each warp takes one group of 32 catalogue events, lane l the
// event 32 g + l, as the index interleaves them.  A lane finds its row entries whose slots lie
// in the layer group (rows hold slots in ascending order, so they form one run), then walks the
// event's list of the block, 8 entries per 16-byte load: for each occurrence it reads the
// trial's class word and adds, per entry, the word's 2-bit field (interior + 2 x above) and its
// bit 1 (2 x above) into two registers, from which the interior and above counts follow.  Up
// to ADJX_K entries per walk; a lane with more walks the list again for the next ADJX_K.  At the
// end it adds its counts into the entry histograms, which no other lane writes in this launch
// (launches follow one another on the stream; the exact path's atomics are the same lane's).
// The counts are the integers the trial-major pass counts.
constexpr int ADJX_LAYERS = 16;    // slots per class word (2 bits each)
constexpr int ADJX_K = 5;          // entries counted per walk of a list
constexpr int ADJX_SMEM = (int)(YX_PAD + 1) * 4;

__global__ void __launch_bounds__(256)
k_adjx_words(int64_t n_trials, int32_t n_sel, int32_t q0, int32_t nq,
             const uint8_t* __restrict__ cls, uint32_t* __restrict__ words) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_trials;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* c = cls + t * n_sel + q0;
    uint32_t w = 0;
    bool eq = false;
    for (int i = 0; i < nq; ++i) {
      const uint32_t ci = c[i];
      w |= (ci != 0u ? 1u : 0u) << (2 * i);
      w |= (ci >= 2u ? 2u : 0u) << (2 * i);
      eq = eq || ci == 3u;
    }
    words[t] = eq ? (w & ~3u) | 2u : w;
  }
}

struct AdjxHistParams {
  const uint16_t* ent16;      // the index's entries
  const int64_t* base;        // [groups] of this block
  const uint32_t* len;        // [groups] of this block
  int64_t groups, catalogue;
  int64_t t0, nb;             // the block's first trial as an index into words (< 0 when the
                              // adjoint's trials start inside the block), trials in the block
  int64_t n_words;            // the adjoint's trials (words and cls rows)
  const uint32_t* words;      // [n_trials] class words of slots [q0, q0 + nq)
  const uint8_t* cls;         // [n_trials][n_sel] classes, for the flagged trials
  int32_t n_sel, q0, nq;
  const uint64_t* rows;       // [catalogue] row descriptors (k_adjb_fill)
  const uint8_t* ent;         // [cap] slot of every row entry
  uint32_t cap;
  uint32_t* h_mean;
  uint32_t* h_gt;
  uint32_t* h_eq;
};

__device__ __forceinline__ uint32_t adjx_slot(uint64_t rw, uint32_t first, uint32_t j, uint32_t cap,
                                              const uint8_t* __restrict__ ent) {
  if (j < 3) return (uint32_t)(rw >> (40 + 8 * j)) & 0xffu;
  const uint32_t x = first + j;
  return x < cap ? (uint32_t)ent[x] : 0xffu;
}

__global__ void __launch_bounds__(1024, 1) k_adjx_hist(AdjxHistParams p) {
  extern __shared__ uint32_t cw[];   // [YX_PAD + 1] class words of the block's trials
  for (int64_t i = threadIdx.x; i <= (int64_t)YX_PAD; i += blockDim.x)
    cw[i] = (i < p.nb && p.t0 + i >= 0 && p.t0 + i < p.n_words) ? __ldg(p.words + p.t0 + i) : 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t qlo = (uint32_t)p.q0, qhi = (uint32_t)(p.q0 + p.nq);
  for (int64_t g = gw; g < p.groups; g += nw) {
    const uint32_t L = __ldg(p.len + g);
    if (L == 0) continue;                                   // uniform over the warp
    const int64_t e = g * 32 + lane;
    const uint64_t rw = e < p.catalogue ? __ldg(p.rows + e) : 0ull;
    const uint32_t first = (uint32_t)rw, rl = (uint32_t)(rw >> 32) & 0xffu;
    uint32_t j0 = 0, j1 = 0;                                // entries with slot < qlo, < qhi
    for (uint32_t j = 0; j < rl; ++j) {
      const uint32_t sl = adjx_slot(rw, first, j, p.cap, p.ent);
      if (first + j >= p.cap) break;
      j0 += sl < qlo ? 1u : 0u;
      j1 += sl < qhi ? 1u : 0u;
    }
    const int n_in = (int)(j1 - j0);
    const int walks = __reduce_max_sync(0xffffffffu, (uint32_t)((n_in + ADJX_K - 1) / ADJX_K));
    const uint4* lst = reinterpret_cast<const uint4*>(p.ent16 + __ldg(p.base + g)) + lane;
    const uint32_t steps = L / 8;                            // 8 entries per lane and load
    for (int c = 0; c < walks; ++c) {
      const int jb = (int)j0 + c * ADJX_K;
      const int have = min(ADJX_K, (int)j1 - jb);           // entries counted by this walk
      const int hv = __reduce_max_sync(0xffffffffu, (uint32_t)max(have, 0));
      uint32_t sh[ADJX_K], m3[ADJX_K], ca[ADJX_K], cb[ADJX_K];
#pragma unroll
      for (int k = 0; k < ADJX_K; ++k) {
        sh[k] = k < have ? 2u * (adjx_slot(rw, first, (uint32_t)(jb + k), p.cap, p.ent) - qlo) : 0u;
        m3[k] = k < have ? 3u : 0u;                         // nothing for unused entries
        ca[k] = cb[k] = 0u;
      }
      auto count = [&](uint32_t off) {
        off = min(off, YX_PAD);
        const uint32_t w = cw[off];
        if ((w & 3u) == 2u) {                               // a trial equal to the threshold
          const uint8_t* c = p.cls + (p.t0 + off) * p.n_sel + p.q0;
#pragma unroll
          for (int k = 0; k < ADJX_K; ++k)
            if (k < have) {
              const uint32_t x = first + (uint32_t)(jb + k), cl = c[sh[k] >> 1];
              if (x < p.cap && cl != 0u) {
                atomicAdd(p.h_mean + x, 1u);
                if (cl == 2u) atomicAdd(p.h_gt + x, 1u);
                if (cl == 3u) atomicAdd(p.h_eq + x, 1u);
              }
            }
          return;
        }
#pragma unroll
        for (int k = 0; k < ADJX_K; ++k)
          if (k < hv) {                                     // uniform over the warp
            const uint32_t f = (w >> sh[k]) & m3[k];
            ca[k] += f;                                     // interior + 2 x above
            cb[k] += f & 2u;                                // 2 x above
          }
      };
#pragma unroll 2
      for (uint32_t i = 0; i < steps; ++i) {
        const uint4 v = __ldcs(lst + (int64_t)i * 32);
        count(v.x & 0xffffu);
        count(v.x >> 16);
        count(v.y & 0xffffu);
        count(v.y >> 16);
        count(v.z & 0xffffu);
        count(v.z >> 16);
        count(v.w & 0xffffu);
        count(v.w >> 16);
      }
#pragma unroll
      for (int k = 0; k < ADJX_K; ++k)
        if (k < have) {
          const uint32_t x = first + (uint32_t)(jb + k);
          if (x < p.cap) {
            p.h_mean[x] += ca[k] - cb[k];
            p.h_gt[x] += cb[k] >> 1;
          }
        }
    }
  }
}

// Sums over catalogue events of every slot's histograms, split by occurrence regime
// (AdjCounts.occ of each slot), from the entry histograms.
__global__ void __launch_bounds__(256)
k_adjb_events(int64_t C, int32_t n_sel, uint32_t cap, const uint64_t* __restrict__ rows,
              const uint8_t* __restrict__ ent, const uint8_t* __restrict__ reg_all,
              const uint32_t* __restrict__ hm, const uint32_t* __restrict__ hg,
              const uint32_t* __restrict__ he, AdjCounts* __restrict__ acc) {
  extern __shared__ unsigned long long sacc[];   // [n_sel][6]
  for (int i = threadIdx.x; i < 6 * n_sel; i += blockDim.x) sacc[i] = 0ull;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < C;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t rw = rows[e];
    const uint32_t first = (uint32_t)rw, len = (uint32_t)(rw >> 32) & 0xffu;
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t x = first + k;
      if (x >= cap) break;
      const int sl = ent[x];
      const uint8_t r = reg_all[(int64_t)sl * C + e];
      const int o = sl * 6 + (r == 1 ? 0 : 3);
      const uint32_t a = hm[x], b = hg[x], c = he[x];
      if (a) atomicAdd(&sacc[o + 0], (unsigned long long)a);
      if (b) atomicAdd(&sacc[o + 1], (unsigned long long)b);
      if (c) atomicAdd(&sacc[o + 2], (unsigned long long)c);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * n_sel; i += blockDim.x)
    if (sacc[i]) atomicAdd(&acc[i / 6].occ[0][0] + (i % 6), sacc[i]);
}

// k_adj_records for every ELT slot of every layer of a multi-layer pass, up to ADJ_MAX_SLOTS ELT
// slots per launch (blockIdx.y): an event's histogram values are those of its row entry for the
// layer (present whenever the event's occurrence regime is not 0).
struct AdjbRecParams {
  const int64_t* rec_off;
  const int32_t* rec_ids;
  const float* loss32;
  const double* loss64;
  const int32_t* rec_orig;
  const double* elt_ret;
  const double* elt_lim;
  const uint8_t* reg_all;            // [n_sel][C]
  int64_t C;
  const uint64_t* rows;
  const uint8_t* ent;
  const uint32_t* hm;
  const uint32_t* hg;
  const uint32_t* he;
  uint32_t cap;
  const unsigned long long* sel_gt;  // [n_sel]
  const unsigned long long* sel_eq;
  int64_t n_trials, m;
  double* grad_loss_mean;
  double* grad_loss_tvar;
  SlotCounts* slots;                 // all ELT slots, layers in selection order
  int32_t slot0;                     // first ELT slot of this launch
  int32_t elt[ADJ_MAX_SLOTS];
  int64_t base[ADJ_MAX_SLOTS];
  uint8_t layer[ADJ_MAX_SLOTS];      // selection index of the slot's layer
};

__global__ void __launch_bounds__(256) k_adjb_records(AdjbRecParams p) {
  const int k = blockIdx.y;
  const int j = p.elt[k];
  const int li = p.layer[k];
  const uint8_t* reg = p.reg_all + (int64_t)li * p.C;
  const double R = p.elt_ret[j], L = p.elt_lim[j];
  const double invN = 1.0 / (double)p.n_trials, invM = 1.0 / (double)p.m;
  const unsigned long long cg = p.sel_gt[li], ce = p.sel_eq[li];
  const double f = ce ? (double)(p.m - (int64_t)cg) / (double)ce : 0.0;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t r = p.rec_off[j] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < p.rec_off[j + 1];
       r += (int64_t)gridDim.x * blockDim.x) {
    const int e = p.rec_ids[r];
    const double x = p.loss32 ? (double)p.loss32[r] : p.loss64[r];
    const double ex = __dsub_rn(x, R);
    const int rj = (ex > 0.0 && ex < L) ? 1 : (ex > L ? 2 : 0);
    double gm = 0.0, gt = 0.0;
    if (reg[e] == 1 && rj != 0) {
      const uint64_t rw = p.rows[e];
      const uint32_t first = (uint32_t)rw, len = (uint32_t)(rw >> 32) & 0xffu;
      uint32_t a = 0, b = 0, c = 0;
      for (uint32_t t = 0; t < len; ++t) {
        const uint32_t xi = first + t;
        if (xi >= p.cap) break;
        if (p.ent[xi] == li) {
          a = p.hm[xi];
          b = p.hg[xi];
          c = p.he[xi];
          break;
        }
      }
      const int o = (rj == 1) ? 0 : 3;
      v[o + 0] += a;
      v[o + 1] += b;
      v[o + 2] += c;
      if (rj == 1) {
        gm = (double)a * invN;
        gt = ((double)b + f * (double)c) * invM;
      }
    }
    const int64_t pos = p.base[k] + p.rec_orig[r];
    p.grad_loss_mean[pos] = gm;
    p.grad_loss_tvar[pos] = gt;
  }
  block_add<6>(v, &p.slots[p.slot0 + k].rl[0][0]);
}

// k_adj_finish for every layer of a multi-layer pass, one block per layer.
struct AdjbFinishParams {
  const AdjCounts* acc;              // [n_sel]
  const SlotCounts* slots;           // all ELT slots
  const unsigned long long* sel_gt;
  const unsigned long long* sel_eq;
  int64_t n, m, total_slots;
  int32_t n_sel;
  double* grad_layer;                // [2][n_sel][4]
  double* grad_elt;                  // [2][total_slots][2]
  int32_t slot_off[ADJB_MAX_SEL + 1];
};

__global__ void __launch_bounds__(256) k_adjb_finish(AdjbFinishParams p) {
  const int i = blockIdx.x;
  const double invN = 1.0 / (double)p.n, invM = 1.0 / (double)p.m;
  const unsigned long long cg = p.sel_gt[i], ce = p.sel_eq[i];
  const double f = ce ? (double)(p.m - (int64_t)cg) / (double)ce : 0.0;
  auto mean_of = [&](const unsigned long long (&c)[3]) { return (double)c[0] * invN; };
  auto tvar_of = [&](const unsigned long long (&c)[3]) {
    return ((double)c[1] + f * (double)c[2]) * invM;
  };
  const AdjCounts& a = p.acc[i];
  if (threadIdx.x == 0) {
    double* gm = p.grad_layer + 4 * (int64_t)i;
    double* gt = p.grad_layer + 4 * (int64_t)(p.n_sel + i);
    gm[0] = -mean_of(a.occ[0]);
    gm[1] = mean_of(a.occ[1]);
    gm[2] = -mean_of(a.agg[0]);
    gm[3] = mean_of(a.agg[1]);
    gt[0] = -tvar_of(a.occ[0]);
    gt[1] = tvar_of(a.occ[1]);
    gt[2] = -tvar_of(a.agg[0]);
    gt[3] = tvar_of(a.agg[1]);
  }
  for (int k = p.slot_off[i] + threadIdx.x; k < p.slot_off[i + 1]; k += blockDim.x) {
    const SlotCounts& c = p.slots[k];
    p.grad_elt[2 * k + 0] = -mean_of(c.rl[0]);
    p.grad_elt[2 * k + 1] = mean_of(c.rl[1]);
    p.grad_elt[2 * (p.total_slots + k) + 0] = -tvar_of(c.rl[0]);
    p.grad_elt[2 * (p.total_slots + k) + 1] = tvar_of(c.rl[1]);
  }
}

// The adjoint of several layers with one histogram pass (the kernels above).  Returns ARA_ERANGE
// without queueing anything when the layers' table would not fit 32-bit entry indices; the
// caller then takes the per-layer path.
static ara_status adjoint_multi(Portfolio& pf, const std::vector<int32_t>& sel, int64_t n_trials,
                                const int64_t* d_offsets, int64_t n_events, const int32_t* d_ids,
                                const YetIndex* yx, int64_t first_trial, const double* d_ylt,
                                const uint8_t* d_regimes,
                                int64_t m, const SelectResult& sr, double* d_grad_elt,
                                double* d_grad_layer, double* d_grad_loss, int64_t total_slots,
                                int64_t total_loss, cudaStream_t s) {
  const int32_t n_sel = (int32_t)sel.size();
  const int64_t C = pf.catalogue, bmw = pf.bm_words;
  int64_t bound = 0;   // every entry is an event of one of the slot's ELTs
  for (int32_t l : sel)
    for (int k = pf.layer_off[l]; k < pf.layer_off[l + 1]; ++k) {
      const int j = pf.layer_elts[k];
      bound += pf.rec_off[j + 1] - pf.rec_off[j];
    }
  if (bound >= (int64_t)UINT32_MAX || n_sel > ADJB_MAX_SEL) return ARA_ERANGE;
  bound = std::max<int64_t>(bound, 1);
  const int64_t n_blocks = (C + 1023) / 1024;
  size_t off = 0;
  auto take = [&](size_t n) { size_t o = (off + 255) / 256 * 256; off = o + n; return o; };
  const size_t o_reg = take((size_t)n_sel * C), o_bits = take(4 * (size_t)n_sel * bmw);
  const size_t o_ptr = take(4 * (size_t)(C + 1)), o_bsum = take(4 * (size_t)n_blocks), o_tot = take(4);
  const size_t o_rows = take(8 * (size_t)C), o_ent = take((size_t)bound);
  const size_t o_cls = take((size_t)n_trials * n_sel);
  const size_t o_hm = take(4 * (size_t)bound), o_hg = take(4 * (size_t)bound), o_he = take(4 * (size_t)bound);
  const size_t o_acc = take(sizeof(AdjCounts) * (size_t)n_sel);
  const size_t o_slots = take(sizeof(SlotCounts) * (size_t)std::max<int64_t>(total_slots, 1));
  const size_t o_words = yx ? take(sizeof(uint32_t) * (size_t)n_trials) : 0;
  char* scratch = nullptr;
  ARA_TRY(dmalloc_async((void**)&scratch, off, s));
  uint8_t* reg_all = (uint8_t*)(scratch + o_reg);
  uint32_t* bits = (uint32_t*)(scratch + o_bits);
  uint32_t* ptr = (uint32_t*)(scratch + o_ptr);
  uint64_t* rows = (uint64_t*)(scratch + o_rows);
  uint8_t* ent = (uint8_t*)(scratch + o_ent);
  uint8_t* cls = (uint8_t*)(scratch + o_cls);
  uint32_t* hm = (uint32_t*)(scratch + o_hm);
  uint32_t* hg = (uint32_t*)(scratch + o_hg);
  uint32_t* he = (uint32_t*)(scratch + o_he);
  AdjCounts* acc = (AdjCounts*)(scratch + o_acc);
  SlotCounts* slots = (SlotCounts*)(scratch + o_slots);
  const uint32_t cap = (uint32_t)bound;
  ara_status st = ARA_OK;
  // 1. occurrence regimes of every catalogue event for every slot, and the bitmaps of regime != 0
  FoldOutHost fo;
  fo.bits = bits;
  fo.regime = reg_all;
  fo.bits_stride = bmw;
  fo.regime_stride = C;
  fo.by_slot = 1;
  fo.bits_from_regime = 1;
  st = launch_fold_to(pf, n_sel, sel.data(), fo, s);
  if (st == ARA_OK && cudaMemsetAsync(scratch + o_hm, 0, off - o_hm, s) != cudaSuccess) st = ARA_ECUDA;
  const int n_rec_launches = (int)((total_slots + ADJ_MAX_SLOTS - 1) / ADJ_MAX_SLOTS);
  const int n_qgroups = (n_sel + ADJX_LAYERS - 1) / ADJX_LAYERS;
  const int64_t n_blocks_used =
      yx ? (first_trial + n_trials - 1) / yx->block - first_trial / yx->block + 1 : 0;
  const int n_hist_launches = yx ? n_qgroups * (int)(1 + n_blocks_used) : 1;
  if (st == ARA_OK && yx &&
      cudaFuncSetAttribute((const void*)k_adjx_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           ADJX_SMEM) != cudaSuccess)
    st = ARA_ECUDA;
  if (st == ARA_OK) {
    LaunchScope ls(ARA_K_ADJOINT, s, 6 + n_hist_launches + n_rec_launches);
    // 2. event-major rows of the slots with a non-zero occurrence regime
    st = launch_event_scan(bits, bmw, n_sel, C, ptr, (uint32_t*)(scratch + o_bsum),
                           (uint32_t*)(scratch + o_tot), s);
    if (st == ARA_OK) {
      k_adjb_fill<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(n_sel, bits, bmw, C, ptr, cap, ent,
                                                             rows, pf.d_err);
      // 3. the class of every (trial, slot) and the trial counts
      const unsigned cb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_trials + 255) / 256, 64));
      k_adjb_class<<<dim3(cb, (unsigned)n_sel), 256, 0, s>>>(n_trials, n_sel, d_regimes, d_ylt,
                                                             sr.thr_key, sr.thr_stride, cls, acc);
      // 4. the histograms: one pass over the trials interior for any slot, or over the
      // event-major index
      if (yx) {
        uint32_t* words = (uint32_t*)(scratch + o_words);
        AdjxHistParams xp{};
        xp.ent16 = yx->d_ent;
        xp.groups = yx->groups;
        xp.catalogue = C;
        xp.words = words;
        xp.cls = cls;
        xp.n_sel = n_sel;
        xp.rows = rows;
        xp.ent = ent;
        xp.cap = cap;
        xp.h_mean = hm;
        xp.h_gt = hg;
        xp.h_eq = he;
        for (int32_t q0 = 0; q0 < n_sel; q0 += ADJX_LAYERS) {
          const int32_t nq = std::min(ADJX_LAYERS, n_sel - q0);
          k_adjx_words<<<(unsigned)std::min<int64_t>((n_trials + 255) / 256, 8 * pf.n_sms), 256, 0, s>>>(
              n_trials, n_sel, q0, nq, cls, words);
          xp.q0 = q0;
          xp.nq = nq;
          const int64_t h_lo = first_trial / yx->block, h_hi = (first_trial + n_trials - 1) / yx->block;
          for (int64_t h = h_lo; h <= h_hi; ++h) {
            xp.base = yx->d_base + (int64_t)h * yx->groups;
            xp.len = yx->d_len + (int64_t)h * yx->groups;
            xp.t0 = h * yx->block - first_trial;
            xp.nb = std::min<int64_t>(yx->block, yx->n_trials - h * yx->block);
            xp.n_words = n_trials;
            k_adjx_hist<<<(unsigned)pf.n_sms, 1024, ADJX_SMEM, s>>>(xp);
          }
        }
      }
      AdjbHistParams hp{};
      hp.n_trials = n_trials;
      hp.offsets = d_offsets;
      hp.n_events = n_events;
      hp.ids = d_ids ? d_ids : reinterpret_cast<const int32_t*>(d_offsets);
      hp.catalogue = C;
      hp.n_sel = n_sel;
      hp.cap = cap;
      hp.cls = cls;
      hp.rows = rows;
      hp.ent = ent;
      hp.h_mean = hm;
      hp.h_gt = hg;
      hp.h_eq = he;
      hp.err = pf.d_err;
      if (!yx) k_adjb_hist<<<(unsigned)(pf.n_sms * 2), ADJB_WARPS * 32, 0, s>>>(hp);
      // 5. per-slot sums of the histograms by occurrence regime
      k_adjb_events<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, 4 * pf.n_sms)),
                      256, (size_t)6 * n_sel * sizeof(unsigned long long), s>>>(C, n_sel, cap, rows, ent,
                                                                                 reg_all, hm, hg, he, acc);
      // 6. record gradients and ELT-slot counts (up to ADJ_MAX_SLOTS slots per launch), then the
      // final combination of every layer
      AdjbRecParams q{};
      q.rec_off = pf.d_rec_off;
      q.rec_ids = pf.d_rec_ids;
      q.loss32 = pf.d_rec_loss32;
      q.loss64 = pf.d_rec_loss;
      q.rec_orig = pf.d_rec_orig;
      q.elt_ret = pf.d_elt_ret;
      q.elt_lim = pf.d_elt_lim;
      q.reg_all = reg_all;
      q.C = C;
      q.rows = rows;
      q.ent = ent;
      q.hm = hm;
      q.hg = hg;
      q.he = he;
      q.cap = cap;
      q.sel_gt = sr.gt;
      q.sel_eq = sr.eq;
      q.n_trials = n_trials;
      q.m = m;
      q.grad_loss_mean = d_grad_loss;
      q.grad_loss_tvar = d_grad_loss + total_loss;
      q.slots = slots;
      AdjbFinishParams fp{};
      fp.acc = acc;
      fp.slots = slots;
      fp.sel_gt = sr.gt;
      fp.sel_eq = sr.eq;
      fp.n = n_trials;
      fp.m = m;
      fp.total_slots = total_slots;
      fp.n_sel = n_sel;
      fp.grad_layer = d_grad_layer;
      fp.grad_elt = d_grad_elt;
      int32_t g = 0, in_launch = 0;
      int64_t b = 0;
      auto flush = [&]() {
        if (in_launch > 0) k_adjb_records<<<dim3(16, (unsigned)in_launch), 256, 0, s>>>(q);
        q.slot0 = g;
        in_launch = 0;
      };
      q.slot0 = 0;
      for (int32_t i = 0; i < n_sel; ++i) {
        const LayerConst& lc = pf.layers[sel[i]];
        fp.slot_off[i] = g + in_launch;
        for (int k = lc.elt_begin; k < lc.elt_end; ++k) {
          const int j = pf.layer_elts[k];
          q.elt[in_launch] = j;
          q.base[in_launch] = b;
          q.layer[in_launch] = (uint8_t)i;
          b += pf.rec_off[j + 1] - pf.rec_off[j];
          if (++in_launch == ADJ_MAX_SLOTS) {
            g += in_launch;
            flush();
          }
        }
      }
      fp.slot_off[n_sel] = g + in_launch;
      g += in_launch;
      flush();
      k_adjb_finish<<<(unsigned)n_sel, 256, 0, s>>>(fp);
      if (cudaGetLastError() != cudaSuccess) st = ARA_ECUDA;
    }
  }
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace ara

using namespace ara;

// ara_adjoint over the trial-major YET (yx null) or over its event-major index (yx set: the
// trials [first_trial, first_trial + n_trials) of the indexed YET; the YET pointers are unused).
static ara_status adjoint_common(ara_portfolio* pf_, const YetIndex* yx, int64_t first_trial,
                                 int64_t n_trials, const int64_t* d_offsets, int64_t n_events,
                                 const int32_t* d_ids,
                                 int32_t n_sel_in, const int32_t* layer_sel, const double* d_ylt,
                                 const uint8_t* d_regimes, double tvar_level, double* d_grad_elt,
                                 double* d_grad_layer, double* d_grad_loss, int32_t* h_ties,
                                 void* stream) {
  Portfolio* pf = static_cast<Portfolio*>(pf_);
  if (!pf || n_trials < 1 || n_events < 0 || !d_ylt || !d_regimes) return ARA_EINVAL;
  if (!yx && (!d_offsets || (n_events > 0 && !d_ids))) return ARA_EINVAL;
  if (!d_grad_elt || !d_grad_layer || !d_grad_loss) return ARA_EINVAL;
  std::vector<int32_t> sel;
  if (n_sel_in == 0 && layer_sel == nullptr) {
    for (int32_t l = 0; l < pf->n_layers; ++l) sel.push_back(l);
  } else {
    if (n_sel_in < 0 || !layer_sel) return ARA_EINVAL;
    for (int32_t i = 0; i < n_sel_in; ++i) {
      if (layer_sel[i] < 0 || layer_sel[i] >= pf->n_layers) return ARA_EINVAL;
      sel.push_back(layer_sel[i]);
    }
  }
  const int32_t n_sel = (int32_t)sel.size();
  if (n_sel == 0) return ARA_OK;
  if (((uintptr_t)d_ids & 3) || ((uintptr_t)d_ylt & 7)) return ARA_EINVAL;
  const int64_t m = tail_count_snap(n_trials, tvar_level);
  if (m < 1) return ARA_EINVAL;
  for (int32_t i = 0; i < n_sel; ++i)
    if (pf->layer_off[sel[i] + 1] - pf->layer_off[sel[i]] > ADJ_MAX_SLOTS) return ARA_ERANGE;
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;

  // TVaR threshold, #{y > v} and #{y == v} of every selected layer
  SelectResult sr;
  ara_status st = select_one_rank(d_ylt, n_trials, n_sel, m, pf->n_sms, s, &sr, pf->d_err);
  if (st != ARA_OK) return st;

  int64_t total_slots = 0, total_loss = 0;
  for (int32_t i = 0; i < n_sel; ++i) {
    const int l = sel[i];
    for (int k = pf->layer_off[l]; k < pf->layer_off[l + 1]; ++k) {
      const int j = pf->layer_elts[k];
      total_loss += pf->rec_off[j + 1] - pf->rec_off[j];
      ++total_slots;
    }
  }
  // Several layers: one histogram pass for all of them (unless a test asks for the per-layer
  // passes, or the layers' table exceeds 32-bit entry indices).  With an index, always that
  // path: the per-layer passes read the trial-major YET.
  if (yx || (n_sel >= 2 && !adjoint_per_layer())) {
    st = adjoint_multi(*pf, sel, n_trials, d_offsets, n_events, d_ids, yx, first_trial, d_ylt, d_regimes, m, sr,
                       d_grad_elt, d_grad_layer, d_grad_loss, total_slots, total_loss, s);
    if (st != ARA_ERANGE || yx) {
      std::vector<unsigned long long> gt(n_sel), eq(n_sel);
      if (st == ARA_OK && h_ties) {
        if (cudaMemcpyAsync(gt.data(), sr.gt, 8 * n_sel, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(eq.data(), sr.eq, 8 * n_sel, cudaMemcpyDeviceToHost, s) != cudaSuccess)
          st = ARA_ECUDA;
      }
      free_select_result(sr, s);
      if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
      if (st == ARA_OK && h_ties)
        for (int32_t i = 0; i < n_sel; ++i) h_ties[i] = (int64_t)(gt[i] + eq[i]) > m ? 1 : 0;
      if (st != ARA_OK) return st;
      return ara_check(pf_, stream);
    }
    st = ARA_OK;
  }

  // scratch
  const int64_t C = pf->catalogue;
  const int64_t bmw = pf->bm_words;
  size_t off = 0;
  auto take = [&](size_t n) { size_t o = (off + 255) / 256 * 256; off = o + n; return o; };
  const size_t o_reg = take((size_t)C), o_bits = take(4 * (size_t)bmw);
  const size_t o_hm = take(4 * (size_t)C), o_hg = take(4 * (size_t)C), o_he = take(4 * (size_t)C);
  const size_t o_acc = take(sizeof(AdjCounts)), o_slots = take(sizeof(SlotCounts) * ADJ_MAX_SLOTS);
  char* scratch = nullptr;
  cudaError_t ce = dmalloc_async((void**)&scratch, off, s);
  if (ce != cudaSuccess) {
    free_select_result(sr, s);
    return ce == cudaErrorMemoryAllocation ? ARA_ENOMEM : ARA_ECUDA;
  }
  uint8_t* reg = (uint8_t*)(scratch + o_reg);
  uint32_t* bits = (uint32_t*)(scratch + o_bits);
  uint32_t* hm = (uint32_t*)(scratch + o_hm);
  uint32_t* hg = (uint32_t*)(scratch + o_hg);
  uint32_t* he = (uint32_t*)(scratch + o_he);
  AdjCounts* acc = (AdjCounts*)(scratch + o_acc);
  SlotCounts* slots = (SlotCounts*)(scratch + o_slots);

  // shared-memory bitmap for the histogram pass
  int shift = 0;
  auto cw = [&](int sh) { return ((C + 31) / 32 + ((int64_t)1 << sh) - 1) >> sh; };   // interleaved words
  const int64_t bm_budget = std::min<int64_t>(pf->max_smem_block, 200 * 1024);
  while (cw(shift) * 4 > bm_budget) ++shift;
  const int smem = (int)(cw(shift) * 4);
  ara_status out_st = ARA_OK;
  if (cudaFuncSetAttribute((const void*)k_adj_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           std::max(smem, 48 * 1024)) != cudaSuccess)
    out_st = ARA_ECUDA;

  int64_t elt_slot0 = 0, loss_base0 = 0;
  for (int32_t i = 0; i < n_sel && out_st == ARA_OK; ++i) {
    const int l = sel[i];
    const LayerConst& lc = pf->layers[l];
    const int n_le = lc.elt_end - lc.elt_begin;
    // 1. occurrence regimes of every catalogue event and the bitmap of regime != 0
    FoldOutHost fo;
    fo.bits = bits;
    fo.regime = reg;
    fo.bits_stride = bmw;
    fo.regime_stride = C;
    fo.by_slot = 1;
    fo.bits_from_regime = 1;
    if ((out_st = launch_fold_to(*pf, 1, &l, fo, s)) != ARA_OK) break;
    // 2. histograms and counters
    if (cudaMemsetAsync(scratch + o_hm, 0, off - o_hm, s) != cudaSuccess) { out_st = ARA_ECUDA; break; }
    AdjHistParams hp{};
    hp.n_trials = n_trials;
    hp.offsets = d_offsets;
    hp.n_events = n_events;
    hp.ids = d_ids ? d_ids : reinterpret_cast<const int32_t*>(d_offsets);
    hp.catalogue = C;
    hp.regimes = d_regimes + (int64_t)i * n_trials;
    hp.ylt = d_ylt + (int64_t)i * n_trials;
    hp.thr_key = sr.thr_key + (int64_t)i * sr.thr_stride;
    hp.bits = bits;
    hp.bm_words = bmw;
    hp.smem_words = cw(shift);
    hp.shift = shift;
    hp.h_mean = hm;
    hp.h_gt = hg;
    hp.h_eq = he;
    hp.err = pf->d_err;
    hp.acc = acc;
    {
      // the histogram pass (which also counts the trials), the event and record reductions,
      // and the final combination
      LaunchScope ls(ARA_K_ADJOINT, s, n_le > 0 ? 4 : 3);
      // the threshold key is read on the device from the selection result
      k_adj_hist<<<pf->n_sms, 1024, smem, s>>>(hp);
      k_adj_events<<<std::max(1, (int)std::min<int64_t>((C + 2047) / 2048, 4 * pf->n_sms)), 256, 0, s>>>(
          C, reg, hm, hg, he, acc);
      AdjRecParams rp{};
      rp.rec_off = pf->d_rec_off;
      rp.rec_ids = pf->d_rec_ids;
      rp.loss32 = pf->d_rec_loss32;
      rp.loss64 = pf->d_rec_loss;
      rp.rec_orig = pf->d_rec_orig;
      rp.elt_ret = pf->d_elt_ret;
      rp.elt_lim = pf->d_elt_lim;
      rp.reg = reg;
      rp.hm = hm;
      rp.hg = hg;
      rp.he = he;
      rp.sel_gt = sr.gt + i;
      rp.sel_eq = sr.eq + i;
      rp.n_trials = n_trials;
      rp.m = m;
      rp.grad_loss_mean = d_grad_loss;
      rp.grad_loss_tvar = d_grad_loss + total_loss;
      rp.slots = slots;
      rp.n_slots = n_le;
      int64_t b = loss_base0;
      for (int k = 0; k < n_le; ++k) {
        const int j = pf->layer_elts[lc.elt_begin + k];
        rp.elt[k] = j;
        rp.base[k] = b;
        b += pf->rec_off[j + 1] - pf->rec_off[j];
      }
      if (n_le > 0) {
        dim3 grid(16, n_le);
        k_adj_records<<<grid, 256, 0, s>>>(rp);
      }
      k_adj_finish<<<1, 256, 0, s>>>(acc, slots, n_le, sr.gt + i, sr.eq + i, n_trials, m,
                                     d_grad_layer + (int64_t)i * 4,
                                     d_grad_layer + (int64_t)(n_sel + i) * 4,
                                     d_grad_elt + 2 * elt_slot0,
                                     d_grad_elt + 2 * (total_slots + elt_slot0));
      if (cudaGetLastError() != cudaSuccess) { out_st = ARA_ECUDA; break; }
      loss_base0 = b;
      elt_slot0 += n_le;
    }
  }
  std::vector<unsigned long long> gt(n_sel), eq(n_sel);
  if (out_st == ARA_OK && h_ties) {
    if (cudaMemcpyAsync(gt.data(), sr.gt, 8 * n_sel, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(eq.data(), sr.eq, 8 * n_sel, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      out_st = ARA_ECUDA;
  }
  cudaFreeAsync(scratch, s);
  free_select_result(sr, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && out_st == ARA_OK) out_st = ARA_ECUDA;
  if (out_st == ARA_OK && h_ties)
    for (int32_t i = 0; i < n_sel; ++i) h_ties[i] = (int64_t)(gt[i] + eq[i]) > m ? 1 : 0;
  if (out_st != ARA_OK) return out_st;
  return ara_check(pf_, stream);
}

extern "C" ara_status ara_adjoint(ara_portfolio* pf, int64_t n_trials, const int64_t* d_offsets,
                                  int64_t n_events, const int32_t* d_ids, int32_t n_sel_in,
                                  const int32_t* layer_sel, const double* d_ylt,
                                  const uint8_t* d_regimes, double tvar_level, double* d_grad_elt,
                                  double* d_grad_layer, double* d_grad_loss, int32_t* h_ties,
                                  void* stream) {
  return adjoint_common(pf, nullptr, 0, n_trials, d_offsets, n_events, d_ids, n_sel_in, layer_sel,
                        d_ylt, d_regimes, tvar_level, d_grad_elt, d_grad_layer, d_grad_loss,
                        h_ties, stream);
}

extern "C" ara_status ara_adjoint_indexed(ara_portfolio* pf, const ara_yet_index* yx,
                                          int64_t first_trial, int64_t n_trials,
                                          int32_t n_sel_in, const int32_t* layer_sel,
                                          const double* d_ylt, const uint8_t* d_regimes,
                                          double tvar_level, double* d_grad_elt,
                                          double* d_grad_layer, double* d_grad_loss,
                                          int32_t* h_ties, void* stream) {
  if (!pf || !yx) return ARA_EINVAL;
  if (yx->catalogue != pf->catalogue || yx->device != pf->device || !yx->d_ent) return ARA_EINVAL;
  if (n_trials == 0 && first_trial == 0) n_trials = yx->n_trials;
  if (first_trial < 0 || n_trials < 1 || first_trial > yx->n_trials - n_trials) return ARA_EINVAL;
  return adjoint_common(pf, yx, first_trial, n_trials, nullptr, yx->n_events, nullptr, n_sel_in, layer_sel,
                        d_ylt, d_regimes, tvar_level, d_grad_elt, d_grad_layer, d_grad_loss,
                        h_ties, stream);
}

extern "C" ara_status ara_adjoint_accumulate(ara_portfolio* pf_, int64_t n_trials,
                                             const int64_t* d_offsets, int64_t n_events,
                                             const int32_t* d_ids, int32_t n_sel_in,
                                             const int32_t* layer_sel, const double* d_ylt,
                                             const uint8_t* d_regimes, double tvar_level,
                                             const double* h_weights, double* d_g_elt_ret,
                                             double* d_g_elt_lim, double* d_g_layer,
                                             double* d_g_loss, void* stream) {
  Portfolio* pf = static_cast<Portfolio*>(pf_);
  if (!pf || !h_weights || !d_g_elt_ret || !d_g_elt_lim || !d_g_layer || !d_g_loss) return ARA_EINVAL;
  std::vector<int32_t> sel;
  if (n_sel_in == 0 && layer_sel == nullptr) {
    for (int32_t l = 0; l < pf->n_layers; ++l) sel.push_back(l);
  } else {
    if (n_sel_in < 0 || !layer_sel) return ARA_EINVAL;
    for (int32_t i = 0; i < n_sel_in; ++i) {
      if (layer_sel[i] < 0 || layer_sel[i] >= pf->n_layers) return ARA_EINVAL;
      sel.push_back(layer_sel[i]);
    }
  }
  const int32_t n_sel = (int32_t)sel.size();
  if (n_sel == 0) return ARA_OK;
  int64_t K = 0, M = 0;
  for (int32_t i = 0; i < n_sel; ++i)
    for (int k = pf->layer_off[sel[i]]; k < pf->layer_off[sel[i] + 1]; ++k) {
      const int j = pf->layer_elts[k];
      M += pf->rec_off[j + 1] - pf->rec_off[j];
      ++K;
    }
  DeviceGuard g(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)(2 * 2 * std::max<int64_t>(K, 1) + 2 * 4 * n_sel +
                                                 2 * std::max<int64_t>(M, 1));
  double* buf = nullptr;
  ARA_TRY(dmalloc_async((void**)&buf, bytes, s));
  double* ge = buf;
  double* gl = ge + 2 * 2 * std::max<int64_t>(K, 1);
  double* gx = gl + 2 * 4 * n_sel;
  ara_status st = ara_adjoint(pf_, n_trials, d_offsets, n_events, d_ids, n_sel, sel.data(), d_ylt,
                              d_regimes, tvar_level, ge, gl, gx, nullptr, stream);
  int64_t slot0 = 0, base0 = 0;
  for (int32_t i = 0; i < n_sel && st == ARA_OK; ++i) {
    const int l = sel[i];
    const LayerConst& lc = pf->layers[l];
    AdjScatterParams sp{};
    sp.w0 = h_weights[2 * i];
    sp.w1 = h_weights[2 * i + 1];
    sp.layer = l;
    sp.n_slots = lc.elt_end - lc.elt_begin;
    sp.gl0 = gl + 4 * i;
    sp.gl1 = gl + 4 * (n_sel + i);
    sp.ge0 = ge + 2 * slot0;
    sp.ge1 = ge + 2 * (K + slot0);
    sp.gx0 = gx;
    sp.gx1 = gx + M;
    sp.rec_off = pf->d_rec_off;
    sp.rec_orig = pf->d_rec_orig;
    sp.g_elt_ret = d_g_elt_ret;
    sp.g_elt_lim = d_g_elt_lim;
    sp.g_layer = d_g_layer;
    sp.g_loss = d_g_loss;
    int64_t b = base0;
    for (int k = 0; k < sp.n_slots; ++k) {
      const int j = pf->layer_elts[lc.elt_begin + k];
      sp.elt[k] = j;
      sp.base[k] = b;
      b += pf->rec_off[j + 1] - pf->rec_off[j];
    }
    if (sp.n_slots > 0) {
      LaunchScope ls(ARA_K_ADJOINT, s);
      k_adj_scatter<<<dim3(8, sp.n_slots), 256, 0, s>>>(sp);
      if (cudaGetLastError() != cudaSuccess) st = ARA_ECUDA;
    }  // a layer without ELTs has S = 0 in every trial: all its gradients are 0
    slot0 += sp.n_slots;
    base0 = b;
  }
  cudaFreeAsync(buf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ARA_OK) st = ARA_ECUDA;
  return st;
}

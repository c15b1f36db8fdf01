// Internal declarations shared by the translation units of libara.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/ara.h"

namespace ara {

// ------------------------------------------------------------------------------------------
// Error plumbing
// ------------------------------------------------------------------------------------------
#define ARA_TRY(expr)                                              \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) {                                       \
      ::ara::note_cuda_error(_e, #expr, __FILE__, __LINE__);       \
      return _e == cudaErrorMemoryAllocation ? ARA_ENOMEM : ARA_ECUDA; \
    }                                                              \
  } while (0)

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Stream-ordered allocations of the library come from its own memory pool on each device, which
// keeps freed memory for reuse instead of returning it at every synchronisation (the default
// pool's behaviour, which made every synchronous call map its scratch again).  Free with
// cudaFreeAsync.  ara_release_memory() returns the idle part to the system.
cudaError_t dmalloc_async(void** ptr, size_t bytes, cudaStream_t s);
// Bytes the library's pool on `dev` holds without using them (reusable by the library).
int64_t pool_idle_bytes(int dev);

// Device-side data error bits (atomicOr into the portfolio's error word).
enum : uint32_t { DERR_EVENT_RANGE = 1u, DERR_OFFSETS = 2u, DERR_TIMEOUT = 4u };

// ------------------------------------------------------------------------------------------
// Launch accounting and per-class event timing
// ------------------------------------------------------------------------------------------
extern std::atomic<int64_t> g_launches;
void timing_begin(int kclass, cudaStream_t s);
void timing_end(int kclass, cudaStream_t s);
// switch event timing off (e.g. while a stream is captured into a graph); returns the old state
bool timing_suspend();
void timing_resume(bool was_on);
// add a host-timed interval (ms) to a timing class (when timing is enabled)
void timing_add_host(int kclass, double ms);

// RAII helper: events around every launch of a kernel class (when timing is enabled) and
// one count per launch.
struct LaunchScope {
  int kclass;
  cudaStream_t s;
  LaunchScope(int k, cudaStream_t st, int n_launches = 1) : kclass(k), s(st) {
    g_launches.fetch_add(n_launches);
    timing_begin(k, s);
  }
  ~LaunchScope() { timing_end(kclass, s); }
};

// ------------------------------------------------------------------------------------------
// Per-layer constants of the folded path
// ------------------------------------------------------------------------------------------
// Occurrence losses o(e) are kept as unsigned fixed point q(e) = round(o(e) * 2^frac_bits),
// q(e) < 2^55, and trial sums are exact 128-bit integer sums of q.  The aggregate terms are
// applied to the exact sum in the same fixed point; only the final year loss is converted to
// double.
struct LayerConst {
  double occ_ret, occ_lim, agg_ret, agg_lim;   // layer terms T (FP64)
  double scale;                                // 2^frac_bits
  double inv_scale;                            // 2^-frac_bits
  uint64_t agg_ret_lo, agg_ret_hi;             // round(AggR * scale) as u128 (saturated)
  uint64_t agg_lim_lo, agg_lim_hi;             // round(AggL * scale) as u128 (saturated)
  int32_t elt_begin, elt_end;                  // slice of layer_elt_ids
  int32_t frac_bits;
  int32_t pad;
};

// Catalogue events per tile of the fold kernel; the portfolio keeps, per ELT, the first record
// of every tile so that the fold reads each tile's record range instead of searching for it.
constexpr int FOLD_TILE = 2048;

struct Portfolio {
  bool borrowed_elts = false;       // a layer set: ELT tables belong to a resident pool
  cudaStream_t owner_stream = nullptr;  // layer sets: stream their buffers were allocated on
  int device = 0;
  int n_sms = 0;
  int max_smem_block = 0;           // opt-in shared memory per block (bytes)
  int64_t catalogue = 0;
  int32_t n_elts = 0, n_layers = 0, flags = 0;
  int64_t n_records = 0;
  // host copies
  std::vector<int64_t> rec_off;
  std::vector<double> elt_ret, elt_lim, elt_max_loss;
  std::vector<int32_t> layer_off, layer_elts;
  std::vector<LayerConst> layers;
  // device tables
  int64_t* d_rec_off = nullptr;     // [n_elts + 1]
  int32_t* d_rec_ids = nullptr;     // [n_records], sorted by event ID within each ELT
  int32_t* d_rec_orig = nullptr;    // [n_records]: position of each sorted record in the order given
  double* d_rec_loss = nullptr;     // [n_records] (FP64 storage) or nullptr
  float* d_rec_loss32 = nullptr;    // [n_records] (FP32 storage) or nullptr
  double* d_elt_ret = nullptr;      // [n_elts]
  double* d_elt_lim = nullptr;      // [n_elts]
  int64_t n_tiles = 0;              // fold tiles: ceil(catalogue / FOLD_TILE)
  int64_t* d_tile_rec = nullptr;    // [n_elts][n_tiles + 1]: first record of each ELT per tile
  int32_t* d_layer_elts = nullptr;  // [layer_off[n_layers]]
  LayerConst* d_layers = nullptr;   // [n_layers]
  void* d_dense = nullptr;          // [n_elts][catalogue] float or double (ARA_DENSE_TABLES)
  // per-layer fold workspace
  uint64_t* d_q = nullptr;          // [n_layers][catalogue]: q(e) (or o(e) bits for F64_SUM)
  uint32_t* d_bits = nullptr;       // [n_layers][bm_words]: bit e set iff q(e) != 0
  int64_t bm_words = 0;             // words per layer (padded to a multiple of 4)
  uint32_t* d_cbits = nullptr;      // [n_layers][cbits_stride]: coarse bitmap (1 bit / 2^k events)
  int64_t cbits_stride = 0;
  // a second fold workspace (slot 1 of ara_prepare_ylt), allocated on first use, so that the
  // fold of one run can proceed while another run streams from the first
  uint64_t* d_q_alt = nullptr;
  uint32_t* d_bits_alt = nullptr;
  uint32_t* d_cbits_alt = nullptr;
  uint32_t* d_err = nullptr;        // device error word
  // host-input pipeline resources (grown on demand)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
  int32_t* d_stage_ids[2] = {nullptr, nullptr};
  int64_t* d_stage_off[2] = {nullptr, nullptr};
  int64_t stage_events = 0, stage_trials = 0;
  double* d_ylt_full = nullptr;     // [n_sel][n_trials] YLT of the host pipeline
  int64_t ylt_full_elems = 0;
  // results of the host pipeline: metrics, selection status and the device error word, in one
  // device block and its pinned host copy (one copy and one synchronisation per call)
  double* d_res = nullptr;
  double* h_res = nullptr;
  int64_t res_elems = 0;
  void* d_sel_scratch = nullptr;    // the host pipeline's selection scratch (grown on demand)
  size_t sel_scratch_bytes = 0;
};

// ------------------------------------------------------------------------------------------
// Kernel entry points (host-side launchers), implemented in ara_ylt.cu / ara_select.cu
// ------------------------------------------------------------------------------------------
struct YltArgs {
  int64_t n_trials;
  const int64_t* offsets;   // [n_trials + 1]
  int64_t id_base;          // subtracted from every offset (host pipeline chunks)
  int64_t n_events;         // valid range of (offset - id_base)
  const int32_t* ids;
  int32_t n_sel;
  const int32_t* sel;       // host [n_sel] layer indices
  double* ylt;              // row i (layer sel[i]) at ylt + i * row_stride
  uint8_t* regimes;         // row i at regimes + i * row_stride, or nullptr
  int64_t row_stride;       // elements between the rows of consecutive selected layers
  int32_t flags;
  int32_t slot = 0;         // fold workspace slot (0 or 1)
  bool prepared = false;    // fold and coarse bitmap already in the slot (ara_prepare_ylt)
};

// The fold workspace of a slot: q tables, exact and coarse hit bitmaps of every layer.
struct FoldSlot {
  uint64_t* q;
  uint32_t* bits;
  uint32_t* cbits;
};
inline FoldSlot fold_slot(const struct Portfolio& pf, int slot) {
  return slot ? FoldSlot{pf.d_q_alt, pf.d_bits_alt, pf.d_cbits_alt} : FoldSlot{pf.d_q, pf.d_bits, pf.d_cbits};
}

ara_status launch_fold(Portfolio& pf, int32_t n_sel, const int32_t* sel_host, int32_t flags,
                       cudaStream_t s, int slot = 0);
// The coarse hit bitmaps the default stream kernel reads (when the exact bitmap does not fit in
// shared memory), built from the slot's exact bitmaps.
ara_status launch_coarsen(Portfolio& pf, int32_t n_sel, const int32_t* sel_host, int32_t flags,
                          cudaStream_t s, int slot);
// Fold into caller-chosen outputs (see k_fold): used by the adjoint for occurrence regimes and
// by the batched plan for every selected layer at once.
struct FoldOutHost {
  uint64_t* q = nullptr;
  uint32_t* bits = nullptr;
  uint8_t* regime = nullptr;
  int64_t q_stride = 0, bits_stride = 0, regime_stride = 0;
  int by_slot = 0, f64_table = 0, bits_from_regime = 0;
  int nonzero_only = 0;   // store only the non-zero entries of q (readers consult the bitmap)
};
// counted = false: the caller counts and times the launch within its own scope.
ara_status launch_fold_to(Portfolio& pf, int32_t n_sel, const int32_t* sel_host,
                          const FoldOutHost& o, cudaStream_t s, bool counted = true);
ara_status launch_ylt(Portfolio& pf, const YltArgs& a, cudaStream_t s);
ara_status run_batched_async(Portfolio& pf, const YltArgs& a, cudaStream_t s);
// One pass of the batched stream for several requests at once (serving): request r owns the
// portfolio's layers (= slots) [slot_first[r], slot_first[r + 1]) and the trials [t0[r], t1[r])
// of a union range of trials; every trial of the union is read once and walks only the table
// entries of the requests that cover it.  Each request's YLT rows go to its own buffer
// ylt[r] ([layers of r][t1[r] - t0[r]], row-major), bitwise equal to a run of that request alone.
constexpr int BT_MAX_REQ = 4;
struct GroupArgs {
  int64_t n_trials = 0;                 // trials of the union range
  const int64_t* offsets = nullptr;     // [n_trials + 1], first trial of the union range
  int64_t n_events = 0;
  const int32_t* ids = nullptr;
  int32_t n_req = 0;                    // 1 .. BT_MAX_REQ
  int32_t slot_first[BT_MAX_REQ + 1] = {0, 0, 0, 0, 0};
  int64_t t0[BT_MAX_REQ] = {0, 0, 0, 0}, t1[BT_MAX_REQ] = {0, 0, 0, 0};   // relative to the union
  double* ylt[BT_MAX_REQ] = {nullptr, nullptr, nullptr, nullptr};
  uint8_t* reg[BT_MAX_REQ] = {nullptr, nullptr, nullptr, nullptr};
};
ara_status run_batched_group_async(Portfolio& pf, const GroupArgs& g, cudaStream_t s);
// Exclusive scan of the per-event count of set bits over n_sel bitmaps (the rows of an
// event-major table): ptr [n + 1], block_sums [ceil(n / 1024)], total [1].
ara_status launch_event_scan(const uint32_t* bits, int64_t bits_stride, int32_t n_sel, int64_t n,
                             uint32_t* ptr, uint32_t* block_sums, uint32_t* total, cudaStream_t s);
ara_status build_dense(Portfolio& pf, cudaStream_t s);
// Compiled shapes (warps per block, ring stages) of the bulk-staged YET stream kernel.
int32_t n_bulk_shapes();
void set_bulk_shape(int32_t i);
void bulk_shape(int32_t i, int32_t* warps, int32_t* stages);
void set_wait_limit_ns(uint64_t ns);
void set_debug_extra_tx(uint32_t bytes);
// Bound of every device-side wait (bulk copies, grid barriers), in nanoseconds.
uint64_t wait_limit_ns();
// Test hook: the selection's blocks skip their grid-barrier arrivals (every wait runs out).
void set_debug_skip_arrival(int32_t on);
int32_t debug_skip_arrival();
// Test hook: the adjoint of several layers takes one histogram pass per layer.
void set_adjoint_per_layer(int32_t on);
int32_t adjoint_per_layer();
// Host check of risk-metric arguments (ranks within [1, n]); ARA_OK or ARA_EINVAL.
ara_status validate_metrics(int64_t n, int32_t n_rp, const double* rps, int32_t n_tvar,
                            const double* levels);
// m = ceil(N (1 - p)) with the library's integer snapping; -1 when p is outside [0, 1).
int64_t tail_count_snap(int64_t n, double p);
// The m-th largest value of each of n_layers device rows: its order key (device, stride
// thr_stride 64-bit words), #{y > v} and #{y == v} (device, one per layer).  Scratch from the
// stream-ordered allocator; release with free_select_result.
struct SelectResult {
  void* scratch = nullptr;
  const uint64_t* thr_key = nullptr;
  int64_t thr_stride = 0;
  const unsigned long long* gt = nullptr;
  const unsigned long long* eq = nullptr;
};
ara_status select_one_rank(const double* d_ylt, int64_t n, int32_t n_layers, int64_t m, int n_sms,
                           cudaStream_t s, SelectResult* out, uint32_t* err);
void free_select_result(SelectResult& r, cudaStream_t s);
// The stream-ordered risk metrics with caller-owned scratch: ARA_ERANGE (and *need) when the
// scratch is too small.
ara_status risk_metrics_queue(const double* d_ylt, int64_t n_trials, int32_t n_layers, int32_t n_rp,
                              const double* rps, int32_t n_tvar, const double* levels,
                              double* d_pml, double* d_tvar, double* d_mean, uint32_t* d_status,
                              void* scratch, size_t scratch_bytes, size_t* need, cudaStream_t s);
// PML / TVaR of n_layers device YLT rows into host arrays (synchronises s); scratch from the
// stream-ordered allocator.
ara_status risk_metrics_device(const double* d_ylt, int64_t n, int32_t n_layers, int32_t n_rp,
                               const double* rps, int32_t n_tvar, const double* levels,
                               double* h_pml, double* h_tvar, double* h_mean, cudaStream_t s);

// Event-major index of a device YET (ara_yet_index_create).  The trials are cut into blocks of
// `block` trials and the catalogue into groups of 32 events.  For block h and group g, the
// trials of the block in which each event of the group occurs are stored as 16-bit offsets
// within the block, in runs of 8 per event interleaved 32 wide (one 16-byte load per lane gives
// 8 entries of its event): entry k of event 32 g + l sits at
// ent[base[h][g] + 256 (k / 8) + 8 l + k % 8] for k < len[h][g], a multiple of 8; lists shorter
// than len[h][g] are padded with YX_PAD, an offset past every block's last trial.  An event
// occurring several times in a trial appears that many times.  Within a list the order is
// unspecified.
constexpr uint32_t YX_PAD = 0xC0C0u;           // the padding offset: bytes 0xC0 0xC0
constexpr int64_t YX_MAX_BLOCK = YX_PAD;       // trials per block at most (offsets < YX_PAD)
struct YetIndex {
  int device = 0;
  int64_t n_trials = 0, n_events = 0, catalogue = 0;
  int64_t block = 0;                 // trials per block
  int32_t n_blocks = 0;
  int64_t groups = 0;                // ceil(catalogue / 32)
  int64_t n_ent = 0;                 // entries, padding included
  uint16_t* d_ent = nullptr;         // [n_ent]
  int64_t* d_base = nullptr;         // [n_blocks][groups]
  uint32_t* d_len = nullptr;         // [n_blocks][groups] list length, a multiple of 8
};

}  // namespace ara

// The opaque handle of the C ABI is the portfolio itself.
struct ara_portfolio : public ara::Portfolio {};
struct ara_yet_index : public ara::YetIndex {};

namespace ara {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace ara

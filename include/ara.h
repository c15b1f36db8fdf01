/*
 * ara.h -- C ABI of the GB300 (sm_103a) Aggregate Risk Analysis library (libara.so).
 *
 * Aggregate Risk Analysis (paper Section IV) streams every trial of a pre-simulated Year
 * Event Table (YET, Eq. 1) through the Event Loss Tables (ELTs, Eq. 2) of a layer (Eq. 3),
 * applies financial terms and writes one Year Loss Table (YLT) entry per trial; PML and
 * TVaR are taken from the YLT (Section IV-A).
 *
 * Financial terms.  Every term pair (retention R, limit L) is applied as the clamp
 *     C(x; R, L) = min(max(x - R, 0), L)
 * (Section IV-B prints this formula with the 0 of max() lost).  Per layer:
 *     a_j(e) = C(x_j(e); R_j, L_j)          x_j(e): loss of event e in ELT j, 0 if absent
 *     o(e)   = C(sum_j a_j(e); OccR, OccL)  occurrence terms, one occurrence at a time
 *     S_t    = sum over the events e of trial t of o(e)
 *     y_t    = C(S_t; AggR, AggL)           aggregate terms -> YLT entry
 * (Algorithm 3 and the two paragraphs after it).
 *
 * Conventions
 *   - Every call returns an ara_status (0 = ARA_OK, negative = error) unless noted.
 *   - "d_" pointers are device memory of the portfolio's device, "h_" pointers host memory.
 *     The library never frees or retains caller memory beyond the call (asynchronous calls
 *     read it until the stream reaches them).
 *   - Streams are cudaStream_t handles passed as void*; NULL is the legacy default stream.
 *   - Argument errors are detected on the host before anything is launched (ARA_EINVAL).
 *     Data errors that only the device can see (an event ID outside the catalogue, trial
 *     offsets that decrease or leave [0, n_events]) are recorded by the kernels, the offending
 *     trial counts as empty, and the next ara_check() on the portfolio returns ARA_EDATA.
 *   - The library is thread-compatible: one portfolio must not run on two streams at once
 *     (its fold workspace is shared); distinct portfolios are independent.
 *   - Scratch that calls allocate in stream order (selections, adjoint, batched runs, layer
 *     sets, serving) comes from the library's own memory pool on each device, which keeps freed
 *     memory for the next call instead of returning it at every synchronisation;
 *     ara_release_memory() returns the idle part to the system.
 */
#ifndef ARA_H
#define ARA_H

#include <stdint.h>

#if defined(__GNUC__)
#define ARA_API __attribute__((visibility("default")))
#else
#define ARA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ara_status;
#define ARA_OK        0
#define ARA_EINVAL   (-1)   /* invalid argument or input table */
#define ARA_ENOMEM   (-2)   /* device or host allocation failed */
#define ARA_ECUDA    (-3)   /* a CUDA runtime call failed (no device, launch failure, ...) */
#define ARA_ETIMEOUT (-4)   /* a bounded device-side wait gave up */
#define ARA_EBUSY    (-5)   /* resource in use */
#define ARA_EDATA    (-6)   /* device-side data check failed in an earlier asynchronous run */
#define ARA_ERANGE   (-7)   /* request exceeds a fixed capacity of the library */

typedef struct ara_portfolio ara_portfolio;

/* ---------------------------------------------------------------------------------------
 * Portfolio: ELTs (Eq. 2) with their terms I = (R_j, L_j), and layers (Eq. 3) with their
 * terms T = (OccR, OccL, AggR, AggL)  [Section IV-A, Section IV-B].
 * --------------------------------------------------------------------------------------- */

/* flags of ara_create_portfolio */
#define ARA_LOSSES_F32   1  /* keep ELT losses in FP32 on the device (each loss must be exactly
                               representable in FP32, else ARA_EINVAL); default FP64 */
#define ARA_DENSE_TABLES 2  /* also build catalogue-indexed direct-access tables
                               [n_elts][catalogue] (Section IV-B), used by ARA_RUN_PER_ELT */

/*
 * Copy a portfolio to the current CUDA device.  Synchronous.
 *   catalogue_size           number of events in the global event catalogue; event IDs are
 *                            0 .. catalogue_size-1  (1 <= catalogue_size <= 2^31 - 1)
 *   n_elts                   number of ELTs (>= 0)
 *   elt_record_offsets       host [n_elts + 1], non-decreasing, [0] = 0: ELT j owns records
 *                            elt_record_offsets[j] .. elt_record_offsets[j+1]-1
 *   record_event_ids         host [total records]: event IDs, unique within an ELT, any order
 *   record_losses            host [total records]: finite losses >= 0
 *   elt_ret, elt_lim         host [n_elts]: per-ELT retention (finite, >= 0) and limit (>= 0,
 *                            +INFINITY allowed)
 *   n_layers                 number of layers (>= 0)
 *   layer_elt_offsets        host [n_layers + 1], non-decreasing, [0] = 0
 *   layer_elt_ids            host [layer_elt_offsets[n_layers]]: ELTs of each layer, in order
 *   occ_ret, occ_lim,        host [n_layers]: occurrence and aggregate retentions (finite,
 *   agg_ret, agg_lim         >= 0) and limits (>= 0, +INFINITY allowed)
 *   flags                    ARA_LOSSES_F32 | ARA_DENSE_TABLES
 *   out                      receives the handle (owned by the library until destroyed)
 * Errors: ARA_EINVAL (any rule above broken; nothing allocated), ARA_ENOMEM, ARA_ECUDA.
 */
ARA_API ara_status ara_create_portfolio(int64_t catalogue_size, int32_t n_elts,
                                const int64_t* elt_record_offsets,
                                const int32_t* record_event_ids, const double* record_losses,
                                const double* elt_ret, const double* elt_lim, int32_t n_layers,
                                const int32_t* layer_elt_offsets, const int32_t* layer_elt_ids,
                                const double* occ_ret, const double* occ_lim,
                                const double* agg_ret, const double* agg_lim, int32_t flags,
                                ara_portfolio** out);

/* Release every device and host resource of the portfolio (synchronises its device; for a
 * layer set, only the stream it was created on). */
ARA_API void ara_destroy_portfolio(ara_portfolio* pf);

/*
 * A layer set: new layers (Eq. 3) over the ELTs of a resident portfolio `pool` (the ELTs and
 * their terms stay where they are; only the layers, their terms and their fold workspace,
 * n_layers x catalogue x ~8.3 bytes, are new).  Allocation and upload are asynchronous on
 * `stream` (stream-ordered allocator), so building a layer set does not stall other streams.
 * The result is used like any portfolio (ara_run_ylt, ara_adjoint, ...) and released with
 * ara_destroy_portfolio; the pool must outlive it.  Layer arguments as in ara_create_portfolio
 * (n_layers >= 1), ELT indices refer to the pool.
 * Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA.
 */
ARA_API ara_status ara_create_layer_set(ara_portfolio* pool, int32_t n_layers,
                                        const int32_t* layer_elt_offsets,
                                        const int32_t* layer_elt_ids, const double* occ_ret,
                                        const double* occ_lim, const double* agg_ret,
                                        const double* agg_lim, void* stream, ara_portfolio** out);

/* ---------------------------------------------------------------------------------------
 * YLT: Algorithm 1 (for each layer) around Algorithm 3 (for each trial, event, ELT).
 * --------------------------------------------------------------------------------------- */

/* flags of ara_run_ylt / ara_run_ylt_host */
#define ARA_RUN_FOLDED    0   /* default: per-ELT and occurrence terms folded once per layer
                                 into a per-event table (occurrence terms depend on nothing but
                                 the event, Section IV-B), then one gather per hit occurrence */
#define ARA_RUN_PER_ELT   1   /* Algorithm 3 literally: every ELT of the layer looked up for
                                 every occurrence (needs ARA_DENSE_TABLES) */
#define ARA_RUN_NO_FILTER 2   /* folded, without the shared-memory hit filter (measurement) */
#define ARA_RUN_F64_SUM   4   /* folded, trial sums in FP64 instead of exact fixed point
                                 (measurement) */
#define ARA_RUN_LDG       8   /* folded, YET read by per-trial 16-byte register loads instead of
                                 the per-warp TMA bulk-copy ring (measurement) */
#define ARA_RUN_BATCHED  32   /* all selected layers in one YET pass (event-major table of every
                                 layer's occurrence losses, one persistent stream kernel); same
                                 results; at most 255 selected layers, no repeats beyond the
                                 portfolio's layer count (ARA_ERANGE) */
#define ARA_RUN_OEP      64   /* occurrence basis: y_t = max_k o(e_{t,k}), the trial's largest
                                 occurrence loss net of ELT and occurrence terms (the loss behind
                                 occurrence exceedance curves); aggregate terms not applied,
                                 regimes all 0.  Only with the default folded path */
#define ARA_RUN_PREPARED 256 /* the fold of the selected layers (per-ELT and occurrence terms,
                                 and the coarse hit bitmap) was queued earlier by
                                 ara_prepare_ylt into fold slot 0 (or 1 with ARA_RUN_SLOT1):
                                 the run only streams the YET.  Folded paths only */
#define ARA_RUN_SLOT1   512   /* with ARA_RUN_PREPARED: use fold slot 1 */
#define ARA_RUN_HOST_DIRECT 16 /* ara_run_ylt_host only: the kernel reads the (pinned, device-
                                 mapped) host YET in place over the CPU-GPU link instead of
                                 staging it with copies; ARA_EINVAL if the host arrays are not
                                 accessible from the device */

/*
 * YLT of n_trials trials for the selected layers.  Asynchronous on `stream`.
 *   d_trial_offsets  device [n_trials + 1] int64: trial t owns events
 *                    d_trial_offsets[t] .. d_trial_offsets[t+1]-1 of d_event_ids
 *                    (0 <= offsets non-decreasing <= n_events, else ARA_EDATA later).
 *                    The default stream kernel splits the trials into one contiguous range
 *                    per warp (n_trials / (SMs x 28) trials each); a range of 2^31 - 512 or
 *                    more events is reported as ARA_EDATA (ARA_RUN_LDG has no such limit)
 *   n_events         number of elements of d_event_ids
 *   d_event_ids      device [n_events] int32, 4-byte aligned: each trial's event IDs in time
 *                    order (Eq. 1)
 *   d_timestamps     device [n_events] float or NULL: accepted for the YET's shape, not read
 *                    (no term of Section IV-B depends on the time of an occurrence)
 *   n_layer_sel      number of layers to run; layer_sel host [n_layer_sel] layer indices,
 *                    or (n_layer_sel = 0, layer_sel = NULL) for all layers in order
 *   d_ylt            device [n_layer_sel][n_trials] double, row-major: the YLT
 *   d_regimes        device [n_layer_sel][n_trials] uint8 or NULL: the aggregate clamp's
 *                    regime per trial (0: S <= AggR or kink, 1: AggR < S < AggR + AggL,
 *                    2: S > AggR + AggL), recorded for ara_adjoint
 *   flags            ARA_RUN_* (one of FOLDED / PER_ELT, optionally NO_FILTER, F64_SUM; PREPARED
 *                    and SLOT1 to stream against a fold queued by ara_prepare_ylt)
 * Errors: ARA_EINVAL (also: ARA_RUN_SLOT1 before slot 1 was ever prepared), ARA_ECUDA; data
 * errors via ara_check().
 */
ARA_API ara_status ara_run_ylt(ara_portfolio* pf, int64_t n_trials, const int64_t* d_trial_offsets,
                       int64_t n_events, const int32_t* d_event_ids, const float* d_timestamps,
                       int32_t n_layer_sel, const int32_t* layer_sel, double* d_ylt,
                       uint8_t* d_regimes, int32_t flags, void* stream);

/*
 * The fold of a run queued on its own: for the selected layers, the per-ELT and occurrence
 * terms of every catalogue event (Algorithm 3's ELT loop and occurrence terms, which depend on
 * the event alone, Section IV-B) into fold slot `slot` (0 or 1) of the portfolio, with the hit
 * bitmaps the stream kernel of `flags` reads.  A later ara_run_ylt with ARA_RUN_PREPARED (and
 * ARA_RUN_SLOT1 for slot 1), the same layers and the same other flags streams the YET against it
 * without folding again; ordering is the caller's (same stream, or an event).  Two slots let the
 * fold of one run proceed on another stream while the previous run streams from the other slot
 * (the paper has no counterpart; this is a pipelining of Algorithm 1's loop over runs).  The
 * first use of slot 1 allocates it (catalogue x ~8.3 bytes per layer; synchronises `stream`).
 * A slot holds the fold of the last prepare (or, slot 0, of the last unprepared run) of each
 * layer: a prepared run after the portfolio's slot was overwritten reads that newer fold.
 *   flags      ARA_RUN_* of the run to come (NO_FILTER, F64_SUM, LDG, OEP); not PER_ELT,
 *              BATCHED, HOST_DIRECT, PREPARED or SLOT1
 * Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA.
 */
ARA_API ara_status ara_prepare_ylt(ara_portfolio* pf, int32_t n_layer_sel, const int32_t* layer_sel,
                                   int32_t slot, int32_t flags, void* stream);

/*
 * The whole analysis from host memory: Algorithm 1 with the transfer of Algorithm 2 and the
 * kernels of Algorithm 3, then the YLT and (optionally) its PML / TVaR back on the host.
 * The YET is copied in chunks on an internal copy stream while earlier chunks are processed
 * on `stream`, so host-to-device traffic overlaps the kernels (pinned host memory gives full
 * link bandwidth); the YLT stays on the device for the risk metrics and is copied back.
 * Synchronous: returns when every output is written.
 *   h_trial_offsets host [n_trials + 1], [0] = 0, non-decreasing (validated: ARA_EINVAL; with
 *                   ARA_RUN_HOST_DIRECT the check runs on the host while the kernels already read
 *                   the YET, whose own bounds checks keep bad offsets harmless; a rejected call
 *                   still waits for them and clears the device error word, as ara_check does)
 *   h_event_ids     host [h_trial_offsets[n_trials]]
 *   h_ylt           host [n_layer_sel][n_trials] or NULL (then only the metrics are returned)
 *   n_rp, return_periods, n_tvar, tvar_levels, h_pml, h_tvar, h_mean: as in
 *                   ara_risk_metrics, or n_rp = n_tvar = 0 and h_mean = NULL for no metrics
 * Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA, ARA_EDATA (event ID outside the catalogue).
 */
ARA_API ara_status ara_run_ylt_host(ara_portfolio* pf, int64_t n_trials,
                                    const int64_t* h_trial_offsets, const int32_t* h_event_ids,
                                    int32_t n_layer_sel, const int32_t* layer_sel, double* h_ylt,
                                    int32_t n_rp, const double* return_periods, int32_t n_tvar,
                                    const double* tvar_levels, double* h_pml, double* h_tvar,
                                    double* h_mean, int32_t flags, void* stream);

/* Synchronise `stream`, then report (and clear) device-side errors recorded by earlier
 * asynchronous runs of this portfolio: ARA_OK, ARA_EDATA (bad event ID or offsets; the YLT of
 * that run is unspecified) or ARA_ETIMEOUT (a bounded wait for a bulk copy gave up). */
ARA_API ara_status ara_check(ara_portfolio* pf, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched portfolio: every selected layer in one pass over the YET, as one CUDA graph.
 * --------------------------------------------------------------------------------------- */

typedef struct ara_plan ara_plan;

#define ARA_PLAN_AUTOTUNE 1   /* time the candidate stream schedules on these inputs, keep the
                                 fastest */

/*
 * Build a plan for the YLT of n_layer_sel layers (<= 255) of a portfolio over one device YET
 * (Algorithm 1's program and layer loops folded into one launch).  The plan owns its scratch
 * (an event-major table of every layer's non-zero occurrence losses, with per-event rows) and a
 * CUDA graph of the whole run: per-layer folds (per-ELT and occurrence terms), the table build,
 * and one persistent stream kernel that reads every occurrence once, accumulates all layers'
 * trial sums exactly, applies their aggregate terms and writes the YLT.  The YET, YLT and
 * regime buffers are bound to the plan: every ara_plan_launch recomputes the YLT from their
 * current contents.  Results equal those of ara_run_ylt bit for bit.  Synchronous.
 *   arguments as ara_run_ylt (layer_sel must not be NULL unless n_layer_sel = 0: all layers)
 *   flags     ARA_PLAN_AUTOTUNE or 0
 * Errors: ARA_EINVAL, ARA_ERANGE (more than 255 layers), ARA_ENOMEM, ARA_ECUDA.
 */
ARA_API ara_status ara_plan_batched(ara_portfolio* pf, int64_t n_trials,
                                    const int64_t* d_trial_offsets, int64_t n_events,
                                    const int32_t* d_event_ids, int32_t n_layer_sel,
                                    const int32_t* layer_sel, double* d_ylt, uint8_t* d_regimes,
                                    int32_t flags, void* stream, ara_plan** out);
/* Replay the plan's graph on `stream` (asynchronous; data errors via ara_check). */
ARA_API ara_status ara_plan_launch(ara_plan* plan, void* stream);
/* The schedule in use: warps per block, blocks per SM, trials per queue grab, the tuned time
 * of one stream kernel in ms (0 without ARA_PLAN_AUTOTUNE), and the copies of each warp's
 * per-layer accumulators in shared memory (1, 2 or 4; a copy per group of 32 / copies lanes).
 * Any output pointer may be NULL.  Errors: ARA_EINVAL (NULL plan). */
ARA_API ara_status ara_plan_info(ara_plan* plan, int32_t* warps, int32_t* blocks_per_sm,
                                 int32_t* trials_per_grab, double* tuned_ms, int32_t* copies);
/* The plan's event-major table, for measurement: d_rows receives its device array of row
 * descriptors [catalogue] (bits 0..31: the event's first table entry; byte 4: the number of its
 * entries, one per selected layer whose occurrence loss for the event is non-zero), valid until
 * the plan is destroyed and rewritten by every launch; n_entries the table's entry count.
 * Synchronises the device.  Errors: ARA_EINVAL, ARA_ECUDA. */
ARA_API ara_status ara_plan_table(ara_plan* plan, const uint64_t** d_rows, int64_t* n_entries);
ARA_API void ara_plan_destroy(ara_plan* plan);

/*
 * Several requests' YLTs in one pass over a shared YET (the batched path serving several
 * requests at once; the paper has no counterpart, it is the single-GPU way for its many tenants
 * to share one reading of the YET).  Request r owns the portfolio's layers
 * [req_layer_first[r], req_layer_first[r + 1]) (every layer of the portfolio belongs to exactly
 * one request, in order) and the trials [req_trial_begin[r], req_trial_end[r]) of the n_trials
 * trials given.  Every trial is read once and walks only the table entries of the requests that
 * cover it.  Request r's YLT goes to d_ylt[r], a device [its layers][its trials] double array
 * (row-major), and its aggregate regimes (as ara_run_ylt) to d_regimes[r] (device, same shape,
 * or NULL; d_regimes itself may be NULL).  Results equal those of ara_run_ylt of each request
 * alone, bit for bit.  Asynchronous on `stream`; scratch from the stream-ordered allocator.
 *   n_req      1..4; the portfolio has at most 255 layers
 *   d_ylt, d_regimes   host arrays [n_req] of device pointers
 * Errors: ARA_EINVAL, ARA_ERANGE, ARA_ENOMEM, ARA_ECUDA; data errors via ara_check().
 */
ARA_API ara_status ara_run_ylt_requests(ara_portfolio* pf, int64_t n_trials,
                                        const int64_t* d_trial_offsets, int64_t n_events,
                                        const int32_t* d_event_ids, int32_t n_req,
                                        const int32_t* req_layer_first,
                                        const int64_t* req_trial_begin,
                                        const int64_t* req_trial_end, double* const* d_ylt,
                                        uint8_t* const* d_regimes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Serving: many risk queries over resident ELTs and a resident YET, on one GPU (the single-GPU
 * form of the paper's multi-tenant GPUs, Section V-D).
 * --------------------------------------------------------------------------------------- */

typedef struct ara_server ara_server;

/* One risk query: layers (Eq. 3) over the server pool's ELTs, evaluated on the trials
 * [trial_begin, trial_end) of the resident YET.  All arrays are host memory, copied at submit. */
typedef struct ara_query {
  int32_t n_layers;                 /* >= 1 */
  const int32_t* layer_elt_offsets; /* [n_layers + 1] */
  const int32_t* layer_elt_ids;     /* ELT indices into the pool */
  const double* occ_ret;            /* [n_layers] each */
  const double* occ_lim;
  const double* agg_ret;
  const double* agg_lim;
  int64_t trial_begin, trial_end;
  int32_t n_rp;                     /* PML return periods */
  const double* return_periods;
  int32_t n_tvar;                   /* TVaR levels */
  const double* tvar_levels;
  int32_t want_mean;                /* mean year loss per layer */
  int32_t want_adjoint;             /* layer-term gradients of mean and TVaR (adjoint_level) */
  double adjoint_level;
  int32_t flags;                    /* ARA_RUN_BATCHED or 0 */
  int32_t tenant;                   /* caller's label, not interpreted */
} ara_query;

/*
 * Start a server over a resident pool portfolio (its ELTs) and a resident device YET.  Up to
 * max_concurrent (1..64) workers run requests at once, each on its own stream.  A free worker
 * admits the oldest queued request when its estimated device memory fits both memory_budget
 * bytes together with the requests already running (<= 0: 80 % of the device's free memory at
 * creation) and the device memory free at that moment; when it does not fit, the first of the
 * next 31 queued requests that fits runs ahead of it (at most 4 times per blocked request).  A
 * request larger than the budget runs alone.  Into the admitted request the worker merges up to
 * three more queued requests (of the next 32) whose trial slices overlap the group's (by at
 * least 60 % of their union by default, see ara_server_set_merging), best overlap first, while their
 * memory fits: the group's layers run in one batched pass over the union of the slices, each
 * trial walking only the table entries of the requests that cover it, so the requests share the
 * reading of the YET (a group's table is kept near L2 size).  The workers' YET passes (batched
 * or single-layer streams, adjoint histograms) run one after the other on the device, each
 * queued behind the previous one; their folds, selections and host work overlap.  Admission
 * counts the library's idle pooled memory (see ara_release_memory) as free.  Creation runs a
 * few small warm-up requests
 * (synchronous), so the first real requests pay no one-time costs.  The pool and the YET must
 * outlive the server.  Results of a request do not depend on what else runs or on the group it
 * ran in (bitwise).
 */
ARA_API ara_status ara_server_create(ara_portfolio* pool, int64_t n_trials,
                                     const int64_t* d_trial_offsets, int64_t n_events,
                                     const int32_t* d_event_ids, int32_t max_concurrent,
                                     int64_t memory_budget, ara_server** out);
/* The device memory the server estimates a query may hold at once (the figure admission uses);
 * the query is validated as by ara_server_submit and not queued.  Errors: ARA_EINVAL. */
ARA_API ara_status ara_server_estimate_bytes(ara_server* server, const ara_query* query,
                                             int64_t* bytes);
/* Queue a query (validated and copied now; ARA_EINVAL on bad arguments); returns a ticket. */
ARA_API ara_status ara_server_submit(ara_server* server, const ara_query* query, int64_t* ticket);
/*
 * Wait for a ticket and collect its results (each pointer may be NULL):
 *   h_pml [n_layers][n_rp], h_tvar [n_layers][n_tvar], h_mean [n_layers],
 *   h_grad_layer [2][n_layers][4] (mean / TVaR objective; d/dOccR, OccL, AggR, AggL),
 *   h_times [3]: seconds queued, running, and from submit to completion.
 * Returns the request's status.  A ticket can be waited for once.
 */
ARA_API ara_status ara_server_wait(ara_server* server, int64_t ticket, double* h_pml,
                                   double* h_tvar, double* h_mean, double* h_grad_layer,
                                   double* h_times);
/* Requests queued or running now, the largest number ever running at once, the largest
 * estimated memory ever admitted at once, and the budget. */
ARA_API ara_status ara_server_stats(ara_server* server, int32_t* queued_or_running,
                                    int32_t* peak_running, int64_t* peak_bytes, int64_t* budget);
/* Merging of queued requests into one pass: at most max_requests_per_pass (1..4; 1 = every
 * request runs its own pass) requests per pass, a request joining a group when its slice
 * overlaps the group's by at least min_overlap (0 < min_overlap <= 1) of their union.  Applies
 * to groups formed after the call.  Default 4 and 0.6.  Errors: ARA_EINVAL. */
ARA_API ara_status ara_server_set_merging(ara_server* server, int32_t max_requests_per_pass,
                                          double min_overlap);
/* Passes run so far (a pass serves one request or a merged group), requests that ran in a merged
 * group of two or more, the times a blocked oldest request was passed by a later one, and the
 * adjoints computed over the server's YET index.  Each pointer may be NULL. */
ARA_API ara_status ara_server_counters(ara_server* server, int64_t* passes,
                                       int64_t* merged_requests, int64_t* head_passed,
                                       int64_t* indexed_adjoints);
/*
 * Build (on != 0) or release (on == 0) an event-major index of the server's resident YET
 * (ara_yet_index_create) for the adjoint requests.  While it exists, a request's adjoint reads
 * the index instead of the YET when its trial slice covers at least half of the index blocks it
 * touches (the indexed pass reads those blocks whole); results are bitwise the same either way.
 * The index's device memory (about 3 bytes per occurrence) is held until released or the server
 * is destroyed; admission sees it as memory in use.  Only while the server is idle: ARA_EBUSY
 * when a request is queued or running.  Synchronous.  Errors as ara_yet_index_create.
 */
ARA_API ara_status ara_server_set_adjoint_index(ara_server* server, int32_t on);
/* Finish every queued request, then stop the workers and release the server. */
ARA_API void ara_server_destroy(ara_server* server);

/* ---------------------------------------------------------------------------------------
 * Adjoint: sensitivities of the risk metrics (Section IV-A) to the financial terms and the
 * ELT losses (Section IV-B).
 * --------------------------------------------------------------------------------------- */

/*
 * For every selected layer, the gradients of two objectives of its YLT row y:
 *   objective 0: the mean year loss (1/N) sum_t y_t
 *   objective 1: TVaR at tvar_level, the mean of the m = ceil(N(1-p)) largest y
 * with respect to every per-ELT retention and limit of the layer's ELTs, the layer's OccR,
 * OccL, AggR, AggL, and every ELT loss record of the layer.  The clamps are piecewise linear;
 * at a kink the derivative is taken as 0.  When the m-th and (m+1)-th largest year losses tie,
 * the trials equal to the m-th share its weight equally (the mean over every choice of the
 * top-m set) and h_ties reports it.  Uses the forward's YLT and recorded regimes instead of
 * recomputing the trial sums.  Synchronous.
 *   YET arguments and layer selection: exactly those of the ara_run_ylt call that produced
 *                  d_ylt and d_regimes (same trials, same layers in the same order)
 *   d_ylt          device [n_layer_sel][n_trials]  (from ara_run_ylt)
 *   d_regimes      device [n_layer_sel][n_trials]  (from ara_run_ylt)
 *   tvar_level     p in [0, 1) with ceil(N(1-p)) >= 1
 *   d_grad_elt     device [2][K][2] double: K = total ELT slots of the selected layers (each
 *                  layer's ELTs in layer order, layers in selection order); (d/dR_j, d/dL_j)
 *   d_grad_layer   device [2][n_layer_sel][4] double: d/dOccR, d/dOccL, d/dAggR, d/dAggL
 *   d_grad_loss    device [2][M] double: M = total records of those slots; slot by slot, each
 *                  ELT's records in the order given to ara_create_portfolio
 *   h_ties         host [n_layer_sel] int32 or NULL
 * Errors: ARA_EINVAL, ARA_ERANGE (a layer with more than 256 ELTs), ARA_ENOMEM, ARA_ECUDA,
 * ARA_EDATA.
 */
ARA_API ara_status ara_adjoint(ara_portfolio* pf, int64_t n_trials, const int64_t* d_trial_offsets,
                               int64_t n_events, const int32_t* d_event_ids, int32_t n_layer_sel,
                               const int32_t* layer_sel, const double* d_ylt,
                               const uint8_t* d_regimes, double tvar_level, double* d_grad_elt,
                               double* d_grad_layer, double* d_grad_loss, int32_t* h_ties,
                               void* stream);

/*
 * ara_adjoint folded into the portfolio's own parameter layout, for reverse-mode automatic
 * differentiation: with upstream weights w[i][o] (selected layer i, objective o as above),
 *   d_g_elt_ret[j], d_g_elt_lim[j]   += sum over (i, o, slots of ELT j) w[i][o] * dJ/d(R_j, L_j)
 *   d_g_layer[l][0..3]               += sum over (i selecting l, o) w[i][o] * dJ/d(OccR..AggL)
 *   d_g_loss[r]                      += the same for every ELT record r, records in the order
 *                                       given to ara_create_portfolio (ELT by ELT)
 *   h_weights   host [n_layer_sel][2]
 *   d_g_elt_ret, d_g_elt_lim  device [n_elts]; d_g_layer device [n_layers][4];
 *   d_g_loss    device [total records]   (accumulated into: zero them first)
 * Synchronous.  Errors as ara_adjoint.
 */
ARA_API ara_status ara_adjoint_accumulate(ara_portfolio* pf, int64_t n_trials,
                                          const int64_t* d_trial_offsets, int64_t n_events,
                                          const int32_t* d_event_ids, int32_t n_layer_sel,
                                          const int32_t* layer_sel, const double* d_ylt,
                                          const uint8_t* d_regimes, double tvar_level,
                                          const double* h_weights, double* d_g_elt_ret,
                                          double* d_g_elt_lim, double* d_g_layer,
                                          double* d_g_loss, void* stream);

/*
 * Event-major index of a device YET, for adjoint passes over the same YET (the trial-major
 * table of Eq. 1, transposed).  The adjoint's histograms count, per catalogue event and
 * layer, the occurrences of the event in trials whose aggregate loss is interior for the layer.
 * Read trial by trial, every occurrence scatters into the histograms.  Read event by event, an
 * event's counts stay in one thread.  The index depends on the YET alone (not on the layers or
 * their terms): build it once, then use it for any number of ara_adjoint_indexed calls.
 *   ara_yet_index_create  reads the YET (same arguments as ara_run_ylt) and builds the index
 *                         on pf's device, for pf's catalogue size.  Synchronous.  Device memory:
 *                         2 bytes per occurrence plus the padding of each group of 32 events
 *                         to its longest list per block of trials (about 1.5x on uniform
 *                         events), and 12 bytes per (block, group).  The index owns its
 *                         memory; the YET may be freed or changed afterwards.
 *                         Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA, ARA_EDATA (an event ID
 *                         outside the catalogue, or offsets that decrease or leave
 *                         [0, n_events]: no index is made).
 *   ara_yet_index_destroy releases it (NULL is accepted).
 */
typedef struct ara_yet_index ara_yet_index;
ARA_API ara_status ara_yet_index_create(ara_portfolio* pf, int64_t n_trials,
                                        const int64_t* d_trial_offsets, int64_t n_events,
                                        const int32_t* d_event_ids, void* stream,
                                        ara_yet_index** out);
ARA_API void ara_yet_index_destroy(ara_yet_index* yx);

/*
 * ara_adjoint over an indexed YET, for its trials [first_trial, first_trial + n_trials)
 * (0 and 0: all of them).  The arguments and results are those of ara_adjoint over those
 * trials of the YET the index was built from (d_ylt, d_regimes: [n_layer_sel][n_trials] of
 * them), with the YET replaced by the index; results are bitwise equal.  The pass reads the
 * index blocks the trials touch whole, so a slice much shorter than a block (49,344 trials at
 * most) costs about as much as the block.  pf must have the catalogue size the index was built
 * for.  Synchronous.
 * Errors as ara_adjoint; also ARA_EINVAL for a catalogue mismatch or trials outside the index,
 * and ARA_ERANGE when the selected layers' tables exceed 32-bit entry indices (ara_adjoint then
 * takes one pass per layer; with an index, call ara_adjoint).
 */
ARA_API ara_status ara_adjoint_indexed(ara_portfolio* pf, const ara_yet_index* yx,
                                       int64_t first_trial, int64_t n_trials,
                                       int32_t n_layer_sel, const int32_t* layer_sel,
                                       const double* d_ylt, const uint8_t* d_regimes,
                                       double tvar_level, double* d_grad_elt, double* d_grad_layer,
                                       double* d_grad_loss, int32_t* h_ties, void* stream);

/* ---------------------------------------------------------------------------------------
 * Risk metrics of Section IV-A (PML, TVaR), read as empirical order statistics of the YLT:
 *   PML(RP)  = the k-th largest year loss, k = ceil(N / RP)
 *   TVaR(p)  = mean of the m largest year losses, m = ceil(N (1 - p))
 * N/RP and N(1-p) within 1e-9 (relative) of an integer are taken as that integer, so that
 * decimal levels such as p = 0.99 give m = N/100 exactly.
 * --------------------------------------------------------------------------------------- */

/*
 * Risk metrics of n_layers YLT rows.  Synchronous (results are host values).
 *   d_ylt         device [n_layers][n_trials] double
 *   return_periods host [n_rp], each >= 1 with 1 <= ceil(N/RP) <= N
 *   tvar_levels   host [n_tvar], each in [0, 1) with ceil(N(1-p)) >= 1
 *   h_pml         host [n_layers][n_rp];  h_tvar host [n_layers][n_tvar]
 *   h_mean        host [n_layers] or NULL: the mean year loss (1/N) sum_t y_t of each row
 * n_rp + n_tvar <= 16 (at least one metric requested), n_trials >= 1.  Allocates its scratch
 * in stream order on `stream`, from the library's memory pool.  The selection is one
 * cooperative launch whose blocks meet at device-side barriers, each wait bounded like the
 * bulk copies' (ara_debug_set ARA_DBG_WAIT_LIMIT_NS).
 * Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA, ARA_ETIMEOUT (a barrier wait ran out).
 */
ARA_API ara_status ara_risk_metrics(const double* d_ylt, int64_t n_trials, int32_t n_layers,
                            int32_t n_rp, const double* return_periods, int32_t n_tvar,
                            const double* tvar_levels, double* h_pml, double* h_tvar,
                            double* h_mean, void* stream);

/*
 * ara_risk_metrics, stream-ordered: the results are written to device memory when the work
 * queued on `stream` completes, and the call returns without waiting, so a caller can queue
 * the next run behind it (the paper has no counterpart; it is the pipelined form of the same
 * computation).  Arguments as ara_risk_metrics, except:
 *   d_pml        device [n_layers][n_rp] double (NULL when n_rp = 0)
 *   d_tvar       device [n_layers][n_tvar] double (NULL when n_tvar = 0)
 *   d_mean       device [n_layers] double or NULL
 *   d_status     device uint32: set to 0 when the work starts; ARA_DEVICE_TIMEOUT is OR-ed
 *                in when a device-side wait runs out (the other outputs are then undefined)
 * Scratch comes from the library's memory pool in stream order and is released in stream order.  Argument
 * errors are returned at once (ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA) and nothing is queued.
 * Scheduling: the selection's blocks, like those of the default stream kernel, each fill an SM's
 * registers, and the selection starts only once every SM is free.  When it runs on another
 * stream than the next ara_run_ylt, order it before that run's stream kernel, e.g.
 * ara_prepare_ylt on the run's stream, a wait on an event recorded after this call, then
 * ara_run_ylt with ARA_RUN_PREPARED: otherwise the next stream kernel may take every SM first and
 * hold the selection back for a whole run.
 */
#define ARA_DEVICE_TIMEOUT 4u
ARA_API ara_status ara_risk_metrics_async(const double* d_ylt, int64_t n_trials, int32_t n_layers,
                                          int32_t n_rp, const double* return_periods,
                                          int32_t n_tvar, const double* tvar_levels, double* d_pml,
                                          double* d_tvar, double* d_mean, uint32_t* d_status,
                                          void* stream);

/*
 * ara_risk_metrics for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment convenience.  Some callers may not call cudaMalloc or
 * the stream-ordered allocator: a process whose device memory is already reserved in full by
 * another allocator (a framework's caching pool, a serving process sized to the whole GPU),
 * where any further allocation fails; or a latency-critical loop that cannot afford an
 * allocation's latency or cudaFree's implicit device synchronisation.  This entry point
 * allocates nothing: its scratch is one fixed array of ARA_STATIC_SELECT_BYTES bytes in
 * device memory, defined in libara itself (every GPU that loads the library holds it until
 * the process exits).  Arguments, results and errors are those of ara_risk_metrics, plus:
 *   - a request whose scratch (about 8 KiB per layer per requested PML/TVaR level) does not
 *     fit in the array returns ARA_ERANGE and launches nothing;
 *   - every call looks up the array's device address on the current device (a cheap host
 *     query), so the address stays right after the device's context is torn down and
 *     recreated (cudaDeviceReset reloads the library's module, possibly elsewhere);
 *   - the call waits for `stream` before it returns, also when a result copy fails, so no
 *     copy queued by it lands in the caller's buffers afterwards;
 *   - every call reuses the same array and clears the part it needs first; calls whose
 *     work overlaps on a device (other streams, other host threads) race on it and must be
 *     serialised by the caller.
 */
#define ARA_STATIC_SELECT_BYTES (4u << 20)
ARA_API ara_status ara_risk_metrics_static(const double* d_ylt, int64_t n_trials,
                                           int32_t n_layers, int32_t n_rp,
                                           const double* return_periods, int32_t n_tvar,
                                           const double* tvar_levels, double* h_pml,
                                           double* h_tvar, double* h_mean, void* stream);

/* ---------------------------------------------------------------------------------------
 * Introspection for measurement.
 * --------------------------------------------------------------------------------------- */

/* Return the memory that the library's pools hold idle (freed scratch kept for reuse) to the
 * system, on every device.  Memory in use is not touched.  Errors: ARA_ECUDA. */
ARA_API ara_status ara_release_memory(void);

/* Kernels launched by this library in this process so far. */
ARA_API int64_t ara_launch_count(void);

/* Launch shapes of the YET-stream kernel (tuning).  ara_stream_shapes writes up to `max`
 * (warps per block, staging-ring stages) pairs into the host arrays and returns how many shapes
 * are compiled in; ara_set_stream_shape selects one for every later run in this process
 * (ARA_EINVAL for an unknown index).  Results do not depend on the shape. */
ARA_API int32_t ara_stream_shapes(int32_t* warps, int32_t* stages, int32_t max);
ARA_API ara_status ara_set_stream_shape(int32_t index);

/* Failure-detection hooks (process-wide; for tests).
 *   ARA_DBG_WAIT_LIMIT_NS  bound of every device-side wait (bulk copies, the risk metrics'
 *                          grid barriers), in ns (default 1e9; >= 1000).  A bulk-copy wait
 *                          that runs out makes the kernel record a timeout, wait (bounded) for
 *                          its own copies in flight and return; ara_check then reports
 *                          ARA_ETIMEOUT.  A barrier wait that runs out ends the selection;
 *                          the risk-metrics call reports ARA_ETIMEOUT.
 *   ARA_DBG_STARVE_COPIES  announce this many bytes more than each bulk copy delivers (a
 *                          multiple of 16, <= 4096; 0 = normal): every wait then runs out,
 *                          which exercises the timeout path without any fault.
 *   ARA_DBG_SKIP_BARRIER_ARRIVAL  1: the selection's blocks do not arrive at its grid
 *                          barriers, so every barrier wait runs out (0 = normal).
 *   ARA_DBG_ADJOINT_PER_LAYER  1: ara_adjoint of several layers takes one histogram pass per
 *                          layer instead of one pass for all (0 = normal); same results.
 * ARA_EINVAL for an unknown key or value. */
#define ARA_DBG_WAIT_LIMIT_NS  1
#define ARA_DBG_STARVE_COPIES  2
#define ARA_DBG_SKIP_BARRIER_ARRIVAL 3
#define ARA_DBG_ADJOINT_PER_LAYER 4
ARA_API ara_status ara_debug_set(int32_t key, int64_t value);

/* kernel classes for timing */
#define ARA_K_FOLD    0   /* per-layer fold of per-ELT and occurrence terms */
#define ARA_K_YLT     1   /* the YET stream: trial sums, aggregate terms, YLT write */
#define ARA_K_SELECT  2   /* PML / TVaR selection (all of its launches) */
#define ARA_K_ADJOINT 3   /* adjoint kernels */
#define ARA_K_BATCHED 4   /* one replay of a batched-portfolio plan (its whole CUDA graph) */
#define ARA_K_TRANSFER 5  /* ara_run_ylt_host's own copies: host-to-device YET chunks (staged
                             mode) and the device-to-host YLT */
#define ARA_K_HOST_CHECK 6 /* ara_run_ylt_host's host-side check of the trial offsets: host wall
                             time, not device time */
#define ARA_K_COUNT   7

/* When enabled, CUDA events are recorded on the launching stream around every launch of
 * each kernel class (and every copy of ARA_K_TRANSFER; ARA_K_HOST_CHECK is timed on the host).
 * ara_timing_read synchronises those events and returns the summed time (ms) and the number of
 * launches (copies, checks) since the last reset. */
ARA_API void ara_timing_enable(int32_t on);
ARA_API void ara_timing_reset(void);
ARA_API ara_status ara_timing_read(int32_t kernel_class, double* total_ms, int64_t* launches);

/* Static description of a status code. */
ARA_API const char* ara_status_string(ara_status s);

#ifdef __cplusplus
}
#endif
#endif /* ARA_H */

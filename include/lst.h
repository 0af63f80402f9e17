/*
 * lst.h -- C-ABI of the GB300 line-segment-tracking (LST) library (liblst.so).
 *
 * The library builds, per collision event, the LST track segments of arXiv 2403.13166
 * (Section 1, Table 1, steps 1-4) on the GPU and scores every quintuplet with the
 * T5-DNN (Sections 2-3):
 *   step 1  mini-doublets (MD): one hit in each sensor of a pT-module, pT > 0.8 GeV;
 *   step 2  line segments (LS): two MDs in modules linked by the module map;
 *   step 3  triplets (T3): two LSs sharing their common MD;
 *   step 4  quintuplets (T5): two T3s sharing their common MD;
 *   score   38 features -> 32 -> 32 -> 1 (ReLU, sigmoid), selected iff score >= wp.
 *
 * Conventions for every call:
 *   - Every function returns an lst_status (0 = LST_OK). No call aborts, exits or traps;
 *     device-side failures are reported through status words that the host reads.
 *   - Pointers documented as DEVICE must be CUDA device (or managed) memory of the
 *     context's device; HOST pointers are ordinary host memory (pinned or not).
 *   - `cuda_stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *   - Input buffers stay owned by the caller and must stay valid until the call's work
 *     on the stream has finished. Everything the library allocates is owned by the
 *     context (geometry, weights, per-event object buffers) and freed by lst_destroy.
 *   - Output hit indices always refer to the caller's original hit order.
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef LST_H
#define LST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lst_status {
    LST_OK = 0,
    LST_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad enum) */
    LST_ERR_CAPACITY = 2,   /* an object buffer or caller buffer was too small; sizes reported */
    LST_ERR_CUDA = 3,       /* a CUDA runtime call failed (message in lst_last_error) */
    LST_ERR_TIMEOUT = 4,    /* a bounded device-side wait ran out */
    LST_ERR_NOT_READY = 5,  /* no geometry loaded / no free event slot / work still running */
    LST_ERR_INPUT = 6,      /* a hit had a sensor id out of range or a non-finite coordinate */
    LST_ERR_NOMEM = 7       /* device allocation failed */
} lst_status;

/* Object kinds (Table 1): steps 1-4, and the track candidates of step 6 (T5s not matched
 * to a pixel seed; no pixel seeds exist here), i.e. the selected T5s after duplicate
 * removal (see lst_get_candidates). */
typedef enum lst_kind { LST_MD = 0, LST_LS = 1, LST_T3 = 2, LST_T5 = 3, LST_TC = 4 } lst_kind;

/* Timed stages of one launch (lst_stage_times): hit grouping, step 1, step 2 (the LS
 * kernel, then the grouping of the LSs by inner MD), steps 3-4, score, track candidates. */
#define LST_N_STAGES 8
/* Arithmetic of the T5-DNN score (Section 2 network). LST_FP32: CUDA cores, FP32
 * operations only, compensated: features in float-float (hi + lo pairs of floats) and
 * every layer a compensated dot product with float-float activations, so that the score
 * is within 1e-6 of an FP64 evaluation even for networks that amplify one FP32 rounding
 * of an input beyond that (about 8x the FP32 operations of a plain evaluation). LST_BF16:
 * tensor cores, BF16 operands, FP32 accumulation. LST_BF16X3: tensor cores, each operand
 * split into BF16 hi + lo parts and hi*hi + lo*hi + hi*lo accumulated in FP32 (about 16
 * significant bits per operand; for networks whose score is sensitive to small input
 * differences). Not in the paper, whose network runs in FP32. */
typedef enum lst_precision { LST_FP32 = 0, LST_BF16 = 1, LST_BF16X3 = 2 } lst_precision;

/* One pT-module (Section 1: two sensors a few mm apart). Sensor ids of module m are
 * 2*m (lower sensor, nearer the interaction point; its hit is the MD anchor, Section 2)
 * and 2*m+1 (upper sensor). */
typedef struct lst_module {
    int32_t layer;    /* 1..6 barrel layers, 7..11 endcap disks (T5-DNN "layer" input) */
    int32_t subdet;   /* 0 = barrel (flat module parallel to z), 1 = endcap (disk module) */
    int32_t side;     /* 0 barrel, -1 / +1 endcap side */
    int32_t ps;       /* 1 = PS module (macro-pixel + strip), 0 = 2S (two strips) */
} lst_module;

/* Cut parameters of the MD/LS/T3/T5 selections (Section 1: "consistency with a
 * continuous, helical trajectory"). All FP32; units cm, GeV, 1/cm. */
typedef struct lst_cuts {
    float kappa_max;        /* curvature of a 0.8 GeV track: k_field / 0.8 */
    float z_lum;            /* luminous-region half length for the z0 road */
    float hit_err;          /* 3-sigma error of a two-hit difference */
    float sensor_gap;       /* distance between the two sensors of a module */
    float t3_kappa_factor;  /* T3 curvature bound = kappa_max * factor */
    float t3_rz_tol;        /* T3 z residual of the middle anchor */
    float t5_kappa_rel;     /* T5 curvature agreement, relative part */
    float t5_kappa_abs;     /* T5 curvature agreement, absolute part */
    float t5_rz_tol;        /* T5 z residual of the inner anchors */
    float t5_chi2_max;      /* > 0: pre-DNN mode, T5s also need the chi2 of an algebraic
                               circle fit to their five anchors (sigma = hit_sigma) <= this;
                               <= 0: DNN mode, no fit selection (Section 2) */
    float hit_sigma;        /* single-hit resolution */
    float k_field;          /* pT [GeV] = k_field * R [cm] */
    float wp;               /* T5-DNN working point: selected iff score >= wp */
} lst_cuts;

/* T5-DNN weights (Section 2), FP32, PyTorch Linear layout W[out][in], flattened as
 * W0(32x38), b0(32), { Wh(32x32), bh(32) } x (n_hidden-1), Wout(32), bout(1). */
typedef struct lst_mlp {
    int32_t n_hidden;       /* hidden layers of width 32: 1..4 (Section 2 compares 1-4) */
    const float *w;         /* HOST pointer, copied by lst_load_geometry */
} lst_mlp;

typedef struct lst_config {
    int32_t precision;          /* lst_precision of the fused T5 score inside lst_run_event */
    int32_t max_events;         /* event slots (events resident at once), >= 1 */
    int32_t use_graphs;         /* 1: batched runs replay a captured CUDA graph */
    int32_t reserved;
    float md_per_hit;           /* initial capacity ratios of the per-event object buffers; */
    float ls_per_md;            /* they grow automatically after an overflow */
    float t3_per_md;
    float t5_per_md;
} lst_config;

typedef struct lst_ctx_s *lst_ctx;
typedef struct lst_event_s *lst_event;

/* Per-event counters after a run. */
typedef struct lst_counts {
    int64_t n_hits, n_md, n_ls, n_t3, n_t5, n_selected;
    int64_t pairs[4];           /* candidate pairs tested by steps 1-4 (MD, LS, T3, T5) */
    int32_t status;             /* lst_status of the event */
    int32_t overflow_mask;      /* bit k set: buffer of kind k overflowed */
    int64_t n_tc;               /* track candidates (selected T5s after duplicate removal) */
} lst_counts;

/* Fills `cfg` with defaults (FP32 score, 1 slot, graphs on, ratios sized for PU200). */
lst_status lst_default_config(lst_config *cfg);

/* Creates a context on CUDA device `cuda_device`. cfg may be NULL (defaults). */
lst_status lst_create(int cuda_device, const lst_config *cfg, lst_ctx *out);

/* Uploads the detector and model once; they stay resident across events.
 *   mods     HOST [n_mod] module table;
 *   map_off  HOST [n_mod+1], map_tgt HOST [map_off[n_mod]]: module map in CSR form
 *            (Section 1: LSs only across adjacent modules passing geometric criteria);
 *   cuts     HOST cut parameters; weights HOST network (may be NULL: scores = 0.5).
 * Everything is copied; the caller keeps ownership. Errors: LST_ERR_ARG for a malformed
 * table (layer/subdet out of range, map not monotonic, target out of range). */
lst_status lst_load_geometry(lst_ctx ctx, const lst_module *mods, int32_t n_mod,
                             const int32_t *map_off, const int32_t *map_tgt,
                             const lst_cuts *cuts, const lst_mlp *weights);

/* Runs steps 1-4 and the T5-DNN score on one event, one launch sequence per event.
 *   x, y, z  DEVICE float32 [n_hits] global hit coordinates (cm);
 *   sensor   DEVICE int32 [n_hits] sensor id (2*module + 0/1).
 * The work is enqueued on `cuda_stream`; the call then waits for the event's counters
 * (one synchronisation per event) and, if an object buffer overflowed, grows it and
 * re-runs the event, so a successful return always carries complete results.
 * Errors: LST_ERR_INPUT for an invalid hit (no results), LST_ERR_NOT_READY without
 * geometry or a free slot, LST_ERR_ARG for n_hits < 0 or null pointers with n_hits > 0. */
lst_status lst_run_event(lst_ctx ctx, const float *x, const float *y, const float *z,
                         const int32_t *sensor, int64_t n_hits, void *cuda_stream,
                         lst_event *out);

/* Batched form: n_events events (each with its own DEVICE arrays, pointer tables on the
 * HOST) go through one persistent launch per stage; with cfg.use_graphs the launch
 * sequence is a CUDA graph captured once. Asynchronous: returns once the work is
 * enqueued. lst_event_counts / lst_get_candidates wait for it. An event whose buffers
 * overflowed reports LST_ERR_CAPACITY (and grows its slot for the next run). Up to three
 * batches are in flight: consecutive calls take three lanes in turn, and a call first
 * waits for the batch that last ran on its lane (the context needs max_events slots for
 * all events in flight). */
lst_status lst_run_batch(lst_ctx ctx, int32_t n_events, const float *const *x,
                         const float *const *y, const float *const *z,
                         const int32_t *const *sensor, const int64_t *n_hits,
                         void *cuda_stream, lst_event *out);

/* Waits for the event and returns its counters. */
lst_status lst_event_counts(lst_event ev, lst_counts *out);

/* Copies the objects of one kind as hit-index tuples:
 *   hit_idx   [n][2|4|6|10] int32 (MD: lower,upper; LS: 2 MDs; T3: 3 MDs; T5 and TC: 5
 *             MDs, each MD as lower,upper), chain order, original hit indices;
 *   score     [n] float T5-DNN score (T5 and TC only, may be NULL);
 *   selected  [n] uint8 (T5 and TC only, may be NULL): DNN mode score >= wp; pre-DNN mode
 *             (cuts.t5_chi2_max > 0) 1 for every T5, the chi2 cut having selected them.
 * Track candidates (LST_TC): the selected T5s without duplicates. Two selected T5s are
 * duplicates when they share >= 3 of their 5 MDs; the one with the smaller circle-fit chi2
 * (NaN as +inf), then the lexicographically smaller hit tuple, ranks above; a selected
 * T5 is a track candidate iff no selected duplicate ranks above it (one pass).
 * Buffers may be HOST or DEVICE memory (detected). *n_out is always set; if
 * capacity < n the call copies nothing and returns LST_ERR_CAPACITY. Objects come in the
 * library's order; compare as sets. */
lst_status lst_get_candidates(lst_event ev, int32_t kind, int32_t *hit_idx, float *score,
                              uint8_t *selected, int64_t capacity, int64_t *n_out);

/* Batched form of lst_get_candidates for n events of one context (typically the events of
 * one lst_run_batch): the objects of every event, concatenated in event order, with
 * offsets[i] .. offsets[i+1] the rows of event i (offsets HOST [n + 1], always set). One
 * synchronisation for the whole batch; with HOST buffers one copy per array (use pinned
 * memory for full link bandwidth). Events whose status is not LST_OK contribute no rows.
 * LST_ERR_CAPACITY (nothing copied) if capacity < offsets[n]. */
lst_status lst_get_candidates_batch(const lst_event *evs, int32_t n, int32_t kind, int32_t *hit_idx,
                                    float *score, uint8_t *selected, int64_t capacity, int64_t *offsets);

/* The event's LS graph, the GNN input that Section 4 proposes to build with LST: nodes are
 * the MDs (ids = the order of lst_get_candidates(LST_MD)), directed edges the LSs from
 * inner to outer MD, in CSR form by inner MD:
 *   row_off   [n_nodes + 1] int32, row_off[n_nodes] = n_edges;
 *   col       [n_edges] int32 outer-MD ids (edges of one node in no particular order);
 *   node_feat [n_nodes][LST_GRAPH_NODE_FEATURES] float or NULL: anchor (lower-sensor) hit
 *             x, y, z, r in cm, MD curvature in 1/cm (0 for endcap MDs), layer 1..11;
 *   edge_feat [n_edges][LST_GRAPH_EDGE_FEATURES] float or NULL: LS curvature in 1/cm, z in cm
 *             of the anchors' chord at r = 0 (z_a - r_a * ((z_b - z_a) / (r_b - r_a))).
 * All buffers are HOST or all DEVICE memory (detected from row_off); node_cap / edge_cap
 * are the node and edge capacities (row_off holds node_cap + 1 values). *n_nodes and
 * *n_edges are always set; LST_ERR_CAPACITY (nothing copied) if a capacity is too small;
 * row_off NULL: size query only. */
#define LST_GRAPH_NODE_FEATURES 6
#define LST_GRAPH_EDGE_FEATURES 2
lst_status lst_get_ls_graph(lst_event ev, int32_t *row_off, int32_t *col, float *node_feat, float *edge_feat,
                            int64_t node_cap, int64_t edge_cap, int64_t *n_nodes, int64_t *n_edges);

/* Copies the 38 T5-DNN input features of every T5 (Section 2 list) as float [n][38]
 * (HOST or DEVICE); same size protocol as lst_get_candidates. These are the FP32 features
 * the tensor-core precisions read (lst_score_t5 on them reproduces those scores); the
 * LST_FP32 event path uses the float-float features. */
lst_status lst_get_t5_features(lst_event ev, float *feat, int64_t capacity, int64_t *n_out);

/* Scores precomputed features with the loaded network (Section 2):
 *   feat DEVICE float [n][38], score_out DEVICE float [n]; precision LST_FP32 (CUDA cores,
 *   compensated network on the given FP32 features),
 *   LST_BF16 or LST_BF16X3 (tensor cores, see lst_precision). Asynchronous on
 *   cuda_stream; a tensor-core wait that ran out is reported by lst_device_errors. */
lst_status lst_score_t5(lst_ctx ctx, const float *feat, int64_t n, int32_t precision,
                        float *score_out, void *cuda_stream);

/* Waits for the device and returns LST_ERR_TIMEOUT if a bounded device-side wait (the
 * tensor-core score kernels wait for their MMAs with an iteration limit) ran out since the
 * last call, else LST_OK; clears the condition. Events of a batch whose score wait ran out
 * report LST_ERR_TIMEOUT themselves. */
lst_status lst_device_errors(lst_ctx ctx);

/* Iteration limit of those device-side waits (default 2^26 polls). */
lst_status lst_set_wait_limit(lst_ctx ctx, int64_t iterations);

/* Test aid for the failure handling above (no counterpart in the paper). With on != 0 the
 * tensor-core score kernels issue no MMA, so nothing ever arrives on the barrier they wait
 * on: after the wait limit each CTA records LST_ERR_TIMEOUT, frees its tensor memory and
 * returns, with nothing left in flight. The events of such a launch report
 * LST_ERR_TIMEOUT, lst_device_errors returns it, and the context stays usable (on = 0
 * restores normal scoring). */
lst_status lst_test_skip_mma(lst_ctx ctx, int32_t on);

/* Test aid for allocation failures (no counterpart in the paper). The next n allocations
 * of event buffers (an event slot's object arena when it is created or grown, and the
 * device staging of host inputs) fail as cudaMalloc fails when the device is out of
 * memory: the call that needed the buffer returns LST_ERR_NOMEM, no event is produced,
 * the slot stays free with no buffer, and the next call allocates normally. n = 0 clears
 * pending failures. */
lst_status lst_test_fail_alloc(lst_ctx ctx, int32_t n);

/* Returns the event's slot to the context. */
lst_status lst_event_release(lst_event ev);

/* Frees everything the context owns (waits for its work first). */
lst_status lst_destroy(lst_ctx ctx);

/* Static text of a status code; never NULL. */
const char *lst_status_str(int32_t status);

/* Last error message of the calling thread (CUDA error string, argument check). */
const char *lst_last_error(void);

/* Launch shapes of the stage kernels (threads per CTA, shared-memory list and staging
 * sizes). lst_set_launch validates (threads a multiple of 32 in 32..256, sizes >= 1, the
 * shared memory within the device limit) and recomputes the persistent grid sizes; the
 * results never depend on these values, only the speed does. */
typedef struct lst_launch {
    int32_t md_threads, md_buf;    /* step 1: CTA size; md_buf is unused (kept for layout) */
    int32_t ls_threads, ls_list;   /* step 2: CTA size; ls_list is unused (kept for layout) */
    int32_t t3_threads;            /* step 3: CTA size */
    int32_t t5_threads;            /* step 4: CTA size */
    int32_t sc_threads;            /* score: CTA size */
    int32_t t3_mds;                /* step 3: middle MDs per warp unit, 1..32; 0 = chosen per
                                      launch from its event count */
} lst_launch;
lst_status lst_get_launch(lst_ctx ctx, lst_launch *out);
lst_status lst_set_launch(lst_ctx ctx, const lst_launch *in);

/* Per-stage device timing. lst_set_timing(ctx, 1) resets the statistics and makes every
 * later launch (lst_run_event and lst_run_batch, graph launches included) record CUDA
 * events at the stage boundaries on the launch stream. lst_stage_times fills ms[LST_N_STAGES]
 * with the mean device time per launch of each stage in ms (0 bin, 1 md, 2 ls, 3 ls_group,
 * 4 t3, 5 t5, 6 score, 7 track candidates) and returns the number of launches averaged. */
lst_status lst_set_timing(lst_ctx ctx, int32_t enable);
lst_status lst_stage_times(lst_ctx ctx, float *ms, int64_t *n_launches);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching of events that arrive one by one (Section 3 runs events
 * concurrently on CUDA streams; here events share batched launches instead).
 * Two worker threads own the context while the server runs (make no other call on it):
 * one admits, stages and launches, the other completes batches and exports their results.
 * Requests are admitted in arrival order when an event slot is free and the estimated
 * object-buffer memory of all admitted events stays within mem_budget_bytes (a single
 * event is always admitted when nothing else is). Admitted events go to the GPU in
 * batches of up to max_batch (one launch per stage, CUDA graph, captured for every batch
 * size when the server starts) on `lanes` streams, so a new batch starts while the
 * previous one is still running.
 *   submit: x, y, z, sensor are HOST arrays that must stay valid until the request's
 *           result has been polled; t_arrival is the request time on lst_clock() (<= 0:
 *           now); the latency of a request is t_done - t_arrival, t_done being the time
 *           its results reached host memory (the library's pinned staging).
 *   poll:   returns up to `max` finished requests (waiting up to wait_ms for the first);
 *           when copy_t5 is set, a result's T5 arrays point into the pinned host staging
 *           its batch was exported to (no copy is made) and stay valid until
 *           lst_serve_free_result(result), which every polled result needs. A batch's
 *           staging (about 45 bytes per T5) is reused once all its results are freed; a
 *           caller that holds results or stops polling makes the library allocate more.
 *   free_result: releases the result's hold on its staging; results may be freed after
 *           lst_serve_stop (the last one frees the staging of a stopped server).
 *   stop:   finishes every submitted request, then joins the workers. */
typedef struct lst_serve_config {
    int32_t max_batch;          /* events per batched launch, 1..max_events */
    int32_t lanes;              /* batches in flight: 1 or 2 */
    int64_t mem_budget_bytes;   /* admission budget (estimated device bytes of admitted events) */
    int32_t copy_t5;            /* 1: results carry the T5 hit tuples, scores, selection */
    int32_t slot_hits;          /* > 0: every event slot is sized at start for this many hits
                                   (growing a slot while serving can pause the workers for
                                   the memory mapping); 0: slots are sized as events need */
} lst_serve_config;

typedef struct lst_serve_result {
    uint64_t tag;               /* the caller's tag */
    int32_t status;             /* lst_status of the event */
    int32_t reserved;
    lst_counts counts;
    double t_arrival, t_admit, t_launch, t_done;   /* lst_clock() seconds */
    int64_t n_t5;
    int32_t *t5_hits;           /* HOST [n_t5][10], in the library's pinned staging */
    float *t5_score;            /* HOST [n_t5], likewise */
    uint8_t *t5_sel;            /* HOST [n_t5], likewise */
    void *owner;                /* the staging the arrays belong to (library use) */
} lst_serve_result;

typedef struct lst_server_s *lst_server;

/* Monotonic clock of the library, seconds. */
double lst_clock(void);
lst_status lst_serve_start(lst_ctx ctx, const lst_serve_config *cfg, lst_server *out);
lst_status lst_serve_submit(lst_server s, const float *x, const float *y, const float *z,
                            const int32_t *sensor, int64_t n_hits, uint64_t tag, double t_arrival);
lst_status lst_serve_poll(lst_server s, lst_serve_result *out, int32_t max, int32_t *n_out,
                          int32_t wait_ms);
lst_status lst_serve_free_result(lst_serve_result *r);
lst_status lst_serve_stop(lst_server s);

/* ---------------------------------------------------------------------------------
 * Pixel seeds: Table 1 steps 0 and 5-8 (Section 1).
 *
 * Step 0 makes pixel seeds (pLSs) upstream from the inner tracker; each is four hits H1..H4
 * (inner first). lst_match_pixel_seeds matches them to the outer-tracker objects of a
 * finished event and forms the four mutually exclusive track-candidate types, longest
 * first:
 *   5 pT5: a track-candidate T5 (LST_TC) matched to a seed;
 *   6 T5:  a track-candidate T5 matched to no seed;
 *   7 pT3: a seed not in a pT5 matched to a T3 that is not in a pT5 (a T3 is in a pT5 when
 *          each of its three MDs is an MD of a pT5's T5);
 *   8 pLS: a seed in neither.
 * A seed matches an object (the T5 by its first T3, or the T3) whose first anchors are P0,
 * P1 and whose curvature is ko when (project specification, FP32):
 *   azimuth window  H4 . P0 > 0 and |H4 x P0| <= (dphi0 + dphi_cm (r(P0) - r4)) r4 r(P0)
 *                   (transverse; the sine of the turn of azimuth from H4 to P0);
 *   slope window    |m_p - m_o| <= dm_abs + dm_rel |m_o|, m_p = (z4 - z1) / (r4 - r1),
 *                   m_o = (z(P1) - z(P0)) / (r(P1) - r(P0));
 *   pT              |kp - ko| <= kappa_rel (|kp| + |ko|) / 2 + kappa_abs, kp the signed
 *                   three-point curvature through H1, H3, H4;
 *   circle          the same for kx, the curvature through H1, H4, P0;
 *   rz              |z4 - zp| <= rz_tol, zp = z1 + (z(P0) - z1) s14 / (s14 + s40) with arc
 *                   lengths s = d (1 + d^2 kbar^2 / 24) of the chords H1H4 and H4P0, kbar =
 *                   (kx + ko) / 2.
 * Matching is one-to-one: the matching pairs in ascending order of (the rz residual |z4 -
 * zp|, |kx - ko|, seed index, the object's hit tuple), each taken when both are still free
 * (first for the T5s, then for the T3s with the seeds left). */
typedef struct lst_pixel_cuts {
    float kappa_rel, kappa_abs, rz_tol, dphi0, dphi_cm, dm_abs, dm_rel;
} lst_pixel_cuts;

typedef struct lst_pixel_counts {
    int64_t n_rows;                 /* track candidates of steps 5-8 */
    int64_t n_pt5, n_t5, n_pt3, n_pls;
    int32_t rounds_pt5, rounds_pt3; /* matching rounds taken (the GPU's one-to-one passes) */
} lst_pixel_counts;

/*   ev        a finished event (lst_run_event or lst_run_batch) with status LST_OK;
 *   seeds     float [n_seeds][4][3]: (x, y, z) of H1..H4 per seed, host or device, read
 *             before the call returns;
 *   pc        matching parameters (copied; all non-negative, else LST_ERR_ARG);
 *   counts    host, may be NULL.
 * Synchronous: returns when the track candidates are ready (lst_get_pixel_candidates); a
 * later call on the same event replaces them. LST_ERR_CAPACITY if more than 8 objects tie
 * at one seed in both ranking measures (the order would then rest on too long a list). */
lst_status lst_match_pixel_seeds(lst_event ev, const float *seeds, int64_t n_seeds, const lst_pixel_cuts *pc,
                                 lst_pixel_counts *counts);

/* The same for n events of one context at once (distinct events; the results are those of
 * n single calls): seeds[i], n_seeds[i] belong to evs[i]; counts, if not NULL, has n
 * entries. One launch per kernel and round covers all n events; rounds go out three at a
 * time and the host then waits once for the whole batch (an event whose round took no pair
 * is done with the stage, and its later rounds return at once). n within 1..max_events,
 * else LST_ERR_ARG. */
lst_status lst_match_pixel_seeds_batch(const lst_event *evs, int32_t n, const float *const *seeds,
                                       const int64_t *n_seeds, const lst_pixel_cuts *pc,
                                       lst_pixel_counts *counts);

/* The track candidates of the event's last lst_match_pixel_seeds call, one row of three
 * int32 each, in no particular order: (type 5..8, seed index or -1 for type 6, object
 * index or -1 for type 8), the object index being the row of the T5 in
 * lst_get_candidates(LST_T5) (types 5, 6) or of the T3 in lst_get_candidates(LST_T3)
 * (type 7). rows host or device; n_out always set; LST_ERR_CAPACITY if capacity < n_out,
 * LST_ERR_NOT_READY if the event was not matched. */
lst_status lst_get_pixel_candidates(lst_event ev, int32_t *rows, int64_t capacity, int64_t *n_out);

/* ---------------------------------------------------------------------------------
 * Mini-doublet finder that allocates nothing (the paper has no counterpart; it is a
 * deployment aid of this library).
 *
 * For callers that cannot call cudaMalloc/cudaFree while they run: a host framework
 * that owns all device memory through its own caching allocator (a foreign cudaFree
 * synchronises the device), trigger or real-time loops whose latency budget cannot
 * absorb that synchronisation, or code that enqueues work while a global-mode stream
 * capture is active elsewhere in the process (allocation is prohibited then).
 *
 * Does steps 0-1 (hit grouping by sensor, then every mini-doublet of the event, with
 * the same FP32 cuts as lst_run_event) using only a fixed scratch array compiled into
 * the library: LST_NOALLOC_SCRATCH_BYTES (about 10.3 MiB) of device memory that every
 * GPU loading the library holds until the process exits. Limits: n_hits <=
 * LST_NOALLOC_MAX_HITS and 2 * n_mod <= LST_NOALLOC_MAX_SENSORS; larger requests return
 * LST_ERR_ARG before any GPU work (lst_last_error says which limit).
 *   ctx       a context with geometry loaded (lst_load_geometry);
 *   x,y,z,sensor  DEVICE hit arrays as in lst_run_event;
 *   md_hits   DEVICE int32 [capacity][2] (lower, upper) original hit indices, caller-owned;
 *   md_kappa  DEVICE float [capacity] MD curvature estimate (0 for endcap), may be NULL;
 *   md_count  DEVICE int64 [1]: number of MDs found (may exceed capacity: then only
 *             `capacity` of them, in unspecified order, were written), or -1 if a hit had
 *             an invalid sensor id or a non-finite coordinate.
 * Asynchronous on cuda_stream; MDs come in no particular order (compare as sets).
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and the device's SM count, which sizes
 * the grids; make that first call before any stream capture. Every call reuses the same scratch and clears what must start at
 * zero; calls that overlap on the GPU (other streams, other threads) race on it and
 * must be serialised by the caller. */
#define LST_NOALLOC_MAX_HITS 524288
#define LST_NOALLOC_MAX_SENSORS 32768
#define LST_NOALLOC_SCRATCH_BYTES 10748416
lst_status lst_find_minidoublets_noalloc(lst_ctx ctx, const float *x, const float *y, const float *z,
                                         const int32_t *sensor, int64_t n_hits, int32_t *md_hits,
                                         float *md_kappa, int64_t capacity, int64_t *md_count,
                                         void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LST_H */

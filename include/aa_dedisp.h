/*
 * aa_dedisp.h -- C ABI of the GB300 (sm_103a) brute-force dedispersion and
 * single-pulse search library (libaa_gb300.so).
 *
 * Pipeline (arXiv:1912.07704, Sec. 1): dedisperse a uint8 filterbank
 * (channels x time) over a multi-range DM plan with per-range time
 * decimation, then run the single-pulse search (boxcar filters + peak
 * finding) on every dedispersed series, keeping the data on the GPU between
 * the two stages.
 *
 * API shape follows the paper's design:
 *   - a plan carries the search parameters and metadata; the library derives
 *     from it an immutable, queryable strategy (Sec. 3.1, 3.2);
 *   - configuration is separate from device memory: every device buffer the
 *     library will use can be queried before anything is allocated
 *     (Sec. 2.3);
 *   - the caller owns the host input and the library never writes it; the
 *     library owns the device buffers and the results it returns (Sec. 2.4);
 *   - every call returns a status code; configuration errors are reported,
 *     never thrown (Sec. 3.1, 3.3).
 *
 * Method (brute force, exact integers):
 *   f_c      = fch1 + c*foff (MHz),  f_top = highest channel frequency
 *   DM_i     = dm_lo + i*dm_step           (double; not accumulated)
 *   s_r(c,i) = round_half_away(((4.148808e3*DM_i)*(f_c^-2 - f_top^-2))
 *                              / (tsamp*dec_r))   (decimated samples; double)
 *   x_r[c][j]= sum_{k<dec_r} x[c][j*dec_r+k],  j < floor(T/dec_r)
 *   y_r[i][t]= sum_c x_r[c][t + s_r(c,i)],      t < L_r = floor(T/dec_r) - max s_r
 *   SNR_w(t) = (sum_{k<w} y[t+k] - w*mu) / (sigma*sqrt(w)),  1 <= w <= min(W, L_r-t)
 *              (mu, sigma: population mean/std of that series)
 *   B(t)     = max_w SNR_w(t);  candidate iff B(t) >= thr, B(t) > B(t-1),
 *              B(t) >= B(t+1) (missing neighbours are -inf).
 *   A series with sigma == 0 yields no candidates.
 *
 * Threading: a plan may be used from one host thread at a time.  Device
 * calls are stream-ordered on the given stream (NULL = legacy default).
 */
#ifndef AA_DEDISP_H
#define AA_DEDISP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* aa_stream_t;

/* Status codes (Sec. 3.3: every iteration/call reports success, pending work
 * or an error). */
typedef enum aa_status {
    AA_OK = 0,
    AA_PENDING = 1,             /* streaming: chunk accepted, more input needed */
    AA_WARN_CAND_OVERFLOW = 2,  /* more candidates than capacity; the count holds
                                   the true total, the first `capacity` stored
                                   (which ones is unspecified) */
    AA_ERR_CONFIG = -1,         /* invalid plan description */
    AA_ERR_NOMEM = -2,          /* device or host allocation failed */
    AA_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    AA_ERR_TIMEOUT = -4,        /* a bounded device-side wait gave up */
    AA_ERR_STATE = -5,          /* call not valid in the object's current state */
    AA_ERR_ARG = -6             /* invalid argument (NULL, size, alignment) */
} aa_status;

/* Static string for a status code (never NULL). */
const char* aa_status_str(aa_status s);

/* Human-readable detail of the last failing call on this host thread
 * (empty string if none).  Valid until the next library call on the thread. */
const char* aa_last_error(void);

/* ------------------------------------------------------------------ plan -- */

/* One DM range: ndm trials DM_i = dm_lo + i*dm_step, searched on the input
 * decimated (summed) by `dec` in time.  Requirements: ndm >= 1, dm_lo >= 0,
 * dm_step >= 0, 1 <= dec <= 16. */
typedef struct aa_dm_range {
    double dm_lo;
    double dm_step;
    int32_t ndm;
    int32_t dec;
} aa_dm_range;

/* Plan description (Sec. 3.1 "plan": search parameters and metadata).
 * nchans >= 1; fch1_mhz > 0 and every channel frequency > 0; foff_mhz != 0;
 * tsamp_s > 0; 1 <= nranges <= 64; nchans*255*max(dec) < 2^24 (so that every
 * dedispersed sample is an exact integer in FP32).  `ranges` is read during
 * aa_plan_create only (the caller keeps ownership). */
typedef struct aa_plan_desc {
    int32_t nchans;
    double fch1_mhz;
    double foff_mhz;
    double tsamp_s;
    int32_t nranges;
    const aa_dm_range* ranges;
} aa_plan_desc;

typedef struct aa_plan aa_plan;
typedef struct aa_dd_result aa_dd_result;    /* library-owned dedispersed output */
typedef struct aa_candidates aa_candidates;  /* library-owned host candidate list */

/* Validate `desc`, build the FP64 delay tables and the strategy (tile shapes,
 * shared-memory sizes).  Host only: no device memory is touched.
 * Returns AA_ERR_ARG if desc/out is NULL, AA_ERR_CONFIG (with
 * aa_last_error() detail) if the description is invalid, AA_ERR_NOMEM on host
 * allocation failure.  On failure *out is set to NULL. */
aa_status aa_plan_create(const aa_plan_desc* desc, aa_plan** out);

/* Release the plan and every device buffer it owns (delay tables).  NULL is a
 * no-op.  Work using the plan must have completed. */
void aa_plan_destroy(aa_plan* plan);

/* Bind the plan to a CUDA device (Sec. 3.1 usage step 4): uploads the delay
 * tables (device memory owned by the plan) and marks the plan ready.  Must be
 * called before any device entry point; the high-level aa_dedisperse binds to
 * the current device itself if needed.  Rebinding to another device is
 * AA_ERR_STATE. */
aa_status aa_plan_bind(aa_plan* plan, int device);

/* Per-range layout for an input of `nsamp` full-rate samples. */
typedef struct aa_range_info {
    int32_t ndm;         /* trials in this range */
    int32_t dec;         /* time decimation */
    int32_t maxshift;    /* largest delay, decimated samples */
    int32_t dm_offset;   /* global index of this range's first trial */
    double dm_lo;
    double dm_step;
    int64_t nsamp_dec;   /* floor(nsamp/dec) */
    int64_t length;      /* L = max(0, nsamp_dec - maxshift): output samples per trial
                            (maxshift: largest effective delay of the strategy in use) */
    int64_t pitch;       /* floats between consecutive output rows (multiple of 64) */
    int64_t row_offset;  /* float offset of this range's row 0 in the output buffer */
    /* strategy (fixed at aa_plan_create) */
    int32_t tile_dms;        /* DM trials per dedispersion CTA */
    int32_t tile_samples;    /* output samples per dedispersion CTA */
    int32_t stage_channels;  /* direct strategy: channel rows per shared-memory stage;
                                grouped: channels per chunk whose delay patterns are
                                grouped (1024 for 8-bit, 4096 for decimated input) */
    int32_t stages;          /* pipeline depth of the staging copies */
    int32_t span_max;        /* largest delay spread across one CTA's trials */
    int32_t smem_bytes;      /* dynamic shared memory per dedispersion CTA */
    int32_t strategy;        /* aa_dedisp_strategy in use for this range */
    int32_t grouped_available;  /* 1 if AA_DEDISP_GROUPED can be selected */
    double grouped_work;     /* adds of the grouped strategy / adds of the direct one */
    int32_t subband_channels;       /* AA_DEDISP_SUBBAND: channels per band (else 0) */
    int32_t subband_coarse_trials;  /* AA_DEDISP_SUBBAND: fine trials per coarse trial */
    double subband_work;     /* adds of the sub-band strategy / adds of the direct one */
    int32_t fdmt_depths;     /* AA_DEDISP_FDMT: merge levels of the channel tree (else 0) */
    int32_t fdmt_max_rows;   /* AA_DEDISP_FDMT: rows of its largest intermediate level */
    double fdmt_work;        /* adds of the FDMT strategy / adds of the direct one */
} aa_range_info;

/* Strategy and memory requests for `nsamp` samples and boxcar widths up to
 * `max_width` (0 if the single-pulse search will not be run).  Pure host
 * computation (Sec. 2.3: memory is requested before it is allocated; Sec. 3.2:
 * the strategy and the ready state can be queried). */
typedef struct aa_plan_info {
    int32_t nchans;
    int32_t nranges;
    int32_t ndm_total;
    int32_t ready;             /* 1 once aa_plan_bind succeeded */
    int32_t device;            /* bound device, -1 if none */
    int32_t max_width;
    int64_t nsamp;
    int64_t in_pitch_min;      /* minimum device input row pitch, bytes (nsamp rounded up to 16) */
    int64_t dd_elems;          /* floats in the dedispersed output buffer */
    int64_t dedisp_ws_bytes;   /* scratch for aa_dedisperse_device */
    int64_t sps_ws_bytes;      /* scratch for aa_sps_search_device at max_width */
    int64_t table_bytes;       /* device delay tables owned by the plan */
    int64_t host_path_bytes;   /* peak device bytes of aa_dedisperse + aa_sps_search */
    int64_t dm_trial_samples;  /* sum over ranges of ndm * L */
    double dm_max;             /* largest trial DM */
    int64_t f32_ws_bytes;      /* scratch for the differentiable-form calls */
} aa_plan_info;

aa_status aa_plan_query(const aa_plan* plan, int64_t nsamp, int32_t max_width,
                        aa_plan_info* info);

/* Layout of range r (0 <= r < nranges) for `nsamp` samples. */
aa_status aa_plan_range(const aa_plan* plan, int64_t nsamp, int32_t r, aa_range_info* info);

/* Effective delay table [ndm][nchans] (decimated samples) of range r under
 * the strategy in use: the brute-force delays for the direct and grouped
 * strategies (= aa_plan_shifts), the band reference's delay plus the
 * channel's delay within its band for sub-band ranges, the delays the tree's
 * splits give for FDMT ranges.  Host only.  AA_ERR_ARG for a bad range, NULL
 * out or cap < ndm x nchans. */
aa_status aa_plan_effective_shifts(const aa_plan* plan, int32_t r, int32_t* out, int64_t cap);

/* Copy range r's delay table, int32 [ndm][nchans] row-major (decimated
 * samples), into caller-owned host memory `out` (capacity `cap` elements). */
aa_status aa_plan_shifts(const aa_plan* plan, int32_t r, int32_t* out, int64_t cap);

/* ----------------------------------------------------- device entry points -- */

/* Candidate record (16 bytes).  dm_index: global trial index (ranges
 * concatenated in plan order); t: sample index in that range's decimated
 * series (start of the boxcar window); width: boxcar width in samples of that
 * series; range: range index; reserved: 0 (beam index in batched runs);
 * snr: B(t). */
typedef struct aa_candidate {
    uint32_t dm_index;
    uint32_t t;
    uint16_t width;
    uint8_t range;
    uint8_t reserved;
    float snr;
} aa_candidate;

/* Dedisperse a device-resident filterbank.
 *   d_in     : uint8 [nchans][in_pitch] device memory, first nsamp bytes of
 *              each row valid; in_pitch % 16 == 0, in_pitch >= nsamp; base
 *              16-byte aligned.  Read only.
 *   d_out    : float [dd_elems] device memory (aa_plan_info.dd_elems);
 *              range r, trial i, sample t is at row_offset_r + i*pitch_r + t
 *              for t < L_r (exact integers); padding is left unwritten.
 *   d_ws     : device scratch of ws_bytes >= dedisp_ws_bytes (may be NULL if
 *              that is 0), 256-byte aligned.
 * The plan must be bound.  Stream-ordered, asynchronous; returns
 * AA_ERR_ARG/AA_ERR_STATE on bad arguments, AA_ERR_CUDA if a launch fails. */
aa_status aa_dedisperse_device(const aa_plan* plan, const uint8_t* d_in, int64_t nsamp,
                               int64_t in_pitch, float* d_out, void* d_ws, size_t ws_bytes,
                               aa_stream_t stream);

/* Single-pulse search over every dedispersed series in d_dd (layout as
 * written by aa_dedisperse_device for the same nsamp).
 *   max_width      : W >= 1, boxcar widths 1..W (in samples of each range);
 *   threshold      : SNR threshold;
 *   d_cands        : device array of cand_capacity records (may be NULL iff
 *                    cand_capacity == 0);
 *   d_count        : device uint64, set to the total number of candidates
 *                    (may exceed cand_capacity); records are unordered;
 *   d_snr_out      : optional float [dd_elems] device buffer receiving B(t)
 *                    for every t < L_r (NULL to skip);
 *   d_ws           : scratch of ws_bytes >= sps_ws_bytes for this max_width.
 * Stream-ordered, asynchronous. */
aa_status aa_sps_search_device(const aa_plan* plan, int64_t nsamp, const float* d_dd,
                               int32_t max_width, float threshold, aa_candidate* d_cands,
                               int64_t cand_capacity, unsigned long long* d_count,
                               float* d_snr_out, void* d_ws, size_t ws_bytes,
                               aa_stream_t stream);

/* Width-samples the last aa_sps_search_device call on this workspace actually
 * evaluated (width blocks whose SNR bound is below the threshold are skipped
 * when no B(t) output is requested).  Synchronises `stream`. */
aa_status aa_sps_workspace_work(const void* d_ws, aa_stream_t stream, int64_t* evaluated);

/* Read and clear the device error word kept at the start of a workspace used
 * by the calls above (synchronises `stream`).  AA_OK, or AA_ERR_TIMEOUT if a
 * bounded device-side wait gave up. */
aa_status aa_workspace_status(void* d_ws, aa_stream_t stream);

/* ------------------------------------------------------------ autotuner -- */

/* How a range's dedispersion is computed; the result is identical (exact
 * integer sums, only their grouping differs).  No counterpart in the paper,
 * which leaves the kernel to the library.
 *   AA_DEDISP_DIRECT:  every trial adds every channel (shift-and-sum).
 *   AA_DEDISP_GROUPED: within a block of 16 trials and a chunk of channels,
 *     channels whose delays differ from the block's first trial by the same
 *     amounts at every trial are first summed once; each trial then adds the
 *     group sums.  Available when the plan could build the group tables. */
typedef enum { AA_DEDISP_DIRECT = 0, AA_DEDISP_GROUPED = 1, AA_DEDISP_SUBBAND = 2,
               AA_DEDISP_FDMT = 3 } aa_dedisp_strategy;

/* Sub-band dedispersion of range r (AA_DEDISP_SUBBAND): an approximation of
 * the brute-force sum with fewer adds, the cheaper-than-brute-force family
 * the dedispersion module's cited work belongs to (Sec. 1).  Channels form
 * bands of band_channels consecutive channels (the last may be shorter), each
 * with a reference channel: its highest-frequency channel c_b.  Fine trials
 * form coarse trials of coarse_trials consecutive trials (the last may be
 * shorter) whose DM D_j is that of their middle trial i_j = j*m + (n_j-1)/2.
 *   stage 1: z[b][j][t] = sum_{c in band b} x[c][t + r(c, j)],
 *            r(c, j) = round_half_away(((k_DM*D_j)*(delta_c - delta_cb))/(tsamp*dec)),
 *            delta_c = f_c^-2 - f_top^-2 (the plan's delay arithmetic);
 *   stage 2: y[i][t] = sum_b z[b][j(i)][t + s(c_b, i)], s the plan's delays,
 * i.e. channel c of trial i is taken at the effective delay
 * s(c_b, i) + r(c, j(i)) instead of s(c, i).  Sums stay exact integers.  The
 * range's maxshift becomes max r + max s(c_b, .) and its length
 * nsamp_dec - maxshift.  Adds per trial-sample: nchans/coarse_trials + nbands.
 * Stage 1 stores 16-bit partial sums; stage 2 adds them in 32 bits.
 * AA_ERR_ARG for a bad range, band_channels outside [1, nchans] or
 * coarse_trials outside [1, 16]; AA_ERR_CONFIG when band_channels * 255 * dec
 * > 65535 (the 16-bit partial sums) or stage 1 does not fit the dedispersion
 * tile.  aa_plan_set_strategy returns the range to an exact strategy.  Not
 * available in batched runs (aa_batch_create returns AA_ERR_CONFIG) nor in
 * the differentiable form; the autotuner leaves such ranges alone.  Like
 * aa_plan_set_strategy, call it while no work of the plan is in flight. */
aa_status aa_plan_set_subband(aa_plan* plan, int32_t r, int32_t band_channels,
                              int32_t coarse_trials);

/* FDMT-style tree dedispersion of range r (AA_DEDISP_FDMT): an
 * approximation of the brute-force sum (the dedispersion module's cited
 * work, Sec. 1) whose adds per output sample grow with log2(nchans) and the
 * range's delay span instead of nchans x ndm: the channels, in
 * falling-frequency order, form a binary tree of subbands (subband [a, b]
 * split at a + ceil((b - a + 1) / 2)); a subband's series at delay delta
 * (its last channel relative to its first) is its upper half's series at
 * delay round(delta (d[m-1] - d[a]) / (d[b] - d[a])) plus its lower half's
 * at delay delta - gap, read gap = round(delta (d[m] - d[a]) / (d[b] - d[a]))
 * samples later (d = f^-2 - f_top^-2, rounding half away from zero, FP64);
 * a single channel has delay 0.  Trial i of the range takes the whole band at
 * delay D_i = its bottom channel's brute-force delay, so the output length
 * is the brute-force one; every other channel's effective delay stays within
 * a closed-form bound of its brute-force delay (about log2(nchans) / 2 + log2(nchans)^2 / 4
 * samples).  Sums are exact integers (32-bit intermediate rows, FP32 output).
 * The workspace grows by two depth buffers (aa_plan_query dedisp_ws_bytes;
 * aa_range_info fdmt_max_rows rows each).  Not available in batched runs.
 * AA_ERR_ARG for a bad range, AA_ERR_CONFIG if sums could exceed 31 bits,
 * AA_ERR_NOMEM if a bound plan cannot upload the tree. */
aa_status aa_plan_set_fdmt(aa_plan* plan, int32_t r);

/* Select the strategy of range r (aa_plan_create picks one from the number
 * of adds each needs).  AA_ERR_ARG for a bad range or strategy value,
 * AA_ERR_CONFIG if the grouped tables are not available for that range.
 * Like aa_plan_autotune, call it while no work of the plan is in flight. */
aa_status aa_plan_set_strategy(aa_plan* plan, int32_t r, int32_t strategy);

/* Sparse width ladder for the single-pulse search: an approximation that
 * evaluates only some boxcar widths when W is large (the cited search method
 * covers large widths sparsely; Sec. 1 names boxcar filters with peak
 * finding).  Widths form chunks of 16 (chunk c = widths 16c+1 .. 16c+16);
 * chunks 0-3 (widths 1..64) always take part, then chunk c_0 = 4 and
 * c_{n+1} = max(c_n + 1, ceil(c_n * growth_x16 / 16)), i.e. chunk starts
 * growing geometrically by growth_x16/16.  B(t) is then the largest SNR over
 * the widths taking part and a candidate's width the smallest of them
 * reaching it.  growth_x16 = 0 restores every width 1..W (the default);
 * otherwise it must lie in [17, 64].  Applies to the searches started (and
 * batches created) after the call.  AA_ERR_ARG for other values,
 * AA_ERR_CONFIG while the decimated ladder (aa_plan_set_sps_decimated) is on. */
aa_status aa_plan_set_sps_ladder(aa_plan* plan, int32_t growth_x16);

/* Decimated width ladder for the single-pulse search: an approximation for
 * wide boxcars (the cited search method evaluates them on the dedispersed
 * series decimated by pairs; Sec. 1 names boxcar filters with peak finding).
 * With base_widths = W0: every width 1..min(W0, W) at every start t
 * (level 0), and for each level k >= 1 with W0 * 2^(k-1) < W the widths
 * m * 2^k, W0/2 < m <= W0, m * 2^k <= W, of the window that starts at the
 * level-k grid point floor(t / 2^k) * 2^k <= t (m samples of the series
 * decimated k times by pairs), each window inside [0, L).  B(t) is the
 * largest SNR over those windows (SNR as in the exhaustive search, with the
 * row's mean and standard deviation), a candidate's width the smallest width
 * reaching it; a wide window's value holds over its level's grid cell, and
 * a candidate sits at the first sample of the cell (peaks as usual: B >= thr,
 * B(t) > B(t-1), B(t) >= B(t+1)).  Evaluates about W0 + W0/2 widths per start
 * instead of W.  base_widths = 0 restores every width (the default);
 * otherwise a power of two in [16, 256].  AA_ERR_ARG for other values,
 * AA_ERR_CONFIG while the sparse ladder (aa_plan_set_sps_ladder) is on.
 * Applies to searches started (and batches created) after the call. */
aa_status aa_plan_set_sps_decimated(aa_plan* plan, int32_t base_widths);

/* Robust statistics for the single-pulse search (outlier rejection).  The
 * mean and standard deviation that normalise each dedispersed series' SNR
 * (Sec. 1: boxcar filters with peak finding) are by default those of all its
 * samples.  With max_iters > 0 they are those of iterative k-sigma clipping,
 * k = c16 / 16 with c16 in [1, 255]: the first pass takes every sample; each
 * further pass keeps the samples y with |y - mu| <= k*sigma of the previous
 * kept set (bounds inclusive, population sigma), decided exactly in integers
 * as 256 (N y - S1)^2 <= c16^2 (N S2 - S1^2) over that set's count N,
 * S1 = sum y and S2 = sum y^2; at most max_iters such passes, ending early at
 * a fixed point (same N, S1, S2); a pass that keeps nothing is dropped.
 * No counterpart in the paper's text, which cites the search method; the
 * clipping rule is this library's.  max_iters = 0 restores the plain
 * statistics.  Applies to the searches started and batches created after the
 * call (device, host, no-allocation, streaming and batched paths).
 * AA_ERR_ARG for max_iters outside [0, 64], or c16 outside [1, 255] with
 * max_iters > 0.  While clipping is on, searches of series of 2^31 samples or
 * more return AA_ERR_CONFIG. */
aa_status aa_plan_set_sps_clip(aa_plan* plan, int32_t c16, int32_t max_iters);

/* Time the dedispersion kernel of every range of a bound plan over a
 * synthetic probe input of nsamp_probe samples for the grouped strategy (if
 * available) and each feasible direct tile shape (channels per shared-memory
 * stage x staging depth) and keep the fastest in the plan's strategy.  Call before the plan's first dedispersion (the
 * strategy is fixed from then on).  cache_path: optional text file; shapes
 * found there (keyed by GPU model, SM count, channels, decimation and the
 * staged row size) are applied without timing, new results are appended.
 * The probe buffers are allocated and freed inside the call. */
aa_status aa_plan_autotune(aa_plan* plan, int64_t nsamp_probe, const char* cache_path);

/* ------------------------------------------------------ batched beams -- */

/* Many independent beams (each with its own plan and length) searched by one
 * CUDA graph.  Beams are grouped into waves whose working set fits
 * wave_budget_bytes (<= 0: half of the free device memory) and waves reuse
 * one buffer region; within a wave the graph issues each beam's kernels on 8
 * concurrent branches (see aa_batch_set_branches for the other form).
 * Plans are bound to the current device if needed; they must stay alive
 * while the batch exists.  The library allocates all device memory at
 * creation (inputs included: see aa_batch_input).  nbeams <= 256. */
typedef struct aa_batch aa_batch;
aa_status aa_batch_create(aa_plan* const* plans, const int64_t* nsamps, int32_t nbeams,
                          int32_t max_width, float threshold, int64_t cand_capacity,
                          int64_t wave_budget_bytes, aa_batch** out);
void aa_batch_destroy(aa_batch* batch);

/* Library-owned device input of a beam: uint8 [nchans][pitch] (first nsamp
 * bytes of each row are read).  The caller fills it before aa_batch_run. */
aa_status aa_batch_input(aa_batch* batch, int32_t beam, uint8_t** d_in, int64_t* pitch);

/* The dedispersed series of a beam after aa_batch_run has completed (until
 * the next run), in the layout aa_dedisperse_device writes for that beam's
 * plan and nsamp (aa_plan_query), library-owned, read-only.  Only beams of
 * the batch's last wave keep their series (earlier waves share the region):
 * AA_ERR_STATE for the others, AA_ERR_ARG for a bad beam or NULL d_dd.
 * (Inspection only, e.g. to check the batched sums against the plain
 * definition; the paper's pipeline searches them in place, Sec. 2.3.) */
aa_status aa_batch_dd_view(const aa_batch* batch, int32_t beam, const float** d_dd);

/* Number of waves and total device bytes held by the batch. */
aa_status aa_batch_info(const aa_batch* batch, int32_t* nwaves, int64_t* device_bytes);

/* How the graph issues each wave (re-records the graph; the buffers, waves
 * and results are unchanged).  branches = 0: one persistent work-queue
 * kernel per stage spanning the wave's beams; branches = k in [1, 64] (8 at
 * creation): each beam's own kernels, as the single-beam path
 * launches them (decimation cascade, one dedispersion launch per range,
 * statistics and boxcar + peaks per range), on k concurrent graph branches,
 * the wave's beams dealt largest first to the least-loaded branch by
 * channel-adds.  The candidate set of a run does not depend on the form.
 * AA_ERR_ARG outside [0, 64]; AA_ERR_CUDA if the graph cannot be recorded
 * (the batch then has no graph until a later call succeeds). */
aa_status aa_batch_set_branches(aa_batch* batch, int32_t branches);

/* Launch the captured graph on `stream` (asynchronous). */
aa_status aa_batch_run(aa_batch* batch, aa_stream_t stream);

/* Candidates of the last run, sorted by (beam, dm_index, t); the record's
 * `reserved` byte holds the beam index.  Synchronises `stream`.  Returns
 * AA_WARN_CAND_OVERFLOW if more than cand_capacity were found. */
aa_status aa_batch_candidates(aa_batch* batch, aa_stream_t stream, aa_candidates** out);

/* --------------------------------------------------- streaming server -- */

/* Continuous-batching search server for streaming beams (Sec. 3.3: the
 * pipeline iterates over the input in chunks and reports a status code per
 * iteration).  Chunk k of a beam carries chunk_nsamp new samples and is
 * searched as the block of full-rate samples [max(0, kN - H), (k+1)N), where
 * the beam's resident history supplies the first samples and
 * H = max_r dec_r * (maxshift_r + W + 2) rounded up to a multiple of 16.  The
 * block runs through the whole pipeline with its own mean and standard
 * deviation; the chunk reports the candidates of range r whose global start
 * index j (decimated samples, record field t) lies in
 * [kN/dec_r - maxshift_r - W - 1, (k+1)N/dec_r - maxshift_r - W - 1).
 * Chunks queue on the host and are admitted into slots (own stream and device
 * workspace; slot count = min(max_slots, what memory_budget allows after the
 * beams' resident buffers)) as slots free up; a beam's chunks run in order,
 * chunks of different beams overlap on the device.  When the plan has no
 * sub-band or FDMT range, a slot runs aa_search_fused_device (same results)
 * and holds its workspace instead of the series of every trial, so a budget
 * admits more slots. */
typedef struct aa_server aa_server;

typedef struct aa_chunk_info {
    int32_t beam;
    int32_t status;        /* AA_PENDING while queued or in flight */
    int64_t chunk;         /* index of the chunk within its beam */
    int64_t block_start;   /* full-rate index of the block's first sample */
    int64_t total;         /* candidates found in the whole block */
    double arrival;        /* caller's submission time (aa_server_clock) */
    double admitted;       /* when the chunk entered a slot */
    double done;           /* when its completion was observed */
} aa_chunk_info;

typedef struct aa_server_report {
    int64_t submitted, completed;
    int32_t slots, max_in_flight;
    int64_t history_nsamp;               /* H */
    double latency_p50, latency_p99, latency_max;  /* done - arrival, seconds */
    double span;                         /* last completion - first arrival, seconds */
} aa_server_report;

/* memory_budget <= 0: half of the free device memory.  chunk_nsamp must be a
 * positive multiple of 16.  The plan is bound to the current device if
 * needed and must outlive the server.  AA_ERR_NOMEM if not even one slot
 * fits. */
aa_status aa_server_create(aa_plan* plan, int32_t nbeams, int64_t chunk_nsamp, int32_t max_width,
                           float threshold, int64_t cand_capacity, int64_t memory_budget,
                           int32_t max_slots, aa_server** out);
void aa_server_destroy(aa_server* server);

/* Queue the next chunk of `beam`: uint8 [nchans][host_pitch] host memory
 * (first chunk_nsamp bytes of each row), read-only, owned by the caller and
 * kept valid until the chunk completes.  arrival_time: the caller's clock
 * (use aa_server_clock).  Returns AA_PENDING and the chunk's ticket;
 * AA_ERR_CONFIG (nothing queued) for a chunk whose samples would pass global
 * sample index 2^32 of its beam (reported start times are 32-bit). */
aa_status aa_server_submit(aa_server* server, int32_t beam, const uint8_t* host_chunk,
                           int64_t host_pitch, double arrival_time, int64_t* ticket);

/* Non-blocking progress: collect finished chunks, admit queued ones.
 * Returns AA_OK when nothing is queued or in flight, AA_PENDING otherwise. */
aa_status aa_server_poll(aa_server* server, int32_t* ncompleted);

/* Block until every submitted chunk has completed. */
aa_status aa_server_drain(aa_server* server);

/* Status and (once complete) the chunk's candidates, library-owned and
 * sorted by (dm_index, t); t is the global start index, `reserved` the beam.
 * Returns the chunk's status (AA_PENDING while not complete). */
aa_status aa_server_result(aa_server* server, int64_t ticket, aa_chunk_info* info,
                           aa_candidates** cands);

/* Latency percentiles and counters of the completed chunks. */
aa_status aa_server_stats(const aa_server* server, aa_server_report* out);

/* Monotonic clock (seconds) used for arrival and completion times. */
double aa_server_clock(void);

/* ------------------------------------------------- differentiable form -- */

/* Float input with per-channel weights (every range must have dec == 1,
 * else AA_ERR_CONFIG):  y[d][t] = sum_c w[c] * x[c][t + s(c,d)]  (FP32 FMA,
 * channels summed in index order).  d_x: float [nchans][x_pitch] (x_pitch >=
 * nsamp), d_w: float [nchans], d_y: float [dd_elems] in the layout of
 * aa_dedisperse_device.  Stream-ordered. */
aa_status aa_dedisperse_f32_device(const aa_plan* plan, const float* d_x, int64_t nsamp,
                                   int64_t x_pitch, const float* d_w, float* d_y,
                                   aa_stream_t stream);

/* Transpose of the float forward: given d_gy (layout of d_y), writes
 * gx[c][u] = w[c] * sum_d gy[d][u - s(c,d)] (float [nchans][x_pitch],
 * overwritten for u < nsamp) and gw[c] = sum_{d,t} gy[d][t] * x[c][t + s(c,d)]
 * (float [nchans], overwritten).  d_ws: aa_plan_info.f32_ws_bytes of scratch. */
aa_status aa_dedisperse_f32_adjoint_device(const aa_plan* plan, const float* d_x, int64_t nsamp,
                                           int64_t x_pitch, const float* d_w, const float* d_gy,
                                           float* d_gx, float* d_gw, void* d_ws, size_t ws_bytes,
                                           aa_stream_t stream);

/* Mean squared error of the float forward against a template (layout of
 * d_y): *d_loss (device double) = mean over every (trial, t < L) of
 * (y - T)^2, reduced in the forward without storing y.  If d_gx and d_gw are
 * both non-NULL the gradients of the loss with respect to x and w are written
 * too; y is then recomputed chunk by chunk of trials (never stored whole).
 * Stream-ordered. */
aa_status aa_dedisperse_f32_mse_device(const aa_plan* plan, const float* d_x, int64_t nsamp,
                                       int64_t x_pitch, const float* d_w, const float* d_template,
                                       double* d_loss, float* d_gx, float* d_gw, void* d_ws,
                                       size_t ws_bytes, aa_stream_t stream);

/* ------------------------------------------ host-buffer (API-owned) path -- */

/* Copy the caller's host filterbank (uint8 [nchans][host_pitch], first nsamp
 * bytes of each row valid; never written) to the device and dedisperse it.
 * The result buffers are allocated and owned by the library (stream-ordered
 * device allocations).  Returns once the host input has been read; the
 * dedispersion runs asynchronously on `stream`.  Binds the plan to the current
 * device if it is not bound. */
aa_status aa_dedisperse(aa_plan* plan, const uint8_t* host_in, int64_t nsamp,
                        int64_t host_pitch, aa_stream_t stream, aa_dd_result** out);

/* Const view of a result: device pointer to the output buffer (layout of
 * aa_dedisperse_device) and the nsamp it was computed for.  Valid until
 * aa_dd_result_destroy. */
aa_status aa_dd_result_view(const aa_dd_result* res, const float** d_out, int64_t* nsamp);

/* Free a result (stream-ordered on the stream it was produced on).  NULL is a
 * no-op. */
void aa_dd_result_destroy(aa_dd_result* res);

/* Run the single-pulse search on a result and bring the candidates to host
 * memory owned by the library, sorted by (dm_index, t).  Blocks until done.
 * Returns AA_WARN_CAND_OVERFLOW if more than cand_capacity were found. */
aa_status aa_sps_search(aa_plan* plan, const aa_dd_result* dd, int32_t max_width,
                        float threshold, int64_t cand_capacity, aa_stream_t stream,
                        aa_candidates** out);

/* Const view of a candidate list: host pointer, records stored, and the
 * total found.  Valid until aa_candidates_destroy. */
aa_status aa_candidates_view(const aa_candidates* c, const aa_candidate** host,
                             int64_t* stored, int64_t* total);

/* Free a candidate list.  NULL is a no-op. */
void aa_candidates_destroy(aa_candidates* c);

/* ------------------------------- fused dedispersion -> search (Sec. 1, 2.3) */

/* Dedispersion and single-pulse search in one call, without the dedispersed
 * series of the whole plan: each range is processed in stripes of
 * stripe_trials consecutive DM trials (0: 256; otherwise a positive multiple
 * of 16), whose series live in one stripe buffer of the workspace while they
 * are searched.  The dedispersion kernels add every row's exact sums (sum y,
 * sum y^2 in 128 bits) as they write it, so the search's mean and sigma need
 * no separate pass over the series; with k-sigma clipped statistics
 * (aa_plan_set_sps_clip) the statistics pass runs on each stripe instead.
 * Candidates (and chunk headers, and B(t) in d_snr_out when non-NULL, in the
 * layout of aa_dedisperse_device's output) are bit for bit those of
 * aa_dedisperse_device followed by aa_sps_search_device.
 *
 * Ranges are searched one after another, each decimated range's input
 * built from the 8-bit input into one buffer shared by the ranges.
 *
 * aa_search_fused_ws_bytes: workspace bytes for (nsamp, max_width,
 * stripe_trials), and the byte offset inside it of the search workspace
 * (what aa_sps_order_device takes as d_sps_ws after the call).  About
 * stripe_trials x the widest range's row pitch x 4 bytes replace the
 * aa_plan_query dd_elems x 4 bytes of the unfused path, and the largest
 * decimated input replaces all of them.
 * aa_search_fused_device: d_in as in aa_dedisperse_device; candidates as in
 * aa_sps_search_device; d_ws 256-byte aligned, >= the bytes above.  Its
 * first word is the error word (aa_workspace_status).  Stream-ordered.
 * AA_ERR_CONFIG for plans with sub-band or FDMT ranges; AA_ERR_ARG on bad
 * arguments. */
aa_status aa_search_fused_ws_bytes(const aa_plan* plan, int64_t nsamp, int32_t max_width,
                                   int32_t stripe_trials, size_t* bytes, size_t* sps_ws_offset);
aa_status aa_search_fused_device(const aa_plan* plan, const uint8_t* d_in, int64_t nsamp,
                                 int64_t in_pitch, int32_t max_width, float threshold,
                                 int32_t stripe_trials, aa_candidate* d_cands,
                                 int64_t cand_capacity, unsigned long long* d_count,
                                 float* d_snr_out, void* d_ws, size_t ws_bytes,
                                 aa_stream_t stream);

/* --------------------------------------- host-buffer pipeline (Sec. 2.3-3.3) */

/* A pipeline searches a sequence of same-sized blocks of caller-owned host
 * data (uint8 [nchans][host_pitch], first nsamp bytes of each row) through
 * the whole path -- decimation, dedispersion, single-pulse search, candidate
 * ordering -- with every device buffer requested once, at creation (Sec. 2.3)
 * and the copies overlapped with the compute: block k+1 is uploaded while
 * block k is searched, and block k's candidates are read back while block
 * k+1 is searched.  The results are those of aa_dedisperse + aa_sps_search
 * on each block.
 *
 * aa_pipeline_create: plan (bound to the current device if needed; it must
 * outlive the pipeline), block length nsamp >= 1, search parameters as in
 * aa_sps_search, depth in [1, 8] = blocks in flight (input slots; 2 overlaps
 * one upload with one search).  Allocates depth x (nchans x in_pitch +
 * cand_capacity x 16) bytes plus one set of working buffers (aa_plan_query
 * with max_width: dd_elems x 4 + dedisp_ws_bytes + sps_ws_bytes, the
 * candidate array and the ordering scratch of aa_postprocess_ws_bytes).
 * AA_ERR_ARG on bad arguments, AA_ERR_NOMEM if memory runs out (nothing is
 * left allocated). */
typedef struct aa_pipeline aa_pipeline;
aa_status aa_pipeline_create(aa_plan* plan, int64_t nsamp, int32_t max_width, float threshold,
                             int64_t cand_capacity, int32_t depth, aa_pipeline** out);

/* Queue the next block.  The host memory is read asynchronously: keep it
 * valid and unchanged until aa_pipeline_wait returns for this ticket
 * (page-locked memory lets the upload overlap the compute; pageable memory
 * works but is copied synchronously by the driver).  Never written.  Returns
 * AA_PENDING and the block's ticket (0, 1, 2, ... in submission order);
 * AA_ERR_STATE if `depth` blocks are already in flight (wait for the oldest
 * first) or another device is current; AA_ERR_ARG on bad arguments. */
aa_status aa_pipeline_submit(aa_pipeline* pipeline, const uint8_t* host_in, int64_t host_pitch,
                             int64_t* ticket);

/* Block until the ticket's search is done and return its candidates
 * (library-owned host memory, sorted by (dm_index, t); free with
 * aa_candidates_destroy).  Tickets may be collected in any order, each once
 * (AA_ERR_STATE for a ticket already collected).  Returns AA_OK,
 * AA_WARN_CAND_OVERFLOW, AA_ERR_TIMEOUT (a bounded device-side wait gave up)
 * or AA_ERR_CUDA; the block's slot is free again in every case. */
aa_status aa_pipeline_wait(aa_pipeline* pipeline, int64_t ticket, aa_candidates** out);

/* Synchronise and free everything the pipeline holds.  NULL is a no-op. */
void aa_pipeline_destroy(aa_pipeline* pipeline);

/* ---------------------------------------------- no-allocation search -- */

/* Size of the fixed scratch area behind aa_sps_search_device_noalloc. */
#define AA_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The single-pulse search of aa_sps_search_device for callers that cannot
 * allocate device memory while running (for example a real-time
 * beam-processing loop whose memory is fixed at start-up, where an
 * allocation could synchronise the device, or a plug-in whose host framework
 * owns all device allocations).  It has no counterpart in the paper.
 * Arguments and results are those of aa_sps_search_device without d_ws and
 * ws_bytes: the scratch is a fixed AA_NOALLOC_SCRATCH_BYTES device array that
 * every GPU loading the library holds until the process exits.  The caller
 * still passes the dedispersed input, the candidate array, the count and the
 * optional B(t) output.  The first call on a device looks up the array's
 * device address (with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture, and do not
 * use this entry point on a device after a cudaDeviceReset of it (the kept
 * address no longer names the array).  All calls share the one array: calls
 * whose GPU work overlaps race.  Returns AA_ERR_ARG if the search needs more scratch than
 * the array holds (aa_plan_query(...).sps_ws_bytes > AA_NOALLOC_SCRATCH_BYTES),
 * otherwise what aa_sps_search_device returns.  Calls no allocation
 * routine. */
aa_status aa_sps_search_device_noalloc(const aa_plan* plan, int64_t nsamp, const float* d_dd,
                                       int32_t max_width, float threshold,
                                       aa_candidate* d_cands, int64_t cand_capacity,
                                       unsigned long long* d_count, float* d_snr_out,
                                       aa_stream_t stream);

/* ------------------------------------- candidate post-processing (Sec. 1) */

/* Device scratch (bytes) needed by aa_sps_order_device and
 * aa_candidates_peaks2d_device for this plan, nsamp, max_width and candidate
 * capacity.  AA_ERR_ARG for NULL/negative arguments, AA_ERR_CONFIG for a plan
 * with more than 64 ranges. */
aa_status aa_postprocess_ws_bytes(const aa_plan* plan, int64_t nsamp, int32_t max_width,
                                  int64_t cand_capacity, size_t* bytes);

/* Order the candidates of one aa_sps_search_device call on the device, by
 * (dm_index, t) -- the order aa_sps_search returns on the host -- with no
 * host round trip.
 *   d_sps_ws      : the workspace that search used, unchanged since (its run
 *                   headers describe where each boxcar CTA wrote its records);
 *   d_cands, d_count, cand_capacity : that search's outputs and capacity;
 *   d_sorted      : device array of cand_capacity records (16-byte aligned)
 *                   receiving min(*d_count, cand_capacity) records in order;
 *   d_tmp         : device scratch (16-byte aligned) of tmp_bytes >=
 *                   aa_postprocess_ws_bytes.
 * nsamp and max_width are those of the search.  Stream-ordered and
 * asynchronous; AA_ERR_ARG on bad arguments, AA_ERR_CUDA if a launch fails. */
aa_status aa_sps_order_device(const aa_plan* plan, int64_t nsamp, int32_t max_width,
                              const void* d_sps_ws, const aa_candidate* d_cands,
                              const unsigned long long* d_count, int64_t cand_capacity,
                              aa_candidate* d_sorted, void* d_tmp, size_t tmp_bytes,
                              aa_stream_t stream);

/* 2-D peak filter over an ordered candidate list (as written by
 * aa_sps_order_device).  The 1-D peak finding of the single-pulse search
 * (Sec. 1) reports a pulse once per trial it shows in; this keeps the local
 * maxima of the DM-time plane.  Candidate c is kept iff no other candidate o
 * of the same range with |o.dm_index - c.dm_index| <= dm_radius and
 * |o.t - c.t| <= t_radius has o.snr > c.snr, or o.snr == c.snr and
 * (o.dm_index, o.t) < (c.dm_index, c.t) lexicographically.  Suppressed
 * candidates still suppress (no chaining).
 *   d_sorted, d_count, cand_capacity : the ordered list; its length is
 *                   min(*d_count, cand_capacity);
 *   d_peaks       : device array of cand_capacity records receiving the kept
 *                   candidates, still in (dm_index, t) order;
 *   d_npeaks      : device uint64 receiving their number;
 *   d_tmp         : as for aa_sps_order_device (may be the same scratch).
 * nsamp and max_width are those of the search.  AA_ERR_ARG for negative radii
 * or bad arguments.  Stream-ordered and asynchronous. */
aa_status aa_candidates_peaks2d_device(const aa_plan* plan, int64_t nsamp, int32_t max_width,
                                       const aa_candidate* d_sorted,
                                       const unsigned long long* d_count, int64_t cand_capacity,
                                       int32_t dm_radius, int32_t t_radius, aa_candidate* d_peaks,
                                       unsigned long long* d_npeaks, void* d_tmp, size_t tmp_bytes,
                                       aa_stream_t stream);

/* ------------------------------------------------------------- profiling -- */

/* Kernel timing (tracing).  While enabled, every kernel the library launches
 * is bracketed by two CUDA events recorded on the stream it is launched on.
 * on = 1 clears the counters and starts recording; on = 0 stops. */
aa_status aa_profile_enable(int32_t on);

/* Launch count and summed device time (ms) of kernel id `kernel` since the
 * last aa_profile_enable(1); waits for the recorded events.  Ids run from 0
 * while aa_profile_kernel_name(id) != NULL.  AA_ERR_ARG for a bad id. */
aa_status aa_profile_read(int32_t kernel, int64_t* launches, double* total_ms);

/* Static name of kernel id `kernel`, NULL past the last id. */
const char* aa_profile_kernel_name(int32_t kernel);

/* ------------------------------------------------- filterbank input (Sec. 4) */

/* SIGPROC filterbank files: the paper's front-end can direct the library to a
 * file on disk (Sec. 4).  A file is a header of keyword/value pairs between
 * "HEADER_START" and "HEADER_END" (each string stored as a little-endian int32
 * length followed by its bytes; integer values int32, real values IEEE
 * double, string values as above), then the samples in time-major order: for
 * each time sample, nifs x nchans values of nbits bits, channel 0 at fch1.
 * Only nbits = 8 and nifs = 1 are read (the library's input type). */
typedef struct aa_fil_header {
    int32_t nchans;
    int32_t nbits;
    int32_t nifs;
    int32_t data_type;     /* 0 if absent */
    int32_t telescope_id;  /* -1 if absent */
    int32_t machine_id;    /* -1 if absent */
    double fch1_mhz;       /* centre frequency of channel 0 */
    double foff_mhz;       /* channel spacing (negative: descending band) */
    double tsamp_s;
    double tstart_mjd;     /* 0 if absent */
    int64_t header_bytes;  /* offset of the first sample in the file */
    int64_t nsamples;      /* complete time samples in the file (from its size) */
    char source_name[80];  /* NUL-terminated, empty if absent */
} aa_fil_header;

/* Parse the header of the file at `path` into *out.  AA_ERR_ARG for NULL
 * arguments or a file that cannot be opened; AA_ERR_CONFIG for a malformed
 * header (no HEADER_START, an unknown keyword, a truncated value, missing
 * nchans/nbits/fch1/foff/tsamp, nbits != 8 or nifs != 1). */
aa_status aa_fil_read_header(const char* path, aa_fil_header* out);

/* Copy time samples [t0, t0 + nsamp) of the file (header `h` as returned by
 * aa_fil_read_header) into the caller-owned host buffer host_tm, time-major:
 * host_tm[t * nchans + c] (may be NULL when nsamp = 0).  AA_ERR_ARG if the range
 * is outside the file or an argument is NULL; AA_ERR_CONFIG if the file is
 * shorter than its header says. */
aa_status aa_fil_read_block(const char* path, const aa_fil_header* h, int64_t t0, int64_t nsamp,
                            uint8_t* host_tm);

/* Corner turn on the device: d_cm[c * cm_pitch + t] = d_tm[t * tm_stride + c]
 * for t < nsamp, c < nchans (time-major block -> the channel-major layout of
 * aa_dedisperse_device).  tm_stride >= nchans and cm_pitch >= nsamp (bytes);
 * the buffers must not overlap.  Asynchronous on `stream`; AA_ERR_ARG for bad
 * sizes or NULL pointers, AA_ERR_CUDA if the launch fails.  No counterpart in
 * the paper (its reader's data layout is internal). */
aa_status aa_corner_turn_device(const uint8_t* d_tm, int64_t nsamp, int32_t nchans,
                                int64_t tm_stride, uint8_t* d_cm, int64_t cm_pitch,
                                aa_stream_t stream);

/* ------------------------------------------------------------ test hooks -- */

/* Fault injection for tests of the bounded device-side waits; affects every
 * later launch in the process.  what = 0: reset all hooks; what = 1: the
 * direct-strategy dedispersion producer never issues the staging copy of
 * channel chunk `value` (that stage's barrier never completes, so every CTA
 * gives up after the wait limit, sets the workspace error word and exits
 * without writing output; the grouped strategy has no staging waits); what =
 * 2: set the wait limit to `value` nanoseconds (default 2 s); what = 3: the
 * boxcar kernel processes `value` consecutive tiles of a series per CTA
 * (0: its own choice; the results do not depend on it).
 * Returns AA_ERR_ARG for an unknown `what`, a non-positive limit or a tile
 * count outside [0, 4096]. */
aa_status aa_debug_inject(int32_t what, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* AA_DEDISP_H */

// Internal declarations shared by the host plan code and the kernel
// translation units of libaa_gb300.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/aa_dedisp.h"

namespace aa {

// ---------------------------------------------------------------- strategy --
// Dedispersion tile: a CTA of kDedispWarps warps covers kDmPerBlock DM trials
// x kTau output samples; channels stream through shared memory in stages of
// `cc` channels (bulk-async copies), each stage reused by all the CTA's DMs.
constexpr int kDedispWarps = 16;
constexpr int kDmPerWarp = 1;
constexpr int kDmPerBlock = kDedispWarps * kDmPerWarp;  // 16
constexpr int kTau = 512;                                // output samples per CTA
constexpr int kDedispThreads = kDedispWarps * 32;

// Boxcar tile: kSpsThreads threads x kSpsSlots consecutive start times each.
constexpr int kSpsThreads = 256;
constexpr int kSpsSlots = 16;
constexpr int kSpsTile = kSpsThreads * kSpsSlots;  // start times per CTA incl. 2 halo
constexpr int kSpsOwned = kSpsTile - 2;              // start times owned per CTA

// Grouped strategy.  Within one (DM block, channel chunk), channels whose
// delays at every trial of the block exceed their delay at the block's first
// trial by the same amounts (the same "delay pattern") are summed once, into a
// group sum z_g[u] = sum_{c in g} x[c][t0 + s(c,d0) + u]; trial d of the block
// then adds z_g[t + delta_g(d)] once per group instead of once per channel.
// Integer sums regrouped: the result is bit-identical.
constexpr int kGroupTau = 512;  // output samples per CTA (grouped strategy)

struct GroupRec {       // one (DM block, channel chunk)
    uint32_t first;     // index of its first GroupDesc
    uint16_t ngroups;
    uint16_t nch;       // channels in the chunk
};
struct GroupDesc {
    uint16_t mstart;    // first member in the record's member list
    uint16_t mcount;
    uint16_t span;      // largest relative delay (delta at the block's last trial)
    uint16_t flush;     // 1: flush the trials' 16-bit sums before adding this group
    uint16_t delta[kDmPerBlock];  // relative delay at each trial of the block
};
struct GroupMember {   // member m of a (DM block, channel chunk), in group order
    int32_t s0;        // its delay at the block's first trial
    uint16_t ch;       // channel within the chunk
    uint16_t span;     // its delay at the block's last trial minus s0
};
static_assert(sizeof(GroupRec) == 8 && sizeof(GroupDesc) == 40 && sizeof(GroupMember) == 8,
              "group table layout");
static_assert(kGroupTau == kTau, "both strategies tile time alike (launch and queue sizing)");

// Tile shape of the direct (shift-and-sum) kernel for one kind of launch.
struct DirectShape {
    int elem = 1, spw = 4;   // bytes per input sample, samples per 32-bit word
    int rw = 0;              // words per shared-memory row copy
    int cc = 2, nstage = 2;  // channels per stage, pipeline depth
    int flush = 2;           // channels between SWAR flushes (multiple of cc)
    size_t smem = 0;
};
// Shape for input samples of `elem` bytes, each at most per_lane_max, and a
// delay spread of `span` samples across a block of trials; false if no
// stage of at least two channels fits.
bool direct_shape(int elem, int32_t span, int per_lane_max, DirectShape& out);

// Sub-band strategy of a range (AA_DEDISP_SUBBAND): channel bands of k
// channels and coarse trials of m fine trials.  Stage 1 (direct kernel) sums
// each band at the coarse trial's relative delays into 16-bit partial series
// z[b][j][t]; stage 2 (its own kernel, 32-bit sums) adds the bands at each
// fine trial's delay of the band's reference (highest-frequency) channel.
struct SubbandPlan {
    int k = 0, m = 0, nsub = 0, ncoarse = 0;
    int32_t rmax = 0;       // largest stage-1 (within-band) delay
    int32_t s2max = 0;      // largest stage-2 (reference channel) delay
    int32_t span2 = 0;      // largest stage-2 delay spread within a coarse trial
    DirectShape shape1;     // stage 1 runs on the direct kernel
    std::vector<int32_t> rel;  // stage 1: per band b, [ncoarse][k_b] (band slices concatenated)
    std::vector<int32_t> s2;   // stage 2: [ndm][nsub]
    double work = 1.0;         // (stage-1 + stage-2 adds) / direct adds
    int32_t* d_rel = nullptr;
    int32_t* d_s2 = nullptr;
};

// Sub-band stage 2 (32-bit accumulation): shared memory for nsub bands and a
// delay span across the coarse trial's fine trials; also the staged window
// length and the bands staged at once.
size_t subband_stage2_smem(int nsub, int span, int& swin, int& nb_chunk);
cudaError_t launch_subband_stage2(const uint16_t* z, int64_t band_stride, int64_t pitch1, int64_t len1, int nsub,
                                  int ncoarse, int m, int ndm, const int32_t* s2, int span, float* out,
                                  int64_t out_pitch, int64_t length, cudaStream_t s);

// FDMT-style tree dedispersion of a range (AA_DEDISP_FDMT, an approximation):
// the channels in falling-frequency order form a binary tree of subbands
// (subband [a, b] split at a + ceil((b - a + 1) / 2)); a subband's sum at
// delay delta (of its last channel relative to its first) adds its upper
// half's sum at delay du(delta) and its lower half's at delta - gap(delta),
// read gap(delta) samples later.  Depths are computed deepest first into
// 32-bit rows; the root's rows are the range's trials (the whole-band delay
// of trial i is the bottom channel's brute-force delay), written as FP32.
struct FdmtRow {
    int32_t u, l;   // rows of the next-deeper depth (>= 0) or channel -(ref + 1) (< 0)
    int32_t gap;    // the lower half is read at t + gap
    int32_t delta;  // this row's delay: valid for t < nsamp_dec - delta
};
static_assert(sizeof(FdmtRow) == 16, "FDMT row layout");
struct FdmtPlan {
    int depths = 0;               // merge levels (the root is depth 0)
    std::vector<FdmtRow> rows;    // deepest depth first, the root's (one per trial) last
    std::vector<int64_t> first;   // [depths + 1]: start of each depth's rows in that order
    int32_t max_rows = 0;         // rows of the largest intermediate depth
    double work = 1.0;            // rows computed / (ndm x nchans): adds relative to direct
    FdmtRow* d_rows = nullptr;
};
cudaError_t launch_fdmt_depth(const FdmtRow* rows, int nrows, int leaf_elem, const void* leaves,
                              int64_t leaf_pitch, const uint32_t* prev, uint32_t* out, int64_t pitch,
                              int64_t nsamp, float* fout, int64_t fpitch, int64_t flen, cudaStream_t s);

// Per-range strategy, derived once at plan creation (immutable afterwards).
struct RangePlan {
    aa_dm_range desc{};
    std::vector<int32_t> shifts;  // [ndm][nchans], decimated samples
    int32_t maxshift = 0;
    int32_t span_max = 0;  // max over DM blocks/channels of s(c,last)-s(c,first)
    int32_t dm_offset = 0;
    int elem = 1;          // bytes per input sample (1: raw uint8, 2: decimated uint16)
    int spw = 4;           // samples per 32-bit word
    int rw = 0;            // words per shared-memory row copy
    int cc = 16;           // channels per stage (even)
    int nstage = 3;        // pipeline depth
    int flush = 256;       // channels between SWAR flushes (multiple of cc)
    size_t smem = 0;       // dynamic shared memory per CTA
    int dec_src = 1;       // decimation source buffer (1 = raw input)
    int f32_span = 0;      // differentiable form: delay spread over any 16 consecutive trials
    int f32_cspan = 0;     // ... and over any 16 consecutive channels
    int32_t* d_shifts = nullptr;  // device copy (inside the plan's table block)
    // grouped strategy (aa_dedisp_strategy AA_DEDISP_GROUPED)
    int strategy = 0;      // 0 direct, 1 grouped
    bool grouped_ok = false;  // the grouped tables exist (spans fit)
    int gcc = 0;           // channels per chunk
    int gz = 0;            // group sums held in shared memory at once
    int gzw = 0;           // 32-bit words per group-sum copy
    int gflush = 1;        // chunks between SWAR flushes (0: flushes placed by the groups' flags)
    int gnj = 3;           // 256-sample blocks covering kGroupTau + span_max
    int gtl = 0;           // lanes per group tail (power of two <= 32), 0: none
    size_t gsmem = 0;      // dynamic shared memory per CTA
    double gwork = 1.0;    // (group adds + pre-sum adds) / direct adds
    std::vector<GroupRec> grec;    // [ndm blocks][chunks]
    std::vector<GroupDesc> gdesc;
    std::vector<GroupMember> gmem; // [ndm blocks][chunks][gcc] members in group order
    GroupRec* d_grec = nullptr;
    GroupDesc* d_gdesc = nullptr;
    GroupMember* d_gmem = nullptr;
    SubbandPlan sb;        // valid once aa_plan_set_subband chose it (strategy 2)
    FdmtPlan fd;           // valid once aa_plan_set_fdmt chose it (strategy 3)
};

}  // namespace aa

struct aa_plan {
    int32_t nchans = 0;
    double fch1 = 0, foff = 0, tsamp = 0, f_top = 0;
    std::vector<aa::RangePlan> ranges;
    std::vector<int> decs;  // distinct decimations > 1, ascending
    int32_t ndm_total = 0;
    double dm_max = 0;
    // single-pulse statistics: iterative k-sigma clipping, k = clip_c16 / 16,
    // at most clip_iters clipping passes (0: plain mean and sigma)
    int32_t clip_c16 = 0, clip_iters = 0;
    // boxcar widths: 0 every width 1..W, else the sparse ladder of growth ladder_g16 / 16
    int32_t ladder_g16 = 0;
    // decimated width ladder with dec_w0 base widths (0: off)
    int32_t dec_w0 = 0;
    int device = -1;
    bool ready = false;
    void* d_tables = nullptr;
    size_t table_bytes = 0;
    void* d_sub = nullptr;  // sub-band and FDMT tables of every range using them
};

namespace aa {

// Layout of every device buffer for one (nsamp, max_width).
struct Layout {
    int64_t nsamp = 0;
    int64_t in_pitch_min = 0;
    std::vector<int64_t> nsamp_dec, length, pitch, row_offset;
    int64_t dd_elems = 0;
    int64_t dm_trial_samples = 0;
    // dedispersion workspace: [error word block][one uint16 buffer per decimation]
    std::vector<int64_t> dec_pitch;   // elements, per entry of plan.decs
    std::vector<int64_t> dec_offset;  // bytes into the workspace
    // sub-band ranges: 16-bit partial series [nsub][ncoarse][sub_pitch] (bytes
    // into the workspace; -1 for other ranges) and their length
    std::vector<int64_t> sub_offset, sub_pitch, sub_len;
    // FDMT ranges: two 32-bit depth buffers of fdmt_rows rows at pitch
    // fdmt_pitch (bytes into the workspace; -1 when no range uses FDMT)
    int64_t fdmt_offset = -1, fdmt_pitch = 0, fdmt_rows = 0;
    int64_t dedisp_ws = 0;
    // single-pulse workspace: [error word + chunk counter][1/sqrt(w)][row stats]
    //                         [width tables][candidate chunk headers]
    int32_t max_width = 0;
    int32_t wpad = 0;
    int64_t stats_offset = 0, table_offset = 0, chunk_offset = 0, chunk_cap = 0, sps_ws = 0;
    // differentiable-form workspace: [loss sum][w-gradient partials][residual chunk]
    int64_t f32_part_offset = 0, f32_resid_offset = 0, f32_ws = 0;
};

constexpr int64_t kErrBlock = 256;  // bytes reserved for the device error word

Layout make_layout(const aa_plan& p, int64_t nsamp, int32_t max_width);

void set_error(const char* fmt, ...);
void clear_error();

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Per-row statistics written by the stats kernel, read by the boxcar kernels.
struct RowStats {
    double mu;        // mean
    double sigma;     // population standard deviation
    double inv_sigma; // 1/sigma (0 if sigma == 0)
    float m0;         // round(mu): integer offset removed before summing
    int32_t zero_sigma;
};
static_assert(sizeof(RowStats) == 32, "RowStats layout");

// Each boxcar CTA appends its candidates as one contiguous run ordered by t;
// the run is described by a chunk header so the host can order the list by
// sorting headers instead of records.
struct CandChunk {
    unsigned long long base;  // index of the run's first record
    uint32_t n;               // records in the run
    uint32_t dm_index;
    uint32_t t0;              // first start time owned by the CTA
    uint32_t reserved;
};
static_assert(sizeof(CandChunk) == 24, "CandChunk layout");
constexpr int64_t kChunkCounterOffset = 8;   // bytes into the error block
constexpr int64_t kEvaluatedOffset = 16;     // evaluated width-samples counter

// ------------------------------------------------------------- profiling --
enum KernelId {
    kKDecimate = 0, kKDedispU8, kKDedispU16, kKRsqrt, kKStats, kKBoxcar, kKF32Fwd, kKF32Adj,
    kKCornerTurn, kKOrder, kKPeaks2d, kKSubband1, kKSubband2, kKFinalize, kKFdmt, kNumKernels
};

// RAII: records CUDA events around a launch on `s` while profiling is on.
class ProfScope {
  public:
    ProfScope(int kernel, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int kernel_;
    cudaStream_t stream_;
    cudaEvent_t start_ = nullptr, stop_ = nullptr;
    bool active_ = false;
};

// ------------------------------------------------------------- launchers --
struct DedispArgs {
    const void* in;          // [nchans][in_pitch] samples (uint8 or uint16)
    int64_t in_pitch;        // elements
    int32_t nchans;
    int64_t nsamp;           // valid samples per row of `in`
    int64_t length;          // output samples per trial
    int32_t ndm;
    const int32_t* shifts;   // [ndm][nchans]
    float* out;              // row 0 of this range
    uint16_t* out16;         // direct strategy only: 16-bit rows instead of `out` (non-NULL)
    int64_t out_pitch;       // elements
    int rw, cc, nstage, flush, elem;
    size_t smem;
    unsigned* err;
    // grouped strategy (used when grouped != 0; cc and smem then describe it)
    int grouped;
    int gz, gzw, gflush, gnj;  // gnj: 256-sample blocks of the longest group sum
    int gtl;                   // lanes per group in phase-1 tail units (0: no tail units)
    const GroupRec* grec;
    const GroupDesc* gdesc;
    const GroupMember* gmem;
    // launches over a stripe of the range's trials: the stripe's first DM
    // block in the range's group tables (out, shifts and ndm already describe
    // the stripe)
    int32_t dmb0;
    // fused statistics (non-NULL): each output row r adds its exact sums to
    // st_acc[3 r .. 3 r + 2] = (sum y, sum y^2 low 64 bits, high 64 bits)
    unsigned long long* st_acc;
};
// Strategy fields of a range's kernel arguments.
void fill_strategy(DedispArgs& a, const RangePlan& r);
cudaError_t launch_dedisperse(const DedispArgs& a, cudaStream_t s);

cudaError_t launch_decimate(const void* in, int in_elem, int64_t in_pitch, int32_t nchans,
                            int64_t nout, int factor, uint16_t* out, int64_t out_pitch,
                            cudaStream_t s);
// Every decimated input of the plan into the dedispersion workspace `ws`
// (layout L), each built from the largest decimation dividing it.
cudaError_t launch_decimation_cascade(const aa_plan& p, const Layout& L, const uint8_t* d_in, int64_t in_pitch,
                                      char* ws, cudaStream_t s);

// ----------------------------------------------------- batched (persistent) --
struct DecimateJob {
    const void* in;
    int32_t in_elem;
    int32_t factor;
    int64_t in_pitch;  // elements
    int64_t nout;      // output samples per channel
    uint16_t* out;
    int64_t out_pitch;  // elements
};
// Work-queue kernels over several descriptors; first[] is the item prefix
// (ndesc + 1 entries, device), queue a device counter cleared beforehand.
cudaError_t launch_dedisperse_batch(const DedispArgs* d_descs, const int64_t* d_first,
                                    const int* d_ndm_blocks, int ndesc, size_t smem,
                                    unsigned long long* d_queue, int grid, bool grouped, int elem,
                                    cudaStream_t s);
cudaError_t launch_decimate_batch(const DecimateJob* d_jobs, const int64_t* d_first, int njobs,
                                  int grid, cudaStream_t s);

struct SpsArgs {
    const float* dd;        // row 0 of this range
    int64_t pitch;          // floats between rows
    int64_t length;         // samples per row
    int32_t nrows;
    int32_t dm_offset;
    int32_t range;
    int32_t max_width;
    int32_t wpad;
    float threshold;
    const double* rsqrt_w;  // [wpad] 1/sqrt(w) for w = 1..wpad (device, FP64)
    RowStats* stats;        // [nrows] of this range
    float2* table;          // [nrows][wpad] (r_w, -c_w)
    aa_candidate* cands;
    int64_t capacity;
    unsigned long long* count;
    float* snr_out;         // optional, row 0 of this range (same pitch)
    unsigned* err;
    int32_t prune;          // skip width blocks bounded below the threshold
    int32_t clip_c16;       // k-sigma clipping of the statistics, k = clip_c16 / 16
    int32_t clip_iters;     // clipping passes (0: plain statistics)
    int32_t ladder_g16;     // sparse width ladder growth x16 (0: every width)
    int32_t dec_w0;         // decimated width ladder base widths (0: off)
    int32_t beam;           // beam id stored in candidate records (batched mode)
    unsigned long long* evaluated;  // width-samples actually evaluated (instrumentation)
    CandChunk* chunks;      // chunk headers (all ranges)
    unsigned long long* nchunks;
    int64_t chunk_cap;
};
cudaError_t launch_sps_stats(const SpsArgs& a, cudaStream_t s);
// mu, sigma and width tables of a.nrows rows from the sums the dedispersion
// kernels accumulated (DedispArgs::st_acc; 3 words per row)
cudaError_t launch_sps_finalize(const SpsArgs& a, const unsigned long long* acc, cudaStream_t s);
cudaError_t launch_sps_boxcar(const SpsArgs& a, cudaStream_t s);
cudaError_t launch_sps_stats_batch(const SpsArgs* d_descs, const int64_t* d_first, int ndesc,
                                   unsigned long long* d_queue, int grid, cudaStream_t s);
cudaError_t launch_sps_boxcar_batch(const SpsArgs* d_descs, const int64_t* d_first,
                                    const int* d_ntiles, int ndesc, size_t smem,
                                    unsigned long long* d_queue, int grid, cudaStream_t s);
int sps_boxcar_tiles(int64_t length);
size_t sps_boxcar_smem(int wpad);
// dynamic shared memory of the boxcar kernel that serves (max_width, wpad,
// dec_w0): the decimated ladder's when dec_w0 > 0
size_t sps_boxcar_smem_for(int32_t max_width, int32_t wpad, int32_t dec_w0);
constexpr size_t kMaxBoxcarSmem = 227 * 1024;
// test hook: boxcar tiles per CTA (0: the launcher's choice)
extern int g_boxcar_seg_tiles;
cudaError_t launch_rsqrt_table(double* t, int wpad, cudaStream_t s);

// Candidate runs moved into their final order: run i copies n[i] records
// from src[i] to dst[i] (record indices).
struct RunCopy {
    int64_t src, dst;
    int64_t n;
};
cudaError_t launch_gather_runs(const aa_candidate* d_in, aa_candidate* d_out, const RunCopy* d_runs,
                               int64_t nruns, cudaStream_t s);

// Host-path candidate list: order the CTA runs (headers `heads`, records
// d_cands[0, stored)) by (beam when by_beam, dm_index, t0) with a counting sort
// of the headers, gather them in that order on the device and copy the ordered
// records into `res` with one device-to-host copy.
aa_status order_candidates(const aa_candidate* d_cands, int64_t stored, std::vector<CandChunk>& heads,
                           bool by_beam, cudaStream_t s, aa_candidates* res);

// ---------------------------------------------------- differentiable form --
struct F32FwdArgs {
    const float* x;
    int64_t x_pitch;
    int32_t nchans;
    int64_t nsamp;
    const float* w;
    const int32_t* shifts;
    int32_t d_begin, d_end;
    int64_t length;
    int32_t rowlen;
    float* y;
    int64_t pitch;
    const float* tmpl;
    double* loss_sum;
    float* resid;
    int64_t rpitch;
    float scale;
};
struct F32AdjArgs {
    const float* x;
    int64_t x_pitch;
    int32_t nchans;
    int64_t nsamp;
    const float* w;
    const int32_t* shifts;
    int32_t d_begin, d_end;
    const float* gy;
    int64_t gpitch;
    int64_t length;
    int32_t rowlen;
    float* gx;
    float* gw_part;
    float* gw;
};
constexpr int kF32Chunk = 256;  // DM trials per recomputation chunk of the loss gradient
int f32_fwd_rowlen(int span);
int f32_adj_rowlen(int cspan);
int f32_adj_tiles(int64_t nsamp);
cudaError_t launch_f32_forward(int mode, const F32FwdArgs& p, cudaStream_t s);
cudaError_t launch_f32_adjoint(const F32AdjArgs& p, cudaStream_t s);
cudaError_t launch_finish_loss(const double* sum, double n, double* loss, cudaStream_t s);

// Host list of n records already in (dm_index, t) order on the device:
// copied on stream s into a page-locked block of the library's pool (the
// call synchronises s); total = candidates found (may exceed n).
aa_status candidates_copy_ordered(const aa_candidate* d_sorted, int64_t n, int64_t total, cudaStream_t s,
                                  aa_candidates** out);

// candidate-list objects shared by the single-beam and batched paths
aa_candidates* candidates_new();
std::vector<aa_candidate>& candidates_list(aa_candidates* c);
void candidates_set_total(aa_candidates* c, int64_t total);

}  // namespace aa

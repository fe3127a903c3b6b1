// Fused dedispersion -> single-pulse search without the [ndm][L] series of
// the whole plan (arXiv:1912.07704 Sec. 1 and 2.3: the data are analysed
// entirely on the GPU, in device memory the plan requests up front).
//
// Ranges are processed one after another, a decimated range's input built
// straight from the 8-bit input into one buffer shared by all ranges (so only
// the largest decimated input is ever held), and each range in stripes of
// consecutive DM trials (whole blocks of kDmPerBlock): the stripe's series
// are dedispersed into one stripe buffer
// while the kernels sum every row exactly (sum y, sum y^2 in 128 bits), a
// finalize kernel turns those sums into mu, sigma and the width table with
// the arithmetic of the statistics kernel, and the boxcar search runs over
// the stripe and appends its candidates.  The next stripe reuses the buffer.
// Results -- candidates, chunk headers, optional B(t) -- are those of
// aa_dedisperse_device followed by aa_sps_search_device, bit for bit; the
// separate statistics pass over the series disappears.  With k-sigma clipped
// statistics the statistics kernel runs on each stripe instead (clipping
// needs several passes over a row).
#include <algorithm>

#include "aa_internal.h"

using namespace aa;

namespace {

aa_status fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? AA_ERR_NOMEM : AA_ERR_CUDA;
}

#define AA_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return fail(e_, (what));  \
    } while (0)

constexpr int32_t kDefaultStripe = 256;  // trials per stripe when the caller passes 0

// Workspace of the fused search: [error word block][decimated input of the
// current range][search workspace][stripe series][row sums], each part
// 256-byte aligned.
struct FusedLayout {
    Layout L;
    int32_t stripe = 0;
    int64_t stripe_pitch = 0;  // floats per stripe row (the widest range's pitch)
    int64_t dec_offset = 0, sps_offset = 0, stripe_offset = 0, acc_offset = 0, bytes = 0;
};

aa_status fused_layout(const aa_plan& p, int64_t nsamp, int32_t max_width, int32_t stripe, FusedLayout& f) {
    if (stripe == 0) stripe = kDefaultStripe;
    if (stripe < kDmPerBlock || stripe % kDmPerBlock) {
        set_error("stripe_trials must be 0 or a positive multiple of %d", kDmPerBlock);
        return AA_ERR_ARG;
    }
    for (size_t r = 0; r < p.ranges.size(); ++r)
        if (p.ranges[r].strategy == 2 || p.ranges[r].strategy == 3) {
            set_error("range %zu uses sub-band or FDMT dedispersion, which the fused search does not stripe", r);
            return AA_ERR_CONFIG;
        }
    f.L = make_layout(p, nsamp, max_width);
    int32_t ndm_max = 0;
    for (const auto& g : p.ranges) ndm_max = std::max(ndm_max, g.desc.ndm);
    f.stripe = std::min(stripe, (int32_t)round_up(std::max(ndm_max, 1), kDmPerBlock));
    for (int64_t pr : f.L.pitch) f.stripe_pitch = std::max(f.stripe_pitch, pr);
    int64_t dec_bytes = 0;
    for (size_t k = 0; k < p.decs.size(); ++k)
        dec_bytes = std::max(dec_bytes, (int64_t)p.nchans * f.L.dec_pitch[k] * 2);
    f.dec_offset = kErrBlock;
    f.sps_offset = f.dec_offset + round_up(dec_bytes, 256);
    f.stripe_offset = f.sps_offset + round_up(f.L.sps_ws, 256);
    f.acc_offset = f.stripe_offset + round_up((int64_t)f.stripe * f.stripe_pitch * 4, 256);
    f.bytes = f.acc_offset + round_up((int64_t)f.stripe * 3 * 8, 256);
    return AA_OK;
}

}  // namespace

extern "C" {

aa_status aa_search_fused_ws_bytes(const aa_plan* p, int64_t nsamp, int32_t max_width, int32_t stripe_trials,
                                   size_t* bytes, size_t* sps_ws_offset) {
    clear_error();
    if (!p || !bytes) { set_error("plan/bytes is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    FusedLayout f;
    const aa_status st = fused_layout(*p, nsamp, max_width, stripe_trials, f);
    if (st != AA_OK) return st;
    *bytes = (size_t)f.bytes;
    if (sps_ws_offset) *sps_ws_offset = (size_t)f.sps_offset;
    return AA_OK;
}

aa_status aa_search_fused_device(const aa_plan* p, const uint8_t* d_in, int64_t nsamp, int64_t in_pitch,
                                 int32_t max_width, float threshold, int32_t stripe_trials,
                                 aa_candidate* d_cands, int64_t cand_capacity, unsigned long long* d_count,
                                 float* d_snr_out, void* d_ws, size_t ws_bytes, aa_stream_t stream) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (!p->ready) { set_error("plan is not bound to a device (aa_plan_bind)"); return AA_ERR_STATE; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->device) {
        set_error("current device %d differs from the plan's device %d", dev, p->device);
        return AA_ERR_STATE;
    }
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    if (cand_capacity < 0 || !d_count || (cand_capacity > 0 && !d_cands)) {
        set_error("candidate array/count invalid");
        return AA_ERR_ARG;
    }
    FusedLayout f;
    aa_status st = fused_layout(*p, nsamp, max_width, stripe_trials, f);
    if (st != AA_OK) return st;
    const Layout& L = f.L;
    if (!d_ws || (int64_t)ws_bytes < f.bytes) {
        set_error("workspace %zu bytes < required %lld", ws_bytes, (long long)f.bytes);
        return AA_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 || (d_in && reinterpret_cast<uintptr_t>(d_in) % 16) ||
        (d_snr_out && reinterpret_cast<uintptr_t>(d_snr_out) % 16)) {
        set_error("d_ws must be 256-byte and d_in/d_snr_out 16-byte aligned");
        return AA_ERR_ARG;
    }
    if (p->clip_iters > 0)
        for (int64_t len : L.length)
            if (len >= (int64_t(1) << 31)) {
                set_error("k-sigma clipping supports series shorter than 2^31 samples");
                return AA_ERR_CONFIG;
            }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AA_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s), "clear count");
    if (L.dd_elems == 0 || L.dm_trial_samples == 0) return AA_OK;
    if (!d_in || in_pitch < nsamp || in_pitch % 16 != 0) {
        set_error("d_in must be non-NULL with in_pitch >= nsamp and a multiple of 16");
        return AA_ERR_ARG;
    }
    char* ws = static_cast<char*>(d_ws);
    char* sps = ws + f.sps_offset;
    float* stripe = reinterpret_cast<float*>(ws + f.stripe_offset);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(ws + f.acc_offset);
    unsigned* err = reinterpret_cast<unsigned*>(ws);  // one error word for both stages
    AA_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s), "clear error word");
    AA_CUDA(cudaMemsetAsync(sps, 0, 24, s), "clear search counters");
    double* rsw = reinterpret_cast<double*>(sps + kErrBlock);
    {
        ProfScope prof(kKRsqrt, s);
        AA_CUDA(launch_rsqrt_table(rsw, L.wpad, s), "rsqrt table launch");
    }
    RowStats* stats = reinterpret_cast<RowStats*>(sps + L.stats_offset);
    float2* table = reinterpret_cast<float2*>(sps + L.table_offset);
    const bool fused_stats = p->clip_iters == 0;
    for (size_t r = 0; r < p->ranges.size(); ++r) {
        const RangePlan& g = p->ranges[r];
        if (L.length[r] <= 0) continue;
        const int C = p->nchans;
        const void* in = d_in;
        int64_t pitch_in = in_pitch;
        if (g.desc.dec > 1) {  // this range's decimated input, from the 8-bit input
            const size_t k = std::find(p->decs.begin(), p->decs.end(), g.desc.dec) - p->decs.begin();
            uint16_t* xd = reinterpret_cast<uint16_t*>(ws + f.dec_offset);
            ProfScope prof(kKDecimate, s);
            AA_CUDA(launch_decimate(d_in, 1, in_pitch, C, nsamp / g.desc.dec, g.desc.dec, xd, L.dec_pitch[k], s),
                    "decimate launch");
            in = xd;
            pitch_in = L.dec_pitch[k];
        }
        for (int32_t s0 = 0; s0 < g.desc.ndm; s0 += f.stripe) {
            const int32_t n = std::min(f.stripe, g.desc.ndm - s0);
            if (fused_stats)
                AA_CUDA(cudaMemsetAsync(acc, 0, (size_t)n * 3 * 8, s), "clear row sums");
            DedispArgs a{};
            a.in = in;
            a.in_pitch = pitch_in;
            a.nchans = C;
            a.nsamp = L.nsamp_dec[r];
            a.length = L.length[r];
            a.ndm = n;
            a.shifts = g.d_shifts + (int64_t)s0 * C;
            a.out = stripe;
            a.out_pitch = L.pitch[r];
            fill_strategy(a, g);
            a.err = err;
            a.dmb0 = s0 / kDmPerBlock;
            a.st_acc = fused_stats ? acc : nullptr;
            {
                ProfScope prof(g.elem == 1 ? kKDedispU8 : kKDedispU16, s);
                AA_CUDA(launch_dedisperse(a, s), "dedisperse launch");
            }
            SpsArgs sa{};
            sa.dd = stripe;
            sa.pitch = L.pitch[r];
            sa.length = L.length[r];
            sa.nrows = n;
            sa.dm_offset = g.dm_offset + s0;
            sa.range = (int32_t)r;
            sa.max_width = max_width;
            sa.wpad = L.wpad;
            sa.threshold = threshold;
            sa.rsqrt_w = rsw;
            sa.stats = stats + g.dm_offset + s0;
            sa.table = table + (int64_t)(g.dm_offset + s0) * L.wpad;
            sa.cands = d_cands;
            sa.capacity = cand_capacity;
            sa.count = d_count;
            sa.snr_out = d_snr_out ? d_snr_out + L.row_offset[r] + (int64_t)s0 * L.pitch[r] : nullptr;
            sa.prune = d_snr_out ? 0 : 1;  // B(t) everywhere requested: exhaustive
            sa.clip_c16 = p->clip_c16;
            sa.clip_iters = p->clip_iters;
            sa.ladder_g16 = p->ladder_g16;
            sa.dec_w0 = p->dec_w0;
            sa.err = err;
            sa.chunks = reinterpret_cast<CandChunk*>(sps + L.chunk_offset);
            sa.nchunks = reinterpret_cast<unsigned long long*>(sps + kChunkCounterOffset);
            sa.chunk_cap = L.chunk_cap;
            sa.evaluated = reinterpret_cast<unsigned long long*>(sps + kEvaluatedOffset);
            if (fused_stats) {
                ProfScope prof(kKFinalize, s);
                AA_CUDA(launch_sps_finalize(sa, acc, s), "statistics finalize launch");
            } else {
                ProfScope prof(kKStats, s);
                AA_CUDA(launch_sps_stats(sa, s), "sps stats launch");
            }
            ProfScope prof(kKBoxcar, s);
            AA_CUDA(launch_sps_boxcar(sa, s), "sps boxcar launch");
        }
    }
    return AA_OK;
}

}  // extern "C"

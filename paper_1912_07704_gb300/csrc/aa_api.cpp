// C-ABI entry points: device-pointer calls (caller-owned device memory) and
// the host-buffer path with library-owned results (arXiv:1912.07704 Sec. 2.3
// memory requests, Sec. 2.4 ownership, Sec. 3.1 usage steps 4-8).
#include <algorithm>
#include <mutex>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "aa_internal.h"

namespace aa {
extern int g_fault_skip_chunk;
extern uint64_t g_wait_limit_ns;
}  // namespace aa

using namespace aa;

struct aa_dd_result {
    const aa_plan* plan = nullptr;
    float* d_out = nullptr;      // dd_elems floats followed by the error word
    unsigned* d_err = nullptr;
    int64_t nsamp = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
};

namespace aa {
namespace {
// Page-locked host blocks for ordered candidate lists, kept for reuse: a list
// of tens of millions of records is then copied at the link's speed into
// memory that is already mapped (a fresh pageable allocation is staged and
// faults in page by page).  Blocks are never returned to the system.
class PinnedPool {
  public:
    void* acquire(size_t bytes, size_t& got) {
        {
            std::lock_guard<std::mutex> g(mu_);
            size_t best = free_.size();
            for (size_t i = 0; i < free_.size(); ++i)
                if (free_[i].first >= bytes && (best == free_.size() || free_[i].first < free_[best].first))
                    best = i;
            if (best < free_.size()) {
                got = free_[best].first;
                void* p = free_[best].second;
                free_.erase(free_.begin() + (long)best);
                return p;
            }
        }
        const size_t want = (bytes + (64u << 20) - 1) / (64u << 20) * (64u << 20);  // 64 MiB steps
        void* p = nullptr;
        if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        got = want;
        return p;
    }
    void release(void* p, size_t bytes) {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu_);
        free_.emplace_back(bytes, p);
    }

  private:
    std::mutex mu_;
    std::vector<std::pair<size_t, void*>> free_;
};
PinnedPool& pinned_pool() {
    static PinnedPool* pool = new PinnedPool();  // outlives every result
    return *pool;
}
}  // namespace
}  // namespace aa

struct aa_candidates {
    std::vector<aa_candidate> list;  // filled by the batch and server paths
    aa_candidate* ordered = nullptr; // filled by order_candidates (pinned pool block)
    size_t ordered_bytes = 0;
    int64_t nordered = 0;
    int64_t total = 0;
    ~aa_candidates() { aa::pinned_pool().release(ordered, ordered_bytes); }
};

namespace aa {
aa_candidates* candidates_new() { return new (std::nothrow) aa_candidates(); }


std::vector<aa_candidate>& candidates_list(aa_candidates* c) { return c->list; }
void candidates_set_total(aa_candidates* c, int64_t total) { c->total = total; }
}  // namespace aa

namespace {

aa_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? AA_ERR_NOMEM : AA_ERR_CUDA;
}

#define AA_CUDA(call, what)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
    } while (0)

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

aa_status check_device(const aa_plan* p) {
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (!p->ready) { set_error("plan is not bound to a device (aa_plan_bind)"); return AA_ERR_STATE; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->device) {
        set_error("current device %d differs from the plan's device %d", dev, p->device);
        return AA_ERR_STATE;
    }
    return AA_OK;
}

// Stream-ordered allocations released together unless kept.
struct AsyncAllocs {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit AsyncAllocs(cudaStream_t st) : s(st) {}
    void* get(size_t bytes) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return p;
    }
    void keep(void* p) { ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end()); }
    ~AsyncAllocs() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

void keep_pool_memory(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[device] = true;
}



}  // namespace

namespace aa {

aa_status order_candidates(const aa_candidate* d_cands, int64_t stored, std::vector<CandChunk>& heads,
                           bool by_beam, cudaStream_t s, aa_candidates* res) {
    // counting sort of the runs by (beam, dm_index), then by t0 inside a bucket
    uint32_t max_dm = 0, max_beam = 0;
    for (const CandChunk& h : heads) {
        max_dm = std::max(max_dm, h.dm_index);
        if (by_beam) max_beam = std::max(max_beam, h.reserved);
    }
    const uint64_t kdm = (uint64_t)max_dm + 1;
    const uint64_t nkeys = ((uint64_t)max_beam + 1) * kdm;
    auto key = [&](const CandChunk& h) { return (by_beam ? (uint64_t)h.reserved * kdm : 0ull) + h.dm_index; };
    std::vector<uint64_t> uk;  // bucket index -> key, used only when keys are sparse
    const bool dense = nkeys <= 4 * (uint64_t)heads.size() + 65536;
    if (!dense) {
        uk.resize(heads.size());
        for (size_t i = 0; i < heads.size(); ++i) uk[i] = key(heads[i]);
        std::sort(uk.begin(), uk.end());
        uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
    }
    const size_t nb = dense ? (size_t)nkeys : uk.size();
    std::vector<int64_t> start(nb + 1, 0);
    std::vector<uint32_t> bucket(heads.size());
    for (size_t i = 0; i < heads.size(); ++i) {
        const uint64_t k = key(heads[i]);
        bucket[i] = dense ? (uint32_t)k : (uint32_t)(std::lower_bound(uk.begin(), uk.end(), k) - uk.begin());
        ++start[bucket[i] + 1];
    }
    for (size_t b = 0; b < nb; ++b) start[b + 1] += start[b];
    std::vector<CandChunk> sorted(heads.size());
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (size_t i = 0; i < heads.size(); ++i) sorted[(size_t)fill[bucket[i]]++] = heads[i];
    }
    for (size_t b = 0; b < nb; ++b)
        if (start[b + 1] - start[b] > 1)
            std::sort(sorted.begin() + start[b], sorted.begin() + start[b + 1],
                  [](const CandChunk& x, const CandChunk& y) { return x.t0 < y.t0; });
    // destinations in that order (records past `stored` were not written)
    std::vector<RunCopy> runs;
    runs.reserve(sorted.size());
    int64_t dst = 0;
    for (const CandChunk& h : sorted) {
        const int64_t src = (int64_t)h.base;
        const int64_t n = std::min<int64_t>((int64_t)h.n, std::max<int64_t>(0, stored - src));
        if (n > 0) {
            runs.push_back(RunCopy{src, dst, n});
            dst += n;
        }
    }
    res->nordered = 0;
    if (dst == 0) return AA_OK;
    pinned_pool().release(res->ordered, res->ordered_bytes);
    res->ordered = static_cast<aa_candidate*>(
        pinned_pool().acquire((size_t)dst * sizeof(aa_candidate), res->ordered_bytes));
    if (!res->ordered) {
        res->ordered_bytes = 0;
        set_error("page-locked host allocation of %lld candidates failed", (long long)dst);
        return AA_ERR_NOMEM;
    }
    AsyncAllocs mem(s);
    aa_candidate* d_out = static_cast<aa_candidate*>(mem.get((size_t)dst * sizeof(aa_candidate)));
    RunCopy* d_runs = static_cast<RunCopy*>(mem.get(runs.size() * sizeof(RunCopy)));
    if (!d_out || !d_runs) { set_error("device allocation failed"); return AA_ERR_NOMEM; }
    AA_CUDA(cudaMemcpyAsync(d_runs, runs.data(), runs.size() * sizeof(RunCopy), cudaMemcpyHostToDevice, s),
            "upload run order");
    AA_CUDA(launch_gather_runs(d_cands, d_out, d_runs, (int64_t)runs.size(), s), "gather candidates");
    AA_CUDA(cudaMemcpyAsync(res->ordered, d_out, (size_t)dst * sizeof(aa_candidate),
                            cudaMemcpyDeviceToHost, s),
            "read candidates");
    AA_CUDA(cudaStreamSynchronize(s), "synchronize");
    res->nordered = dst;
    return AA_OK;
}

aa_status candidates_copy_ordered(const aa_candidate* d_sorted, int64_t n, int64_t total, cudaStream_t s,
                                  aa_candidates** out) {
    *out = nullptr;
    aa_candidates* res = candidates_new();
    if (!res) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
    res->total = total;
    if (n > 0) {
        res->ordered = static_cast<aa_candidate*>(
            pinned_pool().acquire((size_t)n * sizeof(aa_candidate), res->ordered_bytes));
        if (!res->ordered) {
            res->ordered_bytes = 0;
            delete res;
            set_error("page-locked host allocation of %lld candidates failed", (long long)n);
            return AA_ERR_NOMEM;
        }
        cudaError_t e = cudaMemcpyAsync(res->ordered, d_sorted, (size_t)n * sizeof(aa_candidate),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            delete res;
            return cuda_fail(e, "read candidates");
        }
        res->nordered = n;
    }
    *out = res;
    return AA_OK;
}

cudaError_t launch_decimation_cascade(const aa_plan& p, const Layout& L, const uint8_t* d_in, int64_t in_pitch,
                                      char* ws, cudaStream_t s) {
    for (size_t k = 0; k < p.decs.size(); ++k) {
        const int dec = p.decs[k];
        const void* src = d_in;
        int src_elem = 1, src_dec = 1;
        int64_t src_pitch = in_pitch;
        for (size_t j = 0; j < k; ++j)
            if (dec % p.decs[j] == 0) {  // the largest decimation dividing this one
                src = ws + L.dec_offset[j];
                src_elem = 2;
                src_dec = p.decs[j];
                src_pitch = L.dec_pitch[j];
            }
        ProfScope prof(kKDecimate, s);
        const cudaError_t e = launch_decimate(src, src_elem, src_pitch, p.nchans, L.nsamp / dec, dec / src_dec,
                                              reinterpret_cast<uint16_t*>(ws + L.dec_offset[k]), L.dec_pitch[k], s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace aa

// FDMT strategy of range r: the depths of its channel tree, deepest first,
// through two 32-bit depth buffers of the workspace; the root writes the
// range's output rows.
static aa_status launch_fdmt(const aa_plan* p, size_t r, const Layout& L, const void* in, int64_t in_pitch,
                             float* d_out, char* ws, cudaStream_t s) {
    const RangePlan& g = p->ranges[r];
    const FdmtPlan& fd = g.fd;
    if (L.length[r] <= 0 || g.desc.ndm <= 0) return AA_OK;
    if (!fd.d_rows || fd.depths < 1) {
        set_error("range %zu: FDMT tables are not on the device", r);
        return AA_ERR_STATE;
    }
    if (L.fdmt_offset < 0 || L.fdmt_rows < fd.max_rows) {
        set_error("range %zu: FDMT workspace missing from the layout", r);
        return AA_ERR_STATE;
    }
    const int64_t nd = L.nsamp_dec[r];
    uint32_t* buf[2] = {reinterpret_cast<uint32_t*>(ws + L.fdmt_offset),
                        reinterpret_cast<uint32_t*>(ws + L.fdmt_offset +
                                                    round_up(L.fdmt_rows * L.fdmt_pitch * 4, 256))};
    for (int q = 0; q < fd.depths; ++q) {
        const int depth = fd.depths - 1 - q;  // deepest first
        const FdmtRow* rows = fd.d_rows + fd.first[(size_t)q];
        const int nrows = (int)(fd.first[(size_t)q + 1] - fd.first[(size_t)q]);
        const uint32_t* prev = buf[(depth + 1) & 1];  // the next-deeper depth (or unused)
        ProfScope prof(kKFdmt, s);
        const cudaError_t e =
            depth == 0 ? launch_fdmt_depth(rows, nrows, g.elem, in, in_pitch, prev, nullptr, L.fdmt_pitch, nd,
                                           d_out + L.row_offset[r], L.pitch[r], L.length[r], s)
                       : launch_fdmt_depth(rows, nrows, g.elem, in, in_pitch, prev, buf[depth & 1], L.fdmt_pitch,
                                           nd, nullptr, 0, 0, s);
        if (e != cudaSuccess) {
            set_error("FDMT depth %d launch: %s", depth, cudaGetErrorString(e));
            cudaGetLastError();
            return AA_ERR_CUDA;
        }
    }
    return AA_OK;
}

// Sub-band strategy of range r: stage 1 per band into the 16-bit partial
// series (direct kernel), stage 2 over all coarse trials into the range's
// output rows (32-bit sums).
static aa_status launch_subband(const aa_plan* p, size_t r, const Layout& L, const void* in, int64_t in_pitch,
                                float* d_out, char* ws, unsigned* err, cudaStream_t s) {
    const RangePlan& g = p->ranges[r];
    const SubbandPlan& sb = g.sb;
    if (L.length[r] <= 0) return AA_OK;
    if (!sb.d_rel || !sb.d_s2) {
        set_error("range %zu: sub-band tables are not on the device", r);
        return AA_ERR_STATE;
    }
    auto shape = [](DedispArgs& a, const DirectShape& d) {
        a.elem = d.elem;
        a.rw = d.rw;
        a.cc = d.cc;
        a.nstage = d.nstage;
        a.flush = d.flush;
        a.smem = d.smem;
        a.grouped = 0;
    };
    const int C = p->nchans;
    const int64_t pitch1 = L.sub_pitch[r];
    uint16_t* z = reinterpret_cast<uint16_t*>(ws + L.sub_offset[r]);
    {
        size_t off = 0;
        for (int b = 0; b < sb.nsub; ++b) {
            ProfScope prof(kKSubband1, s);  // one record per launch
            const int c0 = b * sb.k, kb = std::min(C, c0 + sb.k) - c0;
            DedispArgs a{};
            a.in = static_cast<const char*>(in) + (int64_t)c0 * in_pitch * g.elem;
            a.in_pitch = in_pitch;
            a.nchans = kb;
            a.nsamp = L.nsamp_dec[r];
            a.length = L.sub_len[r];
            a.ndm = sb.ncoarse;
            a.shifts = sb.d_rel + off;
            a.out16 = z + (int64_t)b * sb.ncoarse * pitch1;
            a.out_pitch = pitch1;
            shape(a, sb.shape1);
            a.err = err;
            AA_CUDA(launch_dedisperse(a, s), "sub-band stage 1 launch");
            off += (size_t)sb.ncoarse * kb;
        }
    }
    ProfScope prof(kKSubband2, s);
    AA_CUDA(launch_subband_stage2(z, (int64_t)sb.ncoarse * pitch1, pitch1, L.sub_len[r], sb.nsub, sb.ncoarse, sb.m,
                                  g.desc.ndm, sb.d_s2, sb.span2, d_out + L.row_offset[r], L.pitch[r],
                                  L.length[r], s),
            "sub-band stage 2 launch");
    return AA_OK;
}

extern "C" {

aa_status aa_dedisperse_device(const aa_plan* p, const uint8_t* d_in, int64_t nsamp,
                               int64_t in_pitch, float* d_out, void* d_ws, size_t ws_bytes,
                               aa_stream_t stream) {
    clear_error();
    aa_status st = check_device(p);
    if (st != AA_OK) return st;
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    const Layout L = make_layout(*p, nsamp, 0);
    if (nsamp == 0 || L.dd_elems == 0) return AA_OK;
    if (!d_in || !d_out || !d_ws) { set_error("d_in, d_out and d_ws must be non-NULL"); return AA_ERR_ARG; }
    if (in_pitch < nsamp || in_pitch % 16 != 0) {
        set_error("in_pitch %lld must be >= nsamp and a multiple of 16", (long long)in_pitch);
        return AA_ERR_ARG;
    }
    if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_ws, 256)) {
        set_error("d_in/d_out must be 16-byte and d_ws 256-byte aligned");
        return AA_ERR_ARG;
    }
    if ((int64_t)ws_bytes < L.dedisp_ws) {
        set_error("workspace %zu bytes < required %lld", ws_bytes, (long long)L.dedisp_ws);
        return AA_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned* err = static_cast<unsigned*>(d_ws);
    AA_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s), "clear error word");
    char* ws = static_cast<char*>(d_ws);
    AA_CUDA(launch_decimation_cascade(*p, L, d_in, in_pitch, ws, s), "decimate launch");
    for (size_t r = 0; r < p->ranges.size(); ++r) {
        const RangePlan& g = p->ranges[r];
        DedispArgs a{};
        if (g.desc.dec == 1) {
            a.in = d_in;
            a.in_pitch = in_pitch;
        } else {
            const size_t k = std::find(p->decs.begin(), p->decs.end(), g.desc.dec) - p->decs.begin();
            a.in = ws + L.dec_offset[k];
            a.in_pitch = L.dec_pitch[k];
        }
        if (g.strategy == 2) {
            st = launch_subband(p, r, L, a.in, a.in_pitch, d_out, ws, err, s);
            if (st != AA_OK) return st;
            continue;
        }
        if (g.strategy == 3) {
            st = launch_fdmt(p, r, L, a.in, a.in_pitch, d_out, ws, s);
            if (st != AA_OK) return st;
            continue;
        }
        a.nchans = p->nchans;
        a.nsamp = L.nsamp_dec[r];
        a.length = L.length[r];
        a.ndm = g.desc.ndm;
        a.shifts = g.d_shifts;
        a.out = d_out + L.row_offset[r];
        a.out_pitch = L.pitch[r];
        fill_strategy(a, g);
        a.err = err;
        if (a.length <= 0) continue;
        ProfScope prof(g.elem == 1 ? kKDedispU8 : kKDedispU16, s);
        AA_CUDA(launch_dedisperse(a, s), "dedisperse launch");
    }
    return AA_OK;
}

aa_status aa_sps_search_device(const aa_plan* p, int64_t nsamp, const float* d_dd, int32_t max_width,
                               float threshold, aa_candidate* d_cands, int64_t cand_capacity,
                               unsigned long long* d_count, float* d_snr_out, void* d_ws,
                               size_t ws_bytes, aa_stream_t stream) {
    clear_error();
    aa_status st = check_device(p);
    if (st != AA_OK) return st;
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    if (cand_capacity < 0 || (cand_capacity > 0 && !d_cands)) { set_error("bad candidate buffer"); return AA_ERR_ARG; }
    if (!d_count || !d_ws) { set_error("d_count and d_ws must be non-NULL"); return AA_ERR_ARG; }
    if (!(threshold == threshold)) { set_error("threshold is NaN"); return AA_ERR_ARG; }
    const Layout L = make_layout(*p, nsamp, max_width);
    if ((int64_t)ws_bytes < L.sps_ws) {
        set_error("workspace %zu bytes < required %lld", ws_bytes, (long long)L.sps_ws);
        return AA_ERR_ARG;
    }
    if (sps_boxcar_smem_for(max_width, L.wpad, p->dec_w0) > kMaxBoxcarSmem) {
        set_error("max_width %d needs %zu bytes of shared memory per boxcar tile (at most %zu)", max_width,
                  sps_boxcar_smem_for(max_width, L.wpad, p->dec_w0), kMaxBoxcarSmem);
        return AA_ERR_CONFIG;
    }
    if (p->clip_iters > 0)
        for (int64_t len : L.length)
            if (len >= (int64_t(1) << 31)) {  // keeps the clipping test inside 128-bit integers
                set_error("k-sigma clipping supports series shorter than 2^31 samples");
                return AA_ERR_CONFIG;
            }
    if (!aligned(d_ws, 256) || (d_dd && !aligned(d_dd, 16)) || (d_snr_out && !aligned(d_snr_out, 16))) {
        set_error("d_ws must be 256-byte and d_dd/d_snr_out 16-byte aligned");
        return AA_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AA_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s), "clear count");
    if (L.dd_elems == 0 || L.dm_trial_samples == 0) return AA_OK;
    if (!d_dd) { set_error("d_dd is NULL"); return AA_ERR_ARG; }
    char* ws = static_cast<char*>(d_ws);
    unsigned* err = reinterpret_cast<unsigned*>(ws);
    AA_CUDA(cudaMemsetAsync(err, 0, 24, s), "clear error word and counters");
    unsigned long long* nchunks = reinterpret_cast<unsigned long long*>(ws + kChunkCounterOffset);
    CandChunk* chunks = reinterpret_cast<CandChunk*>(ws + L.chunk_offset);
    double* rsw = reinterpret_cast<double*>(ws + kErrBlock);
    {
        ProfScope prof(kKRsqrt, s);
        AA_CUDA(launch_rsqrt_table(rsw, L.wpad, s), "rsqrt table launch");
    }
    RowStats* stats = reinterpret_cast<RowStats*>(ws + L.stats_offset);
    float2* table = reinterpret_cast<float2*>(ws + L.table_offset);
    std::vector<SpsArgs> args(p->ranges.size());
    for (size_t r = 0; r < p->ranges.size(); ++r) {
        const RangePlan& g = p->ranges[r];
        SpsArgs& a = args[r];
        a.dd = d_dd + L.row_offset[r];
        a.pitch = L.pitch[r];
        a.length = L.length[r];
        a.nrows = g.desc.ndm;
        a.dm_offset = g.dm_offset;
        a.range = (int32_t)r;
        a.max_width = max_width;
        a.wpad = L.wpad;
        a.threshold = threshold;
        a.rsqrt_w = rsw;
        a.stats = stats + g.dm_offset;
        a.table = table + (int64_t)g.dm_offset * L.wpad;
        a.cands = d_cands;
        a.capacity = cand_capacity;
        a.count = d_count;
        a.snr_out = d_snr_out ? d_snr_out + L.row_offset[r] : nullptr;
        a.prune = d_snr_out ? 0 : 1;  // B(t) everywhere requested: exhaustive
        a.clip_c16 = p->clip_c16;
        a.clip_iters = p->clip_iters;
        a.ladder_g16 = p->ladder_g16;
        a.dec_w0 = p->dec_w0;
        a.err = err;
        a.chunks = chunks;
        a.nchunks = nchunks;
        a.chunk_cap = L.chunk_cap;
        a.evaluated = reinterpret_cast<unsigned long long*>(ws + kEvaluatedOffset);
        if (a.length <= 0) continue;
        {
            ProfScope prof(kKStats, s);
            AA_CUDA(launch_sps_stats(a, s), "sps stats launch");
        }
        ProfScope prof(kKBoxcar, s);
        AA_CUDA(launch_sps_boxcar(a, s), "sps boxcar launch");
    }
    return AA_OK;
}

aa_status aa_sps_workspace_work(const void* d_ws, aa_stream_t stream, int64_t* evaluated) {
    clear_error();
    if (!d_ws || !evaluated) { set_error("d_ws/evaluated is NULL"); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long v = 0;
    AA_CUDA(cudaMemcpyAsync(&v, static_cast<const char*>(d_ws) + kEvaluatedOffset, sizeof v,
                            cudaMemcpyDeviceToHost, s), "read work counter");
    AA_CUDA(cudaStreamSynchronize(s), "synchronize");
    *evaluated = (int64_t)v;
    return AA_OK;
}

aa_status aa_workspace_status(void* d_ws, aa_stream_t stream) {
    clear_error();
    if (!d_ws) { set_error("d_ws is NULL"); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned h = 0;
    AA_CUDA(cudaMemcpyAsync(&h, d_ws, sizeof h, cudaMemcpyDeviceToHost, s), "read error word");
    AA_CUDA(cudaStreamSynchronize(s), "synchronize");
    AA_CUDA(cudaMemsetAsync(d_ws, 0, sizeof h, s), "clear error word");
    if (h) { set_error("a bounded device-side wait gave up (code %u)", h); return AA_ERR_TIMEOUT; }
    return AA_OK;
}

aa_status aa_dedisperse(aa_plan* p, const uint8_t* host_in, int64_t nsamp, int64_t host_pitch,
                        aa_stream_t stream, aa_dd_result** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0 || (nsamp > 0 && (!host_in || host_pitch < nsamp))) {
        set_error("bad host input (nsamp %lld, pitch %lld)", (long long)nsamp, (long long)host_pitch);
        return AA_ERR_ARG;
    }
    if (!p->ready) {
        int dev = 0;
        AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
        aa_status b = aa_plan_bind(p, dev);
        if (b != AA_OK) return b;
    }
    aa_status st = check_device(p);
    if (st != AA_OK) return st;
    keep_pool_memory(p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Layout L = make_layout(*p, nsamp, 0);
    AsyncAllocs mem(s);
    aa_dd_result* res = new (std::nothrow) aa_dd_result();
    if (!res) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
    res->plan = p;
    res->nsamp = nsamp;
    res->stream = s;
    res->device = p->device;
    float* d_out = static_cast<float*>(mem.get((size_t)L.dd_elems * 4 + kErrBlock));
    uint8_t* d_in = static_cast<uint8_t*>(mem.get((size_t)p->nchans * L.in_pitch_min));
    void* d_ws = mem.get((size_t)L.dedisp_ws);
    if (!d_out || !d_in || !d_ws) {
        delete res;
        set_error("device allocation of %lld bytes failed",
                  (long long)(L.dd_elems * 4 + p->nchans * L.in_pitch_min + L.dedisp_ws));
        return AA_ERR_NOMEM;
    }
    if (nsamp > 0) {
        // one contiguous copy when the rows are packed alike on both sides
        cudaError_t e = host_pitch == L.in_pitch_min
                            ? cudaMemcpyAsync(d_in, host_in, (size_t)p->nchans * (size_t)host_pitch,
                                              cudaMemcpyHostToDevice, s)
                            : cudaMemcpy2DAsync(d_in, L.in_pitch_min, host_in, host_pitch, nsamp, p->nchans,
                                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) {
                e = cudaEventRecord(ev, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev);  // host input fully read
                cudaEventDestroy(ev);
            }
        }
        if (e != cudaSuccess) { delete res; return cuda_fail(e, "host-to-device copy"); }
    }
    st = aa_dedisperse_device(p, d_in, nsamp, L.in_pitch_min, d_out, d_ws, (size_t)L.dedisp_ws, stream);
    if (st != AA_OK) { delete res; return st; }
    unsigned* d_err = reinterpret_cast<unsigned*>(d_out + L.dd_elems);
    cudaError_t e = nsamp > 0 ? cudaMemcpyAsync(d_err, d_ws, sizeof(unsigned), cudaMemcpyDeviceToDevice, s)
                              : cudaMemsetAsync(d_err, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) { delete res; return cuda_fail(e, "keep error word"); }
    mem.keep(d_out);
    res->d_out = d_out;
    res->d_err = d_err;
    *out = res;
    return AA_OK;
}

aa_status aa_dd_result_view(const aa_dd_result* r, const float** d_out, int64_t* nsamp) {
    clear_error();
    if (!r) { set_error("result is NULL"); return AA_ERR_ARG; }
    if (d_out) *d_out = r->d_out;
    if (nsamp) *nsamp = r->nsamp;
    return AA_OK;
}

void aa_dd_result_destroy(aa_dd_result* r) {
    if (!r) return;
    if (r->d_out) cudaFreeAsync(r->d_out, r->stream);
    delete r;
}

aa_status aa_sps_search(aa_plan* p, const aa_dd_result* dd, int32_t max_width, float threshold,
                        int64_t cand_capacity, aa_stream_t stream, aa_candidates** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!p || !dd) { set_error("plan/result is NULL"); return AA_ERR_ARG; }
    if (dd->plan != p) { set_error("result was produced by another plan"); return AA_ERR_ARG; }
    if (cand_capacity < 0) { set_error("cand_capacity must be >= 0"); return AA_ERR_ARG; }
    aa_status st = check_device(p);
    if (st != AA_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Layout L = make_layout(*p, dd->nsamp, max_width > 0 ? max_width : 1);
    AsyncAllocs mem(s);
    void* d_ws = mem.get((size_t)L.sps_ws);
    aa_candidate* d_c = static_cast<aa_candidate*>(mem.get((size_t)std::max<int64_t>(cand_capacity, 1) * sizeof(aa_candidate)));
    unsigned long long* d_n = static_cast<unsigned long long*>(mem.get(sizeof(unsigned long long)));
    if (!d_ws || !d_c || !d_n) { set_error("device allocation failed"); return AA_ERR_NOMEM; }
    st = aa_sps_search_device(p, dd->nsamp, dd->d_out, max_width, threshold, d_c, cand_capacity, d_n,
                              nullptr, d_ws, (size_t)L.sps_ws, stream);
    if (st != AA_OK) return st;
    aa_candidates* res = new (std::nothrow) aa_candidates();
    if (!res) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
    unsigned long long total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, d_n, sizeof total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { delete res; return cuda_fail(e, "read candidate count"); }
    const int64_t stored = std::min<int64_t>((int64_t)total, cand_capacity);
    // Records arrive as per-CTA runs (each ordered by t); order the runs by
    // (dm_index, t0) through their headers, gather on the device, copy once.
    unsigned long long nchunks = 0;
    e = cudaMemcpyAsync(&nchunks, static_cast<char*>(d_ws) + kChunkCounterOffset, sizeof nchunks,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { delete res; return cuda_fail(e, "read candidate chunk count"); }
    const int64_t nh = std::min<int64_t>((int64_t)nchunks, L.chunk_cap);
    std::vector<CandChunk> heads((size_t)nh);
    if (nh > 0) {
        e = cudaMemcpyAsync(heads.data(), static_cast<char*>(d_ws) + L.chunk_offset,
                            (size_t)nh * sizeof(CandChunk), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { delete res; return cuda_fail(e, "read candidate chunks"); }
    }
    st = order_candidates(d_c, stored, heads, false, s, res);
    if (st != AA_OK) { delete res; return st; }
    res->total = (int64_t)total;
    unsigned h = 0, h2 = 0;
    e = cudaMemcpyAsync(&h, d_ws, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h2, dd->d_err, sizeof h2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { delete res; return cuda_fail(e, "read error word"); }
    h |= h2;
    if (h) { delete res; set_error("a bounded device-side wait gave up"); return AA_ERR_TIMEOUT; }
    *out = res;
    return (int64_t)total > cand_capacity ? AA_WARN_CAND_OVERFLOW : AA_OK;
}

aa_status aa_candidates_view(const aa_candidates* c, const aa_candidate** host, int64_t* stored,
                             int64_t* total) {
    clear_error();
    if (!c) { set_error("candidates is NULL"); return AA_ERR_ARG; }
    const bool ord = c->nordered > 0;
    const int64_t n = ord ? c->nordered : (int64_t)c->list.size();
    if (host) *host = n == 0 ? nullptr : (ord ? c->ordered : c->list.data());
    if (stored) *stored = n;
    if (total) *total = c->total;
    return AA_OK;
}

void aa_candidates_destroy(aa_candidates* c) { delete c; }

aa_status aa_debug_inject(int32_t what, int64_t value) {
    clear_error();
    switch (what) {
        case 0:  // reset
            g_fault_skip_chunk = -1;
            g_wait_limit_ns = 2000000000ull;
            g_boxcar_seg_tiles = 0;
            return AA_OK;
        case 1:  // never issue the staging copy of this channel chunk
            g_fault_skip_chunk = (int)value;
            return AA_OK;
        case 2:  // bounded-wait limit in nanoseconds
            if (value <= 0) { set_error("limit must be > 0"); return AA_ERR_ARG; }
            g_wait_limit_ns = (uint64_t)value;
            return AA_OK;
        case 3:  // boxcar tiles per CTA (0: the launcher's choice)
            if (value < 0 || value > 4096) { set_error("tiles per CTA must be in [0, 4096]"); return AA_ERR_ARG; }
            g_boxcar_seg_tiles = (int)value;
            return AA_OK;
    }
    set_error("unknown injection %d", what);
    return AA_ERR_ARG;
}

}  // extern "C"

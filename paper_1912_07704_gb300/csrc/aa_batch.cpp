// Batched multi-beam search: many independent beams (each its own bound
// plan and length) searched by one CUDA graph.  Beams are grouped into waves
// whose working set (decimated inputs, dedispersed series, search workspace)
// fits a memory budget; waves reuse one buffer region.  Within a wave the
// graph either issues each beam's own kernels (those of the single-beam path)
// on several concurrent branches, or runs one persistent work-queue kernel
// per stage (decimation, dedispersion, statistics, boxcar + peaks) whose
// queue spans every beam of the wave.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

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

// Concurrent graph branches per wave at creation.  Measured on 32 uneven
// beams of 2^17..2^20 samples and 128 short beams of 2^15..2^16: with 8
// branches the batch runs at 1.00x and 1.05x the speed of the same beams
// issued one after another; the persistent work-queue form at 0.96x / 0.97x.
constexpr int kDefaultBranches = 8;

struct WaveTables {
    // host copies (uploaded into the arena)
    std::vector<DecimateJob> dec_jobs[4];  // one launch per cascade level
    std::vector<int64_t> dec_first[4];
    // one persistent launch per kernel variant: [grouped * 2 + (16-bit input)]
    std::vector<DedispArgs> dd[4];
    std::vector<int64_t> dd_first[4];
    std::vector<int> dd_ndmb[4];
    std::vector<SpsArgs> sps;
    std::vector<int64_t> st_first, bx_first;
    std::vector<int> bx_ntiles;
    // device copies
    DecimateJob* d_dec_jobs[4] = {};
    int64_t* d_dec_first[4] = {};
    DedispArgs* d_dd[4] = {};
    int64_t* d_dd_first[4] = {};
    int* d_dd_ndmb[4] = {};
    SpsArgs* d_sps = nullptr;
    int64_t* d_st_first = nullptr;
    int64_t* d_bx_first = nullptr;
    int* d_bx_ntiles = nullptr;
    unsigned long long* d_queues = nullptr;  // 6 counters: 4 dedispersion variants, stats, boxcar
    size_t dd_smem[4] = {0, 0, 0, 0};
    size_t bx_smem = 0;  // the largest boxcar shared memory of the wave's descriptors
};

}  // namespace

struct aa_batch {
    int device = -1;
    int32_t nbeams = 0;
    std::vector<aa_plan*> plans;
    std::vector<int64_t> nsamps, in_pitch, in_offset;
    int32_t max_width = 0;
    float threshold = 0;
    int64_t capacity = 0;
    int64_t chunk_cap = 0;
    int32_t wpad = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<std::vector<int>> waves;
    std::vector<WaveTables> tables;
    aa_candidate* d_cands = nullptr;
    unsigned long long* d_counts = nullptr;  // [0] candidates, [1] chunks
    CandChunk* d_chunks = nullptr;
    unsigned* d_err = nullptr;
    double* d_rsw = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid_dd = 0, grid_st = 0, grid_bx = 0, grid_dec = 0;
    std::vector<float*> dd_of;    // each beam's dedispersed series (inside its wave's region)
    std::vector<int> wave_of;     // each beam's wave
    // per-beam launch arguments of the branched form (single-beam kernels)
    int32_t branches = 0;  // 0: persistent work-queue kernels; k >= 1: k graph branches
    std::vector<std::vector<DedispArgs>> beam_dd;
    std::vector<std::vector<SpsArgs>> beam_sps;
    std::vector<char*> beam_dec_ws;
    std::vector<double> beam_work;  // channel-adds + boxcar samples, for dealing beams to branches
};

namespace {

struct BeamNeeds {
    int64_t dec_bytes = 0, dd_bytes = 0, sps_bytes = 0;
    int64_t total() const { return dec_bytes + dd_bytes + sps_bytes; }
};

BeamNeeds beam_needs(const aa_plan& p, int64_t nsamp, int32_t W) {
    const Layout L = make_layout(p, nsamp, W);
    BeamNeeds n;
    n.dec_bytes = round_up(L.dedisp_ws, 256);
    n.dd_bytes = round_up(L.dd_elems * 4, 256);
    n.sps_bytes = round_up((int64_t)p.ndm_total * (int64_t)sizeof(RowStats), 256) +
                  round_up((int64_t)p.ndm_total * L.wpad * 8, 256);
    return n;
}

void free_batch(aa_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->arena) cudaFree(b->arena);
    delete b;
}

// One beam's stages as the single-beam path issues them: decimation cascade,
// one dedispersion launch per range, then statistics and boxcar + peaks per
// range.
cudaError_t issue_beam(const aa_batch* b, int bi, cudaStream_t s) {
    const aa_plan& pl = *b->plans[bi];
    const Layout L = make_layout(pl, b->nsamps[bi], b->max_width);
    const uint8_t* d_in = reinterpret_cast<const uint8_t*>(b->arena + b->in_offset[bi]);
    cudaError_t e = launch_decimation_cascade(pl, L, d_in, b->in_pitch[bi], b->beam_dec_ws[bi], s);
    for (const DedispArgs& a : b->beam_dd[bi])
        if (e == cudaSuccess) e = launch_dedisperse(a, s);
    for (const SpsArgs& a : b->beam_sps[bi]) {
        if (e == cudaSuccess) e = launch_sps_stats(a, s);
        if (e == cudaSuccess) e = launch_sps_boxcar(a, s);
    }
    return e;
}

// Records the whole batch (every wave) into b->graph / b->exec: either one
// persistent work-queue kernel per stage and wave, or each beam's own
// launches on b->branches concurrent branches (beams of a wave dealt to the
// least-loaded branch, largest first; a wave starts when every branch of the
// previous one has finished, since it reuses their buffers).
cudaError_t capture_graph(aa_batch* b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    const int nbr = b->branches;
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> bs((size_t)nbr, nullptr);
    std::vector<cudaEvent_t> ev((size_t)nbr + 1, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int k = 0; k < nbr && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&bs[k], cudaStreamNonBlocking);
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (le == cudaSuccess) le = x; };
        chk(cudaMemsetAsync(b->d_counts, 0, 16, cs));
        chk(cudaMemsetAsync(b->d_err, 0, 4, cs));
        chk(launch_rsqrt_table(b->d_rsw, b->wpad, cs));
        for (size_t wi = 0; wi < b->tables.size(); ++wi) {
            WaveTables& T = b->tables[wi];
            if (nbr == 0) {
                chk(cudaMemsetAsync(T.d_queues, 0, 6 * sizeof(unsigned long long), cs));
                for (int lv = 0; lv < 4; ++lv)
                    chk(launch_decimate_batch(T.d_dec_jobs[lv], T.d_dec_first[lv], (int)T.dec_jobs[lv].size(),
                                              b->grid_dec, cs));
                for (int sg = 0; sg < 4; ++sg)
                    chk(launch_dedisperse_batch(T.d_dd[sg], T.d_dd_first[sg], T.d_dd_ndmb[sg], (int)T.dd[sg].size(),
                                                T.dd_smem[sg], &T.d_queues[sg], b->grid_dd, sg >= 2, (sg & 1) + 1, cs));
                chk(launch_sps_stats_batch(T.d_sps, T.d_st_first, (int)T.sps.size(), &T.d_queues[4],
                                           b->grid_st, cs));
                chk(launch_sps_boxcar_batch(T.d_sps, T.d_bx_first, T.d_bx_ntiles, (int)T.sps.size(), T.bx_smem,
                                            &T.d_queues[5], b->grid_bx, cs));
                continue;
            }
            std::vector<int> order(b->waves[wi]);
            std::stable_sort(order.begin(), order.end(),
                             [&](int x, int y) { return b->beam_work[x] > b->beam_work[y]; });
            std::vector<std::vector<int>> lanes((size_t)nbr);
            std::vector<double> load((size_t)nbr, 0.0);
            for (int bi : order) {
                const size_t k = std::min_element(load.begin(), load.end()) - load.begin();
                lanes[k].push_back(bi);
                load[k] += b->beam_work[bi];
            }
            chk(cudaEventRecord(ev[nbr], cs));  // fork
            for (int k = 0; k < nbr; ++k) {
                if (lanes[k].empty()) continue;
                chk(cudaStreamWaitEvent(bs[k], ev[nbr], 0));
                for (int bi : lanes[k]) chk(issue_beam(b, bi, bs[k]));
                chk(cudaEventRecord(ev[k], bs[k]));
                chk(cudaStreamWaitEvent(cs, ev[k], 0));  // join
            }
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess && le != cudaSuccess) {
            cudaGraphDestroy(g);
            e = le;
        } else if (e == cudaSuccess) {
            b->graph = g;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    for (cudaStream_t x : bs)
        if (x) cudaStreamDestroy(x);
    if (cs) cudaStreamDestroy(cs);
    return e;
}

}  // namespace

extern "C" {

aa_status aa_batch_create(aa_plan* const* plans, const int64_t* nsamps, int32_t nbeams,
                          int32_t max_width, float threshold, int64_t cand_capacity,
                          int64_t wave_budget_bytes, aa_batch** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!plans || !nsamps || nbeams < 1 || nbeams > 256) { set_error("need 1..256 beams"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    if (cand_capacity < 1) { set_error("cand_capacity must be >= 1"); return AA_ERR_ARG; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    for (int i = 0; i < nbeams; ++i) {
        if (!plans[i]) { set_error("plan %d is NULL", i); return AA_ERR_ARG; }
        if (nsamps[i] < 0) { set_error("nsamp of beam %d is negative", i); return AA_ERR_ARG; }
        for (const auto& rg : plans[i]->ranges)
            if (rg.strategy == 2 || rg.strategy == 3) {
                set_error("beam %d: sub-band and FDMT ranges are not available in batched runs", i);
                return AA_ERR_CONFIG;
            }
        if (plans[i]->clip_iters > 0 && nsamps[i] >= (int64_t(1) << 31)) {
            set_error("beam %d: k-sigma clipping supports series shorter than 2^31 samples", i);
            return AA_ERR_CONFIG;
        }
        if (!plans[i]->ready) {
            aa_status st = aa_plan_bind(plans[i], dev);
            if (st != AA_OK) return st;
        }
        if (plans[i]->device != dev) { set_error("plan %d is bound to another device", i); return AA_ERR_STATE; }
    }
    aa_batch* b = new (std::nothrow) aa_batch();
    if (!b) return AA_ERR_NOMEM;
    b->device = dev;
    b->nbeams = nbeams;
    b->plans.assign(plans, plans + nbeams);
    b->nsamps.assign(nsamps, nsamps + nbeams);
    b->max_width = max_width;
    b->threshold = threshold;
    b->capacity = cand_capacity;
    b->wpad = (int32_t)round_up(max_width, kSpsSlots);

    // waves by memory
    if (wave_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        wave_budget_bytes = (int64_t)(fr / 2);
    }
    std::vector<BeamNeeds> needs(nbeams);
    int64_t in_bytes = 0, chunk_cap = 0;
    for (int i = 0; i < nbeams; ++i) {
        needs[i] = beam_needs(*plans[i], nsamps[i], max_width);
        const Layout L = make_layout(*plans[i], nsamps[i], max_width);
        b->in_pitch.push_back(L.in_pitch_min);
        b->in_offset.push_back(in_bytes);
        in_bytes += round_up((int64_t)plans[i]->nchans * L.in_pitch_min, 256);
        chunk_cap += L.chunk_cap;
    }
    b->chunk_cap = std::max<int64_t>(chunk_cap, 1);
    int64_t wave_bytes = 0, cur = 0;
    std::vector<int> w;
    for (int i = 0; i < nbeams; ++i) {
        if (!w.empty() && cur + needs[i].total() > wave_budget_bytes) {
            b->waves.push_back(w);
            wave_bytes = std::max(wave_bytes, cur);
            w.clear();
            cur = 0;
        }
        w.push_back(i);
        cur += needs[i].total();
    }
    b->waves.push_back(w);
    wave_bytes = std::max(wave_bytes, cur);

    // descriptor tables: 25 arrays per wave, each padded to 256 bytes
    constexpr int64_t kArraysPerWave = 25;
    size_t table_bytes = 0;
    for (auto& wv : b->waves) {
        int64_t nr = 0;
        for (int i : wv) nr += (int64_t)plans[i]->ranges.size();
        table_bytes += (size_t)(kArraysPerWave * 256 +
                                4 * round_up(nr * (int64_t)sizeof(DedispArgs), 256) +
                                round_up(nr * (int64_t)sizeof(SpsArgs), 256) +
                                6 * round_up((nr + 1) * 8, 256) + 5 * round_up(nr * 4, 256) +
                                4 * round_up(nr * (int64_t)sizeof(DecimateJob), 256) +
                                4 * round_up((nr + 1) * 8, 256));
    }
    const int64_t cand_bytes = round_up(cand_capacity * (int64_t)sizeof(aa_candidate), 256);
    const int64_t chunk_bytes = round_up(b->chunk_cap * (int64_t)sizeof(CandChunk), 256);
    const int64_t small_bytes = 256 + 256 + round_up((int64_t)b->wpad * 8, 256);
    b->arena_bytes = (size_t)(in_bytes + wave_bytes + table_bytes + cand_bytes + chunk_bytes + small_bytes);
    cudaError_t e = cudaMalloc(&b->arena, b->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("batch needs %zu device bytes: %s", b->arena_bytes, cudaGetErrorString(e));
        free_batch(b);
        return AA_ERR_NOMEM;
    }
    char* p = b->arena;
    p += in_bytes;  // beam inputs first (aa_batch_input)
    char* wave_area = p;
    p += wave_bytes;
    b->d_cands = reinterpret_cast<aa_candidate*>(p);
    p += cand_bytes;
    b->d_chunks = reinterpret_cast<CandChunk*>(p);
    p += chunk_bytes;
    b->d_counts = reinterpret_cast<unsigned long long*>(p);
    p += 256;
    b->d_err = reinterpret_cast<unsigned*>(p);
    p += 256;
    b->d_rsw = reinterpret_cast<double*>(p);
    p += round_up((int64_t)b->wpad * 8, 256);
    char* tables = p;

    // per-wave descriptors
    b->tables.resize(b->waves.size());
    b->dd_of.assign(nbeams, nullptr);
    b->wave_of.assign(nbeams, -1);
    b->beam_dd.assign(nbeams, {});
    b->beam_sps.assign(nbeams, {});
    b->beam_dec_ws.assign(nbeams, nullptr);
    b->beam_work.assign(nbeams, 0.0);
    for (size_t wi = 0; wi < b->waves.size(); ++wi) {
        WaveTables& T = b->tables[wi];
        char* q = wave_area;
        for (int v = 0; v < 4; ++v) T.dd_first[v].push_back(0);
        T.st_first.push_back(0);
        T.bx_first.push_back(0);
        for (int lv = 0; lv < 4; ++lv) T.dec_first[lv].push_back(0);
        for (int bi : b->waves[wi]) {
            const aa_plan& pl = *plans[bi];
            const int64_t n = nsamps[bi];
            const Layout L = make_layout(pl, n, max_width);
            const uint8_t* d_in = reinterpret_cast<const uint8_t*>(b->arena + b->in_offset[bi]);
            char* dec_ws = q;
            b->beam_dec_ws[bi] = dec_ws;
            q += needs[bi].dec_bytes;
            float* dd = reinterpret_cast<float*>(q);
            q += needs[bi].dd_bytes;
            b->dd_of[bi] = dd;
            b->wave_of[bi] = (int)wi;
            RowStats* stats = reinterpret_cast<RowStats*>(q);
            q += round_up((int64_t)pl.ndm_total * (int64_t)sizeof(RowStats), 256);
            float2* tab = reinterpret_cast<float2*>(q);
            q += round_up((int64_t)pl.ndm_total * L.wpad * 8, 256);
            // decimation cascade (level = position of the source in the chain)
            std::vector<int> level(pl.decs.size(), 0);
            for (size_t k = 0; k < pl.decs.size(); ++k) {
                const int dec = pl.decs[k];
                const void* src = d_in;
                int src_elem = 1, src_dec = 1;
                int64_t src_pitch = b->in_pitch[bi];
                for (size_t j = 0; j < k; ++j)
                    if (dec % pl.decs[j] == 0) {
                        src = dec_ws + L.dec_offset[j];
                        src_elem = 2;
                        src_dec = pl.decs[j];
                        src_pitch = L.dec_pitch[j];
                        level[k] = level[j] + 1;
                    }
                if (level[k] > 3) {
                    set_error("decimation cascade deeper than 4 levels");
                    free_batch(b);
                    return AA_ERR_CONFIG;
                }
                DecimateJob job{src, src_elem, dec / src_dec, src_pitch, n / dec,
                                reinterpret_cast<uint16_t*>(dec_ws + L.dec_offset[k]), L.dec_pitch[k]};
                if (job.nout > 0) {
                    T.dec_jobs[level[k]].push_back(job);
                    T.dec_first[level[k]].push_back(T.dec_first[level[k]].back() +
                                                    (job.nout + 3) / 4 * pl.nchans);
                }
            }
            for (size_t r = 0; r < pl.ranges.size(); ++r) {
                const RangePlan& g = pl.ranges[r];
                if (L.length[r] <= 0) continue;
                DedispArgs a{};
                if (g.desc.dec == 1) {
                    a.in = d_in;
                    a.in_pitch = b->in_pitch[bi];
                } else {
                    const size_t k = std::find(pl.decs.begin(), pl.decs.end(), g.desc.dec) - pl.decs.begin();
                    a.in = dec_ws + L.dec_offset[k];
                    a.in_pitch = L.dec_pitch[k];
                }
                a.nchans = pl.nchans;
                a.nsamp = L.nsamp_dec[r];
                a.length = L.length[r];
                a.ndm = g.desc.ndm;
                a.shifts = g.d_shifts;
                a.out = dd + L.row_offset[r];
                a.out_pitch = L.pitch[r];
                fill_strategy(a, g);
                a.err = b->d_err;
                const int sg = (a.grouped ? 2 : 0) + (a.elem == 2 ? 1 : 0);
                T.dd_smem[sg] = std::max(T.dd_smem[sg], a.smem);
                const int ndmb = (a.ndm + kDmPerBlock - 1) / kDmPerBlock;
                const int64_t ntiles = (a.length + kTau - 1) / kTau;
                T.dd[sg].push_back(a);
                b->beam_dd[bi].push_back(a);
                b->beam_work[bi] += (double)a.ndm * (double)a.length * (double)a.nchans;
                T.dd_ndmb[sg].push_back(ndmb);
                T.dd_first[sg].push_back(T.dd_first[sg].back() + (int64_t)ndmb * ntiles);
                SpsArgs s{};
                s.dd = dd + L.row_offset[r];
                s.pitch = L.pitch[r];
                s.length = L.length[r];
                s.nrows = g.desc.ndm;
                s.dm_offset = g.dm_offset;
                s.range = (int32_t)r;
                s.max_width = max_width;
                s.wpad = L.wpad;
                s.threshold = threshold;
                s.rsqrt_w = b->d_rsw;
                s.stats = stats + g.dm_offset;
                s.table = tab + (int64_t)g.dm_offset * L.wpad;
                s.cands = b->d_cands;
                s.capacity = cand_capacity;
                s.count = &b->d_counts[0];
                s.snr_out = nullptr;
                s.err = b->d_err;
                s.prune = 1;
                s.clip_c16 = pl.clip_c16;
                s.clip_iters = pl.clip_iters;
                s.ladder_g16 = pl.ladder_g16;
                s.dec_w0 = pl.dec_w0;
                T.bx_smem = std::max(T.bx_smem, sps_boxcar_smem_for(s.max_width, s.wpad, s.dec_w0));
                s.beam = bi;
                s.chunks = b->d_chunks;
                s.nchunks = &b->d_counts[1];
                s.chunk_cap = b->chunk_cap;
                s.evaluated = nullptr;
                T.sps.push_back(s);
                b->beam_sps[bi].push_back(s);
                T.st_first.push_back(T.st_first.back() + s.nrows);
                const int nt = sps_boxcar_tiles(s.length);
                T.bx_ntiles.push_back(nt);
                T.bx_first.push_back(T.bx_first.back() + (int64_t)nt * s.nrows);
            }
        }
        // upload tables
        bool overflow = false;
        auto put = [&](const void* src, size_t bytes) {
            char* dst = tables;
            tables += round_up((int64_t)std::max<size_t>(bytes, 8), 256);
            if (tables > b->arena + b->arena_bytes) {
                overflow = true;  // never copy outside the arena
                return b->arena;
            }
            if (bytes) cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
            return dst;
        };
        for (int lv = 0; lv < 4; ++lv) {
            T.d_dec_jobs[lv] = reinterpret_cast<DecimateJob*>(put(T.dec_jobs[lv].data(), T.dec_jobs[lv].size() * sizeof(DecimateJob)));
            T.d_dec_first[lv] = reinterpret_cast<int64_t*>(put(T.dec_first[lv].data(), T.dec_first[lv].size() * 8));
        }
        for (int sg = 0; sg < 4; ++sg) {
            T.d_dd[sg] = reinterpret_cast<DedispArgs*>(put(T.dd[sg].data(), T.dd[sg].size() * sizeof(DedispArgs)));
            T.d_dd_first[sg] = reinterpret_cast<int64_t*>(put(T.dd_first[sg].data(), T.dd_first[sg].size() * 8));
            T.d_dd_ndmb[sg] = reinterpret_cast<int*>(put(T.dd_ndmb[sg].data(), T.dd_ndmb[sg].size() * 4));
        }
        T.d_sps = reinterpret_cast<SpsArgs*>(put(T.sps.data(), T.sps.size() * sizeof(SpsArgs)));
        T.d_st_first = reinterpret_cast<int64_t*>(put(T.st_first.data(), T.st_first.size() * 8));
        T.d_bx_first = reinterpret_cast<int64_t*>(put(T.bx_first.data(), T.bx_first.size() * 8));
        T.d_bx_ntiles = reinterpret_cast<int*>(put(T.bx_ntiles.data(), T.bx_ntiles.size() * 4));
        T.d_queues = reinterpret_cast<unsigned long long*>(put(nullptr, 0));
        if (overflow) {
            set_error("internal: descriptor tables overflow the arena");
            free_batch(b);
            return AA_ERR_STATE;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { free_batch(b); return fail(e, "upload batch tables"); }
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    const int sms = prop.multiProcessorCount;
    b->grid_dd = sms * 2;  // two 512-thread CTAs per SM (each staging ring <= 113 KB)
    b->grid_st = sms * 4;
    b->grid_bx = sms * 2;
    b->grid_dec = sms * 16;

    // capture the whole batch into one graph (each beam's own kernels on
    // kDefaultBranches concurrent branches; aa_batch_set_branches switches)
    b->branches = kDefaultBranches;
    e = capture_graph(b);
    if (e != cudaSuccess) { free_batch(b); return fail(e, "capture batch graph"); }
    *out = b;
    return AA_OK;
}

void aa_batch_destroy(aa_batch* b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    free_batch(b);
    if (prev >= 0) cudaSetDevice(prev);
}

aa_status aa_batch_set_branches(aa_batch* b, int32_t branches) {
    clear_error();
    if (!b) { set_error("batch is NULL"); return AA_ERR_ARG; }
    if (branches < 0 || branches > 64) { set_error("branches must be in [0, 64]"); return AA_ERR_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    AA_CUDA(cudaSetDevice(b->device), "cudaSetDevice");
    b->branches = branches;
    const cudaError_t e = capture_graph(b);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(e, "capture batch graph");
    return AA_OK;
}

aa_status aa_batch_input(aa_batch* b, int32_t beam, uint8_t** d_in, int64_t* pitch) {
    clear_error();
    if (!b || beam < 0 || beam >= b->nbeams) { set_error("bad batch/beam"); return AA_ERR_ARG; }
    if (d_in) *d_in = reinterpret_cast<uint8_t*>(b->arena + b->in_offset[beam]);
    if (pitch) *pitch = b->in_pitch[beam];
    return AA_OK;
}

aa_status aa_batch_dd_view(const aa_batch* b, int32_t beam, const float** d_dd) {
    clear_error();
    if (!b || !d_dd || beam < 0 || beam >= b->nbeams) { set_error("bad batch/beam/d_dd"); return AA_ERR_ARG; }
    *d_dd = nullptr;
    if (b->wave_of[beam] != (int)b->waves.size() - 1) {
        set_error("beam %d ran in wave %d of %zu: its series were overwritten by later waves", beam,
                  b->wave_of[beam], b->waves.size());
        return AA_ERR_STATE;
    }
    *d_dd = b->dd_of[beam];
    return AA_OK;
}

aa_status aa_batch_info(const aa_batch* b, int32_t* nwaves, int64_t* device_bytes) {
    clear_error();
    if (!b) { set_error("batch is NULL"); return AA_ERR_ARG; }
    if (nwaves) *nwaves = (int32_t)b->waves.size();
    if (device_bytes) *device_bytes = (int64_t)b->arena_bytes;
    return AA_OK;
}

aa_status aa_batch_run(aa_batch* b, aa_stream_t stream) {
    clear_error();
    if (!b) { set_error("batch is NULL"); return AA_ERR_ARG; }
    if (!b->exec) { set_error("the batch has no recorded graph (a failed aa_batch_set_branches)"); return AA_ERR_STATE; }
    AA_CUDA(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)), "batch graph launch");
    return AA_OK;
}

aa_status aa_batch_candidates(aa_batch* b, aa_stream_t stream, aa_candidates** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!b) { set_error("batch is NULL"); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long counts[2] = {0, 0};
    unsigned err = 0;
    AA_CUDA(cudaMemcpyAsync(counts, b->d_counts, 16, cudaMemcpyDeviceToHost, s), "read counts");
    AA_CUDA(cudaMemcpyAsync(&err, b->d_err, 4, cudaMemcpyDeviceToHost, s), "read error word");
    AA_CUDA(cudaStreamSynchronize(s), "synchronize");
    if (err) { set_error("a bounded device-side wait gave up"); return AA_ERR_TIMEOUT; }
    const int64_t stored = std::min<int64_t>((int64_t)counts[0], b->capacity);
    const int64_t nh = std::min<int64_t>((int64_t)counts[1], b->chunk_cap);
    std::vector<CandChunk> heads((size_t)nh);
    if (nh) AA_CUDA(cudaMemcpyAsync(heads.data(), b->d_chunks, nh * sizeof(CandChunk), cudaMemcpyDeviceToHost, s), "read chunks");
    AA_CUDA(cudaStreamSynchronize(s), "synchronize");
    aa_candidates* res = candidates_new();
    if (!res) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
    // runs ordered by (beam, dm_index, t0), gathered on the device, copied once
    const aa_status ost = order_candidates(b->d_cands, stored, heads, true, s, res);
    if (ost != AA_OK) {
        aa_candidates_destroy(res);
        return ost;
    }
    candidates_set_total(res, (int64_t)counts[0]);
    *out = res;
    return (int64_t)counts[0] > b->capacity ? AA_WARN_CAND_OVERFLOW : AA_OK;
}

}  // extern "C"

// Streaming search server with continuous batching (arXiv:1912.07704
// Sec. 3.3: the pipeline iterates over the input in chunks and reports a
// status code per iteration).
//
// Chunk k of a beam (N new samples) is searched as the block of full-rate
// samples [max(0, kN - H), (k+1)N): the resident history of the beam followed
// by the new samples, with H = max_r dec_r (maxshift_r + W + 2) rounded up to a
// multiple of 16 (so decimation bins stay aligned with the whole series).  The
// block runs through the full pipeline (decimation, dedispersion, per-block
// statistics, boxcar search, peaks); the chunk reports the candidates of range
// r whose global start index j (decimated samples) lies in
//   [kN/dec_r - maxshift_r - W - 1, (k+1)N/dec_r - maxshift_r - W - 1),
// regions that tile the series chunk after chunk and where the full W windows
// and both neighbours of every start are inside the block.
//
// Requests queue on the host; the loop admits a queued chunk into a free
// slot (own stream and device workspace; the number of slots is fixed by the
// memory budget) as soon as the chunk's beam has no chunk in flight, so that
// chunks of different beams overlap on the device.  A slot runs the fused
// dedispersion -> search (stripes of trials, statistics from the
// dedispersion kernels) when the plan allows it, so it holds one stripe of
// series instead of every row.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
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

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket;
    int32_t beam;
    int64_t chunk;
    const uint8_t* host;
    int64_t host_pitch;
    double arrival;  // caller's clock (seconds); latency = completion - arrival
    double admitted = 0, done = 0;
    aa_status status = AA_PENDING;
    std::vector<aa_candidate> cands;
    int64_t total = 0;
    int slot = -1;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* dd_ws = nullptr;
    float* dd = nullptr;
    void* sps_ws = nullptr;
    aa_candidate* cands = nullptr;
    unsigned long long* count = nullptr;  // device
    unsigned long long* h_count = nullptr;  // pinned host
    int64_t req = -1;  // index into requests
};

struct Beam {
    uint8_t* buf[2] = {nullptr, nullptr};  // ping-pong blocks [nchans][pitch]
    int64_t next_chunk = 0;                // chunk expected next
    bool in_flight = false;
    cudaEvent_t last = nullptr;            // completion of the previous chunk
    bool has_last = false;
};

}  // namespace

struct aa_server {
    aa_plan* plan = nullptr;
    int32_t nbeams = 0;
    int64_t N = 0, H = 0, pitch = 0;
    int32_t W = 0;
    float thr = 0;
    int64_t cap = 0;
    int device = -1;
    std::vector<Beam> beams;
    std::vector<Slot> slots;
    std::vector<Request> reqs;  // by ticket
    std::deque<int64_t> queue;  // queued tickets (arrival order)
    int64_t completed = 0;
    int32_t max_in_flight = 0;
    double first_arrival = -1, last_done = 0;
    // fused dedispersion -> search (aa_search_fused_device) when the plan
    // allows it: a slot then holds one stripe of series, not every row
    bool fused = false;
    size_t fused_ws = 0;
};

namespace {

int64_t block_start(const aa_server& s, int64_t k) { return std::max<int64_t>(0, k * s.N - s.H); }

aa_status launch_chunk(aa_server& s, Slot& sl, Request& r) {
    Beam& b = s.beams[r.beam];
    const int64_t k = r.chunk;
    const int64_t b0 = block_start(s, k);
    const int64_t len = (k + 1) * s.N - b0;
    const int64_t hist = k * s.N - b0;  // samples carried over
    uint8_t* dst = b.buf[k & 1];
    const int C = s.plan->nchans;
    cudaStream_t st = sl.stream;
    if (hist > 0) {
        const uint8_t* src = b.buf[(k - 1) & 1];
        const int64_t prev_b0 = block_start(s, k - 1);
        const int64_t off = b0 - prev_b0;  // tail of the previous block
        if (b.has_last) AA_CUDA(cudaStreamWaitEvent(st, b.last, 0), "wait previous chunk");
        AA_CUDA(cudaMemcpy2DAsync(dst, s.pitch, src + off, s.pitch, hist, C, cudaMemcpyDeviceToDevice, st),
                "history copy");
    }
    AA_CUDA(cudaMemcpy2DAsync(dst + hist, s.pitch, r.host, r.host_pitch, s.N, C, cudaMemcpyHostToDevice, st),
            "chunk upload");
    if (s.fused) {
        const aa_status e = aa_search_fused_device(s.plan, dst, len, s.pitch, s.W, s.thr, 0, sl.cands, s.cap,
                                                   sl.count, nullptr, sl.dd_ws, s.fused_ws,
                                                   reinterpret_cast<aa_stream_t>(st));
        if (e != AA_OK) return e;
    } else {
        const Layout L = make_layout(*s.plan, len, s.W);
        aa_status e = aa_dedisperse_device(s.plan, dst, len, s.pitch, sl.dd, sl.dd_ws, (size_t)L.dedisp_ws,
                                           reinterpret_cast<aa_stream_t>(st));
        if (e != AA_OK) return e;
        e = aa_sps_search_device(s.plan, len, sl.dd, s.W, s.thr, sl.cands, s.cap, sl.count, nullptr,
                                 sl.sps_ws, (size_t)L.sps_ws, reinterpret_cast<aa_stream_t>(st));
        if (e != AA_OK) return e;
    }
    AA_CUDA(cudaMemcpyAsync(sl.h_count, sl.count, 8, cudaMemcpyDeviceToHost, st), "count readback");
    AA_CUDA(cudaEventRecord(sl.done, st), "record completion");
    AA_CUDA(cudaEventRecord(b.last, st), "record beam progress");
    b.has_last = true;
    return AA_OK;
}

// Completed slot: fetch the stored records, keep the chunk's emitted region.
aa_status harvest(aa_server& s, Slot& sl) {
    Request& r = s.reqs[(size_t)sl.req];
    const int64_t total = (int64_t)*sl.h_count;
    const int64_t stored = std::min(total, s.cap);
    std::vector<aa_candidate> raw((size_t)stored);
    if (stored)
        AA_CUDA(cudaMemcpy(raw.data(), sl.cands, stored * sizeof(aa_candidate), cudaMemcpyDeviceToHost),
                "candidate readback");
    const int64_t k = r.chunk;
    const int64_t b0 = block_start(s, k);
    for (const aa_candidate& c : raw) {
        const RangePlan& g = s.plan->ranges[c.range];
        const int64_t dec = g.desc.dec;
        const int64_t lag = g.maxshift + s.W + 1;
        const int64_t lo = k * s.N / dec - lag, hi = (k + 1) * s.N / dec - lag;
        const int64_t j = b0 / dec + c.t;  // global start index
        if (j >= std::max<int64_t>(lo, 0) && j < hi) {
            aa_candidate o = c;
            o.t = (uint32_t)j;
            o.reserved = (uint8_t)r.beam;
            r.cands.push_back(o);
        }
    }
    std::sort(r.cands.begin(), r.cands.end(), [](const aa_candidate& a, const aa_candidate& b) {
        return a.dm_index != b.dm_index ? a.dm_index < b.dm_index : a.t < b.t;
    });
    r.total = total;
    r.status = total > s.cap ? AA_WARN_CAND_OVERFLOW : AA_OK;
    r.done = now_s();
    s.last_done = std::max(s.last_done, r.done);
    s.beams[r.beam].in_flight = false;
    s.completed++;
    sl.req = -1;
    return AA_OK;
}

void free_server(aa_server* s) {
    if (!s) return;
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFree(sl.dd_ws);
        cudaFree(sl.dd);
        cudaFree(sl.sps_ws);
        cudaFree(sl.cands);
        cudaFree(sl.count);
        if (sl.h_count) cudaFreeHost(sl.h_count);
    }
    for (auto& b : s->beams) {
        cudaFree(b.buf[0]);
        cudaFree(b.buf[1]);
        if (b.last) cudaEventDestroy(b.last);
    }
    delete s;
}

}  // namespace

extern "C" {

aa_status aa_server_create(aa_plan* plan, int32_t nbeams, int64_t chunk_nsamp, int32_t max_width,
                           float threshold, int64_t cand_capacity, int64_t memory_budget,
                           int32_t max_slots, aa_server** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!plan || nbeams < 1 || nbeams > 256 || chunk_nsamp < 16 || chunk_nsamp % 16 != 0) {
        set_error("need a plan, 1..256 beams and chunk_nsamp a positive multiple of 16");
        return AA_ERR_ARG;
    }
    if (max_width < 1 || max_width > 65535 || cand_capacity < 1 || max_slots < 1) {
        set_error("bad max_width / cand_capacity / max_slots");
        return AA_ERR_ARG;
    }
    int dev = 0;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (!plan->ready) {
        aa_status st = aa_plan_bind(plan, dev);
        if (st != AA_OK) return st;
    }
    aa_server* s = new (std::nothrow) aa_server();
    if (!s) return AA_ERR_NOMEM;
    s->plan = plan;
    s->nbeams = nbeams;
    s->N = chunk_nsamp;
    s->W = max_width;
    s->thr = threshold;
    s->cap = cand_capacity;
    s->device = dev;
    int64_t H = 0;
    for (const auto& g : plan->ranges)
        H = std::max<int64_t>(H, (int64_t)g.desc.dec * (g.maxshift + max_width + 2));
    s->H = round_up(H, 16);
    const int64_t block = s->H + s->N;
    const Layout L = make_layout(*plan, block, max_width);
    s->pitch = L.in_pitch_min;
    // resident state: two block buffers per beam
    const int64_t beam_bytes = 2 * (int64_t)plan->nchans * s->pitch;
    s->fused = aa_search_fused_ws_bytes(plan, block, max_width, 0, &s->fused_ws, nullptr) == AA_OK;
    clear_error();  // plans with sub-band or FDMT ranges keep the unfused path
    const int64_t work_bytes = s->fused ? (int64_t)s->fused_ws : L.dedisp_ws + L.dd_elems * 4 + L.sps_ws;
    const int64_t slot_bytes = work_bytes + cand_capacity * (int64_t)sizeof(aa_candidate) + 4096;
    if (memory_budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        memory_budget = (int64_t)(fr / 2);
    }
    const int64_t avail = memory_budget - beam_bytes * nbeams;
    const int64_t nslots = std::min<int64_t>(max_slots, avail / slot_bytes);
    if (nslots < 1) {
        set_error("memory budget %lld too small: %lld resident + %lld per slot",
                  (long long)memory_budget, (long long)(beam_bytes * nbeams), (long long)slot_bytes);
        delete s;
        return AA_ERR_NOMEM;
    }
    s->beams.resize(nbeams);
    for (auto& b : s->beams) {
        cudaError_t e = cudaMalloc(&b.buf[0], (size_t)plan->nchans * s->pitch);
        if (e == cudaSuccess) e = cudaMalloc(&b.buf[1], (size_t)plan->nchans * s->pitch);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.last, cudaEventDisableTiming);
        if (e != cudaSuccess) { free_server(s); return fail(e, "beam state allocation"); }
    }
    s->slots.resize((size_t)nslots);
    for (auto& sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (s->fused) {  // one fused workspace per slot
            if (e == cudaSuccess) e = cudaMalloc(&sl.dd_ws, std::max<size_t>(s->fused_ws, 256));
        } else {
            if (e == cudaSuccess) e = cudaMalloc(&sl.dd_ws, (size_t)L.dedisp_ws);
            if (e == cudaSuccess) e = cudaMalloc(&sl.dd, (size_t)std::max<int64_t>(L.dd_elems * 4, 256));
            if (e == cudaSuccess) e = cudaMalloc(&sl.sps_ws, (size_t)L.sps_ws);
        }
        if (e == cudaSuccess) e = cudaMalloc(&sl.cands, (size_t)cand_capacity * sizeof(aa_candidate));
        if (e == cudaSuccess) e = cudaMalloc(&sl.count, 256);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_count, 64);
        if (e != cudaSuccess) { free_server(s); return fail(e, "slot allocation"); }
    }
    *out = s;
    return AA_OK;
}

void aa_server_destroy(aa_server* s) { free_server(s); }

aa_status aa_server_submit(aa_server* s, int32_t beam, const uint8_t* host_chunk, int64_t host_pitch,
                           double arrival_time, int64_t* ticket) {
    clear_error();
    if (!s || !host_chunk || !ticket) { set_error("server/host_chunk/ticket is NULL"); return AA_ERR_ARG; }
    if (beam < 0 || beam >= s->nbeams) { set_error("beam %d out of range", beam); return AA_ERR_ARG; }
    if (host_pitch < s->N) { set_error("host_pitch must be >= chunk_nsamp"); return AA_ERR_ARG; }
    // Reported start times are global sample indices of the beam, stored in
    // 32 bits: every index this chunk can report is below (chunk + 1) * N
    // (decimation only lowers it), so refuse chunks past 2^32 samples.
    const int64_t chunk = s->beams[beam].next_chunk;
    if ((chunk + 1) * s->N > (int64_t)UINT32_MAX) {
        set_error("beam %d chunk %lld: global sample index would pass 2^32 (start a new beam)", beam,
                  (long long)chunk);
        return AA_ERR_CONFIG;
    }
    Request r;
    r.ticket = (int64_t)s->reqs.size();
    r.beam = beam;
    r.chunk = s->beams[beam].next_chunk++;
    r.host = host_chunk;
    r.host_pitch = host_pitch;
    r.arrival = arrival_time;
    if (s->first_arrival < 0 || arrival_time < s->first_arrival) s->first_arrival = arrival_time;
    s->reqs.push_back(std::move(r));
    s->queue.push_back(s->reqs.back().ticket);
    *ticket = s->reqs.back().ticket;
    return AA_PENDING;
}

aa_status aa_server_poll(aa_server* s, int32_t* ncompleted) {
    clear_error();
    if (!s) { set_error("server is NULL"); return AA_ERR_ARG; }
    int32_t nc = 0;
    // harvest finished slots
    for (auto& sl : s->slots) {
        if (sl.req < 0) continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return fail(q, "chunk completion");
        aa_status st = harvest(*s, sl);
        if (st != AA_OK) return st;
        nc++;
    }
    // admit queued chunks (arrival order; a beam's chunks stay in order)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request& r = s->reqs[(size_t)*it];
        Beam& b = s->beams[r.beam];
        bool earlier_queued = false;
        for (auto jt = s->queue.begin(); jt != it; ++jt)
            if (s->reqs[(size_t)*jt].beam == r.beam) { earlier_queued = true; break; }
        if (b.in_flight || earlier_queued) { ++it; continue; }
        Slot* free_slot = nullptr;
        for (auto& sl : s->slots)
            if (sl.req < 0) { free_slot = &sl; break; }
        if (!free_slot) break;
        free_slot->req = r.ticket;
        r.slot = (int)(free_slot - s->slots.data());
        r.admitted = now_s();
        b.in_flight = true;
        aa_status st = launch_chunk(*s, *free_slot, r);
        if (st != AA_OK) {
            r.status = st;
            free_slot->req = -1;
            b.in_flight = false;
            return st;
        }
        it = s->queue.erase(it);
    }
    int32_t busy = 0;
    for (auto& sl : s->slots) busy += sl.req >= 0;
    s->max_in_flight = std::max(s->max_in_flight, busy);
    if (ncompleted) *ncompleted = nc;
    return (s->queue.empty() && busy == 0) ? AA_OK : AA_PENDING;
}

aa_status aa_server_drain(aa_server* s) {
    clear_error();
    if (!s) { set_error("server is NULL"); return AA_ERR_ARG; }
    for (;;) {
        aa_status st = aa_server_poll(s, nullptr);
        if (st == AA_OK) return AA_OK;
        if (st != AA_PENDING) return st;
        bool waited = false;
        for (auto& sl : s->slots)
            if (sl.req >= 0) {
                AA_CUDA(cudaEventSynchronize(sl.done), "wait chunk");
                waited = true;
                break;
            }
        if (!waited && !s->queue.empty()) {
            set_error("queued chunks cannot be admitted");
            return AA_ERR_STATE;
        }
    }
}

aa_status aa_server_result(aa_server* s, int64_t ticket, aa_chunk_info* info, aa_candidates** cands) {
    clear_error();
    if (!s || ticket < 0 || ticket >= (int64_t)s->reqs.size()) { set_error("bad server/ticket"); return AA_ERR_ARG; }
    const Request& r = s->reqs[(size_t)ticket];
    if (info) {
        info->beam = r.beam;
        info->chunk = r.chunk;
        info->status = r.status;
        info->arrival = r.arrival;
        info->admitted = r.admitted;
        info->done = r.done;
        info->total = r.total;
        info->block_start = block_start(*s, r.chunk);
    }
    if (r.status == AA_PENDING) return AA_PENDING;
    if (cands) {
        aa_candidates* c = candidates_new();
        if (!c) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
        candidates_list(c) = r.cands;
        candidates_set_total(c, (int64_t)r.cands.size());
        *cands = c;
    }
    return r.status;
}

aa_status aa_server_stats(const aa_server* s, aa_server_report* out) {
    clear_error();
    if (!s || !out) { set_error("server/out is NULL"); return AA_ERR_ARG; }
    std::vector<double> lat;
    for (const auto& r : s->reqs)
        if (r.status != AA_PENDING) lat.push_back(r.done - r.arrival);
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        const size_t i = std::min(lat.size() - 1, (size_t)std::ceil(q * lat.size()) - 1);
        return lat[i];
    };
    out->submitted = (int64_t)s->reqs.size();
    out->completed = s->completed;
    out->slots = (int32_t)s->slots.size();
    out->max_in_flight = s->max_in_flight;
    out->history_nsamp = s->H;
    out->latency_p50 = pct(0.50);
    out->latency_p99 = pct(0.99);
    out->latency_max = lat.empty() ? 0.0 : lat.back();
    out->span = (s->first_arrival >= 0 && s->completed) ? s->last_done - s->first_arrival : 0.0;
    return AA_OK;
}

double aa_server_clock(void) { return now_s(); }

}  // extern "C"

// Host-buffer pipeline: the whole search (decimation, dedispersion, single-
// pulse search, candidate ordering) of a sequence of same-sized blocks of
// caller-owned host data, with the copies overlapped with the compute
// (arXiv:1912.07704 Sec. 2.3: device memory requested once, up front;
// Sec. 2.4: host input owned by the caller and never written; Sec. 3.3: the
// pipeline iterates over its input and reports a status per iteration).
//
// Three streams: h2d (block uploads into one of `depth` input slots),
// compute (dedispersion + search + ordering, one block after another, into
// one set of working buffers) and d2h (ordered candidates into page-locked
// host blocks).  Block k+1's upload runs while block k is searched; block k's
// candidates are read while block k+1 is searched.  Every device buffer is
// allocated at creation: a step allocates nothing on the device.
#include <algorithm>
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

// Per-block status words copied back with the block's candidate count.
struct HostInfo {
    unsigned long long count;  // candidates found
    unsigned dd_err;           // dedispersion workspace error word
    unsigned sps_err;          // search workspace error word
};

struct Slot {
    uint8_t* d_in = nullptr;          // [nchans][in_pitch] uploaded block
    aa_candidate* d_sorted = nullptr; // ordered candidates of the block searched from this slot
    HostInfo* h_info = nullptr;       // page-locked
    cudaEvent_t uploaded = nullptr, searched = nullptr;
    int64_t ticket = -1;              // block occupying the slot (-1: free)
};

}  // namespace

struct aa_pipeline {
    aa_plan* plan = nullptr;
    int device = -1;
    int64_t nsamp = 0;
    int32_t max_width = 0;
    float threshold = 0;
    int64_t cap = 0;
    Layout L;
    cudaStream_t h2d = nullptr, compute = nullptr, d2h = nullptr;
    std::vector<Slot> slots;
    float* d_dd = nullptr;
    void* d_ws_dd = nullptr;
    void* d_ws_sps = nullptr;
    aa_candidate* d_cands = nullptr;
    unsigned long long* d_count = nullptr;
    void* d_tmp = nullptr;
    size_t tmp_bytes = 0;
    int64_t next_ticket = 0;
};

namespace {

void free_pipeline(aa_pipeline* pl) {
    if (!pl) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (pl->device >= 0) cudaSetDevice(pl->device);
    for (cudaStream_t s : {pl->h2d, pl->compute, pl->d2h})
        if (s) cudaStreamSynchronize(s);
    for (Slot& sl : pl->slots) {
        cudaFree(sl.d_in);
        cudaFree(sl.d_sorted);
        if (sl.h_info) cudaFreeHost(sl.h_info);
        if (sl.uploaded) cudaEventDestroy(sl.uploaded);
        if (sl.searched) cudaEventDestroy(sl.searched);
    }
    cudaFree(pl->d_dd);
    cudaFree(pl->d_ws_dd);
    cudaFree(pl->d_ws_sps);
    cudaFree(pl->d_cands);
    cudaFree(pl->d_count);
    cudaFree(pl->d_tmp);
    for (cudaStream_t s : {pl->h2d, pl->compute, pl->d2h})
        if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete pl;
}

}  // namespace

extern "C" {

aa_status aa_pipeline_create(aa_plan* p, int64_t nsamp, int32_t max_width, float threshold,
                             int64_t cand_capacity, int32_t depth, aa_pipeline** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (nsamp < 1) { set_error("nsamp must be >= 1"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    if (cand_capacity < 1) { set_error("cand_capacity must be >= 1"); return AA_ERR_ARG; }
    if (depth < 1 || depth > 8) { set_error("depth must be in [1, 8]"); return AA_ERR_ARG; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (!p->ready) {
        const aa_status b = aa_plan_bind(p, dev);
        if (b != AA_OK) return b;
    }
    if (p->device != dev) { set_error("the plan is bound to device %d, current is %d", p->device, dev); return AA_ERR_STATE; }
    aa_pipeline* pl = new (std::nothrow) aa_pipeline();
    if (!pl) { set_error("host allocation failed"); return AA_ERR_NOMEM; }
    pl->plan = p;
    pl->device = dev;
    pl->nsamp = nsamp;
    pl->max_width = max_width;
    pl->threshold = threshold;
    pl->cap = cand_capacity;
    pl->L = make_layout(*p, nsamp, max_width);
    size_t tmp = 0;
    aa_status st = aa_postprocess_ws_bytes(p, nsamp, max_width, cand_capacity, &tmp);
    if (st != AA_OK) { delete pl; return st; }
    pl->tmp_bytes = tmp;
    auto bail = [&](cudaError_t e, const char* what) {
        const aa_status r = fail(e, what);
        free_pipeline(pl);
        return r;
    };
    cudaError_t e;
    for (cudaStream_t* s : {&pl->h2d, &pl->compute, &pl->d2h})
        if ((e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
    const Layout& L = pl->L;
    const size_t in_bytes = (size_t)p->nchans * (size_t)L.in_pitch_min;
    const size_t rec = sizeof(aa_candidate);
    pl->slots.resize((size_t)depth);
    for (Slot& sl : pl->slots) {
        if ((e = cudaMalloc(&sl.d_in, in_bytes)) != cudaSuccess) return bail(e, "input slot");
        if ((e = cudaMalloc(&sl.d_sorted, (size_t)cand_capacity * rec)) != cudaSuccess) return bail(e, "ordered candidates");
        if ((e = cudaHostAlloc(&sl.h_info, sizeof(HostInfo), cudaHostAllocDefault)) != cudaSuccess) return bail(e, "status words");
        if ((e = cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
        if ((e = cudaEventCreateWithFlags(&sl.searched, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    }
    if ((e = cudaMalloc(&pl->d_dd, (size_t)std::max<int64_t>(L.dd_elems, 1) * 4)) != cudaSuccess) return bail(e, "dedispersed series");
    if ((e = cudaMalloc(&pl->d_ws_dd, (size_t)L.dedisp_ws)) != cudaSuccess) return bail(e, "dedispersion workspace");
    if ((e = cudaMalloc(&pl->d_ws_sps, (size_t)L.sps_ws)) != cudaSuccess) return bail(e, "search workspace");
    if ((e = cudaMalloc(&pl->d_cands, (size_t)cand_capacity * rec)) != cudaSuccess) return bail(e, "candidates");
    if ((e = cudaMalloc(&pl->d_count, 256)) != cudaSuccess) return bail(e, "count");
    if ((e = cudaMalloc(&pl->d_tmp, tmp)) != cudaSuccess) return bail(e, "ordering scratch");
    *out = pl;
    return AA_OK;
}

void aa_pipeline_destroy(aa_pipeline* pl) { free_pipeline(pl); }

aa_status aa_pipeline_submit(aa_pipeline* pl, const uint8_t* host_in, int64_t host_pitch, int64_t* ticket) {
    clear_error();
    if (!pl || !host_in || !ticket) { set_error("pipeline/host_in/ticket is NULL"); return AA_ERR_ARG; }
    if (host_pitch < pl->nsamp) { set_error("host_pitch %lld < nsamp %lld", (long long)host_pitch, (long long)pl->nsamp); return AA_ERR_ARG; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != pl->device) { set_error("current device %d differs from the pipeline's %d", dev, pl->device); return AA_ERR_STATE; }
    const int64_t t = pl->next_ticket;
    Slot& sl = pl->slots[(size_t)(t % (int64_t)pl->slots.size())];
    if (sl.ticket >= 0) {
        set_error("block %lld still occupies the slot: aa_pipeline_wait for it first (at most %zu blocks in flight)",
                  (long long)sl.ticket, pl->slots.size());
        return AA_ERR_STATE;
    }
    const aa_plan* p = pl->plan;
    const Layout& L = pl->L;
    // upload (the slot's previous search has finished reading it: it was waited for)
    cudaError_t e = host_pitch == L.in_pitch_min
                        ? cudaMemcpyAsync(sl.d_in, host_in, (size_t)p->nchans * (size_t)host_pitch,
                                          cudaMemcpyHostToDevice, pl->h2d)
                        : cudaMemcpy2DAsync(sl.d_in, (size_t)L.in_pitch_min, host_in, (size_t)host_pitch,
                                            (size_t)pl->nsamp, (size_t)p->nchans, cudaMemcpyHostToDevice, pl->h2d);
    if (e != cudaSuccess) return fail(e, "host-to-device copy");
    AA_CUDA(cudaEventRecord(sl.uploaded, pl->h2d), "record upload");
    // search, in block order on the compute stream
    AA_CUDA(cudaStreamWaitEvent(pl->compute, sl.uploaded, 0), "wait upload");
    const aa_stream_t cs = reinterpret_cast<aa_stream_t>(pl->compute);
    aa_status st = aa_dedisperse_device(p, sl.d_in, pl->nsamp, L.in_pitch_min, pl->d_dd, pl->d_ws_dd,
                                        (size_t)L.dedisp_ws, cs);
    if (st != AA_OK) return st;
    st = aa_sps_search_device(p, pl->nsamp, pl->d_dd, pl->max_width, pl->threshold, pl->d_cands, pl->cap,
                              pl->d_count, nullptr, pl->d_ws_sps, (size_t)L.sps_ws, cs);
    if (st != AA_OK) return st;
    st = aa_sps_order_device(p, pl->nsamp, pl->max_width, pl->d_ws_sps, pl->d_cands, pl->d_count, pl->cap,
                             sl.d_sorted, pl->d_tmp, pl->tmp_bytes, cs);
    if (st != AA_OK) return st;
    AA_CUDA(cudaMemcpyAsync(&sl.h_info->count, pl->d_count, 8, cudaMemcpyDeviceToHost, pl->compute), "read count");
    AA_CUDA(cudaMemcpyAsync(&sl.h_info->dd_err, pl->d_ws_dd, 4, cudaMemcpyDeviceToHost, pl->compute), "read error word");
    AA_CUDA(cudaMemcpyAsync(&sl.h_info->sps_err, pl->d_ws_sps, 4, cudaMemcpyDeviceToHost, pl->compute), "read error word");
    AA_CUDA(cudaEventRecord(sl.searched, pl->compute), "record search");
    sl.ticket = t;
    pl->next_ticket = t + 1;
    *ticket = t;
    return AA_PENDING;
}

aa_status aa_pipeline_wait(aa_pipeline* pl, int64_t ticket, aa_candidates** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!pl) { set_error("pipeline is NULL"); return AA_ERR_ARG; }
    if (ticket < 0 || ticket >= pl->next_ticket) { set_error("ticket %lld was not submitted", (long long)ticket); return AA_ERR_ARG; }
    Slot& sl = pl->slots[(size_t)(ticket % (int64_t)pl->slots.size())];
    if (sl.ticket != ticket) { set_error("ticket %lld was already collected", (long long)ticket); return AA_ERR_STATE; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != pl->device) cudaSetDevice(pl->device);
    aa_status st = AA_OK;
    cudaError_t e = cudaEventSynchronize(sl.searched);
    if (e != cudaSuccess) {
        st = fail(e, "block search");
    } else if (sl.h_info->dd_err | sl.h_info->sps_err) {
        set_error("a bounded device-side wait gave up");
        st = AA_ERR_TIMEOUT;
    } else {
        const int64_t total = (int64_t)sl.h_info->count;
        const int64_t stored = std::min(total, pl->cap);
        st = candidates_copy_ordered(sl.d_sorted, stored, total, pl->d2h, out);
        if (st == AA_OK && total > pl->cap) st = AA_WARN_CAND_OVERFLOW;
    }
    sl.ticket = -1;  // the slot is free whatever the outcome
    if (prev >= 0 && prev != pl->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"

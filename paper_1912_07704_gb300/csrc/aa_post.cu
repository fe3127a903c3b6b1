// Candidate post-processing on the device.
//
// aa_sps_order_device moves the single-pulse search's per-CTA runs into
// (dm_index, t) order without a host round trip: each boxcar CTA owns one
// slot (range, trial, tile) of a dense table, the run lengths are scanned into
// destinations and the runs gathered.
//
// aa_candidates_peaks2d_device keeps the local maxima of the DM-time plane
// among the ordered candidates.  The search of arXiv:1912.07704 Sec. 1
// (boxcar filters with peak finding) leaves one candidate per local maximum
// in time of every trial; a pulse then shows up in many neighbouring trials.
// A candidate is kept when no other candidate of the same range within
// +-dm_radius trials and +-t_radius samples has a larger SNR, equal SNRs
// going to the smaller (dm_index, t).
#include <algorithm>
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanBlock = (int64_t)kScanThreads * kScanItems;
constexpr int kMaxRanges = 64;

struct RangeTable {
    int32_t n;
    int32_t dm_offset[kMaxRanges + 1];  // first global trial of each range (+ the total)
    int32_t ntiles[kMaxRanges];         // boxcar CTAs per trial
    int64_t slot_base[kMaxRanges];      // first run slot of each range
    int32_t nbuckets[kMaxRanges];       // time buckets per trial (peak filter index)
    int64_t bucket_base[kMaxRanges];    // first bucket entry of each range
};

__device__ __forceinline__ int range_of(const RangeTable& rt, uint32_t dm) {
    int r = 0;
    while (r + 1 < rt.n && (uint32_t)rt.dm_offset[r + 1] <= dm) ++r;
    return r;
}

__device__ __forceinline__ int64_t live_count(const unsigned long long* dn, int64_t cap) {
    return dn ? min((int64_t)*dn, cap) : cap;
}

// ---------------------------------------------------------------- scan --
// Exclusive scan of v over the block; returns this thread's offset and the
// block total in `total`.
__device__ __forceinline__ int64_t block_scan(int64_t v, int64_t* sh, int64_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const int64_t before = warp ? sh[warp - 1] : 0;
    return before + x - v;
}

// In-place exclusive scan of each kScanBlock-element block of data[0, n),
// n = live_count(dn, cap); block totals to sums[blockIdx.x] (0 past n).
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(int64_t* data, const unsigned long long* dn,
                                                                   int64_t cap, int64_t* sums) {
    __shared__ int64_t sh[32];
    const int64_t n = live_count(dn, cap);
    const int64_t block0 = (int64_t)blockIdx.x * kScanBlock;
    if (block0 >= n) {
        if (threadIdx.x == 0) sums[blockIdx.x] = 0;
        return;
    }
    const int64_t base = block0 + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? data[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) add_block_offsets_kernel(int64_t* data, const unsigned long long* dn,
                                                                         int64_t cap, const int64_t* offs) {
    const int64_t n = live_count(dn, cap);
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    if (blockIdx.x == 0 || base >= n) return;
    const int64_t off = offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) data[base + k] += off;
}

int64_t scan_blocks(int64_t cap) { return (cap + kScanBlock - 1) / kScanBlock; }

// scratch elements for scanning up to cap values (every level)
int64_t scan_scratch(int64_t cap) {
    int64_t t = 0;
    while (cap > 1) {
        cap = scan_blocks(cap);
        t += cap;
    }
    return t + 1;
}

// Exclusive scan of data[0, live_count(dn, cap)) in place; scratch holds
// scan_scratch(cap) elements.
cudaError_t exclusive_scan(int64_t* data, const unsigned long long* dn, int64_t cap, int64_t* scratch,
                           cudaStream_t s) {
    if (cap <= 0) return cudaSuccess;
    const int64_t nb = scan_blocks(cap);
    scan_blocks_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, dn, cap, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nb == 1) return e;
    // every block wrote its sum (0 past n): scan all nb of them
    if ((e = exclusive_scan(scratch, nullptr, nb, scratch + nb, s)) != cudaSuccess) return e;
    add_block_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, dn, cap, scratch);
    return cudaGetLastError();
}

int grid_for(int64_t work, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
}

// ------------------------------------------------------------ ordering --
__global__ void slot_runs_kernel(const CandChunk* __restrict__ heads, const unsigned long long* __restrict__ nheads,
                                 int64_t head_cap, const unsigned long long* __restrict__ count, int64_t stored_cap,
                                 RangeTable rt, int64_t nslots, int64_t* cnt, int64_t* src) {
    const int64_t nh = live_count(nheads, head_cap);
    const int64_t stored = live_count(count, stored_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += (int64_t)gridDim.x * blockDim.x) {
        const CandChunk h = heads[i];
        const int r = range_of(rt, h.dm_index);
        const int64_t slot = rt.slot_base[r] + (int64_t)(h.dm_index - (uint32_t)rt.dm_offset[r]) * rt.ntiles[r] +
                             h.t0 / kSpsOwned;
        if (slot < 0 || slot >= nslots) continue;  // not a header of this plan's layout
        const int64_t base = (int64_t)h.base;
        // records past the capacity were never written
        cnt[slot] = min((int64_t)h.n, max((int64_t)0, stored - base));
        src[slot] = base;
    }
}

// dst[] holds a copy of cnt[] on entry and the scan of it after exclusive_scan.
// One warp per slot; 16-byte records.
__global__ void gather_slots_kernel(const uint4* __restrict__ in, uint4* __restrict__ out,
                                    const int64_t* __restrict__ cnt, const int64_t* __restrict__ src,
                                    const int64_t* __restrict__ dst, int64_t nslots) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < nslots; g += nw) {
        const int64_t c = cnt[g];
        if (c <= 0) continue;
        const int64_t s = src[g], d = dst[g];
        for (int64_t k = lane; k < c; k += 32) out[d + k] = in[s + k];
    }
}

// --------------------------------------------------------- 2-D peaks --
// row_start/row_end of each global trial in the ordered list (left 0/0 for
// trials without candidates).
__global__ void row_index_kernel(const aa_candidate* __restrict__ c, const unsigned long long* dn, int64_t cap,
                                 int32_t ndm, int64_t* row_start, int64_t* row_end) {
    const int64_t n = live_count(dn, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t d = c[i].dm_index;
        if (d >= (uint32_t)ndm) continue;
        if (i == 0 || c[i - 1].dm_index != d) row_start[d] = i;
        if (i + 1 == n || c[i + 1].dm_index != d) row_end[d] = i + 1;
    }
}

__device__ __forceinline__ bool beats(const aa_candidate& o, const aa_candidate& c) {
    if (o.snr != c.snr) return o.snr > c.snr;
    return o.dm_index != c.dm_index ? o.dm_index < c.dm_index : o.t < c.t;
}

// Time-bucket index of the ordered list: for trial d of range r and bucket b
// (kBucketShift-bit buckets of t, the last one open-ended), the offset from
// the row's first record of its first record with t >= b << kBucketShift.
// Every bucket of a non-empty row is written exactly once: a record fills the
// buckets after its predecessor's, the row's last record the rest.
constexpr int kBucketShift = 8;

__device__ __forceinline__ uint32_t bucket_of(uint32_t t, int32_t nb) {
    return min(t >> kBucketShift, (uint32_t)(nb - 1));
}

__global__ void bucket_index_kernel(const aa_candidate* __restrict__ c, const unsigned long long* dn, int64_t cap,
                                    const int64_t* __restrict__ row_start, const int64_t* __restrict__ row_end,
                                    RangeTable rt, uint32_t* __restrict__ first) {
    const int64_t n = live_count(dn, cap);
    const uint32_t ndm = (uint32_t)rt.dm_offset[rt.n];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const aa_candidate me = c[i];
        if (me.dm_index >= ndm) continue;
        const int r = range_of(rt, me.dm_index);
        const int32_t nb = rt.nbuckets[r];
        uint32_t* row = first + rt.bucket_base[r] + (int64_t)(me.dm_index - (uint32_t)rt.dm_offset[r]) * nb;
        const int64_t rs = row_start[me.dm_index];
        const uint32_t rel = (uint32_t)(i - rs);
        const int64_t b = bucket_of(me.t, nb);
        const int64_t bp = i == rs ? -1 : (int64_t)bucket_of(c[i - 1].t, nb);
        for (int64_t k = bp + 1; k <= b; ++k) row[k] = rel;
        if (i + 1 == row_end[me.dm_index]) {
            const uint32_t len = (uint32_t)(row_end[me.dm_index] - rs);
            for (int64_t k = b + 1; k < nb; ++k) row[k] = len;
        }
    }
}

// The peak test runs in two passes.  Pass 1, one thread per candidate,
// visits rows from the candidate's own trial outwards and each row from the
// candidate's time outwards, four records a side per load round, so that a
// stronger neighbour (on the rising side of a pulse it is usually a few
// samples away) ends the search early; a candidate still undecided after
// kPass1Budget records is queued.  Pass 2 gives each queued candidate a warp
// that walks every row's window 32 records at a time.  flag[i] = 1 iff
// candidate i is a peak; last = flag[n - 1].
constexpr int kPass1Budget = 24;
constexpr int kSide = 4;

struct PeakCtx {
    int64_t dlo, dhi, tlo, thi, d0;
    const uint32_t* rows;  // bucket entries of trial d at rows + d * nb
    int32_t nb;
};

__device__ __forceinline__ PeakCtx peak_ctx(const RangeTable& rt, const uint32_t* first, const aa_candidate& me,
                                            int32_t dm_radius, int32_t t_radius) {
    PeakCtx k;
    const int r = range_of(rt, me.dm_index);
    k.nb = rt.nbuckets[r];
    k.d0 = me.dm_index;
    k.dlo = max((int64_t)rt.dm_offset[r], k.d0 - dm_radius);
    k.dhi = min((int64_t)rt.dm_offset[r + 1] - 1, k.d0 + dm_radius);
    k.rows = first + rt.bucket_base[r] - (int64_t)rt.dm_offset[r] * k.nb;
    k.tlo = (int64_t)me.t - t_radius;
    k.thi = (int64_t)me.t + t_radius;
    return k;
}

// First index of row d (records [rs, end)) with t >= tt: the time index
// bounds it to one bucket, a binary search finds it there.
__device__ __forceinline__ int64_t lower_t(const aa_candidate* __restrict__ c, const PeakCtx& k, int64_t d,
                                           int64_t rs, int64_t end, int64_t tt) {
    if (tt <= 0) return rs;
    const uint32_t b = bucket_of((uint32_t)min(tt, (int64_t)UINT32_MAX), k.nb);
    const uint32_t* row = k.rows + d * k.nb;
    int64_t lo = rs + (int64_t)row[b];
    int64_t hi = b + 1 < (uint32_t)k.nb ? rs + (int64_t)row[b + 1] : end;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)c[mid].t < tt) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// trial visited k-th: d0, d0-1, d0+1, d0-2, d0+2, ...
__device__ __forceinline__ int64_t kth_row(int64_t d0, int64_t k) { return (k & 1) ? d0 - (k + 1) / 2 : d0 + k / 2; }

__global__ void __launch_bounds__(256) peak_pass1_kernel(const aa_candidate* __restrict__ c,
                                                         const unsigned long long* dn, int64_t cap,
                                                         const int64_t* __restrict__ row_start,
                                                         const int64_t* __restrict__ row_end,
                                                         const uint32_t* __restrict__ first, RangeTable rt,
                                                         int32_t dm_radius, int32_t t_radius, int64_t* flag,
                                                         int64_t* last, int64_t* queue,
                                                         unsigned long long* nqueue) {
    const int64_t n = live_count(dn, cap);
    const uint32_t ndm = (uint32_t)rt.dm_offset[rt.n];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const aa_candidate me = c[i];
        bool peak = me.dm_index < ndm;
        bool decided = true;
        if (peak) {
            const PeakCtx k = peak_ctx(rt, first, me, dm_radius, t_radius);
            int budget = kPass1Budget;
            for (int64_t kk = 0; peak && decided && kk <= 2 * (int64_t)dm_radius; ++kk) {
                const int64_t d = kth_row(k.d0, kk);
                if (d < k.dlo || d > k.dhi) continue;
                const int64_t rs = row_start[d], end = row_end[d];
                if (rs == end) continue;
                // in its own row the candidate itself is the first record with t >= its t
                int64_t right = d == k.d0 ? i : lower_t(c, k, d, rs, end, (int64_t)me.t);
                int64_t left = right - 1;
                bool go_r = right < end, go_l = left >= rs;
                while (go_r || go_l) {
                    if (budget <= 0) {
                        decided = false;
                        break;
                    }
                    aa_candidate R[kSide], L[kSide];
#pragma unroll
                    for (int j = 0; j < kSide; ++j) {
                        if (go_r && right + j < end) R[j] = c[right + j];
                        if (go_l && left - j >= rs) L[j] = c[left - j];
                    }
#pragma unroll
                    for (int j = 0; j < kSide; ++j) {
                        if (go_r) {
                            if (right + j >= end || (int64_t)R[j].t > k.thi) go_r = false;
                            else if (right + j != i && beats(R[j], me)) peak = false;
                        }
                        if (go_l) {
                            if (left - j < rs || (int64_t)L[j].t < k.tlo) go_l = false;
                            else if (left - j != i && beats(L[j], me)) peak = false;
                        }
                    }
                    if (!peak) break;
                    right += kSide;
                    left -= kSide;
                    budget -= 2 * kSide;
                }
            }
        }
        if (!decided && peak) {
            queue[atomicAdd(nqueue, 1ull)] = i;
        } else {
            flag[i] = peak ? 1 : 0;
            if (i == n - 1) *last = peak ? 1 : 0;
        }
    }
}

__global__ void __launch_bounds__(256) peak_pass2_kernel(const aa_candidate* __restrict__ c,
                                                         const unsigned long long* dn, int64_t cap,
                                                         const int64_t* __restrict__ row_start,
                                                         const int64_t* __restrict__ row_end,
                                                         const uint32_t* __restrict__ first, RangeTable rt,
                                                         int32_t dm_radius, int32_t t_radius, int64_t* flag,
                                                         int64_t* last, const int64_t* __restrict__ queue,
                                                         const unsigned long long* nqueue) {
    const int64_t n = live_count(dn, cap);
    const int64_t nq = (int64_t)*nqueue;
    const int lane = threadIdx.x & 31;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nq;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t i = queue[w];
        const aa_candidate me = c[i];
        const PeakCtx k = peak_ctx(rt, first, me, dm_radius, t_radius);
        bool peak = true;
        for (int64_t kk = 0; peak && kk <= 2 * (int64_t)dm_radius; ++kk) {
            const int64_t d = kth_row(k.d0, kk);
            if (d < k.dlo || d > k.dhi) continue;
            const int64_t rs = row_start[d], end = row_end[d];
            if (rs == end) continue;
            // the window from its first record, 32 records per step
            for (int64_t q0 = lower_t(c, k, d, rs, end, k.tlo); q0 < end; q0 += 32) {
                const int64_t q = q0 + lane;
                bool past = q >= end, beat = false;
                if (!past) {
                    const aa_candidate o = c[q];
                    past = (int64_t)o.t > k.thi;
                    beat = !past && (int64_t)o.t >= k.tlo && q != i && beats(o, me);
                }
                if (__any_sync(0xffffffffu, beat)) {
                    peak = false;
                    break;
                }
                if (__any_sync(0xffffffffu, past)) break;
            }
        }
        if (lane == 0) {
            flag[i] = peak ? 1 : 0;
            if (i == n - 1) *last = peak ? 1 : 0;
        }
    }
}

// pos = exclusive scan of the flags
__global__ void compact_kernel(const aa_candidate* __restrict__ c, const unsigned long long* dn, int64_t cap,
                               const int64_t* __restrict__ pos, const int64_t* __restrict__ last,
                               aa_candidate* __restrict__ out, unsigned long long* nout) {
    const int64_t n = live_count(dn, cap);
    if (n == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *nout = 0;
        return;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = pos[i];
        const int64_t next = i + 1 < n ? pos[i + 1] : p + *last;
        if (next != p) out[p] = c[i];
        if (i == n - 1) *nout = (unsigned long long)next;
    }
}

RangeTable range_table(const aa_plan& p, const Layout& L, int64_t& nslots, int64_t& nbucket_entries) {
    RangeTable rt{};
    rt.n = (int32_t)p.ranges.size();
    int64_t base = 0, bbase = 0;
    for (int r = 0; r < rt.n; ++r) {
        const int64_t ndm = p.ranges[r].desc.ndm;
        rt.dm_offset[r] = p.ranges[r].dm_offset;
        rt.ntiles[r] = (int32_t)((L.length[r] + kSpsOwned - 1) / kSpsOwned);
        rt.slot_base[r] = base;
        base += ndm * rt.ntiles[r];
        rt.nbuckets[r] = (int32_t)std::max<int64_t>(1, (L.length[r] + (1 << kBucketShift) - 1) >> kBucketShift);
        rt.bucket_base[r] = bbase;
        bbase += ndm * rt.nbuckets[r];
    }
    rt.dm_offset[rt.n] = p.ndm_total;
    nslots = base;
    nbucket_entries = bbase;
    return rt;
}

aa_status post_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return AA_ERR_CUDA;
}

aa_status check_post_args(const aa_plan* p, int64_t nsamp, int32_t max_width, int64_t cap) {
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0 || max_width < 1 || cap < 0) {
        set_error("bad nsamp / max_width / capacity");
        return AA_ERR_ARG;
    }
    if ((int)p->ranges.size() > kMaxRanges) {
        set_error("post-processing supports at most %d ranges", kMaxRanges);
        return AA_ERR_CONFIG;
    }
    return AA_OK;
}

int64_t post_scratch_elems(const aa_plan& p, int64_t nsamp, int32_t max_width, int64_t cap) {
    const Layout L = make_layout(p, nsamp, max_width);
    int64_t nslots = 0, nbe = 0;
    range_table(p, L, nslots, nbe);
    const int64_t ordering = 3 * nslots + scan_scratch(nslots);
    const int64_t peaks = 2 * (int64_t)p.ndm_total + 2 * cap + 2 + scan_scratch(cap) + (nbe + 1) / 2;
    return std::max(ordering, peaks);
}

}  // namespace
}  // namespace aa

using namespace aa;

extern "C" aa_status aa_postprocess_ws_bytes(const aa_plan* p, int64_t nsamp, int32_t max_width,
                                             int64_t cand_capacity, size_t* bytes) {
    clear_error();
    if (!bytes) { set_error("bytes is NULL"); return AA_ERR_ARG; }
    const aa_status st = check_post_args(p, nsamp, max_width, cand_capacity);
    if (st != AA_OK) return st;
    *bytes = (size_t)(8 * post_scratch_elems(*p, nsamp, max_width, cand_capacity) + 256);
    return AA_OK;
}

extern "C" aa_status aa_sps_order_device(const aa_plan* p, int64_t nsamp, int32_t max_width,
                                         const void* d_sps_ws, const aa_candidate* d_cands,
                                         const unsigned long long* d_count, int64_t cand_capacity,
                                         aa_candidate* d_sorted, void* d_tmp, size_t tmp_bytes,
                                         aa_stream_t stream) {
    clear_error();
    aa_status st = check_post_args(p, nsamp, max_width, cand_capacity);
    if (st != AA_OK) return st;
    if (!d_sps_ws || !d_count || !d_tmp || (cand_capacity > 0 && (!d_cands || !d_sorted))) {
        set_error("NULL device pointer");
        return AA_ERR_ARG;
    }
    const int64_t need = 8 * post_scratch_elems(*p, nsamp, max_width, cand_capacity) + 256;
    if ((int64_t)tmp_bytes < need) {
        set_error("scratch of %zu bytes < %lld required", tmp_bytes, (long long)need);
        return AA_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(d_tmp) % 16 || reinterpret_cast<uintptr_t>(d_cands) % 16 ||
        reinterpret_cast<uintptr_t>(d_sorted) % 16) {
        set_error("device buffers must be 16-byte aligned");
        return AA_ERR_ARG;
    }
    const Layout L = make_layout(*p, nsamp, max_width);
    int64_t nslots = 0, nbe = 0;
    const RangeTable rt = range_table(*p, L, nslots, nbe);
    if (cand_capacity == 0 || nslots == 0) return AA_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t* cnt = static_cast<int64_t*>(d_tmp);
    int64_t* src = cnt + nslots;
    int64_t* dst = src + nslots;
    int64_t* scratch = dst + nslots;
    const char* ws = static_cast<const char*>(d_sps_ws);
    const CandChunk* heads = reinterpret_cast<const CandChunk*>(ws + L.chunk_offset);
    const unsigned long long* nheads = reinterpret_cast<const unsigned long long*>(ws + kChunkCounterOffset);
    ProfScope prof(kKOrder, s);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nslots * 8, s);
    if (e != cudaSuccess) return post_fail(e, "clear run table");
    slot_runs_kernel<<<grid_for(L.chunk_cap, 256), 256, 0, s>>>(heads, nheads, L.chunk_cap, d_count,
                                                                cand_capacity, rt, nslots, cnt, src);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "run table");
    if ((e = cudaMemcpyAsync(dst, cnt, (size_t)nslots * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return post_fail(e, "copy run lengths");
    if ((e = exclusive_scan(dst, nullptr, nslots, scratch, s)) != cudaSuccess) return post_fail(e, "scan runs");
    gather_slots_kernel<<<grid_for(nslots * 32, 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(d_cands),
                                                                   reinterpret_cast<uint4*>(d_sorted), cnt, src,
                                                                   dst, nslots);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "gather runs");
    return AA_OK;
}

extern "C" aa_status aa_candidates_peaks2d_device(const aa_plan* p, int64_t nsamp, int32_t max_width,
                                                  const aa_candidate* d_sorted, const unsigned long long* d_count,
                                                  int64_t cand_capacity, int32_t dm_radius, int32_t t_radius,
                                                  aa_candidate* d_peaks, unsigned long long* d_npeaks,
                                                  void* d_tmp, size_t tmp_bytes, aa_stream_t stream) {
    clear_error();
    aa_status st = check_post_args(p, nsamp, max_width, cand_capacity);
    if (st != AA_OK) return st;
    if (!d_count || !d_npeaks || !d_tmp || (cand_capacity > 0 && (!d_sorted || !d_peaks))) {
        set_error("NULL device pointer");
        return AA_ERR_ARG;
    }
    if (dm_radius < 0 || t_radius < 0) {
        set_error("radii must be >= 0");
        return AA_ERR_ARG;
    }
    const int64_t need = 8 * post_scratch_elems(*p, nsamp, max_width, cand_capacity) + 256;
    if ((int64_t)tmp_bytes < need) {
        set_error("scratch of %zu bytes < %lld required", tmp_bytes, (long long)need);
        return AA_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(d_tmp) % 16) {
        set_error("scratch must be 16-byte aligned");
        return AA_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (cand_capacity == 0) {
        e = cudaMemsetAsync(d_npeaks, 0, sizeof(unsigned long long), s);
        return e == cudaSuccess ? AA_OK : post_fail(e, "clear peak count");
    }
    const Layout L = make_layout(*p, nsamp, max_width);
    int64_t nslots = 0, nbe = 0;
    const RangeTable rt = range_table(*p, L, nslots, nbe);
    const int64_t ndm = p->ndm_total;
    int64_t* row_start = static_cast<int64_t*>(d_tmp);
    int64_t* row_end = row_start + ndm;
    int64_t* flag = row_end + ndm;
    int64_t* last = flag + cand_capacity;
    int64_t* scratch = last + 1;
    int64_t* queue = scratch + scan_scratch(cand_capacity);
    unsigned long long* nqueue = reinterpret_cast<unsigned long long*>(queue + cand_capacity);
    uint32_t* first = reinterpret_cast<uint32_t*>(queue + cand_capacity + 1);
    ProfScope prof(kKPeaks2d, s);
    if ((e = cudaMemsetAsync(row_start, 0, (size_t)(2 * ndm) * 8, s)) != cudaSuccess)
        return post_fail(e, "clear row index");
    if ((e = cudaMemsetAsync(nqueue, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return post_fail(e, "clear peak queue");
    row_index_kernel<<<grid_for(cand_capacity, 256), 256, 0, s>>>(d_sorted, d_count, cand_capacity,
                                                                  (int32_t)ndm, row_start, row_end);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "row index");
    bucket_index_kernel<<<grid_for(cand_capacity, 256), 256, 0, s>>>(d_sorted, d_count, cand_capacity, row_start,
                                                                     row_end, rt, first);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "bucket index");
    peak_pass1_kernel<<<grid_for(cand_capacity, 256), 256, 0, s>>>(d_sorted, d_count, cand_capacity, row_start,
                                                                   row_end, first, rt, dm_radius, t_radius, flag,
                                                                   last, queue, nqueue);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "peak flags");
    peak_pass2_kernel<<<grid_for(cand_capacity * 32, 256), 256, 0, s>>>(d_sorted, d_count, cand_capacity,
                                                                         row_start, row_end, first, rt, dm_radius,
                                                                         t_radius, flag, last, queue, nqueue);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "peak flags");
    if ((e = exclusive_scan(flag, d_count, cand_capacity, scratch, s)) != cudaSuccess)
        return post_fail(e, "scan peak flags");
    compact_kernel<<<grid_for(cand_capacity, 256), 256, 0, s>>>(d_sorted, d_count, cand_capacity, flag, last,
                                                                d_peaks, d_npeaks);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_fail(e, "compact peaks");
    return AA_OK;
}

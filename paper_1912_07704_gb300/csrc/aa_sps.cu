// Single-pulse search kernels for sm_103a (arXiv:1912.07704 Sec. 1: boxcar
// filters and peak finding on every dedispersed series, on the GPU).
//
//   stats   : per series exact integer moments (sum y, sum y^2 in 128 bits),
//             mu, sigma (population) and the per-width factors
//             r_w = 1/(sigma sqrt w), c_w = w (mu - m0) r_w  (FP64 -> FP32).
//   boxcar  : for every start t, B(t) = max_{w<=min(W,L-t)} SNR_w(t) with
//             SNR_w = (S'_w - w (mu - m0)) / (sigma sqrt w) = S'_w r_w - c_w,
//             S'_w = sum_{k<w} (y[t+k] - m0) summed exactly (FP32 when every
//             partial sum of the tile fits in 2^24, int64 otherwise); then
//             thresholded local maxima are appended to the candidate list,
//             one atomic per CTA (the CTA's run is contiguous and ordered by t,
//             and is described by a chunk header).
//             The CTA then resolves each of its candidates' width (the
//             smallest maximising w) from the series it staged, with the same
//             arithmetic bit for bit.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr float kSentinel = -1.2676506002282294e30f;  // -2^100: marks t outside [0, L)
constexpr float kSentinelTest = -1e29f;

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__global__ void rsqrt_table_kernel(double* t, int wpad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < wpad) t[i] = 1.0 / sqrt((double)(i + 1));
}

// 128-bit warp reduction on (hi, lo) halves.
__device__ __forceinline__ void add128(unsigned long long& hi, unsigned long long& lo,
                                       unsigned long long h2, unsigned long long l2) {
    const unsigned long long n = lo + l2;
    hi += h2 + (n < lo ? 1ull : 0ull);
    lo = n;
}

constexpr int kStatsThreads = 512;

// Sparse width ladder: width chunk c (widths 16c+1 .. 16c+16) takes part iff
// its bit is set.  Chunks 0-3 always; then c_0 = 4 and
// c_{n+1} = max(c_n + 1, ceil(c_n * g16 / 16)).  Whole CTA; words past
// nchunks are cleared.
__host__ __device__ constexpr int ladder_words(int wpad) { return (wpad / kSpsSlots + 31) / 32; }
__device__ __forceinline__ void fill_ladder(uint32_t* mask, int nchunks, int g16) {
    for (int i = threadIdx.x; i < (nchunks + 31) / 32; i += blockDim.x) mask[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < min(4, nchunks); ++c) mask[c >> 5] |= 1u << (c & 31);
        for (int c = 4; c < nchunks; c = max(c + 1, (c * g16 + 15) / 16)) mask[c >> 5] |= 1u << (c & 31);
    }
}
__device__ __forceinline__ bool ladder_has(const uint32_t* mask, int w) {  // width w >= 1
    const int c = (w - 1) / kSpsSlots;
    return (mask[c >> 5] >> (c & 31)) & 1u;
}

// Statistics of one series (row) and its width table; whole CTA.
//
// Exact integer sums N, S1 = sum y, S2 = sum y^2 (128-bit) over the kept
// samples; pass 0 keeps every sample.  With k-sigma clipping (k = c16/16),
// each further pass keeps the samples with |y - mu| <= k sigma of the previous
// set, i.e. (times 16N, squared) 256 (N y - S1)^2 <= c16^2 (N S2 - S1^2).
// That set is an interval of integers; thread 0 finds its ends exactly (an
// FP64 estimate corrected by the 128-bit test), so each sample needs two
// compares.  Stops after clip_iters passes, at a pass keeping nothing
// (dropped) or at a fixed point (same N, S1, S2).

// 256 (N v - S1)^2 <= R, exactly (|N v - S1| < 2^57 for |v| <= 2^25, N < 2^31)
__device__ __forceinline__ bool clip_keeps(long long N, long long S1, unsigned __int128 R, long long v) {
    const long long d = N * v - S1;
    const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
    return (((unsigned __int128)ad * ad) << 8) <= R;
}

// Ends [lo, hi] of the kept interval, clamped to +-2^25 (every sample lies
// within +-2^24); lo > hi when no integer is kept.
__device__ void clip_interval(long long N, long long S1, unsigned __int128 R, long long& lo, long long& hi) {
    constexpr long long kLim = 1ll << 25;
    const double half = sqrt((double)R) / 16.0;  // |N v - S1| <= half
    const double c = (double)S1 / (double)N, h = half / (double)N;
    lo = (long long)fmax(fmin(ceil(c - h), (double)kLim), (double)-kLim);
    hi = (long long)fmax(fmin(floor(c + h), (double)kLim), (double)-kLim);
    // the estimate is within a few units; move each end onto the exact boundary
    for (int k = 0; k < 64 && lo <= hi && !clip_keeps(N, S1, R, lo); ++k) ++lo;
    for (int k = 0; k < 64 && lo > -kLim && clip_keeps(N, S1, R, lo - 1); ++k) --lo;
    for (int k = 0; k < 64 && hi >= lo && !clip_keeps(N, S1, R, hi); ++k) --hi;
    for (int k = 0; k < 64 && hi < kLim && clip_keeps(N, S1, R, hi + 1); ++k) ++hi;
}

__device__ __forceinline__ void stats_accumulate(float yf, bool clip, float lo, float hi, long long& cnt,
                                                 long long& s1, long long& s2) {
    if (clip && !(yf >= lo && yf <= hi)) return;
    const int v = (int)yf;  // exact: |y| < 2^24
    ++cnt;
    s1 += v;
    s2 += (long long)v * v;
}

// Statistics of a series from the exact sums of its N samples, S1 = sum y
// and S2 = H:Lo = sum y^2 (128 bits); f receives mu - m0.
__device__ RowStats row_stats_from_sums(long long N, long long S1, unsigned long long H, unsigned long long Lo,
                                        double& f) {
    RowStats st{};
    if (N > 0) {
        // N^2 var = N * sum y^2 - (sum y)^2, exact in 128 bits
        const unsigned __int128 S2 = ((unsigned __int128)H << 64) | Lo;
        const __int128 num = (__int128)N * (__int128)S2 - (__int128)S1 * (__int128)S1;
        const unsigned __int128 un = num > 0 ? (unsigned __int128)num : 0;
        const double numd = (double)(unsigned long long)(un >> 64) * 18446744073709551616.0 +
                            (double)(unsigned long long)un;
        st.mu = (double)S1 / (double)N;
        st.sigma = sqrt(numd) / (double)N;
        const long long m0 = llround(st.mu);
        st.m0 = (float)m0;
        st.inv_sigma = st.sigma > 0 ? 1.0 / st.sigma : 0.0;
        st.zero_sigma = st.sigma > 0 ? 0 : 1;
        f = (double)(S1 - m0 * N) / (double)N;  // mu - m0
    } else {
        st.zero_sigma = 1;
        f = 0.0;
    }
    return st;
}

// Width table of one row, whole CTA: r_w = 1/(sigma sqrt w), c_w = w f r_w
// (FP64, stored FP32 as (r_w, -c_w)); widths past max_width never win.
__device__ void write_width_table(const SpsArgs& a, const double* rsw, int row, double f, double inv) {
    float2* tab = a.table + (int64_t)row * a.wpad;
    for (int i = threadIdx.x; i < a.wpad; i += blockDim.x) {
        const int w = i + 1;
        if (w <= a.max_width) {
            const double r = inv * rsw[i];
            const double c = (double)w * f * r;
            tab[i] = make_float2((float)r, (float)(-c));
        } else {
            tab[i] = make_float2(0.0f, -FLT_MAX);
        }
    }
}

__device__ __forceinline__ void stats_row(const SpsArgs& a, const double* rsw, int row) {
    constexpr int NW = kStatsThreads / 32;
    constexpr int64_t kFlush = 4096;  // float4 steps per 128-bit flush: 2^14 samples, s2 < 2^14 * 2^48
    __shared__ long long s1w[NW], cw[NW];
    __shared__ unsigned long long hiw[NW], low[NW];
    __shared__ long long sh_N, sh_S1;           // sums of the accepted set
    __shared__ unsigned long long sh_H, sh_L;   // its S2 (high, low words)
    __shared__ float sh_lo, sh_hi;              // kept interval of the next pass
    __shared__ int sh_go;
    __shared__ double sh_f, sh_inv;
    const float* y = a.dd + (int64_t)row * a.pitch;  // 16-byte aligned rows
    const int64_t n = a.length;
    const int64_t n4 = n >> 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int iters = a.clip_iters;
    for (int pass = 0; pass <= iters; ++pass) {
        const bool clip = pass > 0;
        const float lo_f = clip ? sh_lo : 0.f, hi_f = clip ? sh_hi : 0.f;
        long long cnt = 0, s1 = 0;
        unsigned long long hi = 0, lo = 0;
        const float4* y4 = reinterpret_cast<const float4*>(y);
        for (int64_t b = threadIdx.x; b < n4; b += (int64_t)kStatsThreads * kFlush) {
            const int64_t e = min(n4, b + (int64_t)kStatsThreads * kFlush);
            long long s2 = 0;
            for (int64_t j = b; j < e; j += kStatsThreads) {
                const float4 q = y4[j];
                stats_accumulate(q.x, clip, lo_f, hi_f, cnt, s1, s2);
                stats_accumulate(q.y, clip, lo_f, hi_f, cnt, s1, s2);
                stats_accumulate(q.z, clip, lo_f, hi_f, cnt, s1, s2);
                stats_accumulate(q.w, clip, lo_f, hi_f, cnt, s1, s2);
            }
            add128(hi, lo, 0ull, (unsigned long long)s2);
        }
        if (threadIdx.x < (int)(n - 4 * n4)) {
            long long s2 = 0;
            stats_accumulate(y[4 * n4 + threadIdx.x], clip, lo_f, hi_f, cnt, s1, s2);
            add128(hi, lo, 0ull, (unsigned long long)s2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            add128(hi, lo, h2, l2);
        }
        if (lane == 0) {
            cw[warp] = cnt;
            s1w[warp] = s1;
            hiw[warp] = hi;
            low[warp] = lo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long C = 0, S1 = 0;
            unsigned long long H = 0, Lo = 0;
            for (int w = 0; w < NW; ++w) {
                C += cw[w];
                S1 += s1w[w];
                add128(H, Lo, hiw[w], low[w]);
            }
            int go;
            if (clip && C == 0) {
                go = 0;  // nothing kept: keep the previous set
            } else {
                const bool same = clip && C == sh_N && S1 == sh_S1 && H == sh_H && Lo == sh_L;
                sh_N = C;
                sh_S1 = S1;
                sh_H = H;
                sh_L = Lo;
                go = pass < iters && !same;
            }
            if (go) {
                const unsigned __int128 S2 = ((unsigned __int128)sh_H << 64) | sh_L;
                const __int128 V = (__int128)sh_N * (__int128)S2 - (__int128)sh_S1 * (__int128)sh_S1;
                const unsigned __int128 R =
                    (unsigned __int128)(a.clip_c16 * a.clip_c16) * (V > 0 ? (unsigned __int128)V : 0);
                long long vlo, vhi;
                clip_interval(sh_N, sh_S1, R, vlo, vhi);
                sh_lo = (float)vlo;  // exact: |v| <= 2^25
                sh_hi = (float)vhi;
            }
            sh_go = go;
        }
        __syncthreads();
        if (!sh_go) break;
    }
    if (threadIdx.x == 0) {
        const RowStats st = row_stats_from_sums(sh_N, sh_S1, sh_H, sh_L, sh_f);
        sh_inv = st.inv_sigma;
        a.stats[row] = st;
    }
    __syncthreads();
    write_width_table(a, rsw, row, sh_f, sh_inv);
}

// Fused statistics (the dedispersion kernels summed each row exactly into
// acc[3 r .. 3 r + 2] = (sum y, sum y^2 low, high)): mu, sigma and the width
// table of every row of a range, with the arithmetic of stats_row's plain
// pass (bit for bit the same results).  One CTA per row.
__global__ void __launch_bounds__(256) sps_finalize_kernel(SpsArgs a, const double* rsw,
                                                          const unsigned long long* acc) {
    __shared__ double sh_f, sh_inv;
    const int row = blockIdx.x;
    if (threadIdx.x == 0) {
        const unsigned long long* r = acc + 3 * (int64_t)row;
        const RowStats st = row_stats_from_sums(a.length, (long long)r[0], r[2], r[1], sh_f);
        sh_inv = st.inv_sigma;
        a.stats[row] = st;
    }
    __syncthreads();
    write_width_table(a, rsw, row, sh_f, sh_inv);
}

__global__ void __launch_bounds__(kStatsThreads) sps_stats_kernel(SpsArgs a, const double* rsw) {
    stats_row(a, rsw, blockIdx.x);
}

// Block-wide exclusive scan of one int64 per thread.
template <int NT>
__device__ long long block_exclusive_scan(long long v, long long* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < NT / 32 ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < NT / 32) scratch[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const long long before = warp > 0 ? scratch[warp - 1] : 0;
    return before + inc - v;
}

// Exclusive scan that also returns the block total.
template <int NT>
__device__ long long block_exclusive_scan_total(long long v, long long* scratch, long long& total) {
    const long long ex = block_exclusive_scan<NT>(v, scratch);
    total = scratch[NT / 32 - 1];
    __syncthreads();  // scratch may be reused after this
    return ex;
}

// Block-wide exclusive scan of one int64 `run` per thread, together with the
// block total and the smallest and largest prefix value min(before + mn) /
// max(before + mx) (mn <= 0 <= mx relative to the thread's own start), in two
// barriers.  scratch: 3 * NT / 32 entries.
template <int NT>
__device__ void block_scan_minmax(long long run, long long mn, long long mx, long long* scratch,
                                  long long& before, long long& total, long long& gmn, long long& gmx) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    const long long ex = inc - run;
    long long lmn = ex + mn, lmx = ex + mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lmn = min(lmn, __shfl_xor_sync(0xffffffffu, lmn, o));
        lmx = max(lmx, __shfl_xor_sync(0xffffffffu, lmx, o));
    }
    if (lane == 31) scratch[warp] = inc;
    if (lane == 0) {
        scratch[NW + warp] = lmn;
        scratch[2 * NW + warp] = lmx;
    }
    __syncthreads();
    long long t = 0, wbase = 0, bmn = LLONG_MAX, bmx = LLONG_MIN;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        bmn = min(bmn, t + scratch[NW + w]);
        bmx = max(bmx, t + scratch[2 * NW + w]);
        if (w == warp) wbase = t;
        t += scratch[w];
    }
    before = wbase + ex;
    total = t;
    gmn = bmn;
    gmx = bmx;
    __syncthreads();  // scratch may be reused after this
}

template <int NT>
__device__ void block_minmax(long long& mn, long long& mx, long long* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __syncthreads();
    if (lane == 0) {
        scratch[warp] = mn;
        scratch[NT / 32 + warp] = mx;
    }
    __syncthreads();
    mn = scratch[0];
    mx = scratch[NT / 32];
    for (int w = 1; w < NT / 32; ++w) {
        mn = min(mn, scratch[w]);
        mx = max(mx, scratch[NT / 32 + w]);
    }
}

constexpr int M = kSpsSlots;
constexpr int NT = kSpsThreads;

// Exact-FP32 tiles.  P is the prefix-sum array of the staged series (index
// i <-> start time t0-1+i): P[i] = sum of y - m0 over the valid samples before
// i, -kBig once a window would run past the series end.  Every window sum
// S_w(t) = P[p+w] - P[p] is an exact FP32 integer (the caller checked that
// the prefix range of the tile is <= 2^24), so this is bit for bit the
// running sum.  Thread owns slots p = M*tid + i; base[i] = P[p] (or +kBig for
// a start outside the series).  C[i] receives w0 of the first chunk of M
// widths (w0+1 .. w0+M) whose best SNR equals B[i]: the smallest maximising
// width lies in that chunk, so the candidate's width is found by evaluating
// it alone.
constexpr float kBig = 1.2676506002282294e30f;  // 2^100

// Block maxima of the prefix sums: Q[j] = max P[i] over i in
// [kQSpan j, kQSpan (j+1)), for the pruning bounds of the wide widths.
constexpr int kQSpan = 128;
__host__ __device__ constexpr int sps_q_count(int wpad) {
    return (kSpsTile + wpad + M + kQSpan - 1) / kQSpan;
}

// Bound of one thread's M starts over a width segment [w1, w2].  For a start
// p in [ps, pl] (pl = ps + M - 1) and a width w, the window's end is p + w, so
// S_w(p) <= P[end] - pmin and w >= max(w1, end - pl); -w f <= -wlo f (f >= 0)
// or -w2 f (f < 0).  So SNR_w(p) <= (P[end] - pmin - drift) / (sigma sqrt(wlo))
// for every end, maximised over the ends:
//  * w1 <= kQSpan: the ends [ps + w1, pl + w2] read one by one (as aligned
//    16-byte vectors from ps + w1 - 1, a superset), wlo = w1;
//  * wider: per block j of Q overlapping the ends, Q[j] with
//    wlo = max(w1, kQSpan j - pl).
// FP32 with the rounding of each step bounded and added (|f| <= 1/2 since
// m0 = round(mu); the differences of the exact integer sums P are exact;
// rsqrtf within 2 ulp), then widened by 1e-4 relative and absolute.
struct ThreadBound {
    const float* Q;
    float pmin;       // min of P over the thread's valid starts (FLT_MAX: none)
    float f;          // mu - m0
    float inv_sigma;
    float cut;        // segments bounded below this are skipped (-FLT_MAX: none)
    int max_width, ylen, nq, ps;
    bool active;      // pruning enabled
};

__device__ __forceinline__ float piece_bound(float top, const ThreadBound& b, int wlo, int whi) {
    const float drift = b.f >= 0.0f ? (float)wlo * b.f : (float)whi * b.f;
    const float diff = top - b.pmin;
    const float rs = rsqrtf((float)wlo);
    // 6 roundings of at most 2^-24 relative each on magnitudes <= |diff| + |drift|
    const float slack = (fabsf(diff) + fabsf(drift)) * b.inv_sigma * rs * 1e-6f + 1e-6f;
    return (diff - drift) * b.inv_sigma * rs + slack;
}

__device__ __forceinline__ float thread_segment_bound(const float* __restrict__ P, const ThreadBound& b,
                                                      int w1, int w2) {
    if (b.pmin == FLT_MAX) return -FLT_MAX;
    const int pl = b.ps + M - 1;
    const int hi = min(b.ylen - 1, pl + w2);
    float ub;
    if (w1 <= kQSpan) {
        // ylen is a multiple of 4, so the last vector ends inside the staged series
        float pmax = -FLT_MAX;
        for (int e = (b.ps + w1 - 1) & ~3; e <= hi; e += 4) {
            const float4 v = *reinterpret_cast<const float4*>(P + e);
            pmax = fmaxf(fmaxf(pmax, fmaxf(v.x, v.y)), fmaxf(v.z, v.w));
        }
        ub = piece_bound(pmax, b, w1, w2);
    } else {
        ub = -FLT_MAX;
        const int j1 = min(b.nq - 1, hi / kQSpan);
        for (int j = (b.ps + w1) / kQSpan; j <= j1; ++j)
            ub = fmaxf(ub, piece_bound(b.Q[j], b, max(w1, j * kQSpan - pl), w2));
    }
    return ub + fabsf(ub) * 1e-4f + 1e-4f;
}

// Main loop.  With pruning, the widths after the first chunk are checked in
// power-of-two blocks [w0+1, 2 w0] (w0 = 16, 32, ...), and inside a block
// that survives and spans more than 128 widths, in segments [w0+1, w0+128].
// A thread can skip a block or segment when its bound is below max(cut, min
// over its slots of the running B): below the running B it can change
// neither B nor C of any of its slots (exact for every slot); below the
// threshold cut it can only change sub-threshold values (exact for every
// B >= threshold and for every peak decision).  The warp skips it when all
// of its threads can (the warp evaluates chunks in lockstep; evaluating a
// chunk a thread could skip changes nothing of the above).  Widths are
// visited in increasing order, so the running B of the small widths prunes
// the wide ones; a thread before a bright pulse evaluates the widths whose
// windows end near the pulse, not the wider ones, whose bound the pulse's
// SNR at the narrower width already exceeds.
__device__ __forceinline__ int boxcar_prefix(const float* __restrict__ P,
                                             const float2* __restrict__ tab, int wpad,
                                             const float (&base)[M], const ThreadBound& bnd,
                                             const uint32_t* lmask, float (&B)[M], int (&C)[M]) {
    const float* pb = P + M * threadIdx.x;
    int evaluated = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        B[i] = -FLT_MAX;
        C[i] = 0;
    }
    constexpr int kSeg = 128;  // widths per segment inside the wide power-of-two blocks
    for (int w0 = 0; w0 < wpad; w0 += M) {
        const bool blk = (w0 & (w0 - 1)) == 0;  // first chunk of a power-of-two block
        if (bnd.active && w0 >= 16 && (blk || (w0 >= 2 * kSeg && (w0 & (kSeg - 1)) == 0))) {
            int w_end = blk ? 2 * w0 : w0 + kSeg;
            float bmin = B[0];
#pragma unroll
            for (int i = 1; i < M; ++i) bmin = fminf(bmin, B[i]);
            const float floor_b = fmaxf(bnd.cut, bmin);
            bool skip = !__any_sync(0xffffffffu,
                                    thread_segment_bound(P, bnd, w0 + 1, min(w_end, bnd.max_width)) >= floor_b);
            if (!skip && blk && w0 >= 2 * kSeg) {
                w_end = w0 + kSeg;
                skip = !__any_sync(0xffffffffu,
                                   thread_segment_bound(P, bnd, w0 + 1, min(w_end, bnd.max_width)) >= floor_b);
            }
            if (skip) {
                w0 = w_end - M;  // next block or segment
                continue;
            }
        }
        if (lmask && !ladder_has(lmask, w0 + 1)) continue;  // chunk not on the width ladder
        ++evaluated;
        float win[2 * M];  // win[k] = P[p_thread + w0 + k]
#pragma unroll
        for (int k = 0; k < 2 * M; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(pb + w0 + k);
            win[k] = v.x; win[k + 1] = v.y; win[k + 2] = v.z; win[k + 3] = v.w;
        }
        float Bc[M];  // best SNR of this chunk, per slot
        {
            const float2 rc0 = tab[w0];
            const float2 rc1 = tab[w0 + 1];
#pragma unroll
            for (int i = 0; i < M; ++i)
                Bc[i] = fmaxf(fmaf(win[i + 1] - base[i], rc0.x, rc0.y),
                              fmaf(win[i + 2] - base[i], rc1.x, rc1.y));
        }
#pragma unroll
        for (int s = 2; s < M; s += 2) {
            const float2 rc0 = tab[w0 + s];
            const float2 rc1 = tab[w0 + s + 1];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const float v0 = fmaf(win[i + s + 1] - base[i], rc0.x, rc0.y);
                const float v1 = fmaf(win[i + s + 2] - base[i], rc1.x, rc1.y);
                Bc[i] = max3f(Bc[i], v0, v1);
            }
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (Bc[i] > B[i]) {  // strict: an equal later chunk keeps the earlier one
                B[i] = Bc[i];
                C[i] = w0;
            }
        }
    }
    return evaluated;
}

// Exact int64 running sums for slot i, for tiles whose partial sums may
// exceed 2^24.  Same SNR arithmetic as boxcar_fast (fmaf of the correctly
// rounded sum).
__device__ __noinline__ float boxcar_exact_slot(const float* __restrict__ ys,
                                                const float2* __restrict__ tab, int wpad, int i,
                                                const uint32_t* lmask) {
    const float* yb = ys + M * threadIdx.x + i;
    long long S = 0;
    float best = -FLT_MAX;
    for (int w = 1; w <= wpad; ++w) {
        const float v = yb[w - 1];
        if (v < kSentinelTest) break;  // window left [0, L): later widths invalid too
        S += (long long)v;
        if (lmask && !ladder_has(lmask, w)) continue;
        const float2 rc = tab[w - 1];
        best = fmaxf(best, fmaf(__ll2float_rn(S), rc.x, rc.y));
    }
    return best;
}

// Shared memory after the main loop: the end of the table region is reused
// for B(t) (kSpsTile floats) followed by the candidate entries (kSpsTile u32).
__host__ __device__ constexpr int sps_region_bytes(int wpad) {
    return (wpad * 8 > kSpsTile * 8) ? wpad * 8 : kSpsTile * 8;
}

// One CTA's work: tiles [tile_lo, tile_hi) of series `row`, in order.  `sm`
// is the dynamic shared memory; the caller guarantees that every thread has
// finished any previous work.
//
// Consecutive tiles of a series overlap by ylen - kSpsOwned staged samples
// (the W-sample halo), so after the first tile the staged prefix sums are
// slid down by kSpsOwned and only the kSpsOwned new samples are staged and
// summed, continuing from the exact sum at the old end.  Prefix sums are then
// relative to the first fully staged tile; sliding is allowed while every
// staged prefix sum lies within +-2^23 (so every window sum, a difference of
// two, is an exact FP32 integer); otherwise the tile is staged afresh.
__device__ __forceinline__ void boxcar_block(const SpsArgs& a, int row, int64_t tile_lo, int64_t tile_hi,
                                             float* sm) {
    __shared__ long long scratch[3 * NT / 32];
    __shared__ unsigned long long s_base;
    __shared__ long long s_pend;  // exact prefix sum just past the staged series
    const int wpad = a.wpad;
    const int ylen = kSpsTile + wpad + M;
    float* ys = sm;
    float2* tab = reinterpret_cast<float2*>(sm + ((ylen + 3) & ~3));
    float* Qs = sm + ((ylen + 3) & ~3) + sps_region_bytes(wpad) / 4;
    const int nq = sps_q_count(wpad);
    uint32_t* s_ladder = reinterpret_cast<uint32_t*>(Qs + ((nq + 3) & ~3));
    const uint32_t* lmask = a.ladder_g16 > 0 ? s_ladder : nullptr;
    if (lmask) fill_ladder(s_ladder, wpad / M, a.ladder_g16);  // visible after the staging barrier
    const int64_t L = a.length;
    const float* y = a.dd + (int64_t)row * a.pitch;
    const RowStats st = a.stats[row];
    const float m0 = st.m0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float2* gtab = a.table + (int64_t)row * wpad;
    // B(t) and the candidate list take the last kSpsTile * 8 bytes of the
    // table region after the width loop: the entries of widths up to
    // 2 * lists4 stay in shared memory for the candidates' widths
    const int lists4 = (sps_region_bytes(wpad) - kSpsTile * 8) / 16;
    constexpr int kBatch = 8;
    constexpr long long kSlideMax = 1ll << 23;
    bool slide = false;  // ys holds the previous tile's prefix sums, all within +-2^23

    for (int64_t tile = tile_lo; tile < tile_hi; ++tile) {
        const int64_t t0 = tile * kSpsOwned;
        // valid start/sample positions: i in [va, vb]  (t = t0-1+i in [0, L))
        const int va = t0 == 0 ? 1 : 0;
        const int vb = (int)min((int64_t)ylen - 1, L - t0);
        const int nkeep = ylen - kSpsOwned;  // staged samples shared with the previous tile

        // The width table, then the series: after a slide only the new samples
        // (minus m0, sentinel outside [0, L)), else all of them.  The previous
        // tile's B(t) and candidate list overwrote only the table's last
        // kSpsTile * 8 bytes (from float4 lists4 on), so after a slide only
        // those are staged again.
        {
            const float4* g4 = reinterpret_cast<const float4*>(gtab);  // wpad is even
            float4* t4 = reinterpret_cast<float4*>(tab);
            const int n4 = wpad / 2;
            for (int i0b = (slide ? lists4 : 0) + threadIdx.x; i0b < n4; i0b += NT * kBatch) {
                float4 v[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0b + u * NT;
                    if (i < n4) v[u] = __ldg(g4 + i);
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u)
                    if (i0b + u * NT < n4) t4[i0b + u * NT] = v[u];
            }
        }
        bool fast = false;
        if (slide) {
            // slide P down by kSpsOwned: rounds of NT x 16 values, all loads of a
            // round before its stores (a round's source and destination overlap;
            // a later round's source never meets an earlier round's destination)
            constexpr int kR = 16;
            for (int r0 = 0; r0 < nkeep; r0 += NT * kR) {
                float v[kR];
#pragma unroll
                for (int u = 0; u < kR; ++u) {
                    const int i = r0 + u * NT + threadIdx.x;
                    v[u] = i < nkeep ? ys[i + kSpsOwned] : 0.0f;
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < kR; ++u) {
                    const int i = r0 + u * NT + threadIdx.x;
                    if (i < nkeep) ys[i] = v[u];
                }
            }
            __syncthreads();  // the last round's loads are done before the new samples land
            for (int i0b = nkeep + threadIdx.x; i0b < ylen; i0b += NT * kBatch) {
                float v[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0b + u * NT;
                    const int64_t t = t0 - 1 + i;
                    v[u] = (i < ylen && t >= 0 && t < L) ? __ldg(y + t) - m0 : kSentinel;
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u)
                    if (i0b + u * NT < ylen) ys[i0b + u * NT] = v[u];
            }
            __syncthreads();
            // exact sums of the new samples, continuing from the old end
            const int segn = ((kSpsOwned + NT - 1) / NT) | 1;  // odd: distinct banks
            const int j0 = min(ylen, nkeep + threadIdx.x * segn), j1 = min(ylen, j0 + segn);
            long long run = 0, mn = 0, mx = 0;
            for (int i = j0; i < j1; ++i) {
                const float v = ys[i];
                if (v > kSentinelTest) {
                    run += (long long)(int)v;
                    mn = min(mn, run);
                    mx = max(mx, run);
                }
            }
            long long tot = 0, ex = 0, gmn = 0, gmx = 0;
            const long long pend = s_pend;
            block_scan_minmax<NT>(run, mn, mx, scratch, ex, tot, gmn, gmx);
            const long long before = pend + ex;
            gmn += pend;
            gmx += pend;
            fast = gmn >= -kSlideMax && gmx <= kSlideMax;
            if (fast) {
                float runf = (float)before;
                for (int i = j0; i < j1; ++i) {
                    const float v = ys[i];
                    ys[i] = i > vb + 1 ? -kBig : runf;
                    if (v > kSentinelTest) runf += v;
                }
                if (threadIdx.x == 0) s_pend = pend + tot;
            }
            // (the reads of s_pend above precede this barrier, its write follows it)
            __syncthreads();
        }
        if (!fast) {
            // stage every sample afresh; loads in batches so that latencies overlap
            for (int i0b = threadIdx.x; i0b < ylen; i0b += NT * kBatch) {
                float v[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0b + u * NT;
                    const int64_t t = t0 - 1 + i;
                    v[u] = (i < ylen && t >= 0 && t < L) ? __ldg(y + t) - m0 : kSentinel;
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u)
                    if (i0b + u * NT < ylen) ys[i0b + u * NT] = v[u];
            }
            __syncthreads();

            // Largest |partial sum| of the tile = range of the prefix sums of ys over
            // its valid samples: FP32 sums are exact when it is <= 2^24.
            const int seg = ((ylen + NT - 1) / NT) | 1;  // odd: the threads' segments fall on distinct banks
            const int i0 = min(ylen, threadIdx.x * seg), i1 = min(ylen, i0 + seg);
            long long run = 0, mn = 0, mx = 0;
            for (int i = i0; i < i1; ++i) {
                const float v = ys[i];
                if (v > kSentinelTest) {
                    run += (long long)(int)v;
                    mn = min(mn, run);
                    mx = max(mx, run);
                }
            }
            long long tot = 0, before = 0, gmn = 0, gmx = 0;
            block_scan_minmax<NT>(run, mn, mx, scratch, before, tot, gmn, gmx);
            fast = (gmx - gmn) <= (1ll << 24);
            slide = gmn >= -kSlideMax && gmx <= kSlideMax;  // the next tile may slide
            if (fast) {
                // ys -> prefix sums P, in place (exact FP32 integers)
                __syncthreads();
                float runf = (float)before;
                for (int i = i0; i < i1; ++i) {
                    const float v = ys[i];
                    ys[i] = i > vb + 1 ? -kBig : runf;
                    if (v > kSentinelTest) runf += v;
                }
                if (threadIdx.x == 0) s_pend = tot;
                __syncthreads();
            }
        }
        slide = slide && fast && (tile + 1 < tile_hi);

        float B[M];
        int C[M];  // per slot: w0 of the first width chunk reaching B (0 on the exact path)
        if (fast) {
            const float* P = ys;
            if (a.prune) {  // block maxima Q: a warp reduces 4 blocks at once
                for (int j0 = 4 * warp; j0 < nq; j0 += 4 * (NT / 32)) {
                    float m[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        m[b] = -FLT_MAX;
#pragma unroll
                        for (int u = 0; u < kQSpan / 32; ++u) {
                            const int i = (j0 + b) * kQSpan + u * 32 + lane;
                            if (i < ylen) m[b] = fmaxf(m[b], P[i]);
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int b = 0; b < 4; ++b) m[b] = fmaxf(m[b], __shfl_xor_sync(0xffffffffu, m[b], o));
                    if (lane < 4 && j0 + lane < nq) Qs[j0 + lane] = lane == 0 ? m[0] : lane == 1 ? m[1] : lane == 2 ? m[2] : m[3];
                }
                __syncthreads();
            }
            float base[M];
            float pmin = FLT_MAX;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const int p = M * threadIdx.x + i;
                const bool valid = p >= va && p <= vb;
                base[i] = valid ? P[p] : kBig;
                if (valid) pmin = fminf(pmin, base[i]);
            }
            ThreadBound bnd;
            bnd.Q = Qs;
            bnd.pmin = pmin;
            bnd.f = (float)(st.mu - (double)m0);
            bnd.inv_sigma = (float)st.inv_sigma;
            bnd.cut = a.threshold > 0.0f ? a.threshold - 1e-3f : -FLT_MAX;
            bnd.max_width = a.max_width;
            bnd.ylen = ylen;
            bnd.nq = nq;
            bnd.ps = M * threadIdx.x;
            bnd.active = a.prune != 0;
            const int chunks = boxcar_prefix(P, tab, wpad, base, bnd, lmask, B, C);
            if (a.evaluated && (threadIdx.x & 31) == 0)
                atomicAdd(a.evaluated, (unsigned long long)chunks * 32ull * M * M);
            if (slide) {
                // A warp that finishes its widths early waits for the tile's
                // slowest one: meanwhile it asks L2 for the next tile's new
                // samples (every warp covers them all; later requests hit L2).
                const int64_t t_new = t0 + kSpsOwned - 1 + nkeep;  // first new sample of the next tile
                const int64_t t_end = min(L, t_new + kSpsOwned);
                for (int64_t t = t_new + 32 * lane; t < t_end; t += 32 * 32)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(y + t));
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                B[i] = boxcar_exact_slot(ys, tab, wpad, i, lmask);
                C[i] = 0;
            }
            if (a.evaluated && threadIdx.x == 0)
                atomicAdd(a.evaluated, (unsigned long long)wpad * NT * M);
        }

        __syncthreads();  // everyone done with the table
        float* Bs = reinterpret_cast<float*>(tab) + 4 * lists4;  // B(t) of every slot
        // candidate entries: slot p (bits 0-15) | first chunk w0 / M (bits 16-31)
        uint32_t* plist = reinterpret_cast<uint32_t*>(Bs + kSpsTile);
#pragma unroll
        for (int i = 0; i < M; ++i) Bs[M * threadIdx.x + i] = B[i];
        __syncthreads();

        const bool zero_sigma = st.zero_sigma != 0;
        unsigned cmask = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = M * threadIdx.x + i;
            const int64_t t = t0 - 1 + p;
            if (p >= 1 && p <= kSpsTile - 2 && t < L) {
                const float v = Bs[p];
                if (a.snr_out) a.snr_out[(int64_t)row * a.pitch + t] = zero_sigma ? 0.0f : v;
                if (!zero_sigma && v >= a.threshold && v > Bs[p - 1] && v >= Bs[p + 1]) cmask |= 1u << i;
            }
        }
        // One atomic per tile: the tile's candidates form one contiguous run in t order.
        long long total = 0;
        const long long my_off = block_exclusive_scan_total<NT>(__popc(cmask), scratch, total);
        if (total > 0) {
            const uint32_t dm_index = (uint32_t)(a.dm_offset + row);
            if (threadIdx.x == 0) {
                s_base = atomicAdd(a.count, (unsigned long long)total);
                const unsigned long long ci = atomicAdd(a.nchunks, 1ull);
                if (ci < (unsigned long long)a.chunk_cap)
                    a.chunks[ci] = CandChunk{s_base, (uint32_t)total, dm_index, (uint32_t)t0, (uint32_t)a.beam};
            }
            {
                int j = (int)my_off;
#pragma unroll
                for (int i = 0; i < M; ++i)
                    if ((cmask >> i) & 1u)
                        plist[j++] = (uint32_t)(M * threadIdx.x + i) | ((uint32_t)(C[i] / M) << 16);
            }
            __syncthreads();

            // Width of each candidate: the smallest w reaching B(t), recomputed from
            // the staged series with the main loop's arithmetic (exact running sums,
            // fmaf of the correctly rounded sum), one warp per candidate, widths
            // interleaved over lanes with a warp prefix sum.
            for (int q = warp; q < (int)total; q += NT / 32) {
                const int p = (int)(plist[q] & 0xffffu);
                const int cw0 = (int)(plist[q] >> 16) * M;
                const int64_t t = t0 - 1 + p;
                const int wmax = (int)min((int64_t)a.max_width, L - t);
                const float* yq = ys + p;  // exact path: yq[w-1] = y[t+w-1] - m0
                const float target = Bs[p];
                float best = -FLT_MAX;
                int bw = 0x7fffffff;
                if (fast) {
                    // prefix form: S_w = P[p+w] - P[p], exact
                    const float* P = ys;
                    const float b0 = P[p];
                    for (int w0 = cw0; w0 < wmax; w0 += 32) {
                        const int w = w0 + lane + 1;
                        if (w <= wmax && (!lmask || ladder_has(lmask, w))) {
                            const float2 rc = w <= 2 * lists4 ? tab[w - 1] : __ldg(gtab + w - 1);
                            const float snr = fmaf(P[p + w] - b0, rc.x, rc.y);
                            if (snr > best) { best = snr; bw = w; }
                        }
                        // widths are visited in increasing order: stop at the chunk
                        // where B(t) is first reached
                        if (__any_sync(0xffffffffu, best == target)) break;
                    }
                } else {
                    long long base = 0;
                    for (int w0 = 0; w0 < wmax; w0 += 32) {
                        const int w = w0 + lane + 1;
                        long long v = (w <= wmax) ? (long long)yq[w - 1] : 0;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const long long u = __shfl_up_sync(0xffffffffu, v, o);
                            if (lane >= o) v += u;
                        }
                        const long long S = base + v;
                        base += __shfl_sync(0xffffffffu, v, 31);
                        if (w <= wmax && (!lmask || ladder_has(lmask, w))) {
                            const float2 rc = w <= 2 * lists4 ? tab[w - 1] : __ldg(gtab + w - 1);
                            const float snr = fmaf(__ll2float_rn(S), rc.x, rc.y);
                            if (snr > best) { best = snr; bw = w; }
                        }
                        if (__any_sync(0xffffffffu, best == target)) break;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
                    if (ob > best || (ob == best && ow < bw)) { best = ob; bw = ow; }
                }
                const unsigned long long idx = s_base + (unsigned long long)q;
                if (lane == 0 && idx < (unsigned long long)a.capacity) {
                    aa_candidate c;
                    c.dm_index = dm_index;
                    c.t = (uint32_t)t;
                    c.width = (uint16_t)bw;
                    c.range = (uint8_t)a.range;
                    c.reserved = (uint8_t)a.beam;
                    c.snr = best;
                    a.cands[idx] = c;
                }
            }
        }  // total > 0
        __syncthreads();  // the next tile overwrites the series, table and lists
    }  // tiles
}

// CTA = seg_tiles consecutive tiles of one series (the last segment of a
// series may be shorter).
__global__ void __launch_bounds__(NT, 2) sps_boxcar_kernel(SpsArgs a, int ntiles, int seg_tiles) {
    extern __shared__ __align__(16) float sm[];
    const int nseg = (ntiles + seg_tiles - 1) / seg_tiles;
    const int row = (int)(blockIdx.x / (unsigned)nseg);
    const int64_t lo = (int64_t)(blockIdx.x - (unsigned)row * (unsigned)nseg) * seg_tiles;
    boxcar_block(a, row, lo, min((int64_t)ntiles, lo + seg_tiles), sm);
}

constexpr int kMaxDecLevels = 16;

// ------------------------------------------------------------ decimated ladder
// Approximate search for wide boxcars (the cited search evaluates them on the
// series decimated by pairs, Sec. 1).  Level 0: widths 1..min(W0, W) of the
// windows starting at t, evaluated as the exhaustive search's first chunks.
// Level k >= 1 (while W0 2^(k-1) < W): widths w = m 2^k, W0/2 < m <= W0,
// w <= W, of the window starting at the level-k grid point
// s = floor(t / 2^k) 2^k <= t (m samples of the series decimated k times by
// pairs).  Every level comes from the tile's one full-rate prefix sum P:
// S = P[s + w] - P[s], exact.  B(t) = the largest SNR over level 0 at t and
// each level's window at its grid point, levels in increasing width (ties to
// the smallest width); the width of a level-k maximum is known directly, that
// of a level-0 maximum is resolved as in the exhaustive search.
//
// Shared memory: the staged series with a left halo H >= 2^K (a slot's
// level-K grid point lies up to 2^K - 1 samples before it), the compact width
// table (level 0, then W0/2 entries per level), and a region that holds the
// levels' strided prefix sums P_k and grid maxima B_k, then B(t), the
// candidate list and the direct widths.
struct DecLayout {
    int K, H, W0, W0e, wpad0, ylen4, ntab;
    int npk, nbk;             // entries of all levels' P_k and B_k (upper bounds for any tile)
    int tab_off, reg_off;     // in floats
    size_t bytes;
};
__host__ __device__ inline int dec_level_points(int k) { return ((kSpsTile - 1) >> k) + 2; }
__host__ __device__ inline DecLayout dec_layout(int W, int W0) {
    DecLayout d{};
    d.W0 = W0;
    d.K = 0;
    while ((W0 << d.K) < W) ++d.K;
    d.H = d.K > 0 ? ((1 << d.K) > 16 ? (1 << d.K) : 16) : 0;
    d.W0e = W0 < W ? W0 : W;
    d.wpad0 = (d.W0e + M - 1) / M * M;
    d.ylen4 = (d.H + kSpsTile + W + M + 3) & ~3;
    d.ntab = d.wpad0 + d.K * (W0 / 2);
    d.npk = d.nbk = 0;
    for (int k = 1; k <= d.K; ++k) {
        d.nbk += dec_level_points(k);
        d.npk += dec_level_points(k) + W0;
    }
    const int reg_a = d.npk * 4 + d.nbk * 4 + d.nbk;       // P_k, B_k (float), winning m (u8)
    const int reg_b = kSpsTile * 4 + kSpsTile * 4 + kSpsTile * 2;  // B(t), candidates, direct widths
    d.tab_off = d.ylen4;
    d.reg_off = d.tab_off + ((d.ntab * 2 + 3) & ~3);
    d.bytes = (size_t)d.reg_off * 4 + (size_t)(((reg_a > reg_b ? reg_a : reg_b) + 15) & ~15);
    return d;
}

__device__ __forceinline__ void boxcar_dec_block(const SpsArgs& a, int ntiles, int64_t bid, float* sm) {
    __shared__ long long scratch[2 * NT / 32];
    __shared__ unsigned long long s_base;
    __shared__ int s_lvl[2 * kMaxDecLevels + 2];  // per level: P_k offset, B_k offset
    const DecLayout d = dec_layout(a.max_width, a.dec_w0);
    const int W0 = d.W0, K = d.K, H = d.H, ylen = d.ylen4;
    float* ys = sm;
    float2* tab = reinterpret_cast<float2*>(sm + d.tab_off);
    float* reg = sm + d.reg_off;
    const int row = (int)(bid / ntiles);
    const int64_t tile = bid - (int64_t)row * ntiles;
    const int64_t t0 = tile * kSpsOwned;
    const int64_t L = a.length;
    const int64_t o = t0 - 1 - H;  // t of ys[0]
    const float* y = a.dd + (int64_t)row * a.pitch;
    const RowStats st = a.stats[row];
    const float m0 = st.m0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // stage the series (minus m0, sentinel outside [0, L)) and the table
    constexpr int kBatch = 8;
    for (int i0b = threadIdx.x; i0b < ylen; i0b += NT * kBatch) {
        float v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = i0b + u * NT;
            const int64_t t = o + i;
            v[u] = (i < ylen && t >= 0 && t < L) ? __ldg(y + t) - m0 : kSentinel;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (i0b + u * NT < ylen) ys[i0b + u * NT] = v[u];
    }
    const float2* gtab = a.table + (int64_t)row * a.wpad;
    for (int e = threadIdx.x; e < d.ntab; e += NT) {
        int w;
        if (e < d.wpad0) {
            w = e + 1;
        } else {
            const int k = 1 + (e - d.wpad0) / (W0 / 2);
            w = (W0 / 2 + 1 + (e - d.wpad0) % (W0 / 2)) << k;
        }
        tab[e] = w <= a.max_width ? __ldg(gtab + w - 1) : make_float2(0.0f, -FLT_MAX);
    }
    if (threadIdx.x == 0) {
        int pk = 0, bk = d.npk;
        for (int k = 1; k <= K; ++k) {
            s_lvl[2 * k] = pk;
            s_lvl[2 * k + 1] = bk;
            pk += dec_level_points(k) + W0;
            bk += dec_level_points(k);
        }
    }
    __syncthreads();

    // exact FP32 prefix sums when the tile's partial sums stay within 2^24
    const int seg = ((ylen + NT - 1) / NT) | 1;  // odd: the threads' segments fall on distinct banks
    const int i0 = min(ylen, threadIdx.x * seg), i1 = min(ylen, i0 + seg);
    long long run = 0, mn = 0, mx = 0;
    for (int i = i0; i < i1; ++i) {
        const float v = ys[i];
        if (v > kSentinelTest) {
            run += (long long)(int)v;
            mn = min(mn, run);
            mx = max(mx, run);
        }
    }
    const long long before = block_exclusive_scan<NT>(run, scratch);
    long long gmn = mn + before, gmx = mx + before;
    block_minmax<NT>(gmn, gmx, scratch);
    const bool fast = (gmx - gmn) <= (1ll << 24);
    const int va = (int)max((int64_t)0, -o);                 // ys index of t = 0
    const int vb = (int)min((int64_t)ylen - 1, L - 1 - o);   // ys index of t = L - 1

    float B[M];
    int C[M];  // level 0: w0 of the first width chunk reaching B
    if (fast) {
        __syncthreads();
        float runf = (float)before;
        for (int i = i0; i < i1; ++i) {
            const float v = ys[i];
            ys[i] = i > vb + 1 ? -kBig : runf;
            if (v > kSentinelTest) runf += v;
        }
        __syncthreads();
        const float* P = ys;
        float base[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int q = H + M * threadIdx.x + i;
            base[i] = (q >= va && q <= vb) ? P[q] : kBig;
        }
        ThreadBound bnd{};
        bnd.active = false;
        boxcar_prefix(P + H, tab, d.wpad0, base, bnd, nullptr, B, C);
        // the levels' strided prefix sums: P_k[i] = P at t = (jk0 + i) 2^k
        for (int k = 1; k <= K; ++k) {
            const int64_t jk0 = (t0 - 1) >> k;
            float* Pk = reg + s_lvl[2 * k];
            const int n = dec_level_points(k) + W0;
            for (int i = threadIdx.x; i < n; i += NT) {
                const int64_t q = (jk0 + i) * ((int64_t)1 << k) - o;  // jk0 may be -1
                Pk[i] = q < ylen ? P[q] : -kBig;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            B[i] = boxcar_exact_slot(ys + H, tab, d.wpad0, i, nullptr);
            C[i] = 0;
        }
    }
    __syncthreads();

    // B_k at every grid point of the tile: the best of the level's widths
    int nitems = 0;
    for (int k = 1; k <= K; ++k) nitems += (int)((((t0 + kSpsTile - 2) >> k) - ((t0 - 1) >> k)) + 1);
    for (int it = threadIdx.x; it < nitems; it += NT) {
        int k = 1, jj = it;
        for (;;) {
            const int nk = (int)((((t0 + kSpsTile - 2) >> k) - ((t0 - 1) >> k)) + 1);
            if (jj < nk) break;
            jj -= nk;
            ++k;
        }
        const int64_t j = ((t0 - 1) >> k) + jj;
        const float2* tk = tab + d.wpad0 + (k - 1) * (W0 / 2);
        float best = -FLT_MAX;
        int bm = 0;
        if (j >= 0) {
            if (fast) {
                const float* Pk = reg + s_lvl[2 * k] + jj;
                const float p0 = Pk[0];
                for (int u = 0; u < W0 / 2; ++u) {
                    const float2 rc = tk[u];
                    const float snr = fmaf(Pk[W0 / 2 + 1 + u] - p0, rc.x, rc.y);
                    if (snr > best) { best = snr; bm = u; }
                }
            } else {
                // exact int64 running sums over the window's samples
                const int64_t q0 = (j << k) - o;
                const int step = 1 << k;
                long long S = 0;
                bool ok = true;
                for (int m = 1; m <= W0 && ok; ++m) {
                    for (int r = 0; r < step; ++r) {
                        const int64_t q = q0 + (int64_t)(m - 1) * step + r;
                        const float v = q < ylen ? ys[q] : kSentinel;
                        if (v < kSentinelTest) { ok = false; break; }  // past the series end
                        S += (long long)v;
                    }
                    if (ok && m > W0 / 2) {
                        const float2 rc = tk[m - W0 / 2 - 1];
                        const float snr = fmaf(__ll2float_rn(S), rc.x, rc.y);
                        if (snr > best) { best = snr; bm = m - W0 / 2 - 1; }
                    }
                }
            }
        }
        reg[s_lvl[2 * k + 1] + jj] = best;
        reinterpret_cast<uint8_t*>(reg + d.npk + d.nbk)[s_lvl[2 * k + 1] - d.npk + jj] = (uint8_t)bm;
    }
    __syncthreads();

    // B(t) = max over level 0 and every level's grid point at or before t
    int wdir[M];  // width of a level maximum (0: level 0)
#pragma unroll
    for (int i = 0; i < M; ++i) wdir[i] = 0;
    const int64_t tf = t0 - 1 + M * (int64_t)threadIdx.x;
    unsigned valid = 0;  // slots with t in [0, L): B is defined there only
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (tf + i >= 0 && tf + i < L) valid |= 1u << i;
    for (int k = 1; k <= K; ++k) {
        const int64_t jk0 = (t0 - 1) >> k;
        const float* Bk = reg + s_lvl[2 * k + 1];
        const uint8_t* Mk = reinterpret_cast<const uint8_t*>(reg + d.npk + d.nbk) + (s_lvl[2 * k + 1] - d.npk);
        int64_t jc = -(1ll << 62);
        float bv = -FLT_MAX;
        int wv = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int64_t j = (tf + i) >> k;
            if (j != jc) {
                jc = j;
                bv = Bk[j - jk0];
                wv = (W0 / 2 + 1 + Mk[j - jk0]) << k;
            }
            if (((valid >> i) & 1u) && bv > B[i]) {
                B[i] = bv;
                wdir[i] = wv;
            }
        }
    }
    if (a.evaluated && threadIdx.x == 0)
        atomicAdd(a.evaluated, (unsigned long long)NT * M * d.wpad0 + (unsigned long long)nitems * (W0 / 2));
    __syncthreads();  // everyone done with the level arrays

    float* Bs = reg;                                          // B(t) of every slot
    uint32_t* plist = reinterpret_cast<uint32_t*>(Bs + kSpsTile);  // slot | level-0 chunk << 16
    uint16_t* WS = reinterpret_cast<uint16_t*>(plist + kSpsTile);  // direct widths per slot
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Bs[M * threadIdx.x + i] = B[i];
        WS[M * threadIdx.x + i] = (uint16_t)wdir[i];
    }
    __syncthreads();

    const bool zero_sigma = st.zero_sigma != 0;
    unsigned cmask = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int p = M * threadIdx.x + i;
        const int64_t t = t0 - 1 + p;
        if (p >= 1 && p <= kSpsTile - 2 && t < L) {
            const float v = Bs[p];
            if (a.snr_out) a.snr_out[(int64_t)row * a.pitch + t] = zero_sigma ? 0.0f : v;
            if (!zero_sigma && v >= a.threshold && v > Bs[p - 1] && v >= Bs[p + 1]) cmask |= 1u << i;
        }
    }
    long long total = 0;
    const long long my_off = block_exclusive_scan_total<NT>(__popc(cmask), scratch, total);
    if (total == 0) return;
    const uint32_t dm_index = (uint32_t)(a.dm_offset + row);
    if (threadIdx.x == 0) {
        s_base = atomicAdd(a.count, (unsigned long long)total);
        const unsigned long long ci = atomicAdd(a.nchunks, 1ull);
        if (ci < (unsigned long long)a.chunk_cap)
            a.chunks[ci] = CandChunk{s_base, (uint32_t)total, dm_index, (uint32_t)t0, (uint32_t)a.beam};
    }
    {
        int j = (int)my_off;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if ((cmask >> i) & 1u)
                plist[j++] = (uint32_t)(M * threadIdx.x + i) | ((uint32_t)(C[i] / M) << 16);
    }
    __syncthreads();

    // widths: direct for a level maximum; for level 0 the smallest w reaching
    // B(t) within its first chunk, as in the exhaustive search
    for (int q = warp; q < (int)total; q += NT / 32) {
        const int p = (int)(plist[q] & 0xffffu);
        const int cw0 = (int)(plist[q] >> 16) * M;
        const int64_t t = t0 - 1 + p;
        const float target = Bs[p];
        float best = -FLT_MAX;
        int bw = 0x7fffffff;
        if (WS[p] != 0) {
            best = target;
            bw = WS[p];
        } else {
            const int wmax = (int)min((int64_t)d.W0e, L - t);
            if (fast) {
                const float* P = ys + H;
                const float b0 = P[p];
                for (int w0 = cw0; w0 < wmax; w0 += 32) {
                    const int w = w0 + lane + 1;
                    if (w <= wmax) {
                        const float2 rc = __ldg(gtab + w - 1);
                        const float snr = fmaf(P[p + w] - b0, rc.x, rc.y);
                        if (snr > best) { best = snr; bw = w; }
                    }
                    if (__any_sync(0xffffffffu, best == target)) break;
                }
            } else {
                const float* yq = ys + H + p;
                long long base = 0;
                for (int w0 = 0; w0 < wmax; w0 += 32) {
                    const int w = w0 + lane + 1;
                    long long v = (w <= wmax) ? (long long)yq[w - 1] : 0;
#pragma unroll
                    for (int s = 1; s < 32; s <<= 1) {
                        const long long u = __shfl_up_sync(0xffffffffu, v, s);
                        if (lane >= s) v += u;
                    }
                    const long long S = base + v;
                    base += __shfl_sync(0xffffffffu, v, 31);
                    if (w <= wmax) {
                        const float2 rc = __ldg(gtab + w - 1);
                        const float snr = fmaf(__ll2float_rn(S), rc.x, rc.y);
                        if (snr > best) { best = snr; bw = w; }
                    }
                    if (__any_sync(0xffffffffu, best == target)) break;
                }
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, s);
                const int ow = __shfl_xor_sync(0xffffffffu, bw, s);
                if (ob > best || (ob == best && ow < bw)) { best = ob; bw = ow; }
            }
        }
        const unsigned long long idx = s_base + (unsigned long long)q;
        if (lane == 0 && idx < (unsigned long long)a.capacity) {
            aa_candidate c;
            c.dm_index = dm_index;
            c.t = (uint32_t)t;
            c.width = (uint16_t)bw;
            c.range = (uint8_t)a.range;
            c.reserved = (uint8_t)a.beam;
            c.snr = best;
            a.cands[idx] = c;
        }
    }
}

__global__ void __launch_bounds__(NT, 2) sps_boxcar_dec_kernel(SpsArgs a, int ntiles) {
    extern __shared__ __align__(16) float sm[];
    boxcar_dec_block(a, ntiles, blockIdx.x, sm);
}

__device__ __forceinline__ int find_desc(const int64_t* first, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent forms over several beams/ranges (work queues).
__global__ void __launch_bounds__(kStatsThreads) sps_stats_batch_kernel(
    const SpsArgs* __restrict__ descs, const int64_t* __restrict__ first, int ndesc,
    unsigned long long* queue) {
    __shared__ long long s_item;
    const int64_t total = first[ndesc];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int k = find_desc(first, ndesc, item);
        stats_row(descs[k], descs[k].rsqrt_w, (int)(item - first[k]));
    }
}

__global__ void __launch_bounds__(NT, 2) sps_boxcar_batch_kernel(
    const SpsArgs* __restrict__ descs, const int64_t* __restrict__ first,
    const int* __restrict__ ntiles, int ndesc, unsigned long long* queue) {
    extern __shared__ __align__(16) float sm[];
    __shared__ long long s_item;
    const int64_t total = first[ndesc];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int k = find_desc(first, ndesc, item);
        const int64_t bid = item - first[k];
        if (descs[k].dec_w0 > 0) {
            boxcar_dec_block(descs[k], ntiles[k], bid, sm);
        } else {
            const int row = (int)(bid / ntiles[k]);
            const int64_t tile = bid - (int64_t)row * ntiles[k];
            boxcar_block(descs[k], row, tile, tile + 1, sm);
        }
    }
}

}  // namespace

cudaError_t launch_sps_stats(const SpsArgs& a, cudaStream_t s) {
    if (a.nrows <= 0) return cudaSuccess;
    sps_stats_kernel<<<a.nrows, kStatsThreads, 0, s>>>(a, a.rsqrt_w);
    return cudaGetLastError();
}

cudaError_t launch_sps_finalize(const SpsArgs& a, const unsigned long long* acc, cudaStream_t s) {
    if (a.nrows <= 0) return cudaSuccess;
    sps_finalize_kernel<<<a.nrows, 256, 0, s>>>(a, a.rsqrt_w, acc);
    return cudaGetLastError();
}

namespace {
// One CTA per run; 16-byte records copied as uint4.
__global__ void __launch_bounds__(256) gather_runs_kernel(const uint4* __restrict__ in,
                                                          uint4* __restrict__ out,
                                                          const RunCopy* __restrict__ runs,
                                                          int64_t nruns) {
    for (int64_t r = blockIdx.x; r < nruns; r += gridDim.x) {
        const RunCopy rc = runs[r];
        for (int64_t k = threadIdx.x; k < rc.n; k += blockDim.x) out[rc.dst + k] = in[rc.src + k];
    }
}
}  // namespace

cudaError_t launch_gather_runs(const aa_candidate* d_in, aa_candidate* d_out, const RunCopy* d_runs,
                               int64_t nruns, cudaStream_t s) {
    if (nruns <= 0) return cudaSuccess;
    static_assert(sizeof(aa_candidate) == sizeof(uint4), "candidate records are 16 bytes");
    const unsigned grid = (unsigned)std::min<int64_t>(nruns, 152 * 16);
    gather_runs_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint4*>(d_in),
                                            reinterpret_cast<uint4*>(d_out), d_runs, nruns);
    return cudaGetLastError();
}

cudaError_t launch_rsqrt_table(double* t, int wpad, cudaStream_t s) {
    rsqrt_table_kernel<<<(wpad + 255) / 256, 256, 0, s>>>(t, wpad);
    return cudaGetLastError();
}

size_t sps_boxcar_smem(int wpad) {
    const int ylen = kSpsTile + wpad + M;
    return (size_t)((ylen + 3) & ~3) * 4 + (size_t)sps_region_bytes(wpad) +
           (size_t)((sps_q_count(wpad) + 3) & ~3) * 4 + (size_t)ladder_words(wpad) * 4;
}

int g_boxcar_seg_tiles = 0;

size_t sps_boxcar_smem_for(int32_t max_width, int32_t wpad, int32_t dec_w0) {
    return dec_w0 > 0 ? dec_layout(max_width, dec_w0).bytes : sps_boxcar_smem(wpad);
}

cudaError_t launch_sps_boxcar(const SpsArgs& a, cudaStream_t s) {
    if (a.nrows <= 0 || a.length <= 0) return cudaSuccess;
    const int64_t ntiles = (a.length + kSpsOwned - 1) / kSpsOwned;
    const int64_t nblocks = ntiles * a.nrows;
    if (nblocks >= (1ll << 31)) return cudaErrorInvalidConfiguration;
    const size_t smem = sps_boxcar_smem_for(a.max_width, a.wpad, a.dec_w0);
    if (smem > kMaxBoxcarSmem) return cudaErrorInvalidConfiguration;
    if (a.dec_w0 > 0) {
        cudaError_t e = cudaFuncSetAttribute(sps_boxcar_dec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        sps_boxcar_dec_kernel<<<(unsigned)nblocks, NT, smem, s>>>(a, (int)ntiles);
        return cudaGetLastError();
    }
    // tiles per CTA: up to 16 (sharing the staged halo), keeping at least
    // 16 CTAs per resident CTA slot (2 per SM)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    const int seg = g_boxcar_seg_tiles > 0
                        ? (int)std::min<int64_t>(g_boxcar_seg_tiles, ntiles)
                        : (int)std::max<int64_t>(1, std::min<int64_t>({16, ntiles, nblocks / (sms * 2 * 16)}));
    const int64_t ncta = (int64_t)a.nrows * ((ntiles + seg - 1) / seg);
    cudaError_t e = cudaFuncSetAttribute(sps_boxcar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sps_boxcar_kernel<<<(unsigned)ncta, NT, smem, s>>>(a, (int)ntiles, seg);
    return cudaGetLastError();
}


}  // namespace aa

namespace aa {

cudaError_t launch_sps_stats_batch(const SpsArgs* d_descs, const int64_t* d_first, int ndesc,
                                   unsigned long long* d_queue, int grid, cudaStream_t s) {
    if (ndesc <= 0) return cudaSuccess;
    sps_stats_batch_kernel<<<grid, kStatsThreads, 0, s>>>(d_descs, d_first, ndesc, d_queue);
    return cudaGetLastError();
}

cudaError_t launch_sps_boxcar_batch(const SpsArgs* d_descs, const int64_t* d_first,
                                    const int* d_ntiles, int ndesc, size_t smem,
                                    unsigned long long* d_queue, int grid, cudaStream_t s) {
    if (ndesc <= 0) return cudaSuccess;
    if (smem > kMaxBoxcarSmem) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(sps_boxcar_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sps_boxcar_batch_kernel<<<grid, NT, smem, s>>>(d_descs, d_first, d_ntiles, ndesc, d_queue);
    return cudaGetLastError();
}

int sps_boxcar_tiles(int64_t length) { return (int)((length + kSpsOwned - 1) / kSpsOwned); }

}  // namespace aa

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
//   width   : for each candidate, the smallest maximising width (same
//             arithmetic as the boxcar kernel, bit for bit).
#include <cfloat>
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

__global__ void __launch_bounds__(kStatsThreads) sps_stats_kernel(SpsArgs a, const double* rsw) {
    __shared__ long long s1w[kStatsThreads / 32];
    __shared__ unsigned long long hiw[kStatsThreads / 32], low[kStatsThreads / 32];
    __shared__ double sh_f, sh_inv;
    const int row = blockIdx.x;
    const float* y = a.dd + (int64_t)row * a.pitch;
    const int64_t n = a.length;
    long long s1 = 0;
    unsigned long long hi = 0, lo = 0;
    for (int64_t i = threadIdx.x; i < n; i += kStatsThreads) {
        const long long v = (long long)y[i];
        s1 += v;
        add128(hi, lo, 0ull, (unsigned long long)(v * v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        add128(hi, lo, h2, l2);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s1w[warp] = s1;
        hiw[warp] = hi;
        low[warp] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long S1 = 0;
        unsigned long long H = 0, Lo = 0;
        for (int w = 0; w < kStatsThreads / 32; ++w) {
            S1 += s1w[w];
            add128(H, Lo, hiw[w], low[w]);
        }
        RowStats st{};
        if (n > 0) {
            // N^2 var = N * sum y^2 - (sum y)^2, exact in 128 bits
            const unsigned __int128 S2 = ((unsigned __int128)H << 64) | Lo;
            const __int128 num = (__int128)n * (__int128)S2 - (__int128)S1 * (__int128)S1;
            const unsigned __int128 un = num > 0 ? (unsigned __int128)num : 0;
            const double numd = (double)(unsigned long long)(un >> 64) * 18446744073709551616.0 +
                                (double)(unsigned long long)un;
            st.mu = (double)S1 / (double)n;
            st.sigma = sqrt(numd) / (double)n;
            const long long m0 = llround(st.mu);
            st.m0 = (float)m0;
            st.inv_sigma = st.sigma > 0 ? 1.0 / st.sigma : 0.0;
            st.zero_sigma = st.sigma > 0 ? 0 : 1;
            sh_f = (double)(S1 - m0 * (long long)n) / (double)n;  // mu - m0
        } else {
            st.zero_sigma = 1;
            sh_f = 0.0;
        }
        sh_inv = st.inv_sigma;
        a.stats[row] = st;
    }
    __syncthreads();
    const double f = sh_f, inv = sh_inv;
    float2* tab = a.table + (int64_t)row * a.wpad;
    for (int i = threadIdx.x; i < a.wpad; i += kStatsThreads) {
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

// ys: staged series minus m0 (sentinel outside [0, L)), index i <-> t0-1+i.
// Thread owns slots p = M*tid + i.  Running sums in FP32, exact because the
// caller checked that every partial sum of the tile is an integer of
// magnitude <= 2^24.  Slot i at width w = w0+s+1 adds ys[M*tid + i + w0 + s].
__device__ __forceinline__ void boxcar_fast(const float* __restrict__ ys,
                                            const float2* __restrict__ tab, int wpad,
                                            float (&B)[M]) {
    const float* yb = ys + M * threadIdx.x;
    float win[2 * M];
#pragma unroll
    for (int k = 0; k < M; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(yb + k);
        win[k] = v.x; win[k + 1] = v.y; win[k + 2] = v.z; win[k + 3] = v.w;
    }
    float S[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        S[i] = 0.0f;
        B[i] = -FLT_MAX;
    }
    for (int w0 = 0; w0 < wpad; w0 += M) {
#pragma unroll
        for (int k = 0; k < M; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(yb + w0 + M + k);
            win[M + k] = v.x; win[M + k + 1] = v.y; win[M + k + 2] = v.z; win[M + k + 3] = v.w;
        }
#pragma unroll
        for (int s = 0; s < M; s += 2) {
            const float2 rc0 = tab[w0 + s];
            const float2 rc1 = tab[w0 + s + 1];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                S[i] += win[i + s];
                const float v0 = fmaf(S[i], rc0.x, rc0.y);
                S[i] += win[i + s + 1];
                const float v1 = fmaf(S[i], rc1.x, rc1.y);
                B[i] = max3f(B[i], v0, v1);
            }
        }
#pragma unroll
        for (int k = 0; k < M; ++k) win[k] = win[M + k];
    }
}

// Exact int64 running sums for slot i, for tiles whose partial sums may
// exceed 2^24.  Same SNR arithmetic as boxcar_fast (fmaf of the correctly
// rounded sum).
__device__ __noinline__ float boxcar_exact_slot(const float* __restrict__ ys,
                                                const float2* __restrict__ tab, int wpad, int i) {
    const float* yb = ys + M * threadIdx.x + i;
    long long S = 0;
    float best = -FLT_MAX;
    for (int w = 1; w <= wpad; ++w) {
        const float v = yb[w - 1];
        if (v < kSentinelTest) break;  // window left [0, L): later widths invalid too
        S += (long long)v;
        const float2 rc = tab[w - 1];
        best = fmaxf(best, fmaf(__ll2float_rn(S), rc.x, rc.y));
    }
    return best;
}

__global__ void __launch_bounds__(NT, 2) sps_boxcar_kernel(SpsArgs a, int ntiles) {
    extern __shared__ __align__(16) float sm[];
    __shared__ long long scratch[2 * NT / 32];
    const int wpad = a.wpad;
    const int ylen = kSpsTile + wpad + M;
    float* ys = sm;
    float2* tab = reinterpret_cast<float2*>(sm + ((ylen + 3) & ~3));
    const int row = blockIdx.x / ntiles;
    const int64_t tile = blockIdx.x - (int64_t)row * ntiles;
    const int64_t t0 = tile * kSpsOwned;
    const int64_t L = a.length;
    const float* y = a.dd + (int64_t)row * a.pitch;
    const RowStats st = a.stats[row];
    const float m0 = st.m0;

    for (int i = threadIdx.x; i < ylen; i += NT) {
        const int64_t t = t0 - 1 + i;
        ys[i] = (t >= 0 && t < L) ? __ldg(y + t) - m0 : kSentinel;
    }
    const float2* gtab = a.table + (int64_t)row * wpad;
    for (int i = threadIdx.x; i < wpad; i += NT) tab[i] = __ldg(gtab + i);
    __syncthreads();

    // Largest |partial sum| of the tile = range of the prefix sums of ys over
    // its valid samples: FP32 running sums are exact when it is <= 2^24.
    const int seg = (ylen + NT - 1) / NT;
    const int i0 = min(ylen, threadIdx.x * seg), i1 = min(ylen, i0 + seg);
    long long run = 0, mn = 0, mx = 0;
    for (int i = i0; i < i1; ++i) {
        const float v = ys[i];
        if (v > kSentinelTest) {
            run += (long long)v;
            mn = min(mn, run);
            mx = max(mx, run);
        }
    }
    const long long before = block_exclusive_scan<NT>(run, scratch);
    mn += before;
    mx += before;
    block_minmax<NT>(mn, mx, scratch);
    const bool fast = (mx - mn) <= (1ll << 24);

    float B[M];
    if (fast) {
        boxcar_fast(ys, tab, wpad, B);
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) B[i] = boxcar_exact_slot(ys, tab, wpad, i);
    }

    __syncthreads();  // everyone done with ys / tab
    float* Bs = sm;   // reuse
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
    // One atomic per CTA: the CTA's candidates form one contiguous run in t order.
    long long total = 0;
    const long long my_off = block_exclusive_scan_total<NT>(__popc(cmask), scratch, total);
    if (total > 0) {
        __shared__ unsigned long long s_base;
        const uint32_t dm_index = (uint32_t)(a.dm_offset + row);
        if (threadIdx.x == 0) {
            s_base = atomicAdd(a.count, (unsigned long long)total);
            const unsigned long long ci = atomicAdd(a.nchunks, 1ull);
            if (ci < (unsigned long long)a.chunk_cap)
                a.chunks[ci] = CandChunk{s_base, (uint32_t)total, dm_index, (uint32_t)t0, 0u};
        }
        __syncthreads();
        unsigned long long idx = s_base + (unsigned long long)my_off;
        while (cmask) {
            const int i = __ffs(cmask) - 1;
            cmask &= cmask - 1;
            if (idx < (unsigned long long)a.capacity) {
                const int p = M * threadIdx.x + i;
                aa_candidate c;
                c.dm_index = dm_index;
                c.t = (uint32_t)(t0 - 1 + p);
                c.width = 0;
                c.range = (uint8_t)a.range;
                c.reserved = 0;
                c.snr = Bs[p];
                a.cands[idx] = c;
            }
            ++idx;
        }
    }
}

// One warp per candidate of this range: recompute SNR_w for w = 1..min(W, L-t)
// with the boxcar kernel's arithmetic and keep the smallest maximising w.
__global__ void __launch_bounds__(256) sps_width_kernel(SpsArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nstored = min((long long)*a.count, (long long)a.capacity);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ci = wid; ci < nstored; ci += nw) {
        aa_candidate c = a.cands[ci];
        if (c.range != (uint8_t)a.range) continue;
        const int row = (int)c.dm_index - a.dm_offset;
        const int64_t t = c.t;
        const float* y = a.dd + (int64_t)row * a.pitch;
        const float2* tab = a.table + (int64_t)row * a.wpad;
        const long long m0 = (long long)a.stats[row].m0;
        const int wmax = (int)min((int64_t)a.max_width, a.length - t);
        const int seg = (wmax + 31) / 32;
        const int w_lo = lane * seg + 1, w_hi = min(wmax, (lane + 1) * seg);
        long long part = 0;
        for (int w = w_lo; w <= w_hi; ++w) part += (long long)y[t + w - 1] - m0;
        long long inc = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        long long S = inc - part;
        float best = -FLT_MAX;
        int bw = 0x7fffffff;
        for (int w = w_lo; w <= w_hi; ++w) {
            S += (long long)y[t + w - 1] - m0;
            const float2 rc = tab[w - 1];
            const float v = fmaf(__ll2float_rn(S), rc.x, rc.y);
            if (v > best) { best = v; bw = w; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
            if (ob > best || (ob == best && ow < bw)) { best = ob; bw = ow; }
        }
        if (lane == 0) {
            c.width = (uint16_t)bw;
            c.snr = best;
            a.cands[ci] = c;
        }
    }
}

}  // namespace

cudaError_t launch_sps_stats(const SpsArgs& a, cudaStream_t s) {
    if (a.nrows <= 0) return cudaSuccess;
    sps_stats_kernel<<<a.nrows, kStatsThreads, 0, s>>>(a, a.rsqrt_w);
    return cudaGetLastError();
}

cudaError_t launch_rsqrt_table(double* t, int wpad, cudaStream_t s) {
    rsqrt_table_kernel<<<(wpad + 255) / 256, 256, 0, s>>>(t, wpad);
    return cudaGetLastError();
}

size_t sps_boxcar_smem(int wpad) {
    const int ylen = kSpsTile + wpad + M;
    return (size_t)((ylen + 3) & ~3) * 4 + (size_t)wpad * 8;
}

cudaError_t launch_sps_boxcar(const SpsArgs& a, cudaStream_t s) {
    if (a.nrows <= 0 || a.length <= 0) return cudaSuccess;
    const int64_t ntiles = (a.length + kSpsOwned - 1) / kSpsOwned;
    const int64_t nblocks = ntiles * a.nrows;
    if (nblocks >= (1ll << 31)) return cudaErrorInvalidConfiguration;
    const size_t smem = sps_boxcar_smem(a.wpad);
    cudaError_t e = cudaFuncSetAttribute(sps_boxcar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sps_boxcar_kernel<<<(unsigned)nblocks, NT, smem, s>>>(a, (int)ntiles);
    return cudaGetLastError();
}

cudaError_t launch_sps_width(const SpsArgs& a, cudaStream_t s) {
    if (a.nrows <= 0 || a.length <= 0 || a.capacity <= 0) return cudaSuccess;
    sps_width_kernel<<<152 * 4, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace aa

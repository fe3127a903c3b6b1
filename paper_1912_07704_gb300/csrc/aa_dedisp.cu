// Time decimation and brute-force dedispersion kernels for sm_103a.
//
// Dedispersion (arXiv:1912.07704 Sec. 1, dedispersion module): for every DM
// trial i of a range, y[i][t] = sum_c x[c][t + s(c,i)], exact integers.
//
// Tile: one CTA = 16 DM trials x 512 output samples.  Channels stream through
// shared memory in stages of `cc` channel rows, each row fetched with one
// bulk-async (TMA) copy tracked by an mbarrier; the row holds the samples
// [t0 + s(c,first DM) .. t0 + 512 + s(c,last DM)] rounded out to 16 bytes, so
// every DM of the block reads from the same staged row.  Because per-channel
// delays are arbitrary, the row is also stored shifted by 1..spw-1 samples so
// that every (channel, DM) read is a 32-bit aligned word.  Each lane sums
// 4 words (uint8: 16 samples) per DM in packed 16-bit lanes (two samples per
// 32-bit add), flushing into 32-bit totals before a lane can overflow.
#include <cstdint>

#include <algorithm>

#include "aa_internal.h"

namespace aa {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for a phase with a wall-clock limit; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t start = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - start > limit_ns) return false;
    return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per stage: far beyond any real copy
constexpr int kMaxStages = 4;                      // staging ring depth limit (mbarriers per CTA)

// SPW = samples per 32-bit word: 4 for raw uint8 input, 2 for decimated uint16.
// acc + x through the FMA pipe (integer multiply-add by a runtime 1): the byte
// split already occupies the ALU pipe.
__device__ __forceinline__ uint32_t mad_add(uint32_t x, uint32_t one, uint32_t acc) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(acc));
    return d;
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Fused statistics of the single-pulse search: the warp's exact sums of one
// output row's samples (s1 = sum y, s2 = sum y^2 per lane; y < 2^24, at most
// 16 samples a lane, so every partial fits in 64 bits) are added to the row's
// accumulators acc = (sum y, sum y^2 low, sum y^2 high); a wrap of the low
// word is carried into the high one, so the 128-bit total is exact.
__device__ __forceinline__ void add_row_sums(unsigned long long* acc, unsigned long long s1,
                                             unsigned long long s2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], s1);
        const unsigned long long old = atomicAdd(&acc[1], s2);
        if (old + s2 < old) atomicAdd(&acc[2], 1ull);
    }
}

// One CTA's work item: DM block (bid % ndm_blocks) x time tile (bid / ndm_blocks).
// `smem` is the dynamic shared memory (layout below); the caller guarantees
// that every thread of the CTA has finished any previous item.
template <int SPW>
__device__ __forceinline__ void dedisperse_block(const DedispArgs& a, int ndm_blocks, int64_t bid,
                                                 uint64_t wait_limit_ns, int fault_skip_chunk,
                                                 uint32_t one, unsigned char* smem, uint64_t* bars,
                                                 bool reinit) {
    constexpr int QW = kTau / (32 * SPW);  // words per lane per DM trial
    constexpr int NCOPY = SPW;             // shifted copies of each staged row
    constexpr int EB = 4 / SPW;            // bytes per sample
    constexpr int A16 = 16 / EB;           // samples per 16-byte unit
    constexpr int SWAR = SPW / 2;          // packed accumulators per word

    const int cc = a.cc, nstage = a.nstage, rw = a.rw;
    const size_t stage_w = (size_t)cc * NCOPY * rw;
    uint32_t* stages = reinterpret_cast<uint32_t*>(smem);
    int* offs = reinterpret_cast<int*>(stages + nstage * stage_w);  // [nstage][16][cc]
    int* bases = offs + nstage * kDmPerBlock * cc;                   // [nstage][cc]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dmb = (int)(bid % ndm_blocks);
    const int64_t tile = bid / ndm_blocks;
    const int d0 = dmb * kDmPerBlock;
    const int dlast = min(a.ndm, d0 + kDmPerBlock) - 1;
    const int64_t t0 = tile * kTau;
    const int C = a.nchans;
    const int nchunks = (C + cc - 1) / cc;
    const unsigned char* in_b = static_cast<const unsigned char*>(a.in);
    const int64_t pitch_b = a.in_pitch * EB;

    if (tid == 0) {  // every barrier of the fixed array, whatever the previous item used
        for (int st = 0; st < kMaxStages; ++st) {
            if (reinit) mbar_inval(&bars[st]);
            mbar_init(&bars[st], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();

    // Producer (warp 0): stage chunk k (channels k*cc ..) into stage k % nstage.
    // Lane l < cc handles channel k*cc + l; its first/last-trial delays (lo,
    // hi) are loaded one stage ahead so the global-load latency stays hidden.
    auto load_lohi = [&](int k, int& lo, int& hi) {
        const int c = k * cc + lane;
        if (k < nchunks && lane < cc && c < C) {
            lo = __ldg(&a.shifts[(int64_t)d0 * C + c]);
            hi = __ldg(&a.shifts[(int64_t)dlast * C + c]);
        } else {
            lo = hi = 0;
        }
    };
    auto issue = [&](int k, int s_lo, int s_hi) {
        const int s = k % nstage;
        const int c0 = k * cc;
        uint32_t bytes = 0;
        int64_t src_off = 0;
        if (lane < cc && c0 + lane < C) {
            const int c = c0 + lane;
            const int64_t base = ((t0 + s_lo) / A16) * A16;
            const int64_t end = t0 + kTau + s_hi + SPW;
            int64_t nb = ((end - base) * EB + 15) / 16 * 16;
            nb = min(nb, (int64_t)rw * 4);
            nb = min(nb, pitch_b - base * EB);
            bytes = nb > 0 ? (uint32_t)nb : 0u;
            src_off = (int64_t)c * pitch_b + base * EB;
            bases[s * cc + lane] = (int)(base - t0);
        }
        uint32_t total = bytes;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (k == fault_skip_chunk) return;  // fault injection: this stage never completes
        if (lane == 0) mbar_arrive_expect_tx(&bars[s], total);
        __syncwarp();
        if (bytes)
            bulk_copy_g2s(stages + s * stage_w + (size_t)lane * NCOPY * rw, in_b + src_off, bytes,
                          &bars[s]);
    };

    int pre_lo = 0, pre_hi = 0;  // delays of the next chunk to issue (warp 0)
    if (warp == 0) {
        for (int k = 0; k < min(nstage - 1, nchunks); ++k) {
            int lo, hi;
            load_lohi(k, lo, hi);
            issue(k, lo, hi);
        }
        load_lohi(nstage - 1, pre_lo, pre_hi);
    }
    int next_issue = min(nstage - 1, nchunks);
    // Each thread owns at most one (trial, channel) word offset per chunk;
    // its delay is prefetched one chunk ahead.
    const bool own = tid < kDmPerBlock * cc;
    const int own_dl = own ? tid / cc : 0, own_cl = own ? tid - (tid / cc) * cc : 0;
    const int64_t own_row = (int64_t)min(d0 + own_dl, dlast) * C;
    int sh_next = (own && own_cl < C) ? __ldg(&a.shifts[own_row + own_cl]) : 0;
    __syncthreads();  // bases[] of the first stages visible to all threads

    uint32_t acc[kDmPerWarp][QW][SWAR];
    uint32_t tot[kDmPerWarp][QW][SPW];
#pragma unroll
    for (int kk = 0; kk < kDmPerWarp; ++kk)
#pragma unroll
        for (int j = 0; j < QW; ++j) {
#pragma unroll
            for (int q = 0; q < SWAR; ++q) acc[kk][j][q] = 0;
#pragma unroll
            for (int q = 0; q < SPW; ++q) tot[kk][j][q] = 0;
        }

    auto flush = [&]() {
#pragma unroll
        for (int kk = 0; kk < kDmPerWarp; ++kk)
#pragma unroll
            for (int j = 0; j < QW; ++j) {
                if constexpr (SPW == 4) {
                    const uint32_t e = acc[kk][j][0], o = acc[kk][j][1];
                    tot[kk][j][0] += e & 0xffffu;
                    tot[kk][j][2] += e >> 16;
                    tot[kk][j][1] += o & 0xffffu;
                    tot[kk][j][3] += o >> 16;
                } else {
                    const uint32_t v = acc[kk][j][0];
                    tot[kk][j][0] += v & 0xffffu;
                    tot[kk][j][1] += v >> 16;
                }
#pragma unroll
                for (int q = 0; q < SWAR; ++q) acc[kk][j][q] = 0;
            }
    };

    int since_flush = 0;
    for (int k = 0; k < nchunks; ++k) {
        const int s = k % nstage;
        const uint32_t parity = (uint32_t)(k / nstage) & 1u;
        const int sh_cur = sh_next;
        if (own && k + 1 < nchunks && (k + 1) * cc + own_cl < C)
            sh_next = __ldg(&a.shifts[own_row + (k + 1) * cc + own_cl]);
        const bool ok = mbar_wait_bounded(&bars[s], parity, wait_limit_ns);
        uint32_t* st = stages + s * stage_w;
        const int c0 = k * cc;
        const int cvalid = min(cc, C - c0);
        if (ok) {
            // shifted copies 1..NCOPY-1 of every staged row
            if constexpr (NCOPY > 1) {
                // one warp per row, 4 words per lane (128-bit loads/stores)
                for (int cl = warp; cl < cvalid; cl += kDedispWarps) {
                    uint32_t* row = st + (size_t)cl * NCOPY * rw;
                    for (int j = 4 * lane; j < rw - 1; j += 128) {
                        const uint4 w = *reinterpret_cast<const uint4*>(row + j);
                        const uint32_t w4 = (j + 4 < rw) ? row[j + 4] : 0u;
#pragma unroll
                        for (int q = 1; q < NCOPY; ++q) {
                            const int sh = q * 8 * EB;
                            *reinterpret_cast<uint4*>(row + q * rw + j) =
                                make_uint4(__funnelshift_r(w.x, w.y, sh), __funnelshift_r(w.y, w.z, sh),
                                           __funnelshift_r(w.z, w.w, sh), __funnelshift_r(w.w, w4, sh));
                        }
                    }
                }
            }
            // word offset of every (DM, channel) of this chunk
            if (own && own_cl < cvalid) {
                const int o = sh_cur - bases[s * cc + own_cl];
                offs[(s * kDmPerBlock + own_dl) * cc + own_cl] =
                    (own_cl * NCOPY + o % SPW) * rw + o / SPW;
            }
        }
        if (!__syncthreads_and(ok)) {
            // A stage never arrived: report, drain the copies still in flight
            // (bounded), and leave without touching the output.
            if (tid == 0) atomicOr(a.err, 1u);
            for (int kk = k; kk < next_issue; ++kk)
                mbar_wait_bounded(&bars[kk % nstage], (uint32_t)(kk / nstage) & 1u, wait_limit_ns);
            return;
        }
        if (next_issue < nchunks) {
            if (warp == 0) {
                issue(next_issue, pre_lo, pre_hi);
                load_lohi(next_issue + 1, pre_lo, pre_hi);
            }
            ++next_issue;
        }

        // accumulate: each warp owns kDmPerWarp trials of the block
#pragma unroll
        for (int kk = 0; kk < kDmPerWarp; ++kk) {
            const int* o = offs + (s * kDmPerBlock + warp * kDmPerWarp + kk) * cc;
            int cl = 0;
            for (; cl + 1 < cvalid; cl += 2) {
                const uint32_t* p0 = st + o[cl] + lane;
                const uint32_t* p1 = st + o[cl + 1] + lane;
#pragma unroll
                for (int j = 0; j < QW; ++j) {
                    const uint32_t v0 = p0[32 * j], v1 = p1[32 * j];
                    if constexpr (SPW == 4) {
                        acc[kk][j][0] = mad_add(v0 & 0x00ff00ffu, one, acc[kk][j][0]);
                        acc[kk][j][0] = mad_add(v1 & 0x00ff00ffu, one, acc[kk][j][0]);
                        acc[kk][j][1] = mad_add(__byte_perm(v0, 0u, 0x4341), one, acc[kk][j][1]);
                        acc[kk][j][1] = mad_add(__byte_perm(v1, 0u, 0x4341), one, acc[kk][j][1]);
                    } else {
                        acc[kk][j][0] = mad_add(v0, one, acc[kk][j][0]);
                        acc[kk][j][0] = mad_add(v1, one, acc[kk][j][0]);
                    }
                }
            }
            if (cl < cvalid) {
                const uint32_t* p0 = st + o[cl] + lane;
#pragma unroll
                for (int j = 0; j < QW; ++j) {
                    const uint32_t v0 = p0[32 * j];
                    if constexpr (SPW == 4) {
                        acc[kk][j][0] = mad_add(v0 & 0x00ff00ffu, one, acc[kk][j][0]);
                        acc[kk][j][1] = mad_add(__byte_perm(v0, 0u, 0x4341), one, acc[kk][j][1]);
                    } else {
                        acc[kk][j][0] = mad_add(v0, one, acc[kk][j][0]);
                    }
                }
            }
        }
        since_flush += cc;
        if (since_flush >= a.flush) {
            flush();
            since_flush = 0;
        }
    }
    flush();

    // epilogue: exact integer totals -> FP32 rows (or 16-bit rows: the
    // sub-band partial sums, which the caller keeps below 2^16)
#pragma unroll
    for (int kk = 0; kk < kDmPerWarp; ++kk) {
        const int d = d0 + warp * kDmPerWarp + kk;
        if (d >= a.ndm) continue;
        if (a.out16) {
            uint16_t* row = a.out16 + (int64_t)d * a.out_pitch;
#pragma unroll
            for (int j = 0; j < QW; ++j) {
                const int64_t t = t0 + (int64_t)SPW * (lane + 32 * j);
                if (t + SPW <= a.length) {
                    if constexpr (SPW == 4) {
                        *reinterpret_cast<uint2*>(row + t) =
                            make_uint2(tot[kk][j][0] | (tot[kk][j][1] << 16), tot[kk][j][2] | (tot[kk][j][3] << 16));
                    } else {
                        *reinterpret_cast<uint32_t*>(row + t) = tot[kk][j][0] | (tot[kk][j][1] << 16);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < SPW; ++q)
                        if (t + q < a.length) row[t + q] = (uint16_t)tot[kk][j][q];
                }
            }
            continue;
        }
        float* row = a.out + (int64_t)d * a.out_pitch;
        if (a.st_acc) {
            unsigned long long s1 = 0, s2 = 0;
#pragma unroll
            for (int j = 0; j < QW; ++j)
#pragma unroll
                for (int q = 0; q < SPW; ++q)
                    if (t0 + (int64_t)SPW * (lane + 32 * j) + q < a.length) {
                        const unsigned long long v = tot[kk][j][q];
                        s1 += v;
                        s2 += v * v;
                    }
            add_row_sums(a.st_acc + 3 * (int64_t)d, s1, s2);
        }
#pragma unroll
        for (int j = 0; j < QW; ++j) {
            const int64_t t = t0 + (int64_t)SPW * (lane + 32 * j);
            if (t + SPW <= a.length) {
                if constexpr (SPW == 4) {
                    *reinterpret_cast<float4*>(row + t) =
                        make_float4((float)tot[kk][j][0], (float)tot[kk][j][1],
                                    (float)tot[kk][j][2], (float)tot[kk][j][3]);
                } else {
                    *reinterpret_cast<float2*>(row + t) =
                        make_float2((float)tot[kk][j][0], (float)tot[kk][j][1]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < SPW; ++q)
                    if (t + q < a.length) row[t + q] = (float)tot[kk][j][q];
            }
        }
    }
}

// Five consecutive 32-bit words of a row, starting at the word holding byte
// bo.  vec: as two aligned 16-byte loads, the five words picked by the word
// offset of bo within its 16-byte block (the same for every lane of the warp,
// so the branch does not diverge); the caller guarantees that the 32 bytes
// from bo rounded down to 16 lie inside the buffer.  Otherwise five word
// loads clamped to the row's last word wl (measured faster than unclamped
// word loads, and than 16-byte loads for 16-bit rows).
__device__ __forceinline__ void load_words5(const unsigned char* row, int64_t bo, bool vec, int wl,
                                            uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3,
                                            uint32_t& w4) {
    if (vec) {
        const uint4* q = reinterpret_cast<const uint4*>(row + (bo & ~(int64_t)15));
        const uint4 q0 = __ldg(q), q1 = __ldg(q + 1);
        switch ((int)(bo >> 2) & 3) {
            case 0: w0 = q0.x; w1 = q0.y; w2 = q0.z; w3 = q0.w; w4 = q1.x; break;
            case 1: w0 = q0.y; w1 = q0.z; w2 = q0.w; w3 = q1.x; w4 = q1.y; break;
            case 2: w0 = q0.z; w1 = q0.w; w2 = q1.x; w3 = q1.y; w4 = q1.z; break;
            default: w0 = q0.w; w1 = q1.x; w2 = q1.y; w3 = q1.z; w4 = q1.w; break;
        }
    } else {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(row);
        const int wi = (int)(bo >> 2);
        w0 = __ldg(w + min(wi, wl));
        w1 = __ldg(w + min(wi + 1, wl));
        w2 = __ldg(w + min(wi + 2, wl));
        w3 = __ldg(w + min(wi + 3, wl));
        w4 = __ldg(w + min(wi + 4, wl));
    }
}

// Grouped strategy (see GroupRec in aa_internal.h).  CTA = 16 DM trials x
// kGroupTau output samples.  The channels stream through in chunks of a.cc;
// the groups of a chunk are processed in batches of at most a.gz:
//   phase 1: z_g[u] = sum over the group's members of x[c][t0 + s0_c + u],
//            u < kGroupTau + span_g, read straight from global memory (each
//            member row is read by one warp, coalesced 32-bit words; the rows
//            of a chunk are shared by the CTAs of all DM blocks through L2),
//            as packed 16-bit pairs stored twice: copy A word j =
//            (z[2j], z[2j+1]) and copy B word j = (z[2j+1], z[2j+2]);
//            work unit = (group, 256 consecutive u), units round-robin over
//            the warps;
//   phase 2: warp w (trial d0 + w) adds z_g[t + delta_g(w)] for its 16
//            samples t: copy (delta & 1), word offset delta >> 1, aligned.
// 16-bit lanes never overflow: a group sum has at most 65535 / (255 dec)
// members, and a trial's accumulators are flushed into 32-bit totals every
// a.gflush chunks when a chunk fits the lanes, else (a.gflush = 0) before each
// group flagged by the plan (the members added since the last flush would
// otherwise pass 65535 / (255 dec)).
// `wait_limit_ns` and `fault_skip_chunk` are unused (no device-side waits).
template <int EB, bool FLAGS>
__device__ __forceinline__ void dedisperse_grouped_block(const DedispArgs& a, int ndm_blocks,
                                                         int64_t bid, unsigned char* smem) {
    constexpr int T = kGroupTau;
    constexpr int QW = T / 64;  // packed words (2 samples) per lane per trial
    const int gcc = a.cc, gz = a.gz, gzw = a.gzw, nj = a.gnj;
    uint32_t* zs = reinterpret_cast<uint32_t*>(smem);  // [gz][2][gzw]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dmb = (int)(bid % ndm_blocks);
    const int64_t tile = bid / ndm_blocks;
    const int d0 = dmb * kDmPerBlock;
    const int dlast = min(a.ndm, d0 + kDmPerBlock) - 1;
    const int64_t t0 = tile * T;
    const int C = a.nchans;
    const int nchunks = (C + gcc - 1) / gcc;
    const unsigned char* in_b = static_cast<const unsigned char*>(a.in);
    const int64_t pitch_b = a.in_pitch * EB;
    const GroupRec* recs = a.grec + (size_t)(a.dmb0 + dmb) * nchunks;
    const GroupMember* mems = a.gmem + (size_t)(a.dmb0 + dmb) * nchunks * gcc;
    // tail units: gtl lanes per group (a power of two), gpt groups per warp
    const int gtl = a.gtl, gtl_log = gtl ? __ffs(gtl) - 1 : 0, gpt = gtl ? 32 / gtl : 1;
    // A lane of a main unit reads below byte EB * (nsamp + 256 gnj) + 31 of its
    // row (tile start + member delay <= nsamp - 1), so with rows at least
    // EB * (256 gnj + 64) bytes long a read past a row's end stays inside the
    // next row: outside the chunk holding the buffer's last row, 8-bit main
    // units read their 17 bytes as two aligned 16-byte loads.
    const bool rows_long = pitch_b >= (int64_t)EB * (256 * nj + 64);

    uint32_t acc[QW];
    uint32_t tot[2 * QW];
#pragma unroll
    for (int q = 0; q < QW; ++q) {
        acc[q] = 0;
        tot[2 * q] = tot[2 * q + 1] = 0;
    }
    const bool has_trial = d0 + warp <= dlast;
    int since_flush = 0;

    for (int k = 0; k < nchunks; ++k) {
        const GroupRec rec = recs[k];
        const GroupDesc* gd = a.gdesc + rec.first;
        const GroupMember* mk = mems + (size_t)k * gcc;
        const unsigned char* chunk_in = in_b + (int64_t)(k * gcc) * pitch_b;
        const bool clamp = !(rows_long && (k + 1) * gcc < C);
        const int G = rec.ngroups;
        for (int gb = 0; gb < G; gb += gz) {
            const int ge = min(G, gb + gz);
            // group fields, one group per lane: members (start | count << 16),
            // span, and this warp's phase-2 word offset at its trial's delay
            uint32_t g_ms = 0, g_span = 0;
            int g_p2 = 0;
            if (gb + lane < ge) {
                const GroupDesc& g = gd[gb + lane];
                g_ms = (uint32_t)g.mstart | ((uint32_t)g.mcount << 16);
                g_span = g.span;
                const int dl = g.delta[warp];
                g_p2 = ((lane * 2 + (dl & 1)) * gzw + (dl >> 1)) | (g.flush ? (int)0x80000000u : 0);
            }
            // ---- phase 1: group sums of this batch.  With a.gtl > 0: two full
            // units per group (samples 0..511), then tail units that cover the
            // samples past 511 of 32 / gtl groups at once (gtl lanes each);
            // otherwise gnj full units per group.
            {
                const int ng = ge - gb;
                // 8-bit input with tail units: one unit per group covers samples
                // 0..511 at 16 per lane; otherwise two units of 8 per lane
                constexpr bool kWide = EB == 1;
                const int nmain = gtl ? (kWide ? ng : 2 * ng) : ng * nj;
                const int nunits = gtl ? nmain + (ng + gpt - 1) / gpt : nmain;
                for (int u = warp; u < nunits; u += kDedispWarps) {
                    int gi, idx;  // this lane's group and sample block (samples 8 idx .. 8 idx + 7,
                                  // or 16 idx .. 16 idx + 15 when wide)
                    bool wide = false;
                    if (gtl) {
                        if (u < nmain) {
                            if (kWide) {
                                gi = u;
                                idx = lane;
                                wide = true;
                            } else {
                                gi = u >> 1;
                                idx = 32 * (u & 1) + lane;
                            }
                        } else {
                            gi = (u - nmain) * gpt + (lane >> gtl_log);
                            idx = 64 + (lane & (gtl - 1));
                        }
                    } else {
                        gi = u / nj;
                        idx = 32 * (u - gi * nj) + lane;
                    }
                    // a main unit gives the whole warp one group: every lane's
                    // window starts at the same offset within 16 bytes
                    const bool vec = EB == 1 && !clamp && (!gtl || u < nmain);
                    const bool gvalid = gi < ng;
                    const int gs = gvalid ? gi : 0;
                    const uint32_t ms = __shfl_sync(0xffffffffu, g_ms, gs);
                    const int zlen = T + (int)__shfl_sync(0xffffffffu, g_span, gs);
                    const int mstart = (int)(ms & 0xffffu), mend = mstart + (int)(ms >> 16);
                    uint32_t* zA = zs + gs * 2 * gzw;
                    uint32_t* zB = zA + gzw;
                    const int wl = (int)(pitch_b >> 2) - 1;
                    if constexpr (kWide) {
                        if (wide) {
                            // 16 samples: five words per member (bytes b .. b + 16)
                            uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, A4 = 0, A5 = 0, A6 = 0, A7 = 0, E = 0;
                            if (gvalid) {
#pragma unroll 2
                                for (int m = mstart; m < mend; ++m) {
                                    const int2 rm = __ldg(reinterpret_cast<const int2*>(mk + m));
                                    const int64_t bo = t0 + rm.x + 16 * idx;
                                    const uint32_t sh = (uint32_t)(bo & 3) * 8u;
                                    uint32_t w0, w1, w2, w3, w4;
                                    load_words5(chunk_in + (int64_t)(rm.y & 0xffff) * pitch_b, bo, vec, wl,
                                                w0, w1, w2, w3, w4);
                                    const uint32_t v0 = __funnelshift_r(w0, w1, sh);
                                    const uint32_t v1 = __funnelshift_r(w1, w2, sh);
                                    const uint32_t v2 = __funnelshift_r(w2, w3, sh);
                                    const uint32_t v3 = __funnelshift_r(w3, w4, sh);
                                    A0 += __byte_perm(v0, 0u, 0x4140);
                                    A1 += __byte_perm(v0, 0u, 0x4342);
                                    A2 += __byte_perm(v1, 0u, 0x4140);
                                    A3 += __byte_perm(v1, 0u, 0x4342);
                                    A4 += __byte_perm(v2, 0u, 0x4140);
                                    A5 += __byte_perm(v2, 0u, 0x4342);
                                    A6 += __byte_perm(v3, 0u, 0x4140);
                                    A7 += __byte_perm(v3, 0u, 0x4342);
                                    E += (w4 >> sh) & 0xffu;
                                }
                                uint4* a4 = reinterpret_cast<uint4*>(zA + 8 * idx);
                                uint4* b4 = reinterpret_cast<uint4*>(zB + 8 * idx);
                                a4[0] = make_uint4(A0, A1, A2, A3);
                                a4[1] = make_uint4(A4, A5, A6, A7);
                                b4[0] = make_uint4(__byte_perm(A0, A1, 0x5432), __byte_perm(A1, A2, 0x5432),
                                                   __byte_perm(A2, A3, 0x5432), __byte_perm(A3, A4, 0x5432));
                                b4[1] = make_uint4(__byte_perm(A4, A5, 0x5432), __byte_perm(A5, A6, 0x5432),
                                                   __byte_perm(A6, A7, 0x5432), __byte_perm(A7, E, 0x5432));
                            }
                            continue;
                        }
                    }
                    uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, E = 0;  // (z0,z1) .. (z6,z7), z8
                    if (gvalid && 8 * idx < zlen) {
#pragma unroll 2
                        for (int m = mstart; m < mend; ++m) {
                            const int2 rm = __ldg(reinterpret_cast<const int2*>(mk + m));  // (s0, ch | span << 16)
                            // byte offset of this lane's first sample in the row.
                            // Bytes at or past the row pitch are never used for an
                            // output sample; their words are clamped to the row's
                            // last word so no read leaves the buffer.
                            const int64_t bo = (int64_t)EB * (t0 + rm.x + 8 * idx);
                            const int wi = (int)(bo >> 2);
                            const uint32_t* w = reinterpret_cast<const uint32_t*>(
                                chunk_in + (int64_t)(rm.y & 0xffff) * pitch_b);
                            const uint32_t sh = (uint32_t)(bo & 3) * 8u;
                            if constexpr (EB == 1) {
                                const uint32_t w0 = __ldg(w + min(wi, wl)), w1 = __ldg(w + min(wi + 1, wl)),
                                               w2 = __ldg(w + min(wi + 2, wl));
                                const uint32_t v0 = __funnelshift_r(w0, w1, sh);
                                const uint32_t v1 = __funnelshift_r(w1, w2, sh);
                                A0 += __byte_perm(v0, 0u, 0x4140);
                                A1 += __byte_perm(v0, 0u, 0x4342);
                                A2 += __byte_perm(v1, 0u, 0x4140);
                                A3 += __byte_perm(v1, 0u, 0x4342);
                                E += (w2 >> sh) & 0xffu;
                            } else {
                                uint32_t w0, w1, w2, w3, w4;
                                load_words5(reinterpret_cast<const unsigned char*>(w), bo, false, wl, w0, w1, w2,
                                            w3, w4);
                                A0 += __funnelshift_r(w0, w1, sh);
                                A1 += __funnelshift_r(w1, w2, sh);
                                A2 += __funnelshift_r(w2, w3, sh);
                                A3 += __funnelshift_r(w3, w4, sh);
                                E += (w4 >> sh) & 0xffffu;
                            }
                        }
                        *reinterpret_cast<uint4*>(zA + 4 * idx) = make_uint4(A0, A1, A2, A3);
                        *reinterpret_cast<uint4*>(zB + 4 * idx) =
                            make_uint4(__byte_perm(A0, A1, 0x5432), __byte_perm(A1, A2, 0x5432),
                                       __byte_perm(A2, A3, 0x5432), __byte_perm(A3, E, 0x5432));
                    }
                }
            }
            __syncthreads();  // group sums complete
            // ---- phase 2: every trial adds every group sum at its relative delay
            if (has_trial) {
                const uint32_t* zl = zs + lane;
                // unrolled twice for 8-bit input; once for 16-bit (measured 2.6 ms
                // faster per step on the decimated ranges, equal on range 0)
                constexpr int kP2Unroll = EB == 1 ? 2 : 1;
                if constexpr (!FLAGS) {
#pragma unroll kP2Unroll
                    for (int g = 0; g < ge - gb; ++g) {
                        const uint32_t* src = zl + __shfl_sync(0xffffffffu, g_p2, g);
#pragma unroll
                        for (int q = 0; q < QW; ++q) acc[q] += src[32 * q];
                    }
                } else {
#pragma unroll 1
                    for (int g = 0; g < ge - gb; ++g) {
                        const int off = __shfl_sync(0xffffffffu, g_p2, g);
                        if (off < 0) {  // this group would overflow the 16-bit lanes
#pragma unroll
                            for (int q = 0; q < QW; ++q) {
                                tot[2 * q] += acc[q] & 0xffffu;
                                tot[2 * q + 1] += acc[q] >> 16;
                                acc[q] = 0;
                            }
                        }
                        const uint32_t* src = zl + (off & 0x7fffffff);
#pragma unroll
                        for (int q = 0; q < QW; ++q) acc[q] += src[32 * q];
                    }
                }
            }
            __syncthreads();  // the next batch (or chunk) overwrites the group sums
        }
        if (!FLAGS && ++since_flush >= a.gflush) {
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                tot[2 * q] += acc[q] & 0xffffu;
                tot[2 * q + 1] += acc[q] >> 16;
                acc[q] = 0;
            }
            since_flush = 0;
        }
    }
#pragma unroll
    for (int q = 0; q < QW; ++q) {
        tot[2 * q] += acc[q] & 0xffffu;
        tot[2 * q + 1] += acc[q] >> 16;
    }

    // epilogue: exact integer totals -> FP32 rows (and the fused statistics)
    if (!has_trial) return;
    if (a.st_acc) {
        unsigned long long s1 = 0, s2 = 0;
#pragma unroll
        for (int q = 0; q < 2 * QW; ++q)
            if (t0 + 2 * (lane + 32 * (q >> 1)) + (q & 1) < a.length) {
                const unsigned long long v = tot[q];
                s1 += v;
                s2 += v * v;
            }
        add_row_sums(a.st_acc + 3 * (int64_t)(d0 + warp), s1, s2);
    }
    float* row = a.out + (int64_t)(d0 + warp) * a.out_pitch;
#pragma unroll
    for (int q = 0; q < QW; ++q) {
        const int64_t t = t0 + 2 * (lane + 32 * q);
        if (t + 2 <= a.length) {
            *reinterpret_cast<float2*>(row + t) = make_float2((float)tot[2 * q], (float)tot[2 * q + 1]);
        } else if (t < a.length) {
            row[t] = (float)tot[2 * q];
        }
    }
}

// FLAGS: the plan places the 16-bit flushes group by group (a.gflush == 0)
template <int EB, bool FLAGS>
__global__ void __launch_bounds__(kDedispThreads, 2)
    dedisperse_grouped_kernel(DedispArgs a, int ndm_blocks) {
    extern __shared__ __align__(128) unsigned char smem[];
    dedisperse_grouped_block<EB, FLAGS>(a, ndm_blocks, blockIdx.x, smem);
}

template <int SPW>
__global__ void __launch_bounds__(kDedispThreads, 2)
    dedisperse_kernel(DedispArgs a, int ndm_blocks, uint64_t wait_limit_ns, int fault_skip_chunk,
                      uint32_t one) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxStages];
    dedisperse_block<SPW>(a, ndm_blocks, blockIdx.x, wait_limit_ns, fault_skip_chunk, one, smem,
                          bars, false);
}

// Persistent form over several beams/ranges: CTAs pull work items from a
// queue; item i belongs to descriptor k with first[k] <= i < first[k+1].
__device__ __forceinline__ int find_desc(const int64_t* first, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One instantiation per strategy and input width (every descriptor of a
// launch uses it).
template <bool GROUPED, int EB>
__global__ void __launch_bounds__(kDedispThreads, 2)
    dedisperse_batch_kernel(const DedispArgs* __restrict__ descs, const int64_t* __restrict__ first,
                            const int* __restrict__ ndm_blocks, int ndesc,
                            unsigned long long* queue, uint64_t wait_limit_ns, uint32_t one) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kMaxStages];  // fixed place: re-initialised per work item
    __shared__ long long s_item;
    const int64_t total = first[ndesc];
    bool reinit = false;
    for (;;) {
        __syncthreads();  // previous item finished by every thread
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int k = find_desc(first, ndesc, item);
        const DedispArgs& a = descs[k];
        if constexpr (GROUPED)
            if (a.gflush == 0)
                dedisperse_grouped_block<EB, true>(a, ndm_blocks[k], item - first[k], smem);
            else
                dedisperse_grouped_block<EB, false>(a, ndm_blocks[k], item - first[k], smem);
        else
            dedisperse_block<4 / EB>(a, ndm_blocks[k], item - first[k], wait_limit_ns, -1, one, smem,
                                     bars, reinit);
        reinit = true;
    }
}

// x_out[c][j] = sum_{k<factor} x_in[c][j*factor + k], j < nout.  One thread
// per 4 outputs; grid-stride over (channel, quad).
template <typename Tin>
__global__ void __launch_bounds__(256) decimate_kernel(const Tin* __restrict__ in, int64_t in_pitch,
                                                       int32_t nchans, int64_t nout, int factor,
                                                       uint16_t* __restrict__ out,
                                                       int64_t out_pitch) {
    const int64_t quads = (nout + 3) / 4;
    const int64_t total = quads * nchans;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q / quads;
        const int64_t j0 = (q - c * quads) * 4;
        const Tin* src = in + c * in_pitch + j0 * factor;
        uint16_t* dst = out + c * out_pitch + j0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j0 + u < nout) {
                uint32_t s = 0;
                for (int k = 0; k < factor; ++k) s += src[u * factor + k];
                dst[u] = (uint16_t)s;
            }
        }
    }
}

// Sums of F consecutive samples with 16-byte loads: a thread reads 16 input
// samples (8-bit: one 16-byte load, F = 2, 4 or 8; 16-bit: two, F = 2) and
// writes their 16 / F sums with one store; the last nout % (16 / F) outputs
// of each row one by one.  Rows, pitches and bases are 16-byte aligned (the
// launcher checks).  An 8-bit word (b0, b1, b2, b3) gives the 16-bit lanes
// (b0 + b1, b2 + b3) as (x & 0x00ff00ff) + ((x >> 8) & 0x00ff00ff), and the
// two lanes added give b0 + b1 + b2 + b3; a 16-bit word (a, b) gives a + b.
template <typename Tin, int F>
__global__ void __launch_bounds__(256) decimate_vec_kernel(const Tin* __restrict__ in, int64_t in_pitch,
                                                           int32_t nchans, int64_t nout,
                                                           uint16_t* __restrict__ out, int64_t out_pitch) {
    constexpr int OPT = 16 / F;  // outputs per thread
    static_assert(sizeof(Tin) == 1 || F == 2, "16-bit input: pair sums only");
    const int64_t units = nout / OPT;
    const int64_t total = units * nchans;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int64_t c = q / units;
        const int64_t j0 = (q - c * units) * OPT;
        const Tin* src = in + c * in_pitch + F * j0;
        uint16_t* dst = out + c * out_pitch + j0;
        if constexpr (sizeof(Tin) == 1) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
            const uint32_t p0 = (v.x & 0x00ff00ffu) + ((v.x >> 8) & 0x00ff00ffu);
            const uint32_t p1 = (v.y & 0x00ff00ffu) + ((v.y >> 8) & 0x00ff00ffu);
            const uint32_t p2 = (v.z & 0x00ff00ffu) + ((v.z >> 8) & 0x00ff00ffu);
            const uint32_t p3 = (v.w & 0x00ff00ffu) + ((v.w >> 8) & 0x00ff00ffu);
            if constexpr (F == 2) {
                *reinterpret_cast<uint4*>(dst) = make_uint4(p0, p1, p2, p3);
            } else {
                const uint32_t s0 = (p0 & 0xffffu) + (p0 >> 16), s1 = (p1 & 0xffffu) + (p1 >> 16);
                const uint32_t s2 = (p2 & 0xffffu) + (p2 >> 16), s3 = (p3 & 0xffffu) + (p3 >> 16);
                if constexpr (F == 4)
                    *reinterpret_cast<uint2*>(dst) = make_uint2(s0 | (s1 << 16), s2 | (s3 << 16));
                else
                    *reinterpret_cast<uint32_t*>(dst) = (s0 + s1) | ((s2 + s3) << 16);
            }
        } else {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4*>(src));
            const uint4 v1 = __ldg(reinterpret_cast<const uint4*>(src) + 1);
            auto pair = [](uint32_t x, uint32_t y) {
                return ((x & 0xffffu) + (x >> 16)) | (((y & 0xffffu) + (y >> 16)) << 16);
            };
            *reinterpret_cast<uint4*>(dst) = make_uint4(pair(v0.x, v0.y), pair(v0.z, v0.w), pair(v1.x, v1.y),
                                                         pair(v1.z, v1.w));
        }
    }
    const int64_t rem = nout - units * OPT;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < rem * nchans; q += stride) {
        const int64_t c = q / rem;
        const int64_t j = units * OPT + (q - c * rem);
        const Tin* src = in + c * in_pitch + F * j;
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < F; ++k) sum += src[k];
        out[c * out_pitch + j] = (uint16_t)sum;
    }
}

// Several decimation jobs in one grid-stride launch (jobs of one cascade
// level only: no job reads another's output).
__global__ void __launch_bounds__(256) decimate_batch_kernel(const DecimateJob* __restrict__ jobs,
                                                             const int64_t* __restrict__ first,
                                                             int njobs) {
    const int64_t total = first[njobs];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_desc(first, njobs, q);
        const DecimateJob& j = jobs[k];
        const int64_t quads = (j.nout + 3) / 4;
        const int64_t local = q - first[k];
        const int64_t c = local / quads;
        const int64_t j0 = (local - c * quads) * 4;
        uint16_t* dst = j.out + c * j.out_pitch + j0;
        for (int u = 0; u < 4; ++u) {
            if (j0 + u >= j.nout) break;
            uint32_t sum = 0;
            if (j.in_elem == 1) {
                const uint8_t* src = static_cast<const uint8_t*>(j.in) + c * j.in_pitch + (j0 + u) * j.factor;
                for (int k2 = 0; k2 < j.factor; ++k2) sum += src[k2];
            } else {
                const uint16_t* src = static_cast<const uint16_t*>(j.in) + c * j.in_pitch + (j0 + u) * j.factor;
                for (int k2 = 0; k2 < j.factor; ++k2) sum += src[k2];
            }
            dst[u] = (uint16_t)sum;
        }
    }
}

}  // namespace

int g_fault_skip_chunk = -1;          // test hook: never issue this chunk
uint64_t g_wait_limit_ns = kWaitLimitNs;

cudaError_t launch_dedisperse_batch(const DedispArgs* d_descs, const int64_t* d_first,
                                    const int* d_ndm_blocks, int ndesc, size_t smem,
                                    unsigned long long* d_queue, int grid, bool grouped, int elem,
                                    cudaStream_t s) {
    if (ndesc <= 0) return cudaSuccess;
    auto kern = grouped ? (elem == 1 ? dedisperse_batch_kernel<true, 1> : dedisperse_batch_kernel<true, 2>)
                        : (elem == 1 ? dedisperse_batch_kernel<false, 1> : dedisperse_batch_kernel<false, 2>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kDedispThreads, smem, s>>>(d_descs, d_first, d_ndm_blocks, ndesc, d_queue,
                                            g_wait_limit_ns, 1u);
    return cudaGetLastError();
}

cudaError_t launch_decimate_batch(const DecimateJob* d_jobs, const int64_t* d_first, int njobs,
                                  int grid, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    decimate_batch_kernel<<<grid, 256, 0, s>>>(d_jobs, d_first, njobs);
    return cudaGetLastError();
}


cudaError_t launch_dedisperse(const DedispArgs& a, cudaStream_t s) {
    if (a.length <= 0 || a.ndm <= 0) return cudaSuccess;
    if (a.nstage < 1 || a.nstage > kMaxStages) return cudaErrorInvalidValue;
    const int ndmb = (a.ndm + kDmPerBlock - 1) / kDmPerBlock;
    const int64_t ntiles = (a.length + kTau - 1) / kTau;
    const int64_t nblocks = (int64_t)ndmb * ntiles;
    if (nblocks >= (1ll << 31)) return cudaErrorInvalidConfiguration;
    if (a.grouped) {
        auto kern = a.elem == 1 ? (a.gflush == 0 ? dedisperse_grouped_kernel<1, true> : dedisperse_grouped_kernel<1, false>)
                                : (a.gflush == 0 ? dedisperse_grouped_kernel<2, true> : dedisperse_grouped_kernel<2, false>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nblocks, kDedispThreads, a.smem, s>>>(a, ndmb);
        return cudaGetLastError();
    }
    auto kern = a.elem == 1 ? dedisperse_kernel<4> : dedisperse_kernel<2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nblocks, kDedispThreads, a.smem, s>>>(a, ndmb, g_wait_limit_ns,
                                                            g_fault_skip_chunk, 1u);
    return cudaGetLastError();
}

cudaError_t launch_decimate(const void* in, int in_elem, int64_t in_pitch, int32_t nchans,
                            int64_t nout, int factor, uint16_t* out, int64_t out_pitch,
                            cudaStream_t s) {
    if (nout <= 0) return cudaSuccess;
    const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec_ok = al16(in) && al16(out) && (in_pitch * in_elem) % 16 == 0 && (out_pitch * 2) % 16 == 0 &&
                        (in_elem == 1 ? (factor == 2 || factor == 4 || factor == 8) : factor == 2);
    if (vec_ok) {
        int64_t blocks = (nout / (16 / factor) * nchans + 255) / 256;
        blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 64));
        const uint8_t* in8 = static_cast<const uint8_t*>(in);
        if (in_elem == 2)
            decimate_vec_kernel<uint16_t, 2><<<(unsigned)blocks, 256, 0, s>>>(
                static_cast<const uint16_t*>(in), in_pitch, nchans, nout, out, out_pitch);
        else if (factor == 2)
            decimate_vec_kernel<uint8_t, 2><<<(unsigned)blocks, 256, 0, s>>>(in8, in_pitch, nchans, nout, out, out_pitch);
        else if (factor == 4)
            decimate_vec_kernel<uint8_t, 4><<<(unsigned)blocks, 256, 0, s>>>(in8, in_pitch, nchans, nout, out, out_pitch);
        else
            decimate_vec_kernel<uint8_t, 8><<<(unsigned)blocks, 256, 0, s>>>(in8, in_pitch, nchans, nout, out, out_pitch);
        return cudaGetLastError();
    }
    const int64_t total = (nout + 3) / 4 * nchans;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (in_elem == 1)
        decimate_kernel<uint8_t><<<(unsigned)blocks, 256, 0, s>>>(
            static_cast<const uint8_t*>(in), in_pitch, nchans, nout, factor, out, out_pitch);
    else
        decimate_kernel<uint16_t><<<(unsigned)blocks, 256, 0, s>>>(
            static_cast<const uint16_t*>(in), in_pitch, nchans, nout, factor, out, out_pitch);
    return cudaGetLastError();
}

}  // namespace aa

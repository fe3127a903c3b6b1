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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
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

// Grouped strategy (see GroupRec / GroupBatch in aa_internal.h).  CTA = 16
// DM trials x kGroupTau output samples, 24 warps.  The channels stream through
// in chunks of a.cc; the groups of a chunk are processed in batches of at most
// a.gz (the DM block's batch table lists them chunk after chunk):
//   phase 1 (producer warps 16..23): z_g[u] = sum over the group's members of
//            x[c][t0 + s0_c + u], u < kGroupTau + span_g, read straight from
//            global memory (each member row is read by one warp, coalesced
//            32-bit words; the rows of a chunk are shared by the CTAs of all
//            DM blocks through L2), as packed 16-bit pairs stored twice:
//            copy A word j = (z[2j], z[2j+1]) and copy B word j =
//            (z[2j+1], z[2j+2]); work unit = (group, 256 or 512 consecutive
//            u) or (several groups' samples past 511: tail units), units
//            round-robin over the producer warps;
//   phase 2 (consumer warp w < 16 = trial d0 + w): adds z_g[t + delta_g(w)]
//            for its 16 samples t: copy (delta & 1), word offset delta >> 1,
//            aligned.
// The two phases run concurrently on a ring of a.gnbuf batch buffers: batch j
// lives in buffer j % gnbuf; full[b] completes when every producer thread has
// written its part of the batch, empty[b] when every consumer thread has read
// it.  Every wait is bounded (wait_limit_ns of wall clock); on expiry the
// thread sets the error word and leaves, and the others then run out of time
// too (nothing waits forever).  Returns false in every thread that gave up.
// 16-bit lanes never overflow: a chunk holds at most 65535 / (255 dec)
// channels, and trial accumulators are flushed every a.gflush chunks.
template <int EB>
__device__ __forceinline__ bool dedisperse_grouped_block(const DedispArgs& a, int ndm_blocks,
                                                         int64_t bid, unsigned char* smem,
                                                         uint64_t* bars, bool reinit,
                                                         uint64_t wait_limit_ns, int fault_skip_batch) {
    constexpr int T = kGroupTau;
    constexpr int QW = T / 64;  // packed words (2 samples) per lane per trial
    constexpr unsigned kFull = 0xffffffffu;
    const int gcc = a.cc, gzw = a.gzw, nj = a.gnj, nbuf = a.gnbuf;
    const int buf_words = a.gz * 2 * gzw;
    uint32_t* zs = reinterpret_cast<uint32_t*>(smem);  // [nbuf][gz][2][gzw]
    uint64_t* full = bars;                              // [kMaxGroupBufs]
    uint64_t* empty = bars + kMaxGroupBufs;             // [kMaxGroupBufs]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dmb = (int)(bid % ndm_blocks);
    const int64_t tile = bid / ndm_blocks;
    const int d0 = dmb * kDmPerBlock;
    const int dlast = min(a.ndm, d0 + kDmPerBlock) - 1;
    const int64_t t0 = tile * T;
    const int C = a.nchans;
    const int nchunks = (C + gcc - 1) / gcc;
    const GroupBatch* batches = a.gbatch + a.gboff[dmb];
    const int nbatch = a.gboff[dmb + 1] - a.gboff[dmb];

    // the block's batch records, staged once after the group-sum buffers
    GroupBatch* btab = reinterpret_cast<GroupBatch*>(zs + nbuf * buf_words);
    for (int i = threadIdx.x; i < nbatch; i += kGroupedThreads)
        reinterpret_cast<uint2*>(btab)[i] = __ldg(reinterpret_cast<const uint2*>(batches + i));
    if (threadIdx.x == 0) {  // every barrier of the fixed array, whatever a previous item used
        for (int b = 0; b < kMaxGroupBufs; ++b) {
            if (reinit) {
                mbar_inval(&full[b]);
                mbar_inval(&empty[b]);
            }
            mbar_init(&full[b], kGroupProducers * 32);
            mbar_init(&empty[b], kDmPerBlock * 32);
        }
        mbar_fence_init();
    }
    __syncthreads();  // batch table staged, barriers initialised
    if (nbatch == 0) return true;  // (a plan always gives a DM block at least one batch)

    if (warp < kDmPerBlock) {
        // ================= consumer: trial d0 + warp
        uint32_t acc[QW];
        uint32_t tot[2 * QW];
#pragma unroll
        for (int q = 0; q < QW; ++q) {
            acc[q] = 0;
            tot[2 * q] = tot[2 * q + 1] = 0;
        }
        const bool has_trial = d0 + warp <= dlast;
        // this trial's relative delay of the lane's group (batch j + 1 in flight)
        auto load_dl = [&](const GroupBatch& b) -> uint32_t {
            return lane < b.ngroups ? (uint32_t)__ldg(&a.gdesc[b.first + lane].delta[warp]) : 0u;
        };
        uint32_t dl_next = load_dl(btab[0]);
        int since_flush = 0;
        for (int j = 0; j < nbatch; ++j) {
            const int b = j % nbuf;
            const uint32_t dl = dl_next;
            if (j + 1 < nbatch) dl_next = load_dl(btab[j + 1]);
            const int g_p2 = b * buf_words + (lane * 2 + (int)(dl & 1u)) * gzw + (int)(dl >> 1);
            const GroupBatch bc = btab[j];
            if (!mbar_wait_bounded(&full[b], (uint32_t)(j / nbuf) & 1u, wait_limit_ns)) {
                atomicOr(a.err, 2u);
                return false;
            }
            if (has_trial) {
                const uint32_t* zl = zs + lane;
#pragma unroll 2
                for (int g = 0; g < bc.ngroups; ++g) {
                    const uint32_t* src = zl + __shfl_sync(kFull, g_p2, g);
#pragma unroll
                    for (int q = 0; q < QW; ++q) acc[q] += src[32 * q];
                }
            }
            mbar_arrive(&empty[b]);  // this thread's reads of buffer b are done
            if ((bc.chunk & kBatchLastOfChunk) && ++since_flush >= a.gflush) {
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
        // epilogue: exact integer totals -> FP32 rows
        if (!has_trial) return true;
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
        return true;
    }

    // ================= producer warp pw
    const int pw = warp - kDmPerBlock;
    const unsigned char* in_b = static_cast<const unsigned char*>(a.in);
    const int64_t pitch_b = a.in_pitch * EB;
    const int wl = (int)(pitch_b >> 2) - 1;  // last word of a row
    const GroupMember* mems = a.gmem + (size_t)dmb * nchunks * gcc;
    // tail units: gtl lanes per group (a power of two), gpt groups per warp
    const int gtl = a.gtl, gtl_log = gtl ? __ffs(gtl) - 1 : 0, gpt = gtl ? 32 / gtl : 1;
    // group fields of the lane's group: (mstart | mcount << 16, span | pad << 16)
    auto load_head = [&](const GroupBatch& b) -> uint2 {
        return lane < b.ngroups ? __ldg(reinterpret_cast<const uint2*>(a.gdesc + b.first + lane))
                                : make_uint2(0u, 0u);
    };
    uint2 head_next = load_head(btab[0]);
    for (int j = 0; j < nbatch; ++j) {
        const int b = j % nbuf;
        const uint2 head = head_next;
        const GroupBatch bc = btab[j];
        if (j + 1 < nbatch) head_next = load_head(btab[j + 1]);
        if (j >= nbuf &&  // the consumers have read the batch that used buffer b before
            !mbar_wait_bounded(&empty[b], (uint32_t)(j / nbuf - 1) & 1u, wait_limit_ns)) {
            atomicOr(a.err, 2u);
            return false;
        }
        uint32_t* zb = zs + b * buf_words;
        const int k = bc.chunk & ~kBatchLastOfChunk;
        const GroupMember* mk = mems + (size_t)k * gcc;
        const unsigned char* chunk_in = in_b + (int64_t)(k * gcc) * pitch_b;
        const int ng = bc.ngroups;
        const uint32_t g_ms = head.x, g_span = head.y & 0xffffu;
        // 8-bit input with tail units: one unit per group covers samples
        // 0..511 at 16 per lane; otherwise units of 8 samples per lane
        constexpr bool kWide = EB == 1;
        const int nmain = gtl ? (kWide ? ng : 2 * ng) : ng * nj;
        const int nunits = gtl ? nmain + (ng + gpt - 1) / gpt : nmain;
        for (int u = pw; u < nunits; u += kGroupProducers) {
            if (u < nmain) {
                // main unit: the whole warp sums one group's members; lane m
                // holds member record m, handed round by shuffles
                int gi, idx;
                if (gtl) {
                    gi = kWide ? u : (u >> 1);
                    idx = kWide ? lane : 32 * (u & 1) + lane;
                } else {
                    gi = u / nj;
                    idx = 32 * (u - gi * nj) + lane;
                }
                const uint32_t ms = __shfl_sync(kFull, g_ms, gi);
                const int zlen = T + (int)__shfl_sync(kFull, g_span, gi);
                const int mstart = (int)(ms & 0xffffu), mend = mstart + (int)(ms >> 16);
                uint32_t* zA = zb + gi * 2 * gzw;
                uint32_t* zB = zA + gzw;
                if (kWide && gtl) {
                    // 16 samples: five words per member (bytes b .. b + 16)
                    uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, A4 = 0, A5 = 0, A6 = 0, A7 = 0, E = 0;
                    for (int m0 = mstart; m0 < mend; m0 += 32) {
                        const int nm = min(32, mend - m0);
                        const int2 my = lane < nm ? __ldg(reinterpret_cast<const int2*>(mk + m0 + lane))
                                                  : make_int2(0, 0);
#pragma unroll 4
                        for (int m = 0; m < nm; ++m) {
                            const int rx = __shfl_sync(kFull, my.x, m), ry = __shfl_sync(kFull, my.y, m);
                            const int64_t bo = t0 + rx + 16 * idx;
                            const int wi = (int)(bo >> 2);
                            const uint32_t* w = reinterpret_cast<const uint32_t*>(
                                chunk_in + (int64_t)(ry & 0xffff) * pitch_b);
                            const uint32_t sh = (uint32_t)(bo & 3) * 8u;
                            const uint32_t w0 = __ldg(w + min(wi, wl)), w1 = __ldg(w + min(wi + 1, wl)),
                                           w2 = __ldg(w + min(wi + 2, wl)), w3 = __ldg(w + min(wi + 3, wl)),
                                           w4 = __ldg(w + min(wi + 4, wl));
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
                    }
                    uint4* a4 = reinterpret_cast<uint4*>(zA + 8 * idx);
                    uint4* b4 = reinterpret_cast<uint4*>(zB + 8 * idx);
                    a4[0] = make_uint4(A0, A1, A2, A3);
                    a4[1] = make_uint4(A4, A5, A6, A7);
                    b4[0] = make_uint4(__byte_perm(A0, A1, 0x5432), __byte_perm(A1, A2, 0x5432),
                                       __byte_perm(A2, A3, 0x5432), __byte_perm(A3, A4, 0x5432));
                    b4[1] = make_uint4(__byte_perm(A4, A5, 0x5432), __byte_perm(A5, A6, 0x5432),
                                       __byte_perm(A6, A7, 0x5432), __byte_perm(A7, E, 0x5432));
                } else {
                    // 8 samples per lane; lanes past the group's length compute
                    // (in-bounds, clamped reads) but do not store
                    uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, E = 0;  // (z0,z1) .. (z6,z7), z8
                    for (int m0 = mstart; m0 < mend; m0 += 32) {
                        const int nm = min(32, mend - m0);
                        const int2 my = lane < nm ? __ldg(reinterpret_cast<const int2*>(mk + m0 + lane))
                                                  : make_int2(0, 0);
#pragma unroll 4
                        for (int m = 0; m < nm; ++m) {
                            const int rx = __shfl_sync(kFull, my.x, m), ry = __shfl_sync(kFull, my.y, m);
                            // byte offset of this lane's first sample in the row;
                            // words at or past the row pitch are clamped to the
                            // row's last word (never used for an output sample)
                            const int64_t bo = (int64_t)EB * (t0 + rx + 8 * idx);
                            const int wi = (int)(bo >> 2);
                            const uint32_t* w = reinterpret_cast<const uint32_t*>(
                                chunk_in + (int64_t)(ry & 0xffff) * pitch_b);
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
                                const uint32_t w0 = __ldg(w + min(wi, wl)), w1 = __ldg(w + min(wi + 1, wl)),
                                               w2 = __ldg(w + min(wi + 2, wl)), w3 = __ldg(w + min(wi + 3, wl)),
                                               w4 = __ldg(w + min(wi + 4, wl));
                                A0 += __funnelshift_r(w0, w1, sh);
                                A1 += __funnelshift_r(w1, w2, sh);
                                A2 += __funnelshift_r(w2, w3, sh);
                                A3 += __funnelshift_r(w3, w4, sh);
                                E += (w4 >> sh) & 0xffffu;
                            }
                        }
                    }
                    if (8 * idx < zlen) {
                        *reinterpret_cast<uint4*>(zA + 4 * idx) = make_uint4(A0, A1, A2, A3);
                        *reinterpret_cast<uint4*>(zB + 4 * idx) =
                            make_uint4(__byte_perm(A0, A1, 0x5432), __byte_perm(A1, A2, 0x5432),
                                       __byte_perm(A2, A3, 0x5432), __byte_perm(A3, E, 0x5432));
                    }
                }
            } else {
                // tail unit: samples past 511 of gpt groups, gtl lanes each
                const int gi = (u - nmain) * gpt + (lane >> gtl_log);
                const int idx = 64 + (lane & (gtl - 1));
                const bool gvalid = gi < ng;
                const int gs = gvalid ? gi : 0;
                const uint32_t ms = __shfl_sync(kFull, g_ms, gs);
                const int zlen = T + (int)__shfl_sync(kFull, g_span, gs);
                const int mstart = (int)(ms & 0xffffu), mend = mstart + (int)(ms >> 16);
                uint32_t* zA = zb + gs * 2 * gzw;
                uint32_t* zB = zA + gzw;
                uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, E = 0;
                if (gvalid && 8 * idx < zlen) {
#pragma unroll 2
                    for (int m = mstart; m < mend; ++m) {
                        const int2 rm = __ldg(reinterpret_cast<const int2*>(mk + m));
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
                            const uint32_t w0 = __ldg(w + min(wi, wl)), w1 = __ldg(w + min(wi + 1, wl)),
                                           w2 = __ldg(w + min(wi + 2, wl)), w3 = __ldg(w + min(wi + 3, wl)),
                                           w4 = __ldg(w + min(wi + 4, wl));
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
        if (j == fault_skip_batch) continue;  // fault injection: batch j is never completed
        mbar_arrive(&full[b]);  // this thread's writes of batch j are done
    }
    return true;
}

template <int EB>
__global__ void __launch_bounds__(kGroupedThreads, 1)
    dedisperse_grouped_kernel(DedispArgs a, int ndm_blocks, uint64_t wait_limit_ns, int fault_skip_batch) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t gbars[2 * kMaxGroupBufs];
    dedisperse_grouped_block<EB>(a, ndm_blocks, blockIdx.x, smem, gbars, false, wait_limit_ns,
                                 fault_skip_batch);
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

// One instantiation per input width (every descriptor of a launch uses it).
template <int EB>
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
        dedisperse_block<4 / EB>(descs[k], ndm_blocks[k], item - first[k], wait_limit_ns, -1, one, smem,
                                 bars, reinit);
        reinit = true;
    }
}

template <int EB>
__global__ void __launch_bounds__(kGroupedThreads, 1)
    dedisperse_grouped_batch_kernel(const DedispArgs* __restrict__ descs,
                                    const int64_t* __restrict__ first,
                                    const int* __restrict__ ndm_blocks, int ndesc,
                                    unsigned long long* queue, uint64_t wait_limit_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t gbars[2 * kMaxGroupBufs];  // fixed place: re-initialised per work item
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
        const bool ok = dedisperse_grouped_block<EB>(descs[k], ndm_blocks[k], item - first[k], smem, gbars,
                                                     reinit, wait_limit_ns, -1);
        reinit = true;
        if (__syncthreads_or(!ok)) break;  // a wait gave up: the error word is set
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
int g_fault_skip_batch = -1;          // test hook: grouped producers never complete this batch
uint64_t g_wait_limit_ns = kWaitLimitNs;

cudaError_t launch_dedisperse_batch(const DedispArgs* d_descs, const int64_t* d_first,
                                    const int* d_ndm_blocks, int ndesc, size_t smem,
                                    unsigned long long* d_queue, int grid, bool grouped, int elem,
                                    cudaStream_t s) {
    if (ndesc <= 0) return cudaSuccess;
    if (grouped) {  // one 768-thread CTA per SM (grid counts two 512-thread CTAs per SM)
        auto kern = elem == 1 ? dedisperse_grouped_batch_kernel<1> : dedisperse_grouped_batch_kernel<2>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(grid + 1) / 2, kGroupedThreads, smem, s>>>(d_descs, d_first, d_ndm_blocks, ndesc, d_queue,
                                                            g_wait_limit_ns);
        return cudaGetLastError();
    }
    auto kern = elem == 1 ? dedisperse_batch_kernel<1> : dedisperse_batch_kernel<2>;
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
        auto kern = a.elem == 1 ? dedisperse_grouped_kernel<1> : dedisperse_grouped_kernel<2>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nblocks, kGroupedThreads, a.smem, s>>>(a, ndmb, g_wait_limit_ns,
                                                                 g_fault_skip_batch);
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

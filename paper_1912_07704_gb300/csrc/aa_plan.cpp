// Plan and strategy (arXiv:1912.07704 Sec. 3.1-3.2): validate the user's
// description, build the FP64 delay tables and derive the immutable,
// queryable strategy and memory requests (Sec. 2.3).  Host only, except
// aa_plan_bind which uploads the delay tables.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <new>

#include "aa_internal.h"

namespace aa {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

// Dispersion constant, MHz^2 pc^-1 cm^3 s.
static constexpr double kDM = 4.148808e3;

// Delay of channel c at dispersion measure dm, in samples of a series
// decimated by dec: round half away from zero of ((kDM*dm)*delta_c)/(tsamp*dec)
// with delta_c = f_c^-2 - f_top^-2, every step an IEEE double rounded in the
// order written (this file is compiled without FP contraction).
static int32_t delay_samples(double fch1, double foff, double f_top, int32_t c, double tsamp,
                             double dm, int32_t dec) {
    double fc = fch1 + (double)c * foff;
    double delta = 1.0 / (fc * fc) - 1.0 / (f_top * f_top);
    double v = kDM * dm * delta / (tsamp * (double)dec);
    return (int32_t)std::llround(v);
}

// Delay of channel c relative to channel cref at dispersion measure dm, in
// samples of a series decimated by dec: round half away from zero of
// ((kDM*dm)*(delta_c - delta_ref))/(tsamp*dec), delta as in delay_samples.
static int32_t rel_delay_samples(double fch1, double foff, double f_top, int32_t c, int32_t cref,
                                 double tsamp, double dm, int32_t dec) {
    double fc = fch1 + (double)c * foff;
    double fr = fch1 + (double)cref * foff;
    double dc = 1.0 / (fc * fc) - 1.0 / (f_top * f_top);
    double dr = 1.0 / (fr * fr) - 1.0 / (f_top * f_top);
    double v = kDM * dm * (dc - dr) / (tsamp * (double)dec);
    return (int32_t)std::llround(v);
}

// Shared-memory footprint of one dedispersion CTA for a given channel chunk.
static size_t dedisp_smem(const RangePlan& r, int cc, int nstage) {
    size_t stage = (size_t)cc * r.spw * r.rw * 4;  // spw shifted copies per channel row
    size_t tables = (size_t)kDmPerBlock * cc * 4 + (size_t)cc * 4;  // word offsets + bases
    return (size_t)nstage * (stage + tables) + 64;  // + mbarriers
}

size_t dedisp_smem_bytes(const RangePlan& r, int cc, int nstage) { return dedisp_smem(r, cc, nstage); }

static size_t shape_smem(int spw, int rw, int cc, int nstage) {
    size_t stage = (size_t)cc * spw * rw * 4;
    size_t tables = (size_t)kDmPerBlock * cc * 4 + (size_t)cc * 4;
    return (size_t)nstage * (stage + tables) + 64;
}

bool direct_shape(int elem, int32_t span, int per_lane_max, DirectShape& out) {
    DirectShape d;
    d.elem = elem;
    d.spw = 4 / elem;
    const int a16 = 16 / elem;  // samples per 16-byte alignment unit
    const int64_t window = (int64_t)kTau + span + (a16 - 1) + d.spw;
    d.rw = (int)round_up((window + d.spw - 1) / d.spw, 4);
    // SWAR flush period: 16-bit lanes hold at most 65535
    const int max_flush = 65535 / std::max(per_lane_max, 1);
    const size_t budget = 120 * 1024;
    d.nstage = 2;
    d.cc = std::min(24, (max_flush / 2) * 2);
    while (d.cc > 2 && shape_smem(d.spw, d.rw, d.cc, d.nstage) > budget) d.cc -= 2;
    if (d.cc < 2 || shape_smem(d.spw, d.rw, d.cc, d.nstage) > 200 * 1024) return false;
    d.flush = (std::min(max_flush, 256) / d.cc) * d.cc;
    d.smem = shape_smem(d.spw, d.rw, d.cc, d.nstage);
    out = d;
    return true;
}

// Shared memory of the grouped strategy: the group sums of one batch (two
// copies each; the input rows are read from global memory).
static size_t grouped_smem(int gz, int gzw) { return (size_t)gz * 2 * gzw * 4; }

// Delay-pattern groups of every (DM block, channel chunk) of a range, and the
// grouped tile shape.  Two CTAs per SM must fit (<= kPairSmem each).
static void build_groups(RangePlan& r, int C) {
    constexpr size_t kPairSmem = 113 * 1024 - 512;
    constexpr int B = kDmPerBlock;
    r.grouped_ok = false;
    const int dec = r.desc.dec;
    const int lane_max = 65535 / (255 * dec);          // channels per 16-bit lane
    if (r.span_max > 4096) return;
    const int gzw = (int)round_up((kGroupTau + r.span_max + 3) / 2 + 2, 4);
    // chunks of up to kGroupChunkMax channels (fewer when 16-bit lanes would
    // overflow): larger chunks put more channels with one delay pattern into
    // one group; as many group sums per batch as two CTAs per SM leave room
    // for (<= 32, one per lane of the warps' group-field registers)
    // The 16-bit lanes bound each group sum (at most kGroupSplit members,
    // fewer when lane_max is smaller) and each trial's running sum between
    // two flushes (at most lane_max members' worth of group sums: the
    // flushes are placed group by group, see the flush flags below), not the
    // chunk.
    // Chunks of up to 1024 channels for 8-bit input, 4096 for 16-bit
    // (measured on the 4096-channel plan: larger chunks give fewer, larger
    // groups, but past 1024 channels the 8-bit kernel's member rows no longer
    // stay in L2 across the DM blocks' CTAs).
    const int kGroupChunkMax = r.elem == 1 ? 1024 : 4096;
    if (lane_max < 1) return;
    // members per group sum at most (larger parts mean fewer group sums but a
    // longer phase 1 for the warp that builds one: measured best at 16 for
    // 8-bit input, 32 for 16-bit)
    const int kGroupSplit = std::min(r.elem == 1 ? 16 : 32, lane_max);
    const int gcc = kGroupChunkMax;
    int gz = 0;
    while (grouped_smem(gz + 1, gzw) <= kPairSmem && gz < std::min(gcc, 32)) ++gz;
    if (gcc < 8 || gz < 1) return;
    {   // samples past kGroupTau (the span and the one sample after it) in lanes of 8
        const int need = (r.span_max + 1 + 7) / 8;
        int tl = 1;
        while (tl < need) tl *= 2;
        r.gtl = (kGroupTau % 256 == 0 && tl <= 32) ? tl : 0;
    }
    // phase 1's static unit assignment: with tail units, an 8-bit range gives
    // a group one unit (warp j mod 16 for batch position j), a 16-bit range
    // two (warp pair j mod 8)
    const int kSlots = (r.gtl > 0 && r.elem == 1) ? kDedispWarps : kDedispWarps / 2;
    const int ndm = r.desc.ndm;
    const int nblk = (ndm + B - 1) / B, nchk = (C + gcc - 1) / gcc;
    r.grec.assign((size_t)nblk * nchk, GroupRec{});
    r.gmem.assign((size_t)nblk * nchk * gcc, GroupMember{});
    r.gdesc.clear();
    double direct = 0, grouped = 0;
    std::vector<GroupDesc> local;
    std::vector<std::vector<uint16_t>> members;
    int run = 0;  // members summed into the trials' 16-bit lanes since the last flush
    for (int b = 0; b < nblk; ++b) {
        const int d0 = b * B, nb = std::min(B, ndm - d0);
        for (int k = 0; k < nchk; ++k) {
            const int c0 = k * gcc, nch = std::min(gcc, C - c0);
            local.clear();
            members.clear();
            for (int cl = 0; cl < nch; ++cl) {
                const int c = c0 + cl;
                GroupDesc g{};
                const int32_t s0 = r.shifts[(size_t)d0 * C + c];
                for (int d = 0; d < B; ++d) {
                    const int dd = d0 + std::min(d, nb - 1);  // pad a partial block with its last trial
                    g.delta[d] = (uint16_t)(r.shifts[(size_t)dd * C + c] - s0);
                }
                g.span = g.delta[B - 1];
                size_t gi = 0;
                while (gi < local.size() && std::memcmp(local[gi].delta, g.delta, sizeof g.delta) != 0) ++gi;
                if (gi == local.size()) {
                    local.push_back(g);
                    members.emplace_back();
                }
                members[gi].push_back((uint16_t)cl);
            }
            // Phase 1 of the kernel gives the unit(s) of the group at batch
            // position j to slot j % kSlots (a warp or a warp pair), and a unit
            // costs one pass over the group's members.  Groups larger than
            // kGroupSplit members are split into near-equal parts (same delay
            // pattern, separate sums), the parts sorted by size and, batch by
            // batch, dealt to the slots least loaded so far, so that no warp
            // waits on one large group.
            struct Part { int gi, b, e; };
            std::vector<Part> parts;
            for (size_t gi = 0; gi < local.size(); ++gi) {
                const int n = (int)members[gi].size();
                const int np = (n + kGroupSplit - 1) / kGroupSplit, base = n / np, rem = n % np;
                for (int j = 0, pos = 0; j < np; ++j) {
                    const int sz = base + (j < rem ? 1 : 0);
                    parts.push_back(Part{(int)gi, pos, pos + sz});
                    pos += sz;
                }
            }
            std::stable_sort(parts.begin(), parts.end(),
                             [](const Part& x, const Part& y) { return x.e - x.b > y.e - y.b; });
            std::vector<Part> laid(parts.size());
            for (size_t b0 = 0; b0 < parts.size(); b0 += (size_t)gz) {
                const int n = (int)std::min(parts.size() - b0, (size_t)gz);
                int load[kDedispWarps] = {}, cnt[kDedispWarps] = {};
                for (int i = 0; i < n; ++i) {
                    int best = -1;
                    for (int q = 0; q < kSlots; ++q) {
                        const int cap = n / kSlots + (q < n % kSlots ? 1 : 0);
                        if (cnt[q] < cap && (best < 0 || load[q] < load[best])) best = q;
                    }
                    const Part& pt = parts[b0 + i];
                    laid[b0 + (size_t)(kSlots * cnt[best] + best)] = pt;
                    ++cnt[best];
                    load[best] += pt.e - pt.b;
                }
            }
            GroupRec& rec = r.grec[(size_t)b * nchk + k];
            if (k == 0) run = 0;
            rec.first = (uint32_t)r.gdesc.size();
            rec.ngroups = (uint16_t)laid.size();
            rec.nch = (uint16_t)nch;
            GroupMember* mem = &r.gmem[((size_t)b * nchk + k) * gcc];
            int m = 0;
            for (const Part& pt : laid) {
                GroupDesc g = local[(size_t)pt.gi];
                g.mstart = (uint16_t)m;
                g.mcount = (uint16_t)(pt.e - pt.b);
                // flush flag: the trials' 16-bit sums are emptied into their
                // 32-bit totals before this group when its members would take
                // the members summed since the last flush past lane_max
                // (groups are added in this order: chunk by chunk, batch by
                // batch, in list order)
                g.flush = 0;
                if (gcc > lane_max && run + g.mcount > lane_max) {
                    g.flush = 1;
                    run = 0;
                }
                run += g.mcount;
                for (int j = pt.b; j < pt.e; ++j) {
                    const uint16_t cl = members[(size_t)pt.gi][(size_t)j];
                    const int32_t s0 = r.shifts[(size_t)d0 * C + c0 + cl];
                    const int32_t s1 = r.shifts[(size_t)(d0 + nb - 1) * C + c0 + cl];
                    mem[m++] = GroupMember{s0, (uint16_t)cl, (uint16_t)(s1 - s0)};
                }
                r.gdesc.push_back(g);
            }
            direct += (double)nch * nb;
            grouped += (double)nch + (double)laid.size() * nb;
        }
    }
    r.gcc = gcc;
    r.gz = gz;
    r.gzw = gzw;
    // a chunk that fits the 16-bit lanes is flushed whole (every lane_max /
    // gcc chunks); otherwise gflush = 0 and the groups' flags place the flushes
    r.gflush = gcc <= lane_max ? lane_max / gcc : 0;
    r.gnj = (kGroupTau + r.span_max + 255) / 256;
    r.gsmem = grouped_smem(gz, gzw);
    r.gwork = direct > 0 ? grouped / direct : 1.0;
    r.grouped_ok = true;
}

void fill_strategy(DedispArgs& a, const RangePlan& r) {
    a.elem = r.elem;
    a.rw = r.rw;
    a.flush = r.flush;
    if (r.strategy == 1) {
        a.grouped = 1;
        a.cc = r.gcc;
        a.nstage = 2;
        a.smem = r.gsmem;
        a.gz = r.gz;
        a.gzw = r.gzw;
        a.gflush = r.gflush;
        a.gnj = r.gnj;
        a.gtl = r.gtl;
        a.grec = r.d_grec;
        a.gdesc = r.d_gdesc;
        a.gmem = r.d_gmem;
    } else {
        a.grouped = 0;
        a.cc = r.cc;
        a.nstage = r.nstage;
        a.smem = r.smem;
        a.gz = a.gzw = a.gflush = a.gnj = a.gtl = 0;
        a.grec = nullptr;
        a.gdesc = nullptr;
        a.gmem = nullptr;
    }
}

static aa_status build_strategy(aa_plan& p) {
    for (auto& r : p.ranges) {
        const int dec = r.desc.dec;
        r.elem = dec == 1 ? 1 : 2;
        r.spw = 4 / r.elem;
        const int ndm = r.desc.ndm;
        const int C = p.nchans;
        int32_t span = 0;
        for (int d0 = 0; d0 < ndm; d0 += kDmPerBlock) {
            int d1 = std::min(ndm, d0 + kDmPerBlock) - 1;
            const int32_t* a = &r.shifts[(size_t)d0 * C];
            const int32_t* b = &r.shifts[(size_t)d1 * C];
            for (int c = 0; c < C; ++c) span = std::max(span, b[c] - a[c]);
        }
        r.span_max = span;
        const int a16 = 16 / r.elem;  // samples per 16-byte alignment unit
        int64_t window = (int64_t)kTau + span + (a16 - 1) + r.spw;
        r.rw = (int)round_up((window + r.spw - 1) / r.spw, 4);
        // SWAR flush period: 16-bit lanes hold at most 65535.
        const int per_lane_max = 255 * dec;
        const int max_flush = 65535 / per_lane_max;
        // Two stages (deeper pipelines measured no faster) and as many
        // channels per stage as fit: the per-stage synchronisation cost is
        // fixed, so larger stages amortise it (measured best at 24 channels).
        const size_t budget = 120 * 1024;
        int nstage = 2, cc = std::min(24, (max_flush / 2) * 2);
        while (cc > 2 && dedisp_smem(r, cc, nstage) > budget) cc -= 2;
        if (cc < 2 || dedisp_smem(r, cc, nstage) > 200 * 1024) {
            set_error("range dm_lo=%g: DM step too coarse for the dedispersion tile "
                      "(delay span %d samples over %d trials)", r.desc.dm_lo, span, kDmPerBlock);
            return AA_ERR_CONFIG;
        }
        r.cc = cc;
        r.nstage = nstage;
        r.flush = (std::min(max_flush, 256) / cc) * cc;
        r.smem = dedisp_smem(r, cc, nstage);
        if (dec == 1) {  // spans used by the differentiable (float) form
            int sp = 0, csp = 0;
            for (int d = 0; d < ndm; ++d) {
                const int32_t* a = &r.shifts[(size_t)d * C];
                const int32_t* b = &r.shifts[(size_t)std::min(ndm - 1, d + 15) * C];
                for (int c = 0; c < C; ++c) sp = std::max(sp, std::abs(b[c] - a[c]));
                for (int c = 0; c < C; ++c) csp = std::max(csp, std::abs(a[std::min(C - 1, c + 15)] - a[c]));
            }
            r.f32_span = sp;
            r.f32_cspan = csp;
        }
        // Grouped strategy where it removes enough adds: one pre-sum add per
        // channel plus one add per group and trial, against one add per
        // channel and trial (measured break-even well above 0.6).
        build_groups(r, C);
        r.strategy = (r.grouped_ok && r.gwork <= 0.6) ? 1 : 0;
    }
    // decimation cascade: each decimated buffer is built from the largest
    // already-built decimation that divides it (or from the raw input).
    for (auto& r : p.ranges)
        if (r.desc.dec > 1 && std::find(p.decs.begin(), p.decs.end(), r.desc.dec) == p.decs.end())
            p.decs.push_back(r.desc.dec);
    std::sort(p.decs.begin(), p.decs.end());
    return AA_OK;
}

Layout make_layout(const aa_plan& p, int64_t nsamp, int32_t max_width) {
    Layout L;
    L.nsamp = nsamp;
    L.in_pitch_min = round_up(std::max<int64_t>(nsamp, 1), 16);
    int64_t off = 0;
    for (auto& r : p.ranges) {
        int64_t nd = nsamp / r.desc.dec;
        // sub-band ranges: the effective delay is at most rmax + s2max
        const int64_t ms = r.strategy == 2 ? (int64_t)r.sb.rmax + r.sb.s2max : r.maxshift;
        int64_t len = std::max<int64_t>(0, nd - ms);
        int64_t pitch = round_up(std::max<int64_t>(len, 1), 64);
        L.nsamp_dec.push_back(nd);
        L.length.push_back(len);
        L.pitch.push_back(pitch);
        L.row_offset.push_back(off);
        off += pitch * r.desc.ndm;
        L.dm_trial_samples += len * r.desc.ndm;
    }
    L.dd_elems = off;
    int64_t ws = kErrBlock;
    for (int d : p.decs) {
        int64_t pitch = round_up(std::max<int64_t>(nsamp / d, 1), 64);
        L.dec_pitch.push_back(pitch);
        L.dec_offset.push_back(ws);
        ws += round_up((int64_t)p.nchans * pitch * 2, 256);
    }
    for (size_t q = 0; q < p.ranges.size(); ++q) {
        const RangePlan& r = p.ranges[q];
        if (r.strategy != 2) {
            L.sub_offset.push_back(-1);
            L.sub_pitch.push_back(0);
            L.sub_len.push_back(0);
            continue;
        }
        const int64_t len1 = std::max<int64_t>(0, nsamp / r.desc.dec - r.sb.rmax);
        const int64_t pitch = round_up(std::max<int64_t>(len1, 1), 64);
        L.sub_offset.push_back(ws);
        L.sub_pitch.push_back(pitch);
        L.sub_len.push_back(len1);
        ws += round_up((int64_t)r.sb.nsub * r.sb.ncoarse * pitch * 2, 256);
    }
    for (size_t q = 0; q < p.ranges.size(); ++q) {
        const RangePlan& r = p.ranges[q];
        if (r.strategy != 3) continue;
        L.fdmt_pitch = std::max(L.fdmt_pitch, round_up(std::max<int64_t>(nsamp / r.desc.dec, 1), 64));
        L.fdmt_rows = std::max<int64_t>(L.fdmt_rows, r.fd.max_rows);
    }
    if (L.fdmt_rows > 0) {  // two 32-bit depth buffers shared by the FDMT ranges
        L.fdmt_offset = ws;
        ws += 2 * round_up(L.fdmt_rows * L.fdmt_pitch * 4, 256);
    }
    L.dedisp_ws = ws;  // always holds at least the error word
    L.max_width = max_width;
    if (max_width > 0) {
        L.wpad = (int32_t)round_up(max_width, kSpsSlots);
        int64_t s = kErrBlock;
        s += round_up((int64_t)L.wpad * 8, 256);  // 1/sqrt(w) table
        L.stats_offset = s;
        s += round_up((int64_t)p.ndm_total * (int64_t)sizeof(RowStats), 256);
        L.table_offset = s;
        s += round_up((int64_t)p.ndm_total * L.wpad * 8, 256);
        int64_t chunks = 0;
        for (size_t r = 0; r < p.ranges.size(); ++r)
            chunks += (int64_t)p.ranges[r].desc.ndm * ((L.length[r] + kSpsOwned - 1) / kSpsOwned);
        L.chunk_offset = s;
        L.chunk_cap = chunks;
        s += round_up(std::max<int64_t>(chunks, 1) * (int64_t)sizeof(CandChunk), 256);
        L.sps_ws = s;
    }
    {
        int64_t s = kErrBlock;  // loss accumulator (double) lives at offset 0
        L.f32_part_offset = s;
        s += round_up((int64_t)p.nchans * f32_adj_tiles(std::max<int64_t>(nsamp, 1)) * 4, 256);
        L.f32_resid_offset = s;
        int64_t maxpitch = 0;
        for (size_t r = 0; r < p.ranges.size(); ++r) maxpitch = std::max(maxpitch, L.pitch[r]);
        s += (int64_t)kF32Chunk * maxpitch * 4;
        L.f32_ws = s;
    }
    return L;
}

}  // namespace aa

using namespace aa;

// Upload every sub-band range's tables into one device block (the plan must
// be bound; the previous block is released).
static aa_status upload_subband(aa_plan* p) {
    // the same per-table rounding as the placement below
    auto table_bytes = [](size_t n) { return (size_t)round_up((int64_t)n * 4 + 256, 256); };
    size_t bytes = 0;
    for (const auto& r : p->ranges) {
        if (r.strategy == 2) bytes += table_bytes(r.sb.rel.size()) + table_bytes(r.sb.s2.size());
        if (r.strategy == 3) bytes += table_bytes(r.fd.rows.size() * 4);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    if (p->d_sub) {
        cudaFree(p->d_sub);
        p->d_sub = nullptr;
    }
    for (auto& r : p->ranges) {
        r.sb.d_rel = r.sb.d_s2 = nullptr;
        r.fd.d_rows = nullptr;
    }
    aa_status st = AA_OK;
    if (bytes) {
        void* mem = nullptr;
        cudaError_t e = cudaMalloc(&mem, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc(%zu) for sub-band / FDMT tables: %s", bytes, cudaGetErrorString(e));
            st = AA_ERR_NOMEM;
        } else {
            p->d_sub = mem;
            size_t off = 0;
            for (auto& r : p->ranges) {
                if (r.strategy == 3) {
                    r.fd.d_rows = reinterpret_cast<FdmtRow*>((char*)mem + off);
                    off += table_bytes(r.fd.rows.size() * 4);
                    if (e == cudaSuccess)
                        e = cudaMemcpy(r.fd.d_rows, r.fd.rows.data(), r.fd.rows.size() * sizeof(FdmtRow),
                                       cudaMemcpyHostToDevice);
                    continue;
                }
                if (r.strategy != 2) continue;
                r.sb.d_rel = reinterpret_cast<int32_t*>((char*)mem + off);
                off += table_bytes(r.sb.rel.size());
                r.sb.d_s2 = reinterpret_cast<int32_t*>((char*)mem + off);
                off += table_bytes(r.sb.s2.size());
                if (e == cudaSuccess)
                    e = cudaMemcpy(r.sb.d_rel, r.sb.rel.data(), r.sb.rel.size() * 4, cudaMemcpyHostToDevice);
                if (e == cudaSuccess)
                    e = cudaMemcpy(r.sb.d_s2, r.sb.s2.data(), r.sb.s2.size() * 4, cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) {
                set_error("upload of sub-band / FDMT tables: %s", cudaGetErrorString(e));
                st = AA_ERR_CUDA;
            }
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

extern "C" {

const char* aa_status_str(aa_status s) {
    switch (s) {
        case AA_OK: return "AA_OK";
        case AA_PENDING: return "AA_PENDING";
        case AA_WARN_CAND_OVERFLOW: return "AA_WARN_CAND_OVERFLOW";
        case AA_ERR_CONFIG: return "AA_ERR_CONFIG";
        case AA_ERR_NOMEM: return "AA_ERR_NOMEM";
        case AA_ERR_CUDA: return "AA_ERR_CUDA";
        case AA_ERR_TIMEOUT: return "AA_ERR_TIMEOUT";
        case AA_ERR_STATE: return "AA_ERR_STATE";
        case AA_ERR_ARG: return "AA_ERR_ARG";
    }
    return "AA_UNKNOWN_STATUS";
}

const char* aa_last_error(void) { return g_last_error.c_str(); }

aa_status aa_plan_create(const aa_plan_desc* d, aa_plan** out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return AA_ERR_ARG; }
    *out = nullptr;
    if (!d) { set_error("desc is NULL"); return AA_ERR_ARG; }
    if (d->nchans < 1) { set_error("nchans must be >= 1 (got %d)", d->nchans); return AA_ERR_CONFIG; }
    if (!(d->tsamp_s > 0) || !std::isfinite(d->tsamp_s)) { set_error("tsamp must be > 0"); return AA_ERR_CONFIG; }
    if (!(d->foff_mhz != 0) || !std::isfinite(d->foff_mhz)) { set_error("foff must be non-zero"); return AA_ERR_CONFIG; }
    if (!(d->fch1_mhz > 0) || !std::isfinite(d->fch1_mhz)) { set_error("fch1 must be > 0"); return AA_ERR_CONFIG; }
    double f_last = d->fch1_mhz + (double)(d->nchans - 1) * d->foff_mhz;
    if (!(f_last > 0)) { set_error("lowest channel frequency %g MHz is not positive", f_last); return AA_ERR_CONFIG; }
    if (d->nranges < 1 || d->nranges > 64) { set_error("nranges must be in [1, 64] (got %d)", d->nranges); return AA_ERR_CONFIG; }
    if (!d->ranges) { set_error("ranges is NULL"); return AA_ERR_ARG; }
    int max_dec = 1;
    int64_t ndm_total = 0;
    for (int r = 0; r < d->nranges; ++r) {
        const aa_dm_range& g = d->ranges[r];
        if (g.ndm < 1) { set_error("range %d: ndm must be >= 1", r); return AA_ERR_CONFIG; }
        if (g.dec < 1 || g.dec > 16) { set_error("range %d: dec must be in [1, 16] (got %d)", r, g.dec); return AA_ERR_CONFIG; }
        if (!(g.dm_lo >= 0) || !(g.dm_step >= 0) || !std::isfinite(g.dm_lo) || !std::isfinite(g.dm_step)) {
            set_error("range %d: dm_lo and dm_step must be finite and >= 0", r);
            return AA_ERR_CONFIG;
        }
        max_dec = std::max(max_dec, g.dec);
        ndm_total += g.ndm;
    }
    if (ndm_total > (1 << 24)) { set_error("too many DM trials (%lld)", (long long)ndm_total); return AA_ERR_CONFIG; }
    if ((int64_t)d->nchans * 255 * max_dec >= (1 << 24)) {
        set_error("nchans*255*dec = %lld >= 2^24: sums would not be exact in FP32",
                  (long long)d->nchans * 255 * max_dec);
        return AA_ERR_CONFIG;
    }
    aa_plan* p = new (std::nothrow) aa_plan();
    if (!p) return AA_ERR_NOMEM;
    try {
        p->nchans = d->nchans;
        p->fch1 = d->fch1_mhz;
        p->foff = d->foff_mhz;
        p->tsamp = d->tsamp_s;
        p->f_top = f_last > d->fch1_mhz ? f_last : d->fch1_mhz;
        int32_t off = 0;
        for (int r = 0; r < d->nranges; ++r) {
            RangePlan rp;
            rp.desc = d->ranges[r];
            rp.dm_offset = off;
            off += rp.desc.ndm;
            rp.shifts.resize((size_t)rp.desc.ndm * p->nchans);
            int32_t ms = 0;
            for (int i = 0; i < rp.desc.ndm; ++i) {
                double dm = rp.desc.dm_lo + (double)i * rp.desc.dm_step;
                p->dm_max = std::max(p->dm_max, dm);
                for (int c = 0; c < p->nchans; ++c) {
                    int32_t s = delay_samples(p->fch1, p->foff, p->f_top, c, p->tsamp, dm, rp.desc.dec);
                    rp.shifts[(size_t)i * p->nchans + c] = s;
                    ms = std::max(ms, s);
                }
            }
            rp.maxshift = ms;
            p->ranges.push_back(std::move(rp));
        }
        p->ndm_total = off;
    } catch (const std::bad_alloc&) {
        delete p;
        set_error("host allocation failed");
        return AA_ERR_NOMEM;
    }
    aa_status st = build_strategy(*p);
    if (st != AA_OK) { delete p; return st; }
    for (auto& r : p->ranges) {
        p->table_bytes += round_up((int64_t)r.shifts.size() * 4, 256);
        p->table_bytes += round_up((int64_t)r.grec.size() * sizeof(GroupRec), 256);
        p->table_bytes += round_up((int64_t)r.gdesc.size() * sizeof(GroupDesc), 256);
        p->table_bytes += round_up((int64_t)r.gmem.size() * sizeof(GroupMember), 256);
    }
    *out = p;
    return AA_OK;
}

void aa_plan_destroy(aa_plan* p) {
    if (!p) return;
    if (p->d_tables || p->d_sub) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(p->device);
        if (p->d_tables) cudaFree(p->d_tables);
        if (p->d_sub) cudaFree(p->d_sub);
        if (prev >= 0) cudaSetDevice(prev);
    }
    delete p;
}

aa_status aa_plan_bind(aa_plan* p, int device) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (p->ready) {
        if (p->device == device) return AA_OK;
        set_error("plan already bound to device %d", p->device);
        return AA_ERR_STATE;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { set_error("cudaSetDevice(%d): %s", device, cudaGetErrorString(e)); return AA_ERR_CUDA; }
    void* mem = nullptr;
    e = cudaMalloc(&mem, p->table_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0) cudaSetDevice(prev);
        set_error("cudaMalloc(%zu) for delay tables: %s", p->table_bytes, cudaGetErrorString(e));
        return AA_ERR_NOMEM;
    }
    size_t off = 0;
    auto upload = [&](const void* src, size_t bytes) -> char* {
        char* dst = (char*)mem + off;
        off += round_up((int64_t)bytes, 256);
        if (bytes && e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
        return dst;
    };
    for (auto& r : p->ranges) {
        r.d_shifts = (int32_t*)upload(r.shifts.data(), r.shifts.size() * 4);
        r.d_grec = (GroupRec*)upload(r.grec.data(), r.grec.size() * sizeof(GroupRec));
        r.d_gdesc = (GroupDesc*)upload(r.gdesc.data(), r.gdesc.size() * sizeof(GroupDesc));
        r.d_gmem = (GroupMember*)upload(r.gmem.data(), r.gmem.size() * sizeof(GroupMember));
        if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
        cudaFree(mem);
        for (auto& r : p->ranges) {
            r.d_shifts = nullptr;
            r.d_grec = nullptr;
            r.d_gdesc = nullptr;
            r.d_gmem = nullptr;
        }
        if (prev >= 0) cudaSetDevice(prev);
        set_error("delay table upload: %s", cudaGetErrorString(e));
        return AA_ERR_CUDA;
    }
    p->d_tables = mem;
    p->device = device;
    p->ready = true;
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    for (const auto& r : p->ranges)
        if (r.strategy == 2 || r.strategy == 3) return upload_subband(p);
    return AA_OK;
}

aa_status aa_plan_query(const aa_plan* p, int64_t nsamp, int32_t max_width, aa_plan_info* info) {
    clear_error();
    if (!p || !info) { set_error("plan/info is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    if (max_width < 0 || max_width > 65535) { set_error("max_width must be in [0, 65535]"); return AA_ERR_ARG; }
    Layout L = make_layout(*p, nsamp, max_width);
    std::memset(info, 0, sizeof *info);
    info->nchans = p->nchans;
    info->nranges = (int32_t)p->ranges.size();
    info->ndm_total = p->ndm_total;
    info->ready = p->ready ? 1 : 0;
    info->device = p->device;
    info->max_width = max_width;
    info->nsamp = nsamp;
    info->in_pitch_min = L.in_pitch_min;
    info->dd_elems = L.dd_elems;
    info->dedisp_ws_bytes = L.dedisp_ws;
    info->sps_ws_bytes = L.sps_ws;
    info->table_bytes = (int64_t)p->table_bytes;
    info->host_path_bytes = (int64_t)p->nchans * L.in_pitch_min + L.dedisp_ws + L.dd_elems * 4 +
                            L.sps_ws + 256;
    info->dm_trial_samples = L.dm_trial_samples;
    info->dm_max = p->dm_max;
    info->f32_ws_bytes = L.f32_ws;
    return AA_OK;
}

aa_status aa_plan_range(const aa_plan* p, int64_t nsamp, int32_t r, aa_range_info* info) {
    clear_error();
    if (!p || !info) { set_error("plan/info is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    Layout L = make_layout(*p, nsamp, 0);
    const RangePlan& g = p->ranges[r];
    info->ndm = g.desc.ndm;
    info->dec = g.desc.dec;
    info->maxshift = g.maxshift;
    info->dm_offset = g.dm_offset;
    info->dm_lo = g.desc.dm_lo;
    info->dm_step = g.desc.dm_step;
    info->nsamp_dec = L.nsamp_dec[r];
    info->length = L.length[r];
    info->pitch = L.pitch[r];
    info->row_offset = L.row_offset[r];
    info->tile_dms = kDmPerBlock;
    info->tile_samples = kTau;
    info->stage_channels = g.cc;
    info->stages = g.nstage;
    info->span_max = g.span_max;
    info->smem_bytes = (int32_t)(g.strategy == 1 ? g.gsmem : g.smem);
    if (g.strategy == 1) {
        info->stage_channels = g.gcc;
        info->stages = 2;
        info->tile_samples = kGroupTau;
    }
    if (g.strategy == 2) {
        info->stage_channels = g.sb.shape1.cc;
        info->stages = g.sb.shape1.nstage;
        int swin = 0, nbc = 0;
        info->smem_bytes = (int32_t)std::max(g.sb.shape1.smem, subband_stage2_smem(g.sb.nsub, g.sb.span2, swin, nbc));
        info->maxshift = g.sb.rmax + g.sb.s2max;
    }
    info->strategy = g.strategy;
    info->grouped_available = g.grouped_ok ? 1 : 0;
    info->grouped_work = g.gwork;
    info->subband_channels = g.strategy == 2 ? g.sb.k : 0;
    info->subband_coarse_trials = g.strategy == 2 ? g.sb.m : 0;
    info->subband_work = g.strategy == 2 ? g.sb.work : 0.0;
    info->fdmt_depths = g.strategy == 3 ? g.fd.depths : 0;
    info->fdmt_max_rows = g.strategy == 3 ? g.fd.max_rows : 0;
    info->fdmt_work = g.strategy == 3 ? g.fd.work : 0.0;
    return AA_OK;
}

aa_status aa_plan_set_strategy(aa_plan* p, int32_t r, int32_t strategy) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    if (strategy != AA_DEDISP_DIRECT && strategy != AA_DEDISP_GROUPED) {
        set_error("unknown strategy %d", strategy);
        return AA_ERR_ARG;
    }
    RangePlan& g = p->ranges[r];
    if (strategy == AA_DEDISP_GROUPED && !g.grouped_ok) {
        set_error("range %d: the grouped strategy is not available (delay span %d)", r, g.span_max);
        return AA_ERR_CONFIG;
    }
    g.strategy = strategy;
    return AA_OK;
}

aa_status aa_plan_set_sps_clip(aa_plan* p, int32_t c16, int32_t max_iters) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (max_iters < 0 || max_iters > 64) { set_error("max_iters %d outside [0, 64]", max_iters); return AA_ERR_ARG; }
    if (max_iters > 0 && (c16 < 1 || c16 > 255)) { set_error("c16 %d outside [1, 255]", c16); return AA_ERR_ARG; }
    p->clip_c16 = max_iters > 0 ? c16 : 0;
    p->clip_iters = max_iters;
    return AA_OK;
}

aa_status aa_plan_set_sps_ladder(aa_plan* p, int32_t growth_x16) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (growth_x16 != 0 && (growth_x16 < 17 || growth_x16 > 64)) {
        set_error("growth_x16 %d: 0 or within [17, 64]", growth_x16);
        return AA_ERR_ARG;
    }
    if (growth_x16 != 0 && p->dec_w0 != 0) {
        set_error("the decimated width ladder is on: switch it off first");
        return AA_ERR_CONFIG;
    }
    p->ladder_g16 = growth_x16;
    return AA_OK;
}

aa_status aa_plan_set_sps_decimated(aa_plan* p, int32_t base_widths) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (base_widths != 0 && (base_widths < 16 || base_widths > 256 || (base_widths & (base_widths - 1)))) {
        set_error("base_widths %d: 0 or a power of two within [16, 256]", base_widths);
        return AA_ERR_ARG;
    }
    if (base_widths != 0 && p->ladder_g16 != 0) {
        set_error("the sparse width ladder is on: switch it off first");
        return AA_ERR_CONFIG;
    }
    p->dec_w0 = base_widths;
    return AA_OK;
}

aa_status aa_plan_set_subband(aa_plan* p, int32_t r, int32_t band_channels, int32_t coarse_trials) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    RangePlan& g = p->ranges[r];
    const int C = p->nchans, dec = g.desc.dec, ndm = g.desc.ndm;
    if (band_channels < 1 || band_channels > C) {
        set_error("band_channels %d outside [1, %d]", band_channels, C);
        return AA_ERR_ARG;
    }
    if (coarse_trials < 1 || coarse_trials > kDmPerBlock) {
        set_error("coarse_trials %d outside [1, %d]", coarse_trials, kDmPerBlock);
        return AA_ERR_ARG;
    }
    if ((int64_t)band_channels * 255 * dec > 65535) {
        set_error("band of %d channels at decimation %d: partial sums exceed 16 bits "
                  "(band_channels * 255 * dec must be <= 65535)", band_channels, dec);
        return AA_ERR_CONFIG;
    }
    SubbandPlan sb;
    sb.k = band_channels;
    sb.m = coarse_trials;
    sb.nsub = (C + sb.k - 1) / sb.k;
    sb.ncoarse = (ndm + sb.m - 1) / sb.m;
    std::vector<int32_t> cref(sb.nsub);
    for (int b = 0; b < sb.nsub; ++b) {
        const int c0 = b * sb.k, c1 = std::min(C, c0 + sb.k) - 1;
        cref[b] = p->foff < 0 ? c0 : c1;  // the band's highest frequency
    }
    // stage 1: delay of every channel relative to its band's reference, at
    // the middle fine trial of each coarse trial
    sb.rel.assign((size_t)sb.ncoarse * C, 0);
    int32_t span1 = 0;
    size_t off = 0;
    for (int b = 0; b < sb.nsub; ++b) {
        const int c0 = b * sb.k, kb = std::min(C, c0 + sb.k) - c0;
        for (int j = 0; j < sb.ncoarse; ++j) {
            const int nj = std::min(sb.m, ndm - j * sb.m);
            const int ij = j * sb.m + (nj - 1) / 2;
            const double dm = g.desc.dm_lo + (double)ij * g.desc.dm_step;
            for (int cl = 0; cl < kb; ++cl) {
                const int32_t v = rel_delay_samples(p->fch1, p->foff, p->f_top, c0 + cl, cref[b], p->tsamp, dm, dec);
                sb.rel[off + (size_t)j * kb + cl] = v;
                sb.rmax = std::max(sb.rmax, v);
            }
        }
        for (int j0 = 0; j0 < sb.ncoarse; j0 += kDmPerBlock) {
            const int j1 = std::min(sb.ncoarse, j0 + kDmPerBlock) - 1;
            for (int cl = 0; cl < kb; ++cl)
                span1 = std::max(span1, sb.rel[off + (size_t)j1 * kb + cl] - sb.rel[off + (size_t)j0 * kb + cl]);
        }
        off += (size_t)sb.ncoarse * kb;
    }
    // stage 2: the reference channels' own delays at every fine trial
    sb.s2.assign((size_t)ndm * sb.nsub, 0);
    int32_t span2 = 0;
    for (int i = 0; i < ndm; ++i)
        for (int b = 0; b < sb.nsub; ++b) {
            const int32_t v = g.shifts[(size_t)i * C + cref[b]];
            sb.s2[(size_t)i * sb.nsub + b] = v;
            sb.s2max = std::max(sb.s2max, v);
        }
    for (int j = 0; j < sb.ncoarse; ++j) {
        const int i0 = j * sb.m, i1 = std::min(ndm, i0 + sb.m) - 1;
        for (int b = 0; b < sb.nsub; ++b)
            span2 = std::max(span2, sb.s2[(size_t)i1 * sb.nsub + b] - sb.s2[(size_t)i0 * sb.nsub + b]);
    }
    if (!direct_shape(g.elem, span1, 255 * dec, sb.shape1)) {
        set_error("range %d: sub-band stage 1 does not fit the dedispersion tile (span %d)", r, span1);
        return AA_ERR_CONFIG;
    }
    sb.span2 = span2;
    sb.work = ((double)sb.ncoarse * C + (double)ndm * sb.nsub) / ((double)ndm * C);
    const SubbandPlan old = g.sb;
    const int old_strategy = g.strategy;
    g.sb = std::move(sb);
    g.strategy = 2;
    if (p->ready) {
        const aa_status st = upload_subband(p);
        if (st != AA_OK) {
            g.sb = old;
            g.strategy = old_strategy;
            upload_subband(p);
            return st;
        }
    }
    return AA_OK;
}

aa_status aa_plan_set_fdmt(aa_plan* p, int32_t r) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    RangePlan& g = p->ranges[r];
    const int32_t C = p->nchans, ndm = g.desc.ndm;
    if (C < 2) { set_error("the FDMT tree needs at least two channels"); return AA_ERR_CONFIG; }
    if ((int64_t)C * 255 * g.desc.dec >= (int64_t(1) << 31)) {
        set_error("range %d: sums of %d channels at decimation %d exceed 31 bits", r, C, g.desc.dec);
        return AA_ERR_CONFIG;
    }
    // channels in falling-frequency order and their f^-2 - f_top^-2, in the
    // operation order of the plan's delays
    std::vector<double> dk((size_t)C);
    std::vector<int32_t> chan((size_t)C);
    for (int32_t k = 0; k < C; ++k) {
        const int32_t c = p->foff < 0 ? k : C - 1 - k;
        const double fc = p->fch1 + (double)c * p->foff;
        chan[(size_t)k] = c;
        dk[(size_t)k] = 1.0 / (fc * fc) - 1.0 / (p->f_top * p->f_top);
    }
    // split of subband [a, b] at delay delta: (upper delay, gap, lower delay)
    auto split = [&](int32_t a, int32_t b, int64_t delta, int32_t& m, int64_t& du, int64_t& gap) {
        m = a + (b - a + 2) / 2;
        const double span = dk[(size_t)b] - dk[(size_t)a];
        gap = span > 0.0 ? llround((double)delta * (dk[(size_t)m] - dk[(size_t)a]) / span) : 0;
        du = span > 0.0 ? llround((double)delta * (dk[(size_t)m - 1] - dk[(size_t)a]) / span) : 0;
    };
    const int32_t bottom = p->foff < 0 ? C - 1 : 0;
    struct Node { int32_t a, b; int64_t lo, hi; int32_t row0; };
    FdmtPlan fd;
    // depth by depth from the root: the delays each node must provide (a
    // contiguous range covering what its parent reads)
    std::vector<std::vector<Node>> depth;
    std::vector<int64_t> rootD((size_t)ndm);
    for (int32_t i = 0; i < ndm; ++i) rootD[(size_t)i] = g.shifts[(size_t)i * C + bottom];
    std::vector<Node> cur;
    if (ndm > 0 && C > 1) {
        const int64_t lo = *std::min_element(rootD.begin(), rootD.end());
        const int64_t hi = *std::max_element(rootD.begin(), rootD.end());
        cur.push_back(Node{0, C - 1, lo, hi, 0});
    }
    // children of a node for the delays [lo, hi] it provides; leaves are not nodes
    auto children = [&](const Node& n, std::vector<Node>& out) {
        int32_t m;
        int64_t du, gap;
        int64_t ulo = INT64_MAX, uhi = INT64_MIN, llo = INT64_MAX, lhi = INT64_MIN;
        for (int64_t d = n.lo; d <= n.hi; ++d) {
            split(n.a, n.b, d, m, du, gap);
            ulo = std::min(ulo, du);
            uhi = std::max(uhi, du);
            llo = std::min(llo, d - gap);
            lhi = std::max(lhi, d - gap);
        }
        split(n.a, n.b, n.lo, m, du, gap);
        if (m - 1 > n.a) out.push_back(Node{n.a, m - 1, ulo, uhi, 0});
        if (n.b > m) out.push_back(Node{m, n.b, llo, lhi, 0});
    };
    while (!cur.empty()) {
        depth.push_back(cur);
        std::vector<Node> nxt;
        for (const Node& n : cur) children(n, nxt);
        cur.swap(nxt);
    }
    fd.depths = (int)depth.size();
    // rows of each depth (the root's: one per trial)
    std::vector<int32_t> nrows(depth.size(), 0);
    for (size_t d = 1; d < depth.size(); ++d)
        for (Node& n : depth[d]) {
            n.row0 = nrows[d];
            nrows[d] += (int32_t)(n.hi - n.lo + 1);
        }
    if (!depth.empty()) nrows[0] = ndm;
    // node of each depth by its first channel (the subbands of a depth are disjoint)
    std::vector<std::vector<int32_t>> at(depth.size(), std::vector<int32_t>((size_t)C, -1));
    for (size_t d = 0; d < depth.size(); ++d)
        for (size_t j = 0; j < depth[d].size(); ++j) at[d][(size_t)depth[d][j].a] = (int32_t)j;
    // reference to the row providing subband [a, b] at delay delta, one depth deeper
    auto ref = [&](size_t d, int32_t a, int32_t b, int64_t delta) -> int32_t {
        if (a == b) return -(chan[(size_t)a] + 1);  // leaf: the channel's own row (delay 0)
        const int32_t j = d + 1 < depth.size() ? at[d + 1][(size_t)a] : -1;
        if (j < 0 || depth[d + 1][(size_t)j].b != b) return INT32_MIN;  // unreachable
        const Node& n = depth[d + 1][(size_t)j];
        if (delta < n.lo || delta > n.hi) return INT32_MIN;
        return n.row0 + (int32_t)(delta - n.lo);
    };
    fd.first.assign(depth.size() + 1, 0);
    for (size_t q = 0; q < depth.size(); ++q) {  // deepest first
        const size_t d = depth.size() - 1 - q;
        fd.first[q] = (int64_t)fd.rows.size();
        auto emit = [&](const Node& n, int64_t delta) {
            int32_t m;
            int64_t du, gap;
            split(n.a, n.b, delta, m, du, gap);
            FdmtRow row{ref(d, n.a, m - 1, du), ref(d, m, n.b, delta - gap), (int32_t)gap, (int32_t)delta};
            fd.rows.push_back(row);
        };
        if (d == 0) {
            for (int32_t i = 0; i < ndm; ++i) emit(depth[0][0], rootD[(size_t)i]);
        } else {
            for (const Node& n : depth[d])
                for (int64_t delta = n.lo; delta <= n.hi; ++delta) emit(n, delta);
            fd.max_rows = std::max(fd.max_rows, nrows[d]);
        }
    }
    fd.first[depth.size()] = (int64_t)fd.rows.size();
    for (const FdmtRow& row : fd.rows)
        if (row.u == INT32_MIN || row.l == INT32_MIN) {
            set_error("internal: FDMT tree reference missing");
            return AA_ERR_STATE;
        }
    fd.work = ndm > 0 ? (double)fd.rows.size() / ((double)ndm * C) : 1.0;
    const FdmtPlan old = g.fd;
    const int old_strategy = g.strategy;
    g.fd = std::move(fd);
    g.strategy = 3;
    if (p->ready) {
        const aa_status st = upload_subband(p);
        if (st != AA_OK) {
            g.fd = old;
            g.strategy = old_strategy;
            upload_subband(p);
            return st;
        }
    }
    return AA_OK;
}

aa_status aa_plan_effective_shifts(const aa_plan* p, int32_t r, int32_t* out, int64_t cap) {
    clear_error();
    if (!p || !out) { set_error("plan/out is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    const RangePlan& g = p->ranges[r];
    const int32_t C = p->nchans, ndm = g.desc.ndm;
    if (cap < (int64_t)ndm * C) { set_error("capacity %lld < %lld", (long long)cap, (long long)ndm * C); return AA_ERR_ARG; }
    if (g.strategy == 2) {  // reference channel's delay + the channel's within its band
        const SubbandPlan& sb = g.sb;
        for (int32_t i = 0; i < ndm; ++i) {
            const int32_t j = i / sb.m;
            size_t off = 0;
            for (int b = 0; b < sb.nsub; ++b) {
                const int c0 = b * sb.k, kb = std::min(C, c0 + sb.k) - c0;
                for (int cl = 0; cl < kb; ++cl)
                    out[(int64_t)i * C + c0 + cl] = sb.s2[(size_t)i * sb.nsub + b] + sb.rel[off + (size_t)j * kb + cl];
                off += (size_t)sb.ncoarse * kb;
            }
        }
        return AA_OK;
    }
    if (g.strategy == 3) {  // walk the tree from each trial's root row
        const FdmtPlan& fd = g.fd;
        // rows of depth d start at fd.first[depths - 1 - d]
        auto walk = [&](auto&& self, int d, int32_t row, int64_t base, int32_t* e) -> void {
            const FdmtRow& x = fd.rows[(size_t)(fd.first[(size_t)(fd.depths - 1 - d)] + row)];
            for (int half = 0; half < 2; ++half) {
                const int32_t ref = half ? x.l : x.u;
                const int64_t b = base + (half ? x.gap : 0);
                if (ref < 0) e[-(ref + 1)] = (int32_t)b;
                else self(self, d + 1, ref, b, e);
            }
        };
        for (int32_t i = 0; i < ndm; ++i) walk(walk, 0, i, 0, out + (int64_t)i * C);
        return AA_OK;
    }
    std::memcpy(out, g.shifts.data(), g.shifts.size() * 4);
    return AA_OK;
}

aa_status aa_plan_shifts(const aa_plan* p, int32_t r, int32_t* out, int64_t cap) {
    clear_error();
    if (!p || !out) { set_error("plan/out is NULL"); return AA_ERR_ARG; }
    if (r < 0 || r >= (int32_t)p->ranges.size()) { set_error("range %d out of bounds", r); return AA_ERR_ARG; }
    const auto& s = p->ranges[r].shifts;
    if (cap < (int64_t)s.size()) { set_error("capacity %lld < %zu", (long long)cap, s.size()); return AA_ERR_ARG; }
    std::memcpy(out, s.data(), s.size() * 4);
    return AA_OK;
}

}  // extern "C"

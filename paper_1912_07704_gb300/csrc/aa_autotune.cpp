// Autotuner for the dedispersion tile: for every range of a bound plan, time
// the kernel over a synthetic probe input for the grouped strategy (when the
// plan built its tables) and each feasible direct stage shape (channels per
// shared-memory stage x pipeline depth), and keep the fastest.  Results can
// be cached in a text file keyed by the GPU and the range's shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "aa_internal.h"

using namespace aa;

namespace aa {
size_t dedisp_smem_bytes(const RangePlan& r, int cc, int nstage);
}

namespace {

std::string cache_key(const cudaDeviceProp& prop, const aa_plan& p, const RangePlan& r) {
    std::ostringstream k;
    std::string name = prop.name;
    std::replace(name.begin(), name.end(), ' ', '_');
    k << name << ";sm=" << prop.multiProcessorCount << ";C=" << p.nchans << ";dec=" << r.desc.dec
      << ";rw=" << r.rw << ";ndm=" << std::min(r.desc.ndm, kDmPerBlock * 64)
      << ";dmstep=" << r.desc.dm_step << ";dmlo=" << r.desc.dm_lo;
    return k.str();
}

struct Choice {
    int strategy, cc, ns;
};

// Lines: key strategy cc nstage ms
std::map<std::string, Choice> read_cache(const char* path) {
    std::map<std::string, Choice> m;
    if (!path) return m;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string key;
        Choice c{};
        double ms;
        if (in >> key >> c.strategy >> c.cc >> c.ns >> ms) m[key] = c;
    }
    return m;
}

}  // namespace

extern "C" aa_status aa_plan_autotune(aa_plan* p, int64_t nsamp_probe, const char* cache_path) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (!p->ready) { set_error("bind the plan before tuning it"); return AA_ERR_STATE; }
    if (nsamp_probe <= 0) { set_error("nsamp_probe must be > 0"); return AA_ERR_ARG; }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) { set_error("current device differs from the plan's device"); return AA_ERR_STATE; }
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { set_error("cudaGetDeviceProperties failed"); return AA_ERR_CUDA; }
    auto cache = read_cache(cache_path);
    std::vector<std::string> new_lines;
    const Layout L = make_layout(*p, nsamp_probe, 0);
    // one probe buffer large enough for the raw input and any decimated input
    size_t bytes = 0;
    for (size_t r = 0; r < p->ranges.size(); ++r)
        bytes = std::max(bytes, (size_t)p->nchans * (size_t)round_up(std::max<int64_t>(L.nsamp_dec[r], 1), 64) * 2);
    bytes = std::max(bytes, (size_t)p->nchans * (size_t)L.in_pitch_min);
    size_t out_bytes = 0;
    for (size_t r = 0; r < p->ranges.size(); ++r)
        out_bytes = std::max(out_bytes, (size_t)(L.pitch[r] * p->ranges[r].desc.ndm * 4));
    void* probe = nullptr;
    void* out = nullptr;
    unsigned* err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    aa_status status = AA_OK;
    if (cudaMalloc(&probe, bytes) != cudaSuccess || cudaMalloc(&out, std::max<size_t>(out_bytes, 256)) != cudaSuccess ||
        cudaMalloc(&err, 256) != cudaSuccess) {
        cudaGetLastError();
        set_error("autotune probe allocation failed");
        status = AA_ERR_NOMEM;
    }
    if (status == AA_OK) {
        cudaMemset(probe, 0x35, bytes);  // the kernel's speed does not depend on the values
        cudaMemset(err, 0, 256);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    for (size_t r = 0; status == AA_OK && r < p->ranges.size(); ++r) {
        RangePlan& g = p->ranges[r];
        if (L.length[r] <= 0 || g.strategy == 2) continue;  // sub-band ranges keep their shape
        const std::string key = cache_key(prop, *p, g);
        int best_cc = g.cc, best_ns = g.nstage, best_strategy = g.strategy;
        auto hit = cache.find(key);
        if (hit != cache.end() && (hit->second.strategy == 0 || g.grouped_ok)) {
            best_strategy = hit->second.strategy;
            best_cc = hit->second.cc;
            best_ns = hit->second.ns;
        } else {
            const int max_flush = 65535 / (255 * g.desc.dec);
            float best_ms = 1e30f;
            // candidate list: the grouped strategy first (cc = 0), then the direct shapes
            std::vector<std::pair<int, int>> shapes;
            if (g.grouped_ok) shapes.push_back({0, 0});
            for (int ns : {2, 3})
                for (int cc : {8, 12, 16, 20, 24, 32}) shapes.push_back({cc, ns});
            for (const auto& shape : shapes) {
                {
                    const int cc = shape.first, ns = shape.second;
                    const bool grouped = cc == 0;
                    if (!grouped && (cc > max_flush || kDmPerBlock * cc > kDedispThreads)) continue;
                    const size_t smem = grouped ? g.gsmem : dedisp_smem_bytes(g, cc, ns);
                    if (smem > 227 * 1024) continue;
                    DedispArgs a{};
                    a.in = probe;
                    a.in_pitch = g.elem == 1 ? L.in_pitch_min : round_up(std::max<int64_t>(L.nsamp_dec[r], 1), 64);
                    a.nchans = p->nchans;
                    a.nsamp = L.nsamp_dec[r];
                    a.length = L.length[r];
                    a.ndm = g.desc.ndm;
                    a.shifts = g.d_shifts;
                    a.out = static_cast<float*>(out);
                    a.out_pitch = L.pitch[r];
                    const int saved = g.strategy;
                    g.strategy = grouped ? 1 : 0;
                    fill_strategy(a, g);
                    g.strategy = saved;
                    if (!grouped) {
                        a.cc = cc;
                        a.nstage = ns;
                        a.flush = (std::min(max_flush, 256) / cc) * cc;
                        a.smem = smem;
                    }
                    a.err = err;
                    if (launch_dedisperse(a, nullptr) != cudaSuccess) { cudaGetLastError(); continue; }
                    cudaEventRecord(e0);
                    for (int it = 0; it < 3; ++it) launch_dedisperse(a, nullptr);
                    cudaEventRecord(e1);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_strategy = grouped ? 1 : 0;
                        if (!grouped) {
                            best_cc = cc;
                            best_ns = ns;
                        }
                    }
                }
            }
            std::ostringstream line;
            line << key << " " << best_strategy << " " << best_cc << " " << best_ns << " " << best_ms / 3;
            new_lines.push_back(line.str());
        }
        g.strategy = best_strategy;
        g.cc = best_cc;
        g.nstage = best_ns;
        g.flush = (std::min(65535 / (255 * g.desc.dec), 256) / best_cc) * best_cc;
        g.smem = dedisp_smem_bytes(g, best_cc, best_ns);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (probe) cudaFree(probe);
    if (out) cudaFree(out);
    if (err) cudaFree(err);
    if (status == AA_OK && cache_path && !new_lines.empty()) {
        std::ofstream f(cache_path, std::ios::app);
        for (auto& l : new_lines) f << l << "\n";
    }
    return status;
}

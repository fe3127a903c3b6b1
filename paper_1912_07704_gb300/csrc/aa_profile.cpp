// Kernel timing: while enabled, every library kernel launch is bracketed by
// two CUDA events recorded on its own stream; aa_profile_read sums the
// elapsed times per kernel.  Disabled by default (no events recorded).
#include <mutex>
#include <vector>

#include "aa_internal.h"

namespace aa {

static const char* kKernelNames[kNumKernels] = {
    "decimate", "dedisperse_u8", "dedisperse_u16", "sps_rsqrt_table",
    "sps_stats", "sps_boxcar", "f32_forward", "f32_adjoint", "corner_turn", "sps_order", "peaks2d", "dedisperse_subband_stage1",
    "dedisperse_subband_stage2", "sps_finalize", "dedisperse_fdmt"};

namespace {
struct Pending {
    int kernel;
    cudaEvent_t start, stop;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
int64_t g_launches[kNumKernels] = {};
double g_ms[kNumKernels] = {};

cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            g_launches[p.kernel] += 1;
            g_ms[p.kernel] += ms;
        } else {
            cudaGetLastError();
        }
        g_free.push_back(p.start);
        g_free.push_back(p.stop);
    }
    g_pending.clear();
}
}  // namespace

ProfScope::ProfScope(int kernel, cudaStream_t s) : kernel_(kernel), stream_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    start_ = get_event();
    stop_ = get_event();
    if (start_ && stop_ && cudaEventRecord(start_, s) == cudaSuccess) {
        active_ = true;
    } else {
        cudaGetLastError();
        if (start_) g_free.push_back(start_);
        if (stop_) g_free.push_back(stop_);
    }
}

ProfScope::~ProfScope() {
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaEventRecord(stop_, stream_) == cudaSuccess) {
        g_pending.push_back({kernel_, start_, stop_});
    } else {
        cudaGetLastError();
        g_free.push_back(start_);
        g_free.push_back(stop_);
    }
}

}  // namespace aa

using namespace aa;

extern "C" {

aa_status aa_profile_enable(int32_t on) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_mu);
    if (on) {
        drain_locked();
        for (int k = 0; k < kNumKernels; ++k) {
            g_launches[k] = 0;
            g_ms[k] = 0.0;
        }
    }
    g_on = on != 0;
    return AA_OK;
}

aa_status aa_profile_read(int32_t kernel, int64_t* launches, double* total_ms) {
    clear_error();
    if (kernel < 0 || kernel >= kNumKernels) { set_error("kernel id %d out of range", kernel); return AA_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    if (launches) *launches = g_launches[kernel];
    if (total_ms) *total_ms = g_ms[kernel];
    return AA_OK;
}

const char* aa_profile_kernel_name(int32_t kernel) {
    if (kernel < 0 || kernel >= kNumKernels) return nullptr;
    return kKernelNames[kernel];
}

}  // extern "C"

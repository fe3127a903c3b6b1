// Entry points of the differentiable (float-weighted) form.
#include <algorithm>

#include "aa_internal.h"

using namespace aa;

namespace {

aa_status fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? AA_ERR_NOMEM : AA_ERR_CUDA;
}

#define AA_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return fail(e_, (what));  \
    } while (0)

aa_status check(const aa_plan* p, const float* x, int64_t nsamp, int64_t x_pitch, const float* w) {
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (!p->ready) { set_error("plan is not bound to a device (aa_plan_bind)"); return AA_ERR_STATE; }
    int dev = -1;
    AA_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->device) { set_error("current device differs from the plan's device"); return AA_ERR_STATE; }
    for (const auto& r : p->ranges)
        if (r.desc.dec != 1 || r.strategy == 2) {
            set_error("the differentiable form supports exact dec == 1 ranges only");
            return AA_ERR_CONFIG;
        }
    if (nsamp < 0 || x_pitch < nsamp) { set_error("bad nsamp/x_pitch"); return AA_ERR_ARG; }
    if (nsamp > 0 && (!x || !w)) { set_error("d_x and d_w must be non-NULL"); return AA_ERR_ARG; }
    return AA_OK;
}

F32FwdArgs fwd_args(const aa_plan* p, const Layout& L, size_t r, const float* x, int64_t nsamp,
                    int64_t x_pitch, const float* w) {
    const RangePlan& g = p->ranges[r];
    F32FwdArgs a{};
    a.x = x;
    a.x_pitch = x_pitch;
    a.nchans = p->nchans;
    a.nsamp = nsamp;
    a.w = w;
    a.shifts = g.d_shifts;
    a.d_begin = 0;
    a.d_end = g.desc.ndm;
    a.length = L.length[r];
    a.rowlen = f32_fwd_rowlen(g.f32_span);
    a.pitch = L.pitch[r];
    return a;
}

F32AdjArgs adj_args(const aa_plan* p, const Layout& L, size_t r, const float* x, int64_t nsamp,
                    int64_t x_pitch, const float* w, float* gx, float* gw, char* ws) {
    const RangePlan& g = p->ranges[r];
    F32AdjArgs a{};
    a.x = x;
    a.x_pitch = x_pitch;
    a.nchans = p->nchans;
    a.nsamp = nsamp;
    a.w = w;
    a.shifts = g.d_shifts;
    a.length = L.length[r];
    a.rowlen = f32_adj_rowlen(g.f32_cspan);
    a.gx = gx;
    a.gw = gw;
    a.gw_part = reinterpret_cast<float*>(ws + L.f32_part_offset);
    return a;
}

}  // namespace

extern "C" {

aa_status aa_dedisperse_f32_device(const aa_plan* p, const float* d_x, int64_t nsamp, int64_t x_pitch,
                                   const float* d_w, float* d_y, aa_stream_t stream) {
    clear_error();
    aa_status st = check(p, d_x, nsamp, x_pitch, d_w);
    if (st != AA_OK) return st;
    const Layout L = make_layout(*p, nsamp, 0);
    if (L.dm_trial_samples == 0) return AA_OK;
    if (!d_y) { set_error("d_y is NULL"); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (size_t r = 0; r < p->ranges.size(); ++r) {
        F32FwdArgs a = fwd_args(p, L, r, d_x, nsamp, x_pitch, d_w);
        a.y = d_y + L.row_offset[r];
        ProfScope prof(kKF32Fwd, s);
        AA_CUDA(launch_f32_forward(0, a, s), "f32 forward launch");
    }
    return AA_OK;
}

aa_status aa_dedisperse_f32_adjoint_device(const aa_plan* p, const float* d_x, int64_t nsamp,
                                           int64_t x_pitch, const float* d_w, const float* d_gy,
                                           float* d_gx, float* d_gw, void* d_ws, size_t ws_bytes,
                                           aa_stream_t stream) {
    clear_error();
    aa_status st = check(p, d_x, nsamp, x_pitch, d_w);
    if (st != AA_OK) return st;
    const Layout L = make_layout(*p, nsamp, 0);
    if (!d_gx || !d_gw || !d_ws) { set_error("d_gx, d_gw and d_ws must be non-NULL"); return AA_ERR_ARG; }
    if ((int64_t)ws_bytes < L.f32_ws) { set_error("workspace too small (%lld needed)", (long long)L.f32_ws); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AA_CUDA(cudaMemset2DAsync(d_gx, (size_t)x_pitch * 4, 0, (size_t)std::max<int64_t>(nsamp, 0) * 4,
                              p->nchans, s), "clear gx");
    AA_CUDA(cudaMemsetAsync(d_gw, 0, (size_t)p->nchans * 4, s), "clear gw");
    if (L.dm_trial_samples == 0) return AA_OK;
    if (!d_gy) { set_error("d_gy is NULL"); return AA_ERR_ARG; }
    for (size_t r = 0; r < p->ranges.size(); ++r) {
        if (L.length[r] <= 0) continue;
        F32AdjArgs a = adj_args(p, L, r, d_x, nsamp, x_pitch, d_w, d_gx, d_gw, static_cast<char*>(d_ws));
        a.d_begin = 0;
        a.d_end = p->ranges[r].desc.ndm;
        a.gy = d_gy + L.row_offset[r];
        a.gpitch = L.pitch[r];
        ProfScope prof(kKF32Adj, s);
        AA_CUDA(launch_f32_adjoint(a, s), "f32 adjoint launch");
    }
    return AA_OK;
}

aa_status aa_dedisperse_f32_mse_device(const aa_plan* p, const float* d_x, int64_t nsamp,
                                       int64_t x_pitch, const float* d_w, const float* d_tmpl,
                                       double* d_loss, float* d_gx, float* d_gw, void* d_ws,
                                       size_t ws_bytes, aa_stream_t stream) {
    clear_error();
    aa_status st = check(p, d_x, nsamp, x_pitch, d_w);
    if (st != AA_OK) return st;
    const Layout L = make_layout(*p, nsamp, 0);
    const bool grad = d_gx || d_gw;
    if (grad && !(d_gx && d_gw)) { set_error("pass both d_gx and d_gw, or neither"); return AA_ERR_ARG; }
    if (!d_loss || !d_ws) { set_error("d_loss and d_ws must be non-NULL"); return AA_ERR_ARG; }
    if ((int64_t)ws_bytes < L.f32_ws) { set_error("workspace too small (%lld needed)", (long long)L.f32_ws); return AA_ERR_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_ws);
    double* sum = reinterpret_cast<double*>(ws);
    AA_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), s), "clear loss");
    if (grad) {
        AA_CUDA(cudaMemset2DAsync(d_gx, (size_t)x_pitch * 4, 0, (size_t)std::max<int64_t>(nsamp, 0) * 4,
                                  p->nchans, s), "clear gx");
        AA_CUDA(cudaMemsetAsync(d_gw, 0, (size_t)p->nchans * 4, s), "clear gw");
    }
    const double n = (double)L.dm_trial_samples;
    if (L.dm_trial_samples > 0) {
        if (!d_tmpl) { set_error("d_template is NULL"); return AA_ERR_ARG; }
        float* resid = reinterpret_cast<float*>(ws + L.f32_resid_offset);
        for (size_t r = 0; r < p->ranges.size(); ++r) {
            if (L.length[r] <= 0) continue;
            F32FwdArgs a = fwd_args(p, L, r, d_x, nsamp, x_pitch, d_w);
            a.tmpl = d_tmpl + L.row_offset[r];
            a.loss_sum = sum;
            if (!grad) {
                ProfScope prof(kKF32Fwd, s);
                AA_CUDA(launch_f32_forward(1, a, s), "f32 loss launch");
                continue;
            }
            // chunks of trials: recompute y, form 2(y - T)/N, accumulate its transpose
            const int ndm = p->ranges[r].desc.ndm;
            for (int db = 0; db < ndm; db += kF32Chunk) {
                const int de = std::min(ndm, db + kF32Chunk);
                a.d_begin = db;
                a.d_end = de;
                a.resid = resid;
                a.rpitch = L.pitch[r];
                a.scale = (float)(2.0 / n);
                {
                    ProfScope prof(kKF32Fwd, s);
                    AA_CUDA(launch_f32_forward(2, a, s), "f32 residual launch");
                }
                F32AdjArgs b = adj_args(p, L, r, d_x, nsamp, x_pitch, d_w, d_gx, d_gw, ws);
                b.d_begin = db;
                b.d_end = de;
                b.gy = resid;
                b.gpitch = L.pitch[r];
                ProfScope prof(kKF32Adj, s);
                AA_CUDA(launch_f32_adjoint(b, s), "f32 adjoint launch");
            }
        }
    }
    AA_CUDA(launch_finish_loss(sum, n, d_loss, s), "finish loss");
    return AA_OK;
}

}  // extern "C"

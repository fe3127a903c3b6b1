// Differentiable form of the dedispersion (per-channel float weights):
//   forward  y[d][t]  = sum_c w[c] x[c][t + s(c,d)]              (FP32 FMA)
//   adjoint  gx[c][u] = w[c] A[c][u],  A[c][u] = sum_d gy[d][u - s(c,d)]
//            gw[c]    = sum_u x[c][u] A[c][u]       (= sum_{d,t} gy[d][t] x[c][t+s(c,d)])
// The MSE loss against a template, mean((y - T)^2), is reduced inside the
// forward; its gradient recomputes y one chunk of DM trials at a time (the
// full DM x time residual is never stored).  Dec-1 ranges only.
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr int FD = 16;   // DM trials per forward CTA
constexpr int FT = 256;  // output samples per forward CTA (16 per thread)
constexpr int FC = 16;   // channels per staging round
constexpr int AC = 16;   // channels per adjoint CTA
constexpr int AT = 256;  // samples per adjoint CTA
constexpr int AD = 16;   // DM trials per adjoint staging round
constexpr int NTH = 256;

enum { kWriteY = 0, kLoss = 1, kResidual = 2 };

struct F32Fwd {
    const float* x;
    int64_t x_pitch;
    int32_t nchans;
    int64_t nsamp;
    const float* w;
    const int32_t* shifts;  // [ndm][nchans] of the range
    int32_t d_begin, d_end; // trials handled by this launch
    int64_t length;         // L of the range
    int32_t rowlen;         // staged samples per channel row (FT + span)
    float* y;               // mode kWriteY: row d at y + d*pitch
    int64_t pitch;
    const float* tmpl;      // template, same layout as y (modes kLoss, kResidual)
    double* loss_sum;       // modes kLoss, kResidual
    float* resid;           // mode kResidual: row (d - d_begin) at resid + (d-d_begin)*rpitch
    int64_t rpitch;
    float scale;            // residual scale (2/N)
};

template <int MODE>
__global__ void __launch_bounds__(NTH) f32_forward_kernel(F32Fwd a, int ntiles_t) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ int slo[FC];
    __shared__ int offs[FD][FC];
    __shared__ float wv[FC];
    __shared__ double red[NTH / 32];
    const int tid = threadIdx.x, dl = tid >> 4, g = tid & 15;
    const int tt = blockIdx.x % ntiles_t;
    const int db = blockIdx.x / ntiles_t;
    const int d0 = a.d_begin + db * FD;
    const int dlast = min(a.d_end, d0 + FD) - 1;
    const int64_t t0 = (int64_t)tt * FT;
    const int C = a.nchans;
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
    for (int c0 = 0; c0 < C; c0 += FC) {
        __syncthreads();
        if (tid < FC) {
            const int c = c0 + tid;
            slo[tid] = c < C ? __ldg(&a.shifts[(int64_t)d0 * C + c]) : 0;
            wv[tid] = c < C ? __ldg(&a.w[c]) : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int cl = 0; cl < FC; ++cl) {
            const int c = c0 + cl;
            const float* row = a.x + (int64_t)c * a.x_pitch;
            const int64_t base = t0 + slo[cl];
            for (int j = tid; j < a.rowlen; j += NTH) {
                const int64_t u = base + j;
                fsm[cl * a.rowlen + j] = (c < C && u < a.nsamp) ? __ldg(row + u) : 0.0f;
            }
        }
        {
            const int odl = tid / FC, ocl = tid % FC;  // NTH == FD * FC
            const int c = c0 + ocl;
            const int d = min(d0 + odl, dlast);
            offs[odl][ocl] = c < C ? __ldg(&a.shifts[(int64_t)d * C + c]) - slo[ocl] : 0;
        }
        __syncthreads();
#pragma unroll 4
        for (int cl = 0; cl < FC; ++cl) {
            const float wc = wv[cl];
            const float* r = fsm + cl * a.rowlen + offs[dl][cl] + g;
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = fmaf(wc, r[16 * k], acc[k]);
        }
    }
    const int d = d0 + dl;
    const bool drow = d <= dlast;
    double local = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int64_t t = t0 + g + 16 * k;
        if (!drow || t >= a.length) continue;
        if constexpr (MODE == kWriteY) {
            a.y[(int64_t)d * a.pitch + t] = acc[k];
        } else {
            const float r = acc[k] - __ldg(&a.tmpl[(int64_t)d * a.pitch + t]);
            local += (double)r * (double)r;
            if constexpr (MODE == kResidual)
                a.resid[(int64_t)(d - a.d_begin) * a.rpitch + t] = a.scale * r;
        }
    }
    if constexpr (MODE != kWriteY) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((tid & 31) == 0) red[tid >> 5] = local;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < NTH / 32; ++i) s += red[i];
            atomicAdd(a.loss_sum, s);
        }
    }
}

struct F32Adj {
    const float* x;
    int64_t x_pitch;
    int32_t nchans;
    int64_t nsamp;
    const float* w;
    const int32_t* shifts;  // [ndm][nchans] of the range
    int32_t d_begin, d_end; // trials whose residual rows are in gy
    const float* gy;        // row (d - d_begin) at gy + (d-d_begin)*gpitch
    int64_t gpitch;
    int64_t length;         // L of the range
    int32_t rowlen;         // staged samples per DM row (AT + channel-tile delay span)
    float* gx;              // [nchans][x_pitch], accumulated
    float* gw_part;         // [nchans][ntiles_t], overwritten
};

__global__ void __launch_bounds__(NTH) f32_adjoint_kernel(F32Adj a, int ntiles_t) {
    extern __shared__ __align__(16) float asm_[];
    __shared__ int smax_s[AD];
    __shared__ int offs[AC][AD];
    const int tid = threadIdx.x, cl = tid >> 4, g = tid & 15;
    const int tt = blockIdx.x % ntiles_t;
    const int cb = blockIdx.x / ntiles_t;
    const int c0 = cb * AC;
    const int C = a.nchans;
    const int clast = min(C, c0 + AC) - 1;
    const int64_t u0 = (int64_t)tt * AT;
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
    for (int dd0 = a.d_begin; dd0 < a.d_end; dd0 += AD) {
        __syncthreads();
        if (tid < AD) {
            const int d = dd0 + tid;
            int sm = 0;
            if (d < a.d_end) {
                const int s_first = __ldg(&a.shifts[(int64_t)d * C + c0]);
                const int s_last = __ldg(&a.shifts[(int64_t)d * C + clast]);
                sm = max(s_first, s_last);  // delays are monotone in the channel index
            }
            smax_s[tid] = sm;
        }
        __syncthreads();
#pragma unroll 4
        for (int dl = 0; dl < AD; ++dl) {
            const int d = dd0 + dl;
            const int64_t base = u0 - smax_s[dl];
            const float* row = a.gy + (int64_t)(d - a.d_begin) * a.gpitch;
            for (int j = tid; j < a.rowlen; j += NTH) {
                const int64_t t = base + j;
                asm_[dl * a.rowlen + j] =
                    (d < a.d_end && t >= 0 && t < a.length) ? __ldg(row + t) : 0.0f;
            }
        }
        {
            const int ocl = tid / AD, odl = tid % AD;  // NTH == AC * AD
            const int c = min(c0 + ocl, clast);
            const int d = dd0 + odl;
            offs[ocl][odl] = d < a.d_end ? smax_s[odl] - __ldg(&a.shifts[(int64_t)d * C + c]) : 0;
        }
        __syncthreads();
#pragma unroll 4
        for (int dl = 0; dl < AD; ++dl) {
            const float* r = asm_ + dl * a.rowlen + offs[cl][dl] + g;
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] += r[16 * k];
        }
    }
    const int c = c0 + cl;
    float part = 0.0f;
    if (c < C) {
        const float wc = __ldg(&a.w[c]);
        const float* xr = a.x + (int64_t)c * a.x_pitch;
        float* gr = a.gx + (int64_t)c * a.x_pitch;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int64_t u = u0 + g + 16 * k;
            if (u < a.nsamp) {
                gr[u] += wc * acc[k];
                part = fmaf(__ldg(xr + u), acc[k], part);
            }
        }
    }
    // the 16 lanes of one channel are consecutive lanes of a warp
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (g == 0 && c < C) a.gw_part[(int64_t)c * ntiles_t + tt] = part;
}

// gw[c] += sum over time tiles of the partials (fixed order: deterministic)
__global__ void gw_reduce_kernel(const float* part, int32_t nchans, int ntiles_t, float* gw) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchans) return;
    float s = 0.0f;
    for (int i = 0; i < ntiles_t; ++i) s += part[(int64_t)c * ntiles_t + i];
    gw[c] += s;
}

__global__ void finish_loss_kernel(const double* sum, double n, double* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *loss = n > 0 ? *sum / n : 0.0;
}

}  // namespace

int f32_fwd_rowlen(int span) { return FT + span + 1; }
int f32_adj_rowlen(int cspan) { return AT + cspan + 1; }
int f32_adj_tiles(int64_t nsamp) { return (int)((nsamp + AT - 1) / AT); }

cudaError_t launch_f32_forward(int mode, const F32FwdArgs& p, cudaStream_t s) {
    const int ndm = p.d_end - p.d_begin;
    if (ndm <= 0 || p.length <= 0) return cudaSuccess;
    F32Fwd a{p.x, p.x_pitch, p.nchans, p.nsamp, p.w, p.shifts, p.d_begin, p.d_end, p.length,
             p.rowlen, p.y, p.pitch, p.tmpl, p.loss_sum, p.resid, p.rpitch, p.scale};
    const int ntiles_t = (int)((p.length + FT - 1) / FT);
    const int64_t nblocks = (int64_t)ntiles_t * ((ndm + FD - 1) / FD);
    const size_t smem = (size_t)FC * p.rowlen * 4;
    if (nblocks >= (1ll << 31)) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    switch (mode) {
        case kWriteY:
            e = cudaFuncSetAttribute(f32_forward_kernel<kWriteY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            f32_forward_kernel<kWriteY><<<(unsigned)nblocks, NTH, smem, s>>>(a, ntiles_t);
            break;
        case kLoss:
            e = cudaFuncSetAttribute(f32_forward_kernel<kLoss>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            f32_forward_kernel<kLoss><<<(unsigned)nblocks, NTH, smem, s>>>(a, ntiles_t);
            break;
        default:
            e = cudaFuncSetAttribute(f32_forward_kernel<kResidual>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            f32_forward_kernel<kResidual><<<(unsigned)nblocks, NTH, smem, s>>>(a, ntiles_t);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_f32_adjoint(const F32AdjArgs& p, cudaStream_t s) {
    if (p.d_end <= p.d_begin || p.length <= 0) return cudaSuccess;
    F32Adj a{p.x, p.x_pitch, p.nchans, p.nsamp, p.w, p.shifts, p.d_begin, p.d_end, p.gy, p.gpitch,
             p.length, p.rowlen, p.gx, p.gw_part};
    const int ntiles_t = f32_adj_tiles(p.nsamp);
    const int64_t nblocks = (int64_t)ntiles_t * ((p.nchans + AC - 1) / AC);
    const size_t smem = (size_t)AD * p.rowlen * 4;
    cudaError_t e = cudaFuncSetAttribute(f32_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    f32_adjoint_kernel<<<(unsigned)nblocks, NTH, smem, s>>>(a, ntiles_t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gw_reduce_kernel<<<(p.nchans + 127) / 128, 128, 0, s>>>(p.gw_part, p.nchans, ntiles_t, p.gw);
    return cudaGetLastError();
}

cudaError_t launch_finish_loss(const double* sum, double n, double* loss, cudaStream_t s) {
    finish_loss_kernel<<<1, 32, 0, s>>>(sum, n, loss);
    return cudaGetLastError();
}

}  // namespace aa

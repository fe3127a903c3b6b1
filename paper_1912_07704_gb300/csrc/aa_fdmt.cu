// FDMT-style tree dedispersion (arXiv:1912.07704 Sec. 1, the dedispersion
// module's cited work): one launch per depth of the channel tree, deepest
// first.  Row r of a depth holds a subband's series at one delay:
//   out[r][t] = U[t] + Lo[t + gap],   t < nsamp - delta_r,
// where U and Lo are rows of the next-deeper depth (32-bit) or input channel
// rows (8- or 16-bit leaves).  The root depth writes one FP32 row per trial
// of the range (t < the range's output length).  Sums are exact integers.
// HBM-bound: each output sample reads two samples and writes one; CTA = one
// row x 1024 samples, consecutive threads on consecutive samples.
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr int kFdmtThreads = 256;
constexpr int kFdmtPerThread = 4;
constexpr int kFdmtTile = kFdmtThreads * kFdmtPerThread;

template <int EB>
__device__ __forceinline__ uint32_t fdmt_leaf(const void* leaves, int64_t pitch, int32_t c, int64_t t) {
    if constexpr (EB == 1) return static_cast<const uint8_t*>(leaves)[(int64_t)c * pitch + t];
    else return static_cast<const uint16_t*>(leaves)[(int64_t)c * pitch + t];
}

template <int EB, bool FINAL>
__global__ void __launch_bounds__(kFdmtThreads)
    fdmt_depth_kernel(const FdmtRow* __restrict__ rows, const void* __restrict__ leaves, int64_t leaf_pitch,
                      const uint32_t* __restrict__ prev, uint32_t* __restrict__ out, int64_t pitch, int64_t nsamp,
                      float* __restrict__ fout, int64_t fpitch, int64_t flen) {
    const FdmtRow r = rows[blockIdx.y];
    const int64_t n = FINAL ? flen : nsamp - r.delta;
    const int64_t t0 = (int64_t)blockIdx.x * kFdmtTile;
    if (t0 >= n) return;
    const bool uleaf = r.u < 0, lleaf = r.l < 0;
    const uint32_t* up = uleaf ? nullptr : prev + (int64_t)r.u * pitch;
    const uint32_t* lp = lleaf ? nullptr : prev + (int64_t)r.l * pitch + r.gap;
    const int32_t uc = uleaf ? -(r.u + 1) : 0, lc = lleaf ? -(r.l + 1) : 0;
#pragma unroll
    for (int k = 0; k < kFdmtPerThread; ++k) {
        const int64_t t = t0 + threadIdx.x + k * kFdmtThreads;
        if (t < n) {
            const uint32_t a = uleaf ? fdmt_leaf<EB>(leaves, leaf_pitch, uc, t) : __ldg(up + t);
            const uint32_t b = lleaf ? fdmt_leaf<EB>(leaves, leaf_pitch, lc, t + r.gap) : __ldg(lp + t);
            if constexpr (FINAL) fout[(int64_t)blockIdx.y * fpitch + t] = (float)(a + b);
            else out[(int64_t)blockIdx.y * pitch + t] = a + b;
        }
    }
}

}  // namespace

cudaError_t launch_fdmt_depth(const FdmtRow* rows, int nrows, int leaf_elem, const void* leaves,
                              int64_t leaf_pitch, const uint32_t* prev, uint32_t* out, int64_t pitch,
                              int64_t nsamp, float* fout, int64_t fpitch, int64_t flen, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    if (nrows > 65535) return cudaErrorInvalidConfiguration;
    const bool fin = fout != nullptr;
    const int64_t n = fin ? flen : nsamp;
    if (n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + kFdmtTile - 1) / kFdmtTile), (unsigned)nrows);
    if (leaf_elem == 1) {
        if (fin) fdmt_depth_kernel<1, true><<<grid, kFdmtThreads, 0, s>>>(rows, leaves, leaf_pitch, prev, out, pitch, nsamp, fout, fpitch, flen);
        else fdmt_depth_kernel<1, false><<<grid, kFdmtThreads, 0, s>>>(rows, leaves, leaf_pitch, prev, out, pitch, nsamp, fout, fpitch, flen);
    } else {
        if (fin) fdmt_depth_kernel<2, true><<<grid, kFdmtThreads, 0, s>>>(rows, leaves, leaf_pitch, prev, out, pitch, nsamp, fout, fpitch, flen);
        else fdmt_depth_kernel<2, false><<<grid, kFdmtThreads, 0, s>>>(rows, leaves, leaf_pitch, prev, out, pitch, nsamp, fout, fpitch, flen);
    }
    return cudaGetLastError();
}

}  // namespace aa

// Stage 2 of sub-band dedispersion: the fine trials of one coarse trial sum
// the bands' 16-bit partial series at their reference channels' delays,
//   y[i][t] = sum_b z[b][j][t + s2[i][b]],
// accumulated in 32-bit registers (the partial sums reach 2^15, so 16-bit
// SWAR lanes would need a flush every two bands).  CTA = one coarse trial x
// kSb2Tau output samples; warp w takes fine trial j*m + w, 16 samples a lane
// (lane + 32 q).  Band windows are staged in shared memory in chunks of
// `nb_chunk` bands with 16-byte loads; a band's window starts at the coarse
// trial's first fine trial's delay (delays grow with the trial) rounded down
// to 8 samples and holds kSb2Tau + span + 7 samples.
#include <algorithm>
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr int kSb2Tau = 512;
constexpr int kSb2Warps = kDmPerBlock;  // one warp per fine trial of a coarse trial
constexpr int kSb2Q = kSb2Tau / 32;

__global__ void __launch_bounds__(kSb2Warps * 32) subband_stage2_kernel(
    const uint16_t* __restrict__ z, int64_t band_stride, int64_t pitch1, int nsub, int ncoarse, int m, int ndm,
    const int32_t* __restrict__ s2, int swin, int nb_chunk, int head_bytes, float* __restrict__ out,
    int64_t out_pitch, int64_t length) {
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_lo = reinterpret_cast<int*>(smem);                    // [nsub] window delays
    uint16_t* win = reinterpret_cast<uint16_t*>(smem + head_bytes);  // [nb_chunk][swin], 16-byte rows
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = (int)(blockIdx.x % ncoarse);
    const int64_t t0 = (int64_t)(blockIdx.x / ncoarse) * kSb2Tau;
    const int i0 = j * m, nj = min(m, ndm - i0);
    for (int b = threadIdx.x; b < nsub; b += blockDim.x) s_lo[b] = s2[(int64_t)i0 * nsub + b];
    const bool active = warp < nj;
    const int32_t* my_s2 = s2 + (int64_t)(i0 + (active ? warp : 0)) * nsub;
    const uint16_t* zj = z + (int64_t)j * pitch1;
    uint32_t acc[kSb2Q];
#pragma unroll
    for (int q = 0; q < kSb2Q; ++q) acc[q] = 0;
    const int nv = swin / 8;  // 16-byte vectors per staged row
    for (int b0 = 0; b0 < nsub; b0 += nb_chunk) {
        const int nbc = min(nb_chunk, nsub - b0);
        __syncthreads();  // s_lo visible; the previous chunk's windows consumed
        // a band's window starts at its delay rounded down to 8 samples (16
        // bytes: rows are 128-byte aligned); vectors at or past the row pitch
        // are zero (they only feed outputs at or past `length`)
        for (int v = threadIdx.x; v < nbc * nv; v += blockDim.x) {
            const int bl = v / nv, k = v - bl * nv;
            const int b = b0 + bl;
            const int64_t a = t0 + (s_lo[b] & ~7) + 8 * (int64_t)k;
            const uint16_t* row = zj + (int64_t)b * band_stride;
            const uint4 q = a < pitch1 ? __ldg(reinterpret_cast<const uint4*>(row + a)) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(win + (size_t)bl * swin + 8 * k) = q;
        }
        __syncthreads();
        if (active) {
            for (int bl = 0; bl < nbc; ++bl) {
                const int b = b0 + bl;
                const int off = my_s2[b] - (s_lo[b] & ~7);  // 0 .. span + 7
                const uint16_t* src = win + (size_t)bl * swin + off + lane;
#pragma unroll
                for (int q = 0; q < kSb2Q; ++q) acc[q] += src[32 * q];
            }
        }
    }
    if (!active) return;
    float* row = out + (int64_t)(i0 + warp) * out_pitch;
#pragma unroll
    for (int q = 0; q < kSb2Q; ++q) {
        const int64_t t = t0 + lane + 32 * q;
        if (t < length) row[t] = (float)acc[q];
    }
}

}  // namespace

size_t subband_stage2_smem(int nsub, int span, int& swin, int& nb_chunk) {
    // 512 outputs + span + 7 (the start rounded down to 8 samples), in 8-sample vectors
    swin = (kSb2Tau + span + 7 + 7) / 8 * 8;
    constexpr size_t kBudget = 96 * 1024;  // two CTAs per SM
    const size_t head = ((size_t)4 * nsub + 15) / 16 * 16;
    nb_chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)nsub, (kBudget - std::min(kBudget / 2, head)) /
                                                                             ((size_t)swin * 2)));
    return head + (size_t)nb_chunk * swin * 2;
}

cudaError_t launch_subband_stage2(const uint16_t* z, int64_t band_stride, int64_t pitch1, int64_t len1, int nsub,
                                  int ncoarse, int m, int ndm, const int32_t* s2, int span, float* out,
                                  int64_t out_pitch, int64_t length, cudaStream_t s) {
    (void)len1;  // rows are read up to their pitch; samples past len1 only feed t >= length
    if (length <= 0 || ndm <= 0) return cudaSuccess;
    int swin = 0, nbc = 0;
    const size_t smem = subband_stage2_smem(nsub, span, swin, nbc);
    const int head = (int)(((size_t)4 * nsub + 15) / 16 * 16);
    const int64_t ntiles = (length + kSb2Tau - 1) / kSb2Tau;
    const int64_t nblocks = ntiles * ncoarse;
    if (nblocks >= (1ll << 31) || m > kSb2Warps || pitch1 % 8 || band_stride % 8)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(subband_stage2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    subband_stage2_kernel<<<(unsigned)nblocks, kSb2Warps * 32, smem, s>>>(
        z, band_stride, pitch1, nsub, ncoarse, m, ndm, s2, swin, nbc, head, out, out_pitch, length);
    return cudaGetLastError();
}

}  // namespace aa

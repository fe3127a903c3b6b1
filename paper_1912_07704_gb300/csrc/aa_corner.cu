// Corner turn of a time-major filterbank block into the channel-major layout
// the dedispersion reads: cm[c * pitch + t] = tm[t * stride + c].
// HBM-bound (one byte read and one written per sample): 64 x 64-byte tiles
// through shared memory, 16-byte global accesses where aligned, a grid of
// persistent CTAs striding over the tiles.
#include <cstdint>

#include "aa_internal.h"

namespace aa {
namespace {

constexpr int kTile = 64;
constexpr int kPad = 4;  // row padding (bytes) of the shared tile

__global__ void __launch_bounds__(256) corner_turn_kernel(const uint8_t* __restrict__ tm,
                                                          int64_t nsamp, int nchans, int64_t stride,
                                                          uint8_t* __restrict__ cm, int64_t pitch,
                                                          int64_t ntile_t, int64_t ntiles) {
    __shared__ __align__(16) uint8_t tile[kTile][kTile + kPad];  // [t][c]
    const int row = threadIdx.x >> 2, seg = (threadIdx.x & 3) * 16;
    for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x) {
        const int64_t t0 = (it % ntile_t) * kTile;
        const int c0 = (int)(it / ntile_t) * kTile;
        // load: time sample t0 + row, channels c0 + seg .. + 15
        {
            const int64_t t = t0 + row;
            const int c = c0 + seg;
            uint8_t* dst = &tile[row][seg];
            if (t < nsamp) {
                const uint8_t* src = tm + t * stride + c;
                if (c + 16 <= nchans && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    const uint4 v = *reinterpret_cast<const uint4*>(src);
                    uint32_t* d4 = reinterpret_cast<uint32_t*>(dst);
                    d4[0] = v.x; d4[1] = v.y; d4[2] = v.z; d4[3] = v.w;
                } else {
                    for (int k = 0; k < 16; ++k) dst[k] = c + k < nchans ? src[k] : 0;
                }
            }
        }
        __syncthreads();
        // store: channel c0 + row, time samples t0 + seg .. + 15
        {
            const int c = c0 + row;
            const int64_t t = t0 + seg;
            if (c < nchans && t < nsamp) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = (uint32_t)tile[seg + 4 * q][row] | ((uint32_t)tile[seg + 4 * q + 1][row] << 8) |
                           ((uint32_t)tile[seg + 4 * q + 2][row] << 16) |
                           ((uint32_t)tile[seg + 4 * q + 3][row] << 24);
                uint8_t* dst = cm + (int64_t)c * pitch + t;
                if (t + 16 <= nsamp && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    for (int k = 0; k < 16 && t + k < nsamp; ++k) dst[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace aa

using namespace aa;

extern "C" aa_status aa_corner_turn_device(const uint8_t* d_tm, int64_t nsamp, int32_t nchans,
                                           int64_t tm_stride, uint8_t* d_cm, int64_t cm_pitch,
                                           aa_stream_t stream) {
    clear_error();
    if (!d_tm || !d_cm) { set_error("device pointer is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0 || nchans < 1 || tm_stride < nchans || cm_pitch < nsamp) {
        set_error("bad sizes (nsamp %lld, nchans %d, stride %lld, pitch %lld)", (long long)nsamp,
                  nchans, (long long)tm_stride, (long long)cm_pitch);
        return AA_ERR_ARG;
    }
    if (nsamp == 0) return AA_OK;
    const int64_t ntile_t = (nsamp + kTile - 1) / kTile;
    const int64_t ntiles = ntile_t * ((nchans + kTile - 1) / kTile);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)std::max(sms, 1) * 8);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        ProfScope prof(kKCornerTurn, s);
        corner_turn_kernel<<<(unsigned)grid, 256, 0, s>>>(d_tm, nsamp, nchans, tm_stride, d_cm, cm_pitch,
                                                           ntile_t, ntiles);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("corner turn launch: %s", cudaGetErrorString(e));
        return AA_ERR_CUDA;
    }
    return AA_OK;
}

// Single-pulse search for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a real-time
// beam-processing loop whose device memory is fixed at start-up (an
// allocation can implicitly synchronise the device and break its latency
// budget), or a plug-in hosted by a framework that owns every device
// allocation and hands the plug-in no workspace.  For them this entry point
// runs the same search as aa_sps_search_device with its scratch taken from a
// fixed-size array that is part of the library's device image.
//
// In host code the name of the array below is only its host-side shadow,
// not a device address: the kernels get the address that
// cudaGetSymbolAddress returns, looked up once per device, with that device
// current, on the first call made on that device (and cached: a
// cudaDeviceReset of that device invalidates it, so this entry point must not
// be used on a device after it was reset).  The array occupies
// AA_NOALLOC_SCRATCH_BYTES on every GPU that loads the library, until the
// process exits.  Every call shares it: calls whose work overlaps on the GPU
// (other streams, other host threads) race on it.
#include <mutex>

#include "aa_internal.h"

namespace {

constexpr size_t kScratchBytes = AA_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_sps_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

using namespace aa;

extern "C" aa_status aa_sps_search_device_noalloc(const aa_plan* p, int64_t nsamp,
                                                  const float* d_dd, int32_t max_width,
                                                  float threshold, aa_candidate* d_cands,
                                                  int64_t cand_capacity,
                                                  unsigned long long* d_count, float* d_snr_out,
                                                  aa_stream_t stream) {
    clear_error();
    if (!p) { set_error("plan is NULL"); return AA_ERR_ARG; }
    if (nsamp < 0) { set_error("nsamp must be >= 0"); return AA_ERR_ARG; }
    if (max_width < 1 || max_width > 65535) { set_error("max_width must be in [1, 65535]"); return AA_ERR_ARG; }
    const Layout L = make_layout(*p, nsamp, max_width);
    if (L.sps_ws > (int64_t)kScratchBytes) {
        set_error("this search needs %lld bytes of scratch; the built-in area holds %zu bytes "
                  "(use aa_sps_search_device with a caller workspace)",
                  (long long)L.sps_ws, kScratchBytes);
        return AA_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error("cudaGetDevice: %s", cudaGetErrorString(e)); return AA_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { set_error("device %d out of range", dev); return AA_ERR_ARG; }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_sps_scratch);  // device `dev` is current
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                set_error("cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
                return AA_ERR_CUDA;
            }
            g_scratch_addr[dev] = addr;
        }
        scratch = g_scratch_addr[dev];
    }
    // The search clears the error word, chunk counter and candidate count
    // itself and rewrites every other scratch byte it reads.
    return aa_sps_search_device(p, nsamp, d_dd, max_width, threshold, d_cands, cand_capacity,
                                d_count, d_snr_out, scratch, kScratchBytes, stream);
}

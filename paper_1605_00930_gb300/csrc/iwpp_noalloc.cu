// iwpp_noalloc.cu — single-image reconstruction that allocates nothing (include/iwpp.h,
// iwpp_reconstruct_noalloc).
//
// Some callers cannot allocate device memory at the point where they reconstruct: code
// that runs under a fixed memory budget reserved at start-up, plug-ins hosted by a
// framework that owns every allocation, or real-time loops where a cudaMalloc (which may
// synchronise the device) is not allowed. For them this entry point uses a workspace that
// lives in the library itself: a file-scope device array of kScratchBytes, which every
// GPU that loads the library holds until the process exits. The caller still passes the
// marker (overwritten by the result) and the mask.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/iwpp.h"
#include "iwpp_host.h"

namespace {

constexpr size_t kScratchBytes = (size_t)IWPP_NOALLOC_SCRATCH_BYTES;

// The workspace of every iwpp_reconstruct_noalloc call on a device. Host code must not pass
// this name to a kernel (in host code it is only a stand-in symbol): the device address is
// obtained with cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up on the first call per device).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IWPP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return IWPP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return IWPP_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return IWPP_OK;
}

}  // namespace

extern "C" int iwpp_reconstruct_noalloc(void *marker_inout, const void *mask, int64_t H, int64_t W,
                                        int connectivity, int op, int dtype, void *stream, int *status_out) {
    if (!marker_inout || !mask) return IWPP_ERR_ARG;
    if (H < 1 || W < 1 || H >= (1ll << 31) || W >= (1ll << 31) || (uint64_t)H * (uint64_t)W >= (1ull << 40))
        return IWPP_ERR_ARG;
    if (dtype != IWPP_U8 && dtype != IWPP_U16) return IWPP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (status_out != nullptr) {   // waiting for the status would break a capture of `stream`
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return IWPP_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return IWPP_ERR_ARG;
    }
    // default plan; with valid sizes and dtype a zero here means a CUDA query failed
    const size_t need = iwpp::workspace_bytes(H, W, dtype, nullptr);
    if (need == 0) return IWPP_ERR_CUDA;
    if (need > kScratchBytes) return IWPP_ERR_WORKSPACE;               // image too large for the scratch
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != IWPP_OK) return rc;
    // The call resets the parts of the scratch that must start at zero (header, tile states)
    // and the tile queue itself, on `stream`, before its kernels run.
    const int r = iwpp::reconstruct_one(marker_inout, mask, H, W, connectivity, op, dtype, nullptr, ws,
                                        kScratchBytes, s, 3);
    if (r != IWPP_OK || status_out == nullptr) return r;
    uint32_t st = 0;
    if (cudaMemcpyAsync(&st, ws, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return IWPP_ERR_CUDA;
    *status_out = (int)st;
    return IWPP_OK;
}

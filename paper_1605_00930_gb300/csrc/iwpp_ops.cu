// iwpp_ops.cu — operators built on reconstruction by dilation (include/iwpp.h): the
// h-maxima transform, the h-dome (regional maxima of height below h, as the contrast
// that remains), and the regional maxima. The paper names further IWPP operators as future
// work; these are the reconstruction-based ones, each a marker built on the device, one
// reconstruction through the same path as iwpp_reconstruct, and an elementwise finish.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/iwpp.h"
#include "iwpp_host.h"

namespace iwpp {
namespace {

// out = max(f - h, 0)
template <typename T>
__global__ void sub_sat_kernel(const T *f, T *out, size_t n, uint32_t h) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t v = f[i];
        out[i] = (T)(v > h ? v - h : 0u);
    }
}

// out = f - out (out <= f after a reconstruction under f)
template <typename T>
__global__ void dome_kernel(const T *f, T *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (T)((uint32_t)f[i] - (uint32_t)out[i]);
}

// mask = 1 where f rises above the reconstruction of f - 1 under f
template <typename T>
__global__ void rmax_kernel(const T *f, const T *r, uint8_t *mask, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mask[i] = f[i] > r[i] ? 1 : 0;
}

int grid_of(size_t n) {
    const int sms = device_sm_count();
    size_t g = (n + 255) / 256;
    const size_t cap = (size_t)(sms > 0 ? sms : 1) * 8;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

int check_args(const void *a, const void *b, int64_t H, int64_t W, int dtype) {
    if (!a || !b || H < 1 || W < 1) return IWPP_ERR_ARG;
    if (dtype != IWPP_U8 && dtype != IWPP_U16) return IWPP_ERR_ARG;
    if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return IWPP_ERR_ARG;
    return IWPP_OK;
}

// marker = max(f - h, 0) into `marker`, then reconstruction by dilation under f
int hmax_into(const void *f, void *marker, int64_t H, int64_t W, uint32_t h, int conn, int dtype, void *ws,
              size_t ws_bytes, cudaStream_t s) {
    const size_t n = (size_t)H * (size_t)W;
    if (dtype == IWPP_U8)
        sub_sat_kernel<uint8_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint8_t *>(f),
                                                            static_cast<uint8_t *>(marker), n, h);
    else
        sub_sat_kernel<uint16_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint16_t *>(f),
                                                             static_cast<uint16_t *>(marker), n, h);
    if (cudaGetLastError() != cudaSuccess) return IWPP_ERR_CUDA;
    return reconstruct_one(marker, f, H, W, conn, IWPP_DILATE, dtype, nullptr, ws, ws_bytes, s, 3);
}

}  // namespace
}  // namespace iwpp

extern "C" int iwpp_hmaxima(const void *image, void *out, int64_t H, int64_t W, uint32_t h, int connectivity,
                            int dtype, void *workspace, size_t ws_bytes, void *stream) {
    const int rc = iwpp::check_args(image, out, H, W, dtype);
    if (rc != IWPP_OK) return rc;
    return iwpp::hmax_into(image, out, H, W, h, connectivity, dtype, workspace, ws_bytes,
                           static_cast<cudaStream_t>(stream));
}

extern "C" int iwpp_hdome(const void *image, void *out, int64_t H, int64_t W, uint32_t h, int connectivity,
                          int dtype, void *workspace, size_t ws_bytes, void *stream) {
    using namespace iwpp;
    int rc = check_args(image, out, H, W, dtype);
    if (rc != IWPP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = hmax_into(image, out, H, W, h, connectivity, dtype, workspace, ws_bytes, s);
    if (rc != IWPP_OK) return rc;
    const size_t n = (size_t)H * (size_t)W;
    if (dtype == IWPP_U8)
        dome_kernel<uint8_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint8_t *>(image),
                                                         static_cast<uint8_t *>(out), n);
    else
        dome_kernel<uint16_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint16_t *>(image),
                                                          static_cast<uint16_t *>(out), n);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

extern "C" int iwpp_regional_maxima(const void *image, void *scratch, uint8_t *out, int64_t H, int64_t W,
                                    int connectivity, int dtype, void *workspace, size_t ws_bytes, void *stream) {
    using namespace iwpp;
    int rc = check_args(image, scratch, H, W, dtype);
    if (rc != IWPP_OK) return rc;
    if (!out) return IWPP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = hmax_into(image, scratch, H, W, 1, connectivity, dtype, workspace, ws_bytes, s);
    if (rc != IWPP_OK) return rc;
    const size_t n = (size_t)H * (size_t)W;
    if (dtype == IWPP_U8)
        rmax_kernel<uint8_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint8_t *>(image),
                                                         static_cast<const uint8_t *>(scratch), out, n);
    else
        rmax_kernel<uint16_t><<<grid_of(n), 256, 0, s>>>(static_cast<const uint16_t *>(image),
                                                          static_cast<const uint16_t *>(scratch), out, n);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

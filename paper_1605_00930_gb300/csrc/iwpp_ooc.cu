// iwpp_ooc.cu — reconstruction of an image held in host memory, band by band
// (include/iwpp.h, iwpp_reconstruct_host).
//
// Sec. 4.5 splits an image too large for the accelerator into tasks, reconstructs each task
// on its own and then corrects the propagation across the task borders. Here the tasks are
// horizontal bands of `band_rows` rows and the correction is iterative: each band is copied
// to the device with one halo row above and below, the halo rows are fixed (their mask is set
// to their marker, so they act as sources that cannot change), the band is reconstructed by
// the single-image path, and the band's rows go back to host memory. Bands are visited top to
// bottom and then bottom to top, each again only after a neighbour changed; when no band is
// left to visit, every band is a fixed point given its neighbours' rows, i.e. the whole image
// a fixed point of J <- min(delta(J), I), which above the marker and below the mask is the
// reconstruction (every value produced on the way is a lower bound of it). The result is
// therefore bit-identical to iwpp_reconstruct.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/iwpp.h"
#include "iwpp_bands.h"
#include "iwpp_host.h"

namespace iwpp {
namespace {

// After a band: flag a change of the band's rows (compared with their copy from before the
// band's reconstruction) and keep the first device error of any band.
template <typename T>
__global__ void band_done_kernel(const T *before, const T *after, size_t n, const uint32_t *band_status,
                                 uint32_t *acc) {
    bool diff = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        diff |= before[i] != after[i];
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(acc + 1, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0 && *band_status != 0) atomicCAS(acc, 0u, *band_status);
}

struct OocLayout {
    size_t acc, jb, ib, j0, rws, total;
    size_t rws_bytes;
    int64_t band;
};

bool ooc_layout(int64_t H, int64_t W, int dtype, int64_t band_rows, OocLayout &L) {
    if (H < 1 || W < 1 || band_rows < 1 || (dtype != IWPP_U8 && dtype != IWPP_U16)) return false;
    if (H >= (1ll << 31) || W >= (1ll << 31) || (uint64_t)H * (uint64_t)W >= (1ull << 40)) return false;
    L.band = band_rows < H ? band_rows : H;
    const int64_t rows = L.band + 2;
    if ((uint64_t)rows * (uint64_t)W >= (1ull << 40)) return false;
    const size_t s = dtype == IWPP_U16 ? 2 : 1;
    const size_t plane = (size_t)rows * (size_t)W * s;
    L.rws_bytes = workspace_bytes(rows, W, dtype, nullptr);
    if (L.rws_bytes == 0) return false;
    L.acc = 0;
    L.jb = 256;
    L.ib = L.jb + align256(plane);
    L.j0 = L.ib + align256(plane);
    L.rws = L.j0 + align256((size_t)L.band * (size_t)W * s);
    L.total = L.rws + align256(L.rws_bytes);
    return true;
}

}  // namespace
}  // namespace iwpp

extern "C" size_t iwpp_host_workspace_bytes(int64_t H, int64_t W, int dtype, int64_t band_rows) {
    iwpp::OocLayout L;
    return iwpp::ooc_layout(H, W, dtype, band_rows, L) ? L.total : 0;
}

extern "C" int iwpp_reconstruct_host(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                                     int op, int dtype, int64_t band_rows, void *workspace, size_t ws_bytes,
                                     void *stream, int32_t *visits_out) {
    using namespace iwpp;
    if (!marker_inout || !mask) return IWPP_ERR_ARG;
    if (connectivity != 4 && connectivity != 8) return IWPP_ERR_ARG;
    if (op != IWPP_DILATE && op != IWPP_ERODE) return IWPP_ERR_ARG;
    OocLayout L;
    if (!ooc_layout(H, W, dtype, band_rows, L)) return IWPP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return IWPP_ERR_WORKSPACE;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    uint32_t *acc = reinterpret_cast<uint32_t *>(base + L.acc);   // [0] first error, [1] changed
    uint8_t *jb = base + L.jb, *ib = base + L.ib, *j0 = base + L.j0, *rws = base + L.rws;
    uint8_t *hm = static_cast<uint8_t *>(marker_inout);
    const uint8_t *hi = static_cast<const uint8_t *>(mask);
    const size_t es = dtype == IWPP_U16 ? 2 : 1, rowb = (size_t)W * es;
    const int64_t nb = (H + L.band - 1) / L.band;
    const int sms = device_sm_count();
    if (sms <= 0) return IWPP_ERR_CUDA;
    if (cudaMemsetAsync(acc, 0, 8, s) != cudaSuccess) return IWPP_ERR_CUDA;

    auto do_band = [&](int64_t b) -> int {
        const int64_t y0 = b * L.band, y1 = y0 + L.band < H ? y0 + L.band : H;
        const int64_t top = y0 > 0 ? 1 : 0, bot = y1 < H ? 1 : 0;
        const int64_t r0 = y0 - top, rows = (y1 - y0) + top + bot;
        const size_t nbytes = (size_t)rows * rowb, band_bytes = (size_t)(y1 - y0) * rowb;
        if (cudaMemcpyAsync(jb, hm + (size_t)r0 * rowb, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(ib, hi + (size_t)r0 * rowb, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        // halo rows: mask := marker, so they feed the band and cannot change
        if (top && cudaMemcpyAsync(ib, jb, rowb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return IWPP_ERR_CUDA;
        if (bot && cudaMemcpyAsync(ib + (size_t)(rows - 1) * rowb, jb + (size_t)(rows - 1) * rowb, rowb,
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (cudaMemcpyAsync(j0, jb + (size_t)top * rowb, band_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        const int rc = reconstruct_one(jb, ib, rows, W, connectivity, op, dtype, nullptr, rws, L.rws_bytes, s, 3);
        if (rc != IWPP_OK) return rc;
        const size_t n = (size_t)(y1 - y0) * (size_t)W;
        size_t g = (n + 255) / 256;
        if (g > (size_t)sms * 8) g = (size_t)sms * 8;
        if (g < 1) g = 1;
        const uint32_t *st = reinterpret_cast<const uint32_t *>(rws);
        if (dtype == IWPP_U8)
            band_done_kernel<uint8_t><<<(unsigned)g, 256, 0, s>>>(j0, jb + (size_t)top * rowb, n, st, acc);
        else
            band_done_kernel<uint16_t><<<(unsigned)g, 256, 0, s>>>(reinterpret_cast<const uint16_t *>(j0),
                                                                   reinterpret_cast<const uint16_t *>(jb + top * rowb),
                                                                   n, st, acc);
        if (cudaGetLastError() != cudaSuccess) return IWPP_ERR_CUDA;
        if (cudaMemcpyAsync(hm + (size_t)y0 * rowb, jb + (size_t)top * rowb, band_bytes, cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        return IWPP_OK;
    };

    // A band is a fixed point given its halo rows once reconstructed; it needs another visit
    // only when a neighbour band changed afterwards (iwpp_bands.h).
    BandSchedule order(nb);
    int32_t visits = 0;
    for (int64_t b = order.next(); b >= 0; b = order.next()) {
        if (cudaMemsetAsync(acc + 1, 0, 4, s) != cudaSuccess) return IWPP_ERR_CUDA;
        const int rc = do_band(b);
        if (rc != IWPP_OK) return rc;
        uint32_t h[2] = {0, 0};
        if (cudaMemcpyAsync(h, acc, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return IWPP_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return IWPP_ERR_CUDA;
        visits++;
        if (h[0] != 0) {
            if (visits_out) *visits_out = visits;
            return (int)h[0];
        }
        order.visited(b, h[1] != 0);
    }
    if (visits_out) *visits_out = visits;
    return IWPP_OK;
}

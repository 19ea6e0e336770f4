// iwpp_ooc.cu — reconstruction of an image held in host memory, band by band
// (include/iwpp.h, iwpp_reconstruct_host).
//
// Sec. 4.5 splits an image too large for the accelerator into tasks, reconstructs each task
// on its own and then corrects the propagation across the task borders. Here the tasks are
// horizontal bands of `band_rows` rows and the correction is iterative: each band is copied
// to the device together with `ov` rows of each neighbour band (the overlap, ov < band_rows)
// and one halo row beyond them; the halo rows are fixed (their mask is set to their marker,
// so they act as sources that cannot change), the extended band is reconstructed by the
// single-image path, and only the band's own rows go back to host memory. Bands are visited
// top to bottom and then bottom to top, each again only after a neighbour's rows changed.
// Every value produced is a lower bound of the reconstruction (a reconstruction with fixed
// sources that are lower bounds). When no band is left to visit, take neighbours b and c,
// and say c's last visit came first: c's visits after b's last one (if any) changed nothing,
// and b's last visit changed nothing of c's rows on the host, so both last visits saw the
// other's final rows. A value that b's last visit computed for an overlap pixel q of c comes
// along a path from a source; its last entry into c's rows is from b's border row (or starts
// at b's halo row, which lies in c), a pixel that c's last visit also held with its final
// value, so c's last visit reached at least that value at q: the overlap values b used are
// c's final rows. Hence each band's own rows are a fixed point of J <- min(delta(J), I)
// given its neighbours' final rows, i.e. the whole image is a fixed point, which above the
// marker and below the mask is the reconstruction: the result is bit-identical to
// iwpp_reconstruct. The overlap lets a path that crosses a border and comes back within ov
// rows be followed in one visit (measured on a 32768^2 sparse-seed image, bands of 4096 rows:
// 66 band visits without overlap, 27 with 32 rows, 15 with 256).
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

// Workspace: flags (256 B) | two band buffers, each: marker plane and mask plane of
// (band_rows + 2 ov + 2) x W (band, overlaps and halo rows) and a band_rows x W copy of the
// band from before its reconstruction | a single-image workspace for band_rows + 2 ov + 2 rows.
struct OocLayout {
    size_t acc, buf[2], plane, jcopy, rws, total;
    size_t rws_bytes;
    int64_t band, ov;
};

bool ooc_layout(int64_t H, int64_t W, int dtype, int64_t band_rows, OocLayout &L) {
    if (H < 1 || W < 1 || band_rows < 1 || (dtype != IWPP_U8 && dtype != IWPP_U16)) return false;
    if (H >= (1ll << 31) || W >= (1ll << 31) || (uint64_t)H * (uint64_t)W >= (1ull << 40)) return false;
    L.band = band_rows < H ? band_rows : H;
    L.ov = band_overlap(L.band);
    const int64_t rows = L.band + 2 * L.ov + 2;
    if ((uint64_t)rows * (uint64_t)W >= (1ull << 40)) return false;
    const size_t s = dtype == IWPP_U16 ? 2 : 1;
    L.plane = align256((size_t)rows * (size_t)W * s);
    L.jcopy = align256((size_t)L.band * (size_t)W * s);
    L.rws_bytes = workspace_bytes(rows, W, dtype, nullptr);
    if (L.rws_bytes == 0) return false;
    L.acc = 0;
    L.buf[0] = 256;
    L.buf[1] = L.buf[0] + 2 * L.plane + L.jcopy;
    L.rws = L.buf[1] + 2 * L.plane + L.jcopy;
    L.total = L.rws + align256(L.rws_bytes);
    return true;
}

// One device band buffer and the band it holds.
struct BandBuf {
    uint8_t *jb, *ib, *j0;
    int64_t band = -1;
    cudaEvent_t loaded = nullptr, free = nullptr;
};

// CUDA objects of one call, released on every return path.
struct OocRes {
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t *flags = nullptr;   // pinned host [0] first error, [1] changed
    ~OocRes() {
        if (copy) cudaStreamDestroy(copy);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (flags) cudaFreeHost(flags);
    }
};

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
    uint8_t *rws = base + L.rws;
    uint8_t *hm = static_cast<uint8_t *>(marker_inout);
    const uint8_t *hi = static_cast<const uint8_t *>(mask);
    const size_t es = dtype == IWPP_U16 ? 2 : 1, rowb = (size_t)W * es;
    const int64_t nb = (H + L.band - 1) / L.band;
    const int sms = device_sm_count();
    if (sms <= 0) return IWPP_ERR_CUDA;

    // Copies of the next band run on a stream of their own while the current band is
    // reconstructed on `stream`; events order the two.
    OocRes R;
    if (cudaStreamCreateWithFlags(&R.copy, cudaStreamNonBlocking) != cudaSuccess) return IWPP_ERR_CUDA;
    for (cudaEvent_t &e : R.ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaHostAlloc(reinterpret_cast<void **>(&R.flags), 8, cudaHostAllocDefault) != cudaSuccess) return IWPP_ERR_CUDA;
    BandBuf buf[2];
    for (int k = 0; k < 2; k++) {
        buf[k].jb = base + L.buf[k];
        buf[k].ib = buf[k].jb + L.plane;
        buf[k].j0 = buf[k].ib + L.plane;
        buf[k].loaded = R.ev[k];
        buf[k].free = R.ev[2 + k];
        if (cudaEventRecord(buf[k].free, s) != cudaSuccess) return IWPP_ERR_CUDA;
    }
    cudaEvent_t done = R.ev[4];
    if (cudaMemsetAsync(acc, 0, 8, s) != cudaSuccess) return IWPP_ERR_CUDA;

    // Band b: own rows [y0, y1); the buffer holds rows [r0, r1) = the extended band
    // [e0, e1) (own rows and overlaps) and a fixed halo row on each side inside the image.
    struct Geo {
        int64_t y0, y1, e0, e1, top, bot, r0, r1;
    };
    auto geometry = [&](int64_t b) {
        Geo g;
        g.y0 = b * L.band;
        g.y1 = g.y0 + L.band < H ? g.y0 + L.band : H;
        g.e0 = g.y0 - L.ov > 0 ? g.y0 - L.ov : 0;
        g.e1 = g.y1 + L.ov < H ? g.y1 + L.ov : H;
        g.top = g.e0 > 0 ? 1 : 0;
        g.bot = g.e1 < H ? 1 : 0;
        g.r0 = g.e0 - g.top;
        g.r1 = g.e1 + g.bot;
        return g;
    };
    // Copy band b (with its overlaps and halo rows) from host memory into buffer B, on the
    // copy stream, once B's previous band is done with it.
    auto upload = [&](BandBuf &B, int64_t b) -> int {
        const Geo g = geometry(b);
        const int64_t r0 = g.r0, rows = g.r1 - g.r0;
        const size_t nbytes = (size_t)rows * rowb;
        if (cudaStreamWaitEvent(R.copy, B.free, 0) != cudaSuccess) return IWPP_ERR_CUDA;
        if (cudaMemcpyAsync(B.jb, hm + (size_t)r0 * rowb, nbytes, cudaMemcpyHostToDevice, R.copy) != cudaSuccess ||
            cudaMemcpyAsync(B.ib, hi + (size_t)r0 * rowb, nbytes, cudaMemcpyHostToDevice, R.copy) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (cudaEventRecord(B.loaded, R.copy) != cudaSuccess) return IWPP_ERR_CUDA;
        B.band = b;
        return IWPP_OK;
    };
    // Reconstruct the band in B on `stream`. P holds the band visited just before (pb); when
    // pb is a neighbour, B's rows of pb (overlap and halo row) may have been copied from host
    // memory before pb's result reached it, so they are taken from P instead.
    auto compute = [&](BandBuf &B, BandBuf &P, int64_t pb) -> int {
        const int64_t b = B.band;
        const Geo g = geometry(b);
        const int64_t rows = g.r1 - g.r0, own = g.y0 - g.r0;   // own: index of row y0 in B
        const size_t band_bytes = (size_t)(g.y1 - g.y0) * rowb;
        if (cudaStreamWaitEvent(s, B.loaded, 0) != cudaSuccess) return IWPP_ERR_CUDA;
        if (pb >= 0 && P.band == pb && (pb == b - 1 || pb == b + 1)) {
            const Geo pg = geometry(pb);
            // rows of pb's own range inside B's buffer (ov + 1 <= band_rows: all of them are pb's)
            const int64_t lo = g.r0 > pg.y0 ? g.r0 : pg.y0, hi = g.r1 < pg.y1 ? g.r1 : pg.y1;
            if (hi > lo &&
                cudaMemcpyAsync(B.jb + (size_t)(lo - g.r0) * rowb, P.jb + (size_t)(lo - pg.r0) * rowb,
                                (size_t)(hi - lo) * rowb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return IWPP_ERR_CUDA;
            if (cudaEventRecord(P.free, s) != cudaSuccess) return IWPP_ERR_CUDA;   // P is read up to here
        }
        // halo rows: mask := marker, so they feed the band and cannot change
        if (g.top && cudaMemcpyAsync(B.ib, B.jb, rowb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (g.bot && cudaMemcpyAsync(B.ib + (size_t)(rows - 1) * rowb, B.jb + (size_t)(rows - 1) * rowb, rowb,
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (cudaMemcpyAsync(B.j0, B.jb + (size_t)own * rowb, band_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (cudaMemsetAsync(acc + 1, 0, 4, s) != cudaSuccess) return IWPP_ERR_CUDA;
        const int rc = reconstruct_one(B.jb, B.ib, rows, W, connectivity, op, dtype, nullptr, rws, L.rws_bytes, s, 3);
        if (rc != IWPP_OK) return rc;
        const size_t n = (size_t)(g.y1 - g.y0) * (size_t)W;
        size_t grid = (n + 255) / 256;
        if (grid > (size_t)sms * 8) grid = (size_t)sms * 8;
        if (grid < 1) grid = 1;
        const uint32_t *st = reinterpret_cast<const uint32_t *>(rws);
        if (dtype == IWPP_U8)
            band_done_kernel<uint8_t><<<(unsigned)grid, 256, 0, s>>>(B.j0, B.jb + (size_t)own * rowb, n, st, acc);
        else
            band_done_kernel<uint16_t><<<(unsigned)grid, 256, 0, s>>>(reinterpret_cast<const uint16_t *>(B.j0),
                                                                      reinterpret_cast<const uint16_t *>(B.jb + own * rowb),
                                                                      n, st, acc);
        if (cudaGetLastError() != cudaSuccess) return IWPP_ERR_CUDA;
        if (cudaMemcpyAsync(R.flags, acc, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hm + (size_t)g.y0 * rowb, B.jb + (size_t)own * rowb, band_bytes, cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return IWPP_ERR_CUDA;
        if (cudaEventRecord(B.free, s) != cudaSuccess || cudaEventRecord(done, s) != cudaSuccess) return IWPP_ERR_CUDA;
        return IWPP_OK;
    };

    // A band is a fixed point given its halo rows once reconstructed; it needs another visit
    // only when a neighbour band changed afterwards (iwpp_bands.h). While a band is
    // reconstructed, the band expected next (the next one in sweep order if this one changes)
    // is copied into the other buffer; a wrong guess costs one more copy, never a result.
    BandSchedule order(nb);
    int32_t visits = 0;
    int64_t cur = order.next(), prev = -1;
    int k = 0;
    if (cur >= 0) {
        const int rc = upload(buf[0], cur);
        if (rc != IWPP_OK) return rc;
    }
    while (cur >= 0) {
        BandBuf &B = buf[k & 1], &O = buf[(k + 1) & 1];
        int rc = compute(B, O, prev);
        if (rc != IWPP_OK) return rc;
        const int64_t guess = order.peek_after_change(cur);
        if (guess >= 0) {
            rc = upload(O, guess);
            if (rc != IWPP_OK) return rc;
        }
        if (cudaEventSynchronize(done) != cudaSuccess) return IWPP_ERR_CUDA;
        visits++;
        if (R.flags[0] != 0) {
            if (cudaStreamSynchronize(R.copy) != cudaSuccess) return IWPP_ERR_CUDA;
            if (visits_out) *visits_out = visits;
            return (int)R.flags[0];
        }
        order.visited(cur, R.flags[1] != 0);
        const int64_t nxt = order.next();
        if (nxt >= 0 && nxt != guess) {   // wrong guess: copy the band that is due
            rc = upload(O, nxt);
            if (rc != IWPP_OK) return rc;
        }
        prev = cur;
        cur = nxt;
        k++;
    }
    if (cudaStreamSynchronize(R.copy) != cudaSuccess) return IWPP_ERR_CUDA;
    if (visits_out) *visits_out = visits;
    return IWPP_OK;
}

// iwpp_api.cu — C ABI of the single-image reconstruction path (include/iwpp.h).
//
// Host side only validates arguments, carves the caller's workspace and enqueues
// three steps on the caller's stream: a workspace reset (memsets), the
// tile-parallel scan kernel (precondition check, tile-local raster / anti-raster
// sweeps of Algorithm 7, frontier initialisation), and the persistent drain
// kernel (Algorithm 7's irregular propagation phase). No host synchronisation,
// no allocation.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/iwpp.h"
#include "iwpp_engine.cuh"

namespace iwpp {

// ---- compiled tile shapes -------------------------------------------------------------------
struct ShapeInfo {
    int th, tw;
};
static const ShapeInfo kShapes[] = {{32, 32}, {32, 64}, {64, 64}};
static constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int shape_index(int th, int tw) {
    for (int i = 0; i < kNumShapes; i++)
        if (kShapes[i].th == th && kShapes[i].tw == tw) return i;
    return -1;
}

// Kernel table: [shape][dtype][conn4/8]
struct KernelSet {
    void (*scan)(EngineArgs);
    void (*drain)(EngineArgs);
    size_t (*smem)(uint32_t);
    int npix;
};

template <typename T, int CONN, int TH, int TW>
static KernelSet make_set() {
    KernelSet k;
    k.scan = scan_kernel<T, CONN, TH, TW>;
    k.drain = drain_kernel<T, CONN, TH, TW>;
    k.smem = &Tile<T, CONN, TH, TW>::smem_bytes;
    k.npix = TH * TW;
    return k;
}

template <int TH, int TW>
static void fill_shape(KernelSet (&row)[2][2]) {
    row[0][0] = make_set<uint8_t, 4, TH, TW>();
    row[0][1] = make_set<uint8_t, 8, TH, TW>();
    row[1][0] = make_set<uint16_t, 4, TH, TW>();
    row[1][1] = make_set<uint16_t, 8, TH, TW>();
}

static KernelSet g_sets[kNumShapes][2][2];
static int g_maxsmem_set[kNumShapes][2][2];
static std::once_flag g_once;
static std::mutex g_mu;

static void init_sets() {
    fill_shape<32, 32>(g_sets[0]);
    fill_shape<32, 64>(g_sets[1]);
    fill_shape<64, 64>(g_sets[2]);
}

const KernelSet &kernels(int shape, int dtype, int conn) {
    std::call_once(g_once, init_sets);
    return g_sets[shape][dtype][conn == 8 ? 1 : 0];
}

// Opt the kernels of one set into the dynamic shared memory they need (per device
// the attribute is per function; set it once with a generous bound).
static cudaError_t ensure_smem_attr(int shape, int dtype, int conn, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    int &done = g_maxsmem_set[shape][dtype][conn == 8 ? 1 : 0];
    if ((size_t)done >= bytes) return cudaSuccess;
    const KernelSet &k = kernels(shape, dtype, conn);
    const int want = (int)(bytes < 100 * 1024 ? 100 * 1024 : bytes);
    cudaError_t e = cudaFuncSetAttribute((const void *)k.scan, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k.drain, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e != cudaSuccess) return e;
    done = want;
    return cudaSuccess;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Persistent CTAs for a plan: blocks_per_sm (or the occupancy maximum) x SMs,
// never more CTAs than needed to give every tile its own warp.
int drain_grid(const iwpp_plan &p, int dtype, int conn, uint32_t ntiles) {
    const int shape = shape_index(p.tile_h, p.tile_w);
    const KernelSet &k = kernels(shape, dtype, conn);
    const size_t smem = k.smem((uint32_t)p.smem_queue_cap);
    if (ensure_smem_attr(shape, dtype, conn, smem) != cudaSuccess) return 0;
    int bps = p.blocks_per_sm;
    if (bps <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k.drain, kThreads, smem) != cudaSuccess)
            return 0;
    }
    const int sms = device_sm_count();
    long long g = (long long)bps * sms;
    const long long need = ((long long)ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    if (g > need) g = need;
    return g < 1 ? 1 : (int)g;
}

bool plan_valid(const iwpp_plan &p) {
    const int shape = shape_index(p.tile_h, p.tile_w);
    if (shape < 0) return false;
    if (p.sweeps < 0 || p.sweeps > 64 || p.revisit_sweeps < 0 || p.revisit_sweeps > 64) return false;
    if (p.smem_queue_cap < 16 || p.smem_queue_cap > p.tile_h * p.tile_w) return false;
    if (p.blocks_per_sm < 0 || p.blocks_per_sm > 32) return false;
    if (p.watchdog_ns < 0) return false;
    return true;
}

void default_plan(iwpp_plan *p) {
    p->tile_h = 32;
    p->tile_w = 32;
    p->sweeps = 1;
    p->revisit_sweeps = 0;
    p->smem_queue_cap = 512;
    p->blocks_per_sm = 0;
    p->watchdog_ns = 0;
}

// Workspace layout of a single-image call.
struct Layout {
    size_t hdr, state, queue, ovf, total;
    uint32_t ntiles, ovcap;
    int grid;
};

static bool image_ok(int64_t H, int64_t W) {
    return H >= 1 && W >= 1 && H < (1ll << 31) && W < (1ll << 31) &&
           (uint64_t)H * (uint64_t)W < (1ull << 32);
}

static bool make_layout(int64_t H, int64_t W, int dtype, int conn, const iwpp_plan &p, Layout &L) {
    if (!image_ok(H, W)) return false;
    const uint64_t tx = (W + p.tile_w - 1) / p.tile_w, ty = (H + p.tile_h - 1) / p.tile_h;
    if (tx * ty >= (1ull << 31)) return false;
    L.ntiles = (uint32_t)(tx * ty);
    L.grid = drain_grid(p, dtype, conn, L.ntiles);
    if (L.grid <= 0) return false;
    const uint32_t npix = (uint32_t)(p.tile_h * p.tile_w);
    L.ovcap = npix - (uint32_t)p.smem_queue_cap;
    L.hdr = 0;
    L.state = 256;
    L.queue = L.state + align256((size_t)L.ntiles * 4);
    L.ovf = L.queue + align256((size_t)L.ntiles * 4);
    L.total = L.ovf + align256((size_t)L.grid * kWarpsPerCta * 2 * L.ovcap * sizeof(uint16_t) + 16);
    return true;
}

// Phases of one call: bit 0 = workspace reset + scan kernel, bit 1 = persistent drain.
enum { kPhaseScan = 1, kPhaseDrain = 2 };

int reconstruct_one(void *marker, const void *mask, int64_t H, int64_t W, int conn, int op, int dtype,
                    const iwpp_plan *plan_in, void *ws, size_t ws_bytes, cudaStream_t stream,
                    int phases) {
    if (!marker || !mask) return IWPP_ERR_ARG;
    if (((uintptr_t)marker & 15) || ((uintptr_t)mask & 15)) return IWPP_ERR_ARG;
    if (!image_ok(H, W)) return IWPP_ERR_ARG;
    if (conn != 4 && conn != 8) return IWPP_ERR_ARG;
    if (op != IWPP_DILATE && op != IWPP_ERODE) return IWPP_ERR_ARG;
    if (dtype != IWPP_U8 && dtype != IWPP_U16) return IWPP_ERR_ARG;
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_plan(&p);
    if (!plan_valid(p)) return IWPP_ERR_ARG;
    if (!ws || ((uintptr_t)ws & 255)) return IWPP_ERR_WORKSPACE;
    Layout L;
    if (!make_layout(H, W, dtype, conn, p, L)) return IWPP_ERR_CUDA;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;

    uint8_t *base = static_cast<uint8_t *>(ws);
    EngineArgs a;
    a.img.J = static_cast<uint8_t *>(marker);
    a.img.I = static_cast<const uint8_t *>(mask);
    a.img.H = (int)H;
    a.img.W = (int)W;
    a.img.tiles_x = (int)((W + p.tile_w - 1) / p.tile_w);
    a.img.tiles_y = (int)((H + p.tile_h - 1) / p.tile_h);
    a.img.flip = op == IWPP_ERODE ? (dtype == IWPP_U8 ? 0xFFu : 0xFFFFu) : 0u;
    a.hdr = reinterpret_cast<WsHeader *>(base + L.hdr);
    a.state = reinterpret_cast<uint32_t *>(base + L.state);
    a.queue = reinterpret_cast<uint32_t *>(base + L.queue);
    a.ovf = reinterpret_cast<uint16_t *>(base + L.ovf);
    a.ntiles = L.ntiles;
    a.qcap = (uint32_t)p.smem_queue_cap;
    a.ovcap = L.ovcap;
    a.sweeps = p.sweeps;
    a.revisit_sweeps = p.revisit_sweeps;
    a.watchdog_ns = p.watchdog_ns > 0 ? p.watchdog_ns : 10ll * 1000 * 1000 * 1000;

    const int shape = shape_index(p.tile_h, p.tile_w);
    const KernelSet &k = kernels(shape, dtype, conn);
    const size_t smem = k.smem(a.qcap);
    if (ensure_smem_attr(shape, dtype, conn, smem) != cudaSuccess) return IWPP_ERR_CUDA;

    if (phases & kPhaseScan) {
        if (cudaMemsetAsync(base, 0, L.queue, stream) != cudaSuccess) return IWPP_ERR_CUDA;  // header + state
        if (cudaMemsetAsync(base + L.queue, 0xFF, (size_t)L.ntiles * 4, stream) != cudaSuccess)
            return IWPP_ERR_CUDA;
        const int sms = device_sm_count();
        const uint32_t ctas = (L.ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
        const uint32_t scan_grid = ctas < (uint32_t)(sms * 16) ? ctas : (uint32_t)(sms * 16);
        k.scan<<<scan_grid, kThreads, smem, stream>>>(a);
    }
    if (phases & kPhaseDrain) k.drain<<<L.grid, kThreads, smem, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

size_t workspace_bytes(int64_t H, int64_t W, int dtype, const iwpp_plan *plan_in) {
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_plan(&p);
    if (!plan_valid(p) || (dtype != 0 && dtype != 1)) return 0;
    Layout L;
    // conn does not change the layout; use the 8-connected kernels for the occupancy query
    if (!make_layout(H, W, dtype, 8, p, L)) return 0;
    Layout L4;
    if (!make_layout(H, W, dtype, 4, p, L4)) return 0;
    return L.total > L4.total ? L.total : L4.total;
}

}  // namespace iwpp

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" int iwpp_default_plan(iwpp_plan *plan) {
    if (!plan) return IWPP_ERR_ARG;
    iwpp::default_plan(plan);
    return IWPP_OK;
}

extern "C" int iwpp_tile_shape_supported(int32_t tile_h, int32_t tile_w) {
    return iwpp::shape_index(tile_h, tile_w) >= 0 ? 1 : 0;
}

extern "C" size_t iwpp_workspace_bytes(int64_t H, int64_t W, int dtype, const iwpp_plan *plan) {
    return iwpp::workspace_bytes(H, W, dtype, plan);
}

extern "C" int iwpp_reconstruct(void *marker_inout, const void *mask, int64_t H, int64_t W,
                                int connectivity, int op, int dtype, void *workspace, size_t ws_bytes,
                                void *stream) {
    return iwpp::reconstruct_one(marker_inout, mask, H, W, connectivity, op, dtype, nullptr, workspace,
                                 ws_bytes, static_cast<cudaStream_t>(stream), 3);
}

extern "C" int iwpp_reconstruct_plan(void *marker_inout, const void *mask, int64_t H, int64_t W,
                                     int connectivity, int op, int dtype, const iwpp_plan *plan,
                                     void *workspace, size_t ws_bytes, void *stream) {
    return iwpp::reconstruct_one(marker_inout, mask, H, W, connectivity, op, dtype, plan, workspace,
                                 ws_bytes, static_cast<cudaStream_t>(stream), 3);
}

extern "C" int iwpp_scan(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                         int op, int dtype, const iwpp_plan *plan, void *workspace, size_t ws_bytes,
                         void *stream) {
    return iwpp::reconstruct_one(marker_inout, mask, H, W, connectivity, op, dtype, plan, workspace,
                                 ws_bytes, static_cast<cudaStream_t>(stream), iwpp::kPhaseScan);
}

extern "C" int iwpp_drain(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                          int op, int dtype, const iwpp_plan *plan, void *workspace, size_t ws_bytes,
                          void *stream) {
    return iwpp::reconstruct_one(marker_inout, mask, H, W, connectivity, op, dtype, plan, workspace,
                                 ws_bytes, static_cast<cudaStream_t>(stream), iwpp::kPhaseDrain);
}

extern "C" int iwpp_sync_status(const void *workspace, void *stream) {
    if (!workspace) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t st = 0;
    if (cudaMemcpyAsync(&st, workspace, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return IWPP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return IWPP_ERR_CUDA;
    return (int)st;
}

extern "C" int iwpp_work_counters(const void *workspace, void *stream, uint64_t out[6]) {
    if (!workspace || !out) return IWPP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    iwpp::WsHeader h;
    if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return IWPP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return IWPP_ERR_CUDA;
    out[0] = h.visits;
    out[1] = h.pops;
    out[2] = h.seeds;
    out[3] = h.waves;
    out[4] = h.idle_ns;
    out[5] = h.busy_ns;
    return IWPP_OK;
}

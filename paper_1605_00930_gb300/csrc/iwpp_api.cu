// iwpp_api.cu — C ABI of the reconstruction paths (include/iwpp.h).
//
// Host code only validates arguments, carves the caller's workspace and enqueues
// kernels on the caller's stream:
//   single image: workspace reset (memsets) -> tile-parallel scan kernel
//     (precondition check, tile-local raster / anti-raster sweeps of Algorithm 7,
//     frontier initialisation) -> persistent drain kernel (Algorithm 7's irregular
//     propagation phase);
//   batch: image-table upload (descriptors as kernel parameters) -> reset -> mixed
//     scan kernel over every tile of every image (per-tile sweep counts) -> compact
//     kernel (initial frontier queued in schedule order) -> one persistent drain
//     over the whole batch.
// No host synchronisation and no allocation on these paths, so they can be captured
// in a CUDA graph.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_engine.cuh"
#include "iwpp_host.h"

#ifndef IWPP_SINGLE_SPREAD
#define IWPP_SINGLE_SPREAD 1   // single images queue their initial frontier in the spread order
#endif

namespace iwpp {

// ---- compiled tile shapes ---------------------------------------------------------------------
struct ShapeInfo {
    int th, tw;
};
static const ShapeInfo kShapes[] = {{32, 32}, {32, 64}, {64, 64}, {16, 32}, {16, 64}};
static constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int shape_index(int th, int tw) {
    for (int i = 0; i < kNumShapes; i++)
        if (kShapes[i].th == th && kShapes[i].tw == tw) return i;
    return -1;
}

// A scan / drain kernel pair with its shared-memory size function. Index [shape][v]:
// v = 0..3 single-image kinds (bit 0 = u16, bit 1 = 8-connectivity), v = 4 mixed batch,
// v = 5 / 6 batches of one connectivity (4 / 8) with both pixel types (cooperative solver
// only: its kernels read the pixel size from each image at run time).
struct KernelSet {
    void (*scan)(EngineArgs);
    void (*drain)(EngineArgs);
    size_t (*smem)(uint32_t);
    RegKernelSet reg;                // register local solver (16 x 64 tiles), else null
    RegKernelSet coop;               // cooperative local solver (64 x 64 tiles), else null
};
static constexpr int kMixed = 4, kAnyPix4 = 5, kAnyPix8 = 6, kVariants = 7;

template <typename T, int CONN, int TH, int TW>
static KernelSet make_set() {
    KernelSet k;
    k.scan = scan_kernel<T, CONN, TH, TW>;
    k.drain = drain_kernel<T, CONN, TH, TW>;
    k.smem = &Tile<T, CONN, TH, TW>::smem_bytes;
    k.reg = reg_kernel_set(TH, TW, (sizeof(T) == 2 ? 1 : 0) | (CONN == 8 ? 2 : 0));
    k.coop = coop_kernel_set(TH, TW, (sizeof(T) == 2 ? 1 : 0) | (CONN == 8 ? 2 : 0));
    return k;
}

template <int TH, int TW>
static size_t mixed_smem_bytes(uint32_t qcap) {
    return mixed_smem_per_warp<TH, TW>(qcap) * kWarpsPerCta;
}

template <int TH, int TW>
static void fill_shape(KernelSet (&row)[kVariants]) {
    row[0] = make_set<uint8_t, 4, TH, TW>();
    row[1] = make_set<uint16_t, 4, TH, TW>();
    row[2] = make_set<uint8_t, 8, TH, TW>();
    row[3] = make_set<uint16_t, 8, TH, TW>();
    row[kMixed].scan = scan_mixed_kernel<TH, TW>;
    row[kMixed].drain = drain_mixed_kernel<TH, TW>;
    row[kMixed].smem = &mixed_smem_bytes<TH, TW>;
    row[kMixed].reg = reg_kernel_set(TH, TW, kMixed);
    row[kMixed].coop = coop_kernel_set(TH, TW, kMixed);
    for (int v : {kAnyPix4, kAnyPix8}) {
        row[v].scan = nullptr;
        row[v].drain = nullptr;
        row[v].smem = nullptr;
        row[v].reg = reg_kernel_set(TH, TW, v);
        row[v].coop = coop_kernel_set(TH, TW, v);
    }
}

static KernelSet g_sets[kNumShapes][kVariants];
static int g_smem_set[kNumShapes][kVariants];
static std::once_flag g_once;
static std::mutex g_mu;

static void init_sets() {
    fill_shape<32, 32>(g_sets[0]);
    fill_shape<32, 64>(g_sets[1]);
    fill_shape<64, 64>(g_sets[2]);
    fill_shape<16, 32>(g_sets[3]);
    fill_shape<16, 64>(g_sets[4]);
}

static int kind_of(int dtype, int conn) { return (dtype == IWPP_U16 ? 1 : 0) | (conn == 8 ? 2 : 0); }

const KernelSet &kernels(int shape, int v) {
    std::call_once(g_once, init_sets);
    return g_sets[shape][v];
}

// Opt a kernel pair into the dynamic shared memory it needs (set once per process with
// a generous bound; the attribute belongs to the function).
static cudaError_t ensure_smem_attr(int shape, int v, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    int &done = g_smem_set[shape][v];
    if ((size_t)done >= bytes) return cudaSuccess;
    const KernelSet &k = kernels(shape, v);
    const int want = (int)(bytes < 100 * 1024 ? 100 * 1024 : bytes);
    cudaError_t e;
    for (void (*f)(EngineArgs) : {k.scan, k.drain, k.reg.scan, k.reg.drain, k.reg.drain_hi, k.coop.scan, k.coop.drain,
                                  k.coop.scan_sweeps, k.coop.scan_feats}) {
        if (!f) continue;
        e = cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e != cudaSuccess) return e;
    }
    done = want;
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// The scan and persistent kernels of a plan (queue or register local solver) and their
// shared memory. Register plans asking for more than kRegBlocks CTAs per SM get the
// high-occupancy build of the persistent kernel.
static void (*drain_fn(const iwpp_plan &p, const KernelSet &k))(EngineArgs) {
    if (p.local_solver == IWPP_SOLVER_COOP) return k.coop.drain;
    if (p.local_solver != IWPP_SOLVER_REGISTER) return k.drain;
    return p.blocks_per_sm > kRegBlocks ? k.reg.drain_hi : k.reg.drain;
}
static void (*scan_fn(const iwpp_plan &p, const KernelSet &k, bool sweeps))(EngineArgs) {
    if (p.local_solver == IWPP_SOLVER_COOP) return sweeps && k.coop.scan_sweeps ? k.coop.scan_sweeps : k.coop.scan;
    return p.local_solver == IWPP_SOLVER_REGISTER ? k.reg.scan : k.scan;
}
static size_t drain_smem(const iwpp_plan &p, const KernelSet &k) {
    if (p.local_solver == IWPP_SOLVER_COOP) return k.coop.smem((uint32_t)p.smem_queue_cap);
    return p.local_solver == IWPP_SOLVER_REGISTER ? k.reg.smem((uint32_t)p.smem_queue_cap)
                                                  : k.smem((uint32_t)p.smem_queue_cap);
}
// Whether the plan's solver has kernels for this set (the cooperative solver has none for
// mixed batches, the register solver none for shapes other than 16 x 64).
static bool has_kernels(const iwpp_plan &p, const KernelSet &k) {
    if (p.local_solver == IWPP_SOLVER_COOP) return k.coop.scan && k.coop.drain && k.coop.smem;
    if (p.local_solver == IWPP_SOLVER_REGISTER)
        return k.reg.scan && k.reg.smem && (p.blocks_per_sm > kRegBlocks ? k.reg.drain_hi : k.reg.drain);
    return k.scan && k.drain && k.smem;
}

// Tiles one persistent CTA works on at a time: one per warp, or one per CTA (cooperative).
static int tiles_per_cta(const iwpp_plan &p) { return p.local_solver == IWPP_SOLVER_COOP ? 1 : kWarpsPerCta; }

// Persistent CTAs for a plan: blocks_per_sm (or the occupancy maximum) x SMs, never more
// CTAs than needed to give every tile its own warp.
static int drain_grid(const iwpp_plan &p, int v, uint32_t ntiles) {
    const int shape = shape_index(p.tile_h, p.tile_w);
    if (shape < 0) return 0;
    const KernelSet &k = kernels(shape, v);
    if (!has_kernels(p, k)) return 0;
    const size_t smem = drain_smem(p, k);
    if (ensure_smem_attr(shape, v, k.smem ? k.smem((uint32_t)p.smem_queue_cap) : smem) != cudaSuccess) return 0;
    int bps = p.blocks_per_sm;
    if (bps <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, drain_fn(p, k), kThreads, smem) != cudaSuccess)
            return 0;
        if (bps <= 0) return 0;
    }
    const int sms = device_sm_count();
    long long g = (long long)bps * sms;
    const long long need = ((long long)ntiles + tiles_per_cta(p) - 1) / tiles_per_cta(p);
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
    if (p.local_solver != IWPP_SOLVER_QUEUE && p.local_solver != IWPP_SOLVER_REGISTER &&
        p.local_solver != IWPP_SOLVER_COOP)
        return false;
    if (p.local_solver == IWPP_SOLVER_COOP &&
        (!coop_kernel_set(p.tile_h, p.tile_w, 0).drain || p.value_levels > 1 || p.blocks_per_sm > kCoopBlocks ||
         p.revisit_sweeps != 0))
        return false;
    if (p.local_solver == IWPP_SOLVER_REGISTER && !reg_kernel_set(p.tile_h, p.tile_w, 0).drain) return false;
    if (p.value_levels < 0 || p.value_levels > kMaxLevels) return false;
    if (p.value_levels > 1 && p.local_solver != IWPP_SOLVER_REGISTER) return false;
    return true;
}

// The measured best static plan, for single images and batches alike: 64 x 64 tiles
// settled by the cooperative solver (one tile per CTA of four warps), no sweeps before the
// persistent kernel (the scan kernel still checks the precondition and collects the
// frontier). The autotuner picked it on every batch measured.
void default_plan(iwpp_plan *p) {
    p->tile_h = 64;
    p->tile_w = 64;
    p->sweeps = 0;
    p->revisit_sweeps = 0;
    p->smem_queue_cap = 512;
    p->blocks_per_sm = 0;
    p->local_solver = IWPP_SOLVER_COOP;
    p->value_levels = 0;
    p->watchdog_ns = 0;
}

void default_batch_plan(iwpp_plan *p) { default_plan(p); }

// Pixel offsets are 64-bit everywhere; sides stay below 2^31 (ints in the kernels) and
// the pixel count below 2^40, which keeps the tile count of any plan below 2^31.
static bool image_ok(int64_t H, int64_t W) {
    return H >= 1 && W >= 1 && H < (1ll << 31) && W < (1ll << 31) &&
           (uint64_t)H * (uint64_t)W < (1ull << 40);
}

static ImageView make_view(void *marker, const void *mask, int64_t H, int64_t W, int conn, int op, int dtype,
                           const iwpp_plan &p, uint32_t tile_base) {
    ImageView v;
    v.J = static_cast<uint8_t *>(marker);
    v.I = static_cast<const uint8_t *>(mask);
    v.H = (int)H;
    v.W = (int)W;
    v.tiles_x = (int)((W + p.tile_w - 1) / p.tile_w);
    v.tiles_y = (int)((H + p.tile_h - 1) / p.tile_h);
    v.flip = op == IWPP_ERODE ? (dtype == IWPP_U8 ? 0xFFu : 0xFFFFu) : 0u;
    v.tile_base = tile_base;
    v.kind = (uint32_t)kind_of(dtype, conn);
    v.pad = 0;
    return v;
}

static void fill_common(EngineArgs &a, const iwpp_plan &p, uint8_t *base, size_t off_state, size_t off_queue,
                        size_t off_ovf, uint32_t ntiles, uint32_t ovcap) {
    a.hdr = reinterpret_cast<WsHeader *>(base);
    a.state = reinterpret_cast<uint32_t *>(base + off_state);
    a.queue = reinterpret_cast<uint32_t *>(base + off_queue);
    a.ovf = reinterpret_cast<uint16_t *>(base + off_ovf);
    a.ntiles = ntiles;
    a.qcap = (uint32_t)p.smem_queue_cap;
    a.ovcap = ovcap;
    a.sweeps = p.sweeps;
    a.revisit_sweeps = p.revisit_sweeps;
    a.tile_sweeps = nullptr;
    a.order = nullptr;
    a.spread = 0;
    a.tile_work = nullptr;
    a.defer_push = 0;
    a.watchdog_ns = p.watchdog_ns > 0 ? p.watchdog_ns : 10ll * 1000 * 1000 * 1000;
    a.imgs = nullptr;
    a.nimg = 0;
    a.nlevels = p.value_levels > 1 ? (uint32_t)p.value_levels : 1u;
    a.lvl = nullptr;
    a.tile_img = nullptr;
    a.feats = nullptr;
    a.sweep_only = 0;
}

// ---- single image ------------------------------------------------------------------------------
// Workspace: header (256 B) | tile states | level counters | tile-queue slots (one ring per
// value level) | per-warp overflow queues.
struct Layout {
    size_t state, lvl, queue, ovf, total;
    uint32_t ntiles, ovcap, nlevels;
    int grid;
};

static bool make_layout(int64_t H, int64_t W, int v, const iwpp_plan &p, Layout &L) {
    if (!image_ok(H, W)) return false;
    const uint64_t tx = (W + p.tile_w - 1) / p.tile_w, ty = (H + p.tile_h - 1) / p.tile_h;
    if (tx * ty >= (1ull << 31)) return false;
    L.ntiles = (uint32_t)(tx * ty);
    L.grid = drain_grid(p, v, L.ntiles);
    if (L.grid <= 0) return false;
    // per-warp overflow queues: the queue solver's only
    L.ovcap = p.local_solver == IWPP_SOLVER_QUEUE ? (uint32_t)(p.tile_h * p.tile_w - p.smem_queue_cap) : 0u;
    L.nlevels = p.value_levels > 1 ? (uint32_t)p.value_levels : 1u;
    L.state = 256;
    L.lvl = L.state + align256((size_t)L.ntiles * 4);
    L.queue = L.lvl + align256(sizeof(LevelCtr) * kMaxLevels);
    L.ovf = L.queue + align256((size_t)L.ntiles * 4 * L.nlevels);
    L.total = L.ovf + align256((size_t)L.grid * kWarpsPerCta * 2 * L.ovcap * sizeof(uint16_t) + 16);
    return true;
}


int reconstruct_one(void *marker, const void *mask, int64_t H, int64_t W, int conn, int op, int dtype,
                    const iwpp_plan *plan_in, void *ws, size_t ws_bytes, cudaStream_t stream, int phases) {
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
    const int v = kind_of(dtype, conn);
    Layout L;
    if (!make_layout(H, W, v, p, L)) return IWPP_ERR_CUDA;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;

    uint8_t *base = static_cast<uint8_t *>(ws);
    EngineArgs a;
    fill_common(a, p, base, L.state, L.queue, L.ovf, L.ntiles, L.ovcap);
    a.img0 = make_view(marker, mask, H, W, conn, op, dtype, p, 0);
    a.lvl = reinterpret_cast<LevelCtr *>(base + L.lvl);

    const int shape = shape_index(p.tile_h, p.tile_w);
    const KernelSet &k = kernels(shape, v);
    const size_t smem = k.smem(a.qcap);
    if (ensure_smem_attr(shape, v, smem) != cudaSuccess) return IWPP_ERR_CUDA;

    if (phases & kPhaseScan) {
        // header, tile states, level counters
        if (cudaMemsetAsync(base, 0, L.queue, stream) != cudaSuccess) return IWPP_ERR_CUDA;
        if (cudaMemsetAsync(base + L.queue, 0xFF, (size_t)L.ntiles * 4 * L.nlevels, stream) != cudaSuccess)
            return IWPP_ERR_CUDA;
        const int sms = device_sm_count();
        const uint32_t ctas = (L.ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
        const uint32_t scan_grid = ctas < (uint32_t)(sms * 16) ? ctas : (uint32_t)(sms * 16);
        // one FIFO: the scan marks tiles PENDING and the initial frontier is queued in the
        // spread order, as in batches; value levels: the scan queues each tile as it finds it
        const bool spread = IWPP_SINGLE_SPREAD && L.nlevels <= 1;
        if (spread) {
            a.defer_push = 1;
            a.spread = spread_multiplier(L.ntiles);
        }
        scan_fn(p, k, p.sweeps > 0)<<<scan_grid, kThreads, drain_smem(p, k), stream>>>(a);
        if (spread) {
            const uint32_t cgrid = (L.ntiles + 255) / 256 < (uint32_t)(sms * 8) ? (L.ntiles + 255) / 256
                                                                                 : (uint32_t)(sms * 8);
            compact_kernel<<<cgrid, 256, 0, stream>>>(a);
            finalize_queue_kernel<<<cgrid, 256, 0, stream>>>(a);
            a.defer_push = 0;
        }
    }
    if (phases & kPhaseDrain) drain_fn(p, k)<<<L.grid, kThreads, drain_smem(p, k), stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

size_t workspace_bytes(int64_t H, int64_t W, int dtype, const iwpp_plan *plan_in) {
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_plan(&p);
    if (!plan_valid(p) || (dtype != 0 && dtype != 1)) return 0;
    size_t best = 0;
    for (int conn = 4; conn <= 8; conn += 4) {   // the layout is the larger of the two kernels'
        Layout L;
        if (!make_layout(H, W, kind_of(dtype, conn), p, L)) return 0;
        if (L.total > best) best = L.total;
    }
    return best;
}

// ---- batch -------------------------------------------------------------------------------------
// Workspace: header (256 B) | image table | tile states | tile-queue slots | tile -> image map |
// overflow queues. Tiles are numbered image by image, row-major inside an image.
struct BatchLayout {
    size_t table, state, queue, timg, ovf, total;
    uint32_t ntiles, ovcap;
    int grid;
};

static int check_image(const iwpp_image &d) {
    if (!d.marker_inout || !d.mask) return IWPP_ERR_ARG;
    if (((uintptr_t)d.marker_inout & 15) || ((uintptr_t)d.mask & 15)) return IWPP_ERR_ARG;
    if (!image_ok(d.H, d.W)) return IWPP_ERR_ARG;
    if (d.connectivity != 4 && d.connectivity != 8) return IWPP_ERR_ARG;
    if (d.op != IWPP_DILATE && d.op != IWPP_ERODE) return IWPP_ERR_ARG;
    if (d.dtype != IWPP_U8 && d.dtype != IWPP_U16) return IWPP_ERR_ARG;
    return IWPP_OK;
}

// Total tiles of a batch (or -1 on a bad argument); bases[i] = first tile of image i.
int64_t batch_tiles(const iwpp_image *imgs, int n, const iwpp_plan &p, std::vector<uint32_t> *bases) {
    if (!imgs || n < 1) return -1;
    uint64_t total = 0;
    if (bases) bases->resize(n);
    for (int i = 0; i < n; i++) {
        if (check_image(imgs[i]) != IWPP_OK) return -1;
        if (bases) (*bases)[i] = (uint32_t)total;
        total += (uint64_t)((imgs[i].W + p.tile_w - 1) / p.tile_w) * (uint64_t)((imgs[i].H + p.tile_h - 1) / p.tile_h);
        if (total >= (1ull << 31)) return -1;
    }
    return (int64_t)total;
}

// Kernel variant of a batch: the specialised one when every image has the same pixel
// type and connectivity; under the cooperative solver, the one of the batch's
// connectivity when only the pixel types differ; else the mixed one.
static int batch_variant(const iwpp_image *imgs, int n, const iwpp_plan &p) {
    const int v = kind_of(imgs[0].dtype, imgs[0].connectivity);
    bool same_kind = true, same_conn = true;
    for (int i = 1; i < n; i++) {
        same_kind = same_kind && kind_of(imgs[i].dtype, imgs[i].connectivity) == v;
        same_conn = same_conn && imgs[i].connectivity == imgs[0].connectivity;
    }
    if (same_kind) return v;
    if (same_conn && p.local_solver == IWPP_SOLVER_COOP) return imgs[0].connectivity == 8 ? kAnyPix8 : kAnyPix4;
    return kMixed;
}

static bool make_batch_layout(const iwpp_image *imgs, int n, const iwpp_plan &p, BatchLayout &L,
                              std::vector<uint32_t> *bases) {
    const int64_t nt = batch_tiles(imgs, n, p, bases);
    if (nt < 1) return false;
    L.ntiles = (uint32_t)nt;
    L.grid = drain_grid(p, batch_variant(imgs, n, p), L.ntiles);
    if (L.grid <= 0) return false;
    L.ovcap = p.local_solver == IWPP_SOLVER_QUEUE ? (uint32_t)(p.tile_h * p.tile_w - p.smem_queue_cap) : 0u;
    L.table = 256;
    L.state = L.table + align256((size_t)n * sizeof(ImageView));
    L.queue = L.state + align256((size_t)L.ntiles * 4);
    L.timg = L.queue + align256((size_t)L.ntiles * 4);
    L.ovf = L.timg + align256((size_t)L.ntiles * 4);
    L.total = L.ovf + align256((size_t)L.grid * kWarpsPerCta * 2 * L.ovcap * sizeof(uint16_t) + 16);
    return true;
}

size_t batch_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan_in) {
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_batch_plan(&p);
    if (!plan_valid(p)) return 0;
    BatchLayout L;
    if (!make_batch_layout(imgs, n, p, L, nullptr)) return 0;
    return L.total;
}

int reconstruct_batch(const iwpp_image *imgs, int n, const iwpp_plan *plan_in, const uint32_t *order,
                      const uint8_t *tile_sweeps, uint32_t *tile_work, void *ws, size_t ws_bytes,
                      cudaStream_t stream, int phases, const LearnedCall *learned) {
    if (phases < 1 || phases > 3) return IWPP_ERR_ARG;
    if (learned && (!learned->params || !learned->order || !learned->sweeps || !learned->sws)) return IWPP_ERR_ARG;
    if (learned) {   // the schedule the call makes is the one it queues and sweeps by
        order = learned->order;
        tile_sweeps = learned->sweeps;
    }
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_batch_plan(&p);
    if (!plan_valid(p) || p.value_levels > 1) return IWPP_ERR_ARG;   // batches: one FIFO
    if (!imgs || n < 1) return IWPP_ERR_ARG;
    for (int i = 0; i < n; i++)
        if (check_image(imgs[i]) != IWPP_OK) return IWPP_ERR_ARG;
    if (!ws || ((uintptr_t)ws & 255)) return IWPP_ERR_WORKSPACE;
    std::vector<uint32_t> bases;
    BatchLayout L;
    if (!make_batch_layout(imgs, n, p, L, &bases)) return IWPP_ERR_ARG;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;

    uint8_t *base = static_cast<uint8_t *>(ws);
    EngineArgs a;
    fill_common(a, p, base, L.state, L.queue, L.ovf, L.ntiles, L.ovcap);
    ImageView *table = reinterpret_cast<ImageView *>(base + L.table);
    a.imgs = table;
    a.nimg = n;
    a.img0 = make_view(imgs[0].marker_inout, imgs[0].mask, imgs[0].H, imgs[0].W, imgs[0].connectivity,
                       imgs[0].op, imgs[0].dtype, p, 0);
    a.tile_sweeps = tile_sweeps;
    a.order = order;
    a.spread = spread_multiplier(L.ntiles);
    a.tile_work = tile_work;
    a.defer_push = 1;
    a.tile_img = reinterpret_cast<const uint32_t *>(base + L.timg);

    const int shape = shape_index(p.tile_h, p.tile_w);
    const int variant = batch_variant(imgs, n, p);
    const KernelSet &k = kernels(shape, variant);
    const size_t smem = k.smem ? k.smem(a.qcap) : drain_smem(p, k);
    if (ensure_smem_attr(shape, variant, smem) != cudaSuccess) return IWPP_ERR_CUDA;
    // learned: features from the scan kernel when the plan's tiles are the feature blocks
    // (cooperative 64 x 64 tiles; not the mixed-kind build), else a features pass first
    const bool fused = learned && p.local_solver == IWPP_SOLVER_COOP && k.coop.scan_feats &&
                       p.tile_h == IWPP_FEATURE_BLOCK && p.tile_w == IWPP_FEATURE_BLOCK;

    if ((phases & kPhaseScan) == 0) {   // drain only: the prepared workspace is reused
        drain_fn(p, k)<<<L.grid, kThreads, drain_smem(p, k), stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
    }
    // image table: descriptors travel as kernel parameters (no host-to-device copy)
    for (int first = 0; first < n; first += kDescChunk) {
        DescChunk c;
        c.first = first;
        c.count = n - first < kDescChunk ? n - first : kDescChunk;
        for (int j = 0; j < c.count; j++) {
            const iwpp_image &d = imgs[first + j];
            c.v[j] = make_view(d.marker_inout, d.mask, d.H, d.W, d.connectivity, d.op, d.dtype, p, bases[first + j]);
        }
        upload_descs_kernel<<<1, kDescChunk, 0, stream>>>(table, c);
    }
    {
        const int sms = device_sm_count();
        const int g = n < sms * 4 ? n : sms * 4;
        tile_image_kernel<<<g, 256, 0, stream>>>(table, n, reinterpret_cast<uint32_t *>(base + L.timg));
    }
    if (cudaMemsetAsync(base, 0, 256, stream) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaMemsetAsync(base + L.state, 0, (size_t)L.ntiles * 4, stream) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaMemsetAsync(base + L.queue, 0xFF, (size_t)L.ntiles * 4, stream) != cudaSuccess) return IWPP_ERR_CUDA;
    const int sms = device_sm_count();
    const uint32_t ctas = (L.ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    const uint32_t scan_grid = ctas < (uint32_t)(sms * 16) ? ctas : (uint32_t)(sms * 16);
    if (learned && !fused) {   // features, MLP and order before the scan, which runs the sweeps
        const int rc = schedule_batch(imgs, n, p, learned->params, learned->order, learned->sweeps, learned->sws,
                                      learned->sws_bytes, stream, 7);
        if (rc != IWPP_OK) return rc;
    }
    if (fused) {
        // scan that also writes every tile's features (no sweeps yet) -> MLP and order ->
        // sweeps-only pass
        float *feats = sched_features(imgs, n, p, learned->sws, learned->sws_bytes);
        if (!feats) return IWPP_ERR_WORKSPACE;
        a.feats = feats;
        a.tile_sweeps = nullptr;
        k.coop.scan_feats<<<scan_grid, kThreads, drain_smem(p, k), stream>>>(a);
        if (cudaGetLastError() != cudaSuccess) return IWPP_ERR_CUDA;
        a.feats = nullptr;
        int rc = schedule_batch(imgs, n, p, learned->params, learned->order, learned->sweeps, learned->sws,
                            learned->sws_bytes, stream, 6);
        if (rc != IWPP_OK) return rc;
        a.tile_sweeps = learned->sweeps;
        a.sweep_only = 1;
        k.coop.scan_sweeps<<<scan_grid, kThreads, drain_smem(p, k), stream>>>(a);
        a.sweep_only = 0;
    } else {
        scan_fn(p, k, p.sweeps > 0 || tile_sweeps != nullptr)<<<scan_grid, kThreads, drain_smem(p, k), stream>>>(a);
    }
    const uint32_t cgrid = (L.ntiles + 255) / 256 < (uint32_t)(sms * 8) ? (L.ntiles + 255) / 256 : (uint32_t)(sms * 8);
    compact_kernel<<<cgrid, 256, 0, stream>>>(a);
    finalize_queue_kernel<<<cgrid, 256, 0, stream>>>(a);
    if (phases & kPhaseDrain) drain_fn(p, k)<<<L.grid, kThreads, drain_smem(p, k), stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

// Kernel launches one batch call makes (for launch accounting by callers); bit 2 of
// `phases`: a learned call with the features in the scan (the schedule's table chunks, MLP,
// keys, bucket scan and scatter, and the sweeps-only pass come on top).
int batch_launches(int n, int phases) {
    const int chunks = (n + kDescChunk - 1) / kDescChunk;
    int prep = chunks + 4;   // table chunks, tile map, scan, compact, finalize
    if (phases & 4) prep += chunks + 5;   // schedule table chunks, MLP, keys, bucket scan, scatter, sweeps
    return ((phases & kPhaseScan) ? prep : 0) + ((phases & kPhaseDrain) ? 1 : 0);
}

}  // namespace iwpp

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" int iwpp_default_plan(iwpp_plan *plan) {
    if (!plan) return IWPP_ERR_ARG;
    iwpp::default_plan(plan);
    return IWPP_OK;
}

extern "C" int iwpp_default_batch_plan(iwpp_plan *plan) {
    if (!plan) return IWPP_ERR_ARG;
    iwpp::default_batch_plan(plan);
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

extern "C" int64_t iwpp_batch_tile_count(const iwpp_image *imgs, int n, const iwpp_plan *plan) {
    iwpp_plan p;
    if (plan) p = *plan; else iwpp::default_batch_plan(&p);
    if (!iwpp::plan_valid(p)) return -1;
    return iwpp::batch_tiles(imgs, n, p, nullptr);
}

extern "C" size_t iwpp_batch_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan) {
    return iwpp::batch_workspace_bytes(imgs, n, plan);
}

extern "C" int iwpp_reconstruct_batch(const iwpp_image *imgs, int n, const iwpp_plan *plan, void *workspace,
                                      size_t ws_bytes, void *stream) {
    return iwpp::reconstruct_batch(imgs, n, plan, nullptr, nullptr, nullptr, workspace, ws_bytes,
                                   static_cast<cudaStream_t>(stream), iwpp::kPhaseScan | iwpp::kPhaseDrain);
}

extern "C" int iwpp_reconstruct_batch_sched(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                            const uint32_t *tile_order, const uint8_t *tile_sweeps,
                                            uint32_t *tile_work, void *workspace, size_t ws_bytes,
                                            void *stream) {
    return iwpp::reconstruct_batch(imgs, n, plan, tile_order, tile_sweeps, tile_work, workspace, ws_bytes,
                                   static_cast<cudaStream_t>(stream), iwpp::kPhaseScan | iwpp::kPhaseDrain);
}

extern "C" int iwpp_reconstruct_batch_phase(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                            const uint32_t *tile_order, const uint8_t *tile_sweeps,
                                            uint32_t *tile_work, int phases, void *workspace, size_t ws_bytes,
                                            void *stream) {
    return iwpp::reconstruct_batch(imgs, n, plan, tile_order, tile_sweeps, tile_work, workspace, ws_bytes,
                                   static_cast<cudaStream_t>(stream), phases);
}

extern "C" int iwpp_batch_launch_count(int n, int phases) {
    if (n < 1 || (phases & 3) == 0 || phases > 7) return -1;
    return iwpp::batch_launches(n, phases);
}

extern "C" int iwpp_reconstruct_batch_learned(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                              const float *params, uint32_t *tile_order, uint8_t *tile_sweeps,
                                              void *sched_ws, size_t sws_bytes, int phases, void *workspace,
                                              size_t ws_bytes, void *stream) {
    const iwpp::LearnedCall lc = {params, tile_order, tile_sweeps, sched_ws, sws_bytes};
    return iwpp::reconstruct_batch(imgs, n, plan, nullptr, nullptr, nullptr, workspace, ws_bytes,
                                   static_cast<cudaStream_t>(stream), phases, &lc);
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

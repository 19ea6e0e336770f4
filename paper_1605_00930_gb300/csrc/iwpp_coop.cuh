// iwpp_coop.cuh — the cooperative local solver (plan local_solver = IWPP_SOLVER_COOP): one
// CTA settles a 64 x 64 tile. Each of its four warps holds a 16-row strip in registers (the
// register solver's layout: two columns per lane, packed u16x2) and runs the register
// solver's down / up passes on it; after every pass pair the strips exchange their first and
// last rows through shared memory, and the CTA iterates until no strip can change. A path
// that crosses the tile vertically then costs a few passes instead of several trips through
// the tile queue, which is what bounds the drain when one chain of tile hops is the critical
// path. The tile queue protocol (pop, notify, finish) is the persistent engine's, run by warp 0
// on behalf of the CTA. Kernels specialised on pixel type and connectivity serve single
// images and uniform batches; the mixed build dispatches on each tile's image kind.
#pragma once

#include "iwpp_regtile.cuh"

namespace iwpp {

constexpr int kCoopStrip = 16;                        // rows per warp
constexpr int kCoopRows = kCoopStrip * kWarpsPerCta;  // rows per CTA tile

struct CoopShared {
    uint32_t rows[kWarpsPerCta][2][32];   // each strip's first and last row, per lane
    uint32_t misc[16];                    // the CTA tile's notification values (3 x 3 grid)
    uint32_t tile, redo;
    // Run statistics, kept here rather than in registers that would stay live through every
    // visit's passes (measured: fewer spills, drains 2-3 % faster); flushed at the end.
    unsigned long long k0, idle, visits, waves[kWarpsPerCta];   // start time, pop waits (warp 0), visits, passes
    long long c0;                                               // warp 0: the visit's start clock
};

#ifndef IWPP_CHG_XOR
#define IWPP_CHG_XOR 1   // 1: passes track "this lane changed something"; a lane that did stores all its rows
#endif

#ifndef IWPP_SCAN_VEC
#define IWPP_SCAN_VEC 0   // 1: the scan kernels copy strips with 16-byte asynchronous copies where rows allow
#endif

template <typename T, int CONN>
__host__ __device__ constexpr size_t coop_smem_bytes() {
    return RegTile<T, CONN, kCoopStrip>::smem_per_warp(0) * kWarpsPerCta + sizeof(CoopShared);
}
// The scan kernels' staging area for 16-byte copies follows the drain's layout (16-byte aligned).
template <typename T, int CONN>
__host__ __device__ constexpr size_t coop_scan_stage_offset() {
    return (coop_smem_bytes<T, CONN>() + 15) & ~(size_t)15;
}
template <typename T, int CONN>
size_t coop_smem_fn(uint32_t) {
    return IWPP_SCAN_VEC ? coop_scan_stage_offset<T, CONN>() + kWarpsPerCta * RegTile<T, CONN, kCoopStrip>::kStageBytes
                         : coop_smem_bytes<T, CONN>();
}

// Fold one strip's notification values (3 x 3 grid around the strip) into the CTA tile's:
// the strip's top side is the tile's only for warp 0 (inside the tile otherwise, where the
// strips already agree), its bottom side only for the last warp, and a strip's corner
// pixels outside the tile's top / bottom rows lie in the tile's west / east neighbours.
__device__ __forceinline__ void coop_fold_misc(CoopShared &C, const uint32_t *m, int w) {
    if (w == 0) {
        atomicMax(&C.misc[0], m[0]);
        atomicMax(&C.misc[1], m[1]);
        atomicMax(&C.misc[2], m[2]);
    } else {
        atomicMax(&C.misc[3], m[0]);
        atomicMax(&C.misc[5], m[2]);
    }
    if (w == kWarpsPerCta - 1) {
        atomicMax(&C.misc[6], m[6]);
        atomicMax(&C.misc[7], m[7]);
        atomicMax(&C.misc[8], m[8]);
    } else {
        atomicMax(&C.misc[3], m[6]);
        atomicMax(&C.misc[5], m[8]);
    }
    atomicMax(&C.misc[3], m[3]);
    atomicMax(&C.misc[5], m[5]);
}

#if IWPP_PHASE_TIMING
#define IWPP_CO_MARK(k)                                  \
    do {                                                 \
        if (w == 0) {                                    \
            const long long _n = clock64();              \
            ph[k] += (unsigned long long)(_n - pt);      \
            pt = _n;                                     \
        }                                                \
    } while (0)
#else
#define IWPP_CO_MARK(k) \
    do {                \
    } while (0)
#endif

// One visit of CTA tile t by the whole CTA (every thread calls it with the same t), including
// the re-processing rounds when the tile is notified while the CTA holds it.
template <typename T, int CONN>
__device__ void visit_tile_coop(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem,
                                CoopShared &C, unsigned long long *ph, int w, int lane) {
    (void)ph;
#if IWPP_PHASE_TIMING
    long long pt = clock64();
#endif
    if (w == 0 && lane == 0) C.c0 = clock64();
    constexpr int TH = kCoopStrip;
    using RT = RegTile<T, CONN, TH>;
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = RT::halo_words(s, lane);
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * kCoopRows + TH * w, x0 = tx * RT::TW;
    if (lane < 16) s.misc[lane] = 0;
    if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
    IWPP_CO_MARK(6);
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    IWPP_CO_MARK(0);
    uint32_t passes = 0;
    // settled: the strip is a fixed point of J <- min(I, max over the neighbourhood) for
    // its current halo
    bool settled = false;
    for (;;) {
        uint32_t rows = 0;
        bool up_fresh = false;   // the strip's last pass was an up pass run with its current halo
        for (;;) {   // joint iterations of the strips
            if (!settled) {
                const uint32_t chd = RT::template pass_down<IWPP_CHG_XOR>(hx, J, I, jt, lane);
                passes++;
                rows |= chd;
                // A down pass that changes nothing right after an up pass with the same halo
                // leaves every pixel checked, with final values, against its neighbours below
                // (by the up pass) and above and beside it (by the down pass): settled.
                if (up_fresh && !__any_sync(0xffffffffu, chd != 0)) {
                    settled = true;
                } else {
                    const uint32_t chu = RT::template pass_up<IWPP_CHG_XOR>(hx, J, I, jb, lane);
                    passes++;
                    rows |= chu;
                    // likewise an up pass that changes nothing after a down pass with the same
                    // halo (a strip that changed may still be short of its fixed point: its
                    // next pass finds out, measured cheaper than a residual check here)
                    settled = !__any_sync(0xffffffffu, chu != 0);
                    up_fresh = true;
                }
            }
            C.rows[w][0][lane] = J[0];
            C.rows[w][1][lane] = J[TH - 1];
            __syncthreads();
            const uint32_t njt = w > 0 ? C.rows[w - 1][1][lane] : jt;
            const uint32_t njb = w < kWarpsPerCta - 1 ? C.rows[w + 1][0][lane] : jb;
            const bool tchg = __any_sync(0xffffffffu, njt != jt), bchg = __any_sync(0xffffffffu, njb != jb);
            if (tchg || bchg) {   // a neighbour strip's boundary row changed: new work possible
                up_fresh = false;
                settled = false;
            }
            jt = njt;
            jb = njb;
            if (!__syncthreads_or(!settled)) break;
        }
        if (w == 0 && lane == 0) C.visits++;
        IWPP_CO_MARK(1);
        if (__syncthreads_or(rows != 0)) {
#if IWPP_CHG_XOR
            // a lane that changed a pixel writes all its rows inside the image
            const int nin = im.H - y0;
            rows = rows == 0 || nin <= 0 ? 0u : (nin >= TH ? 0xFFFFu : (1u << nin) - 1u);
#endif
            RT::store(im, y0, x0, J, rows, lane);
            RT::notify_scan(s, J, jt, jb, it, ib, lane);
            if (lane == 0) coop_fold_misc(C, s.misc, w);
            fence_protocol();
            __syncthreads();
            IWPP_CO_MARK(2);
            if (w == 0 && lane < 9 && lane != 4 && C.misc[lane]) {
                const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
                if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                    notify_tile(a, im.tile_base + (uint32_t)(ny * im.tiles_x + nx));
            }
            IWPP_CO_MARK(3);
        }
        if (w == 0) {
            const bool r = finish_tile(a, t, lane);
            if (lane == 0) C.redo = r;
        }
        IWPP_CO_MARK(4);
        __syncthreads();
        const bool redo = C.redo != 0;
        if (!redo) break;
        // re-process: J and I stay in registers; only the tile's halo can have changed
        if (lane < 16) s.misc[lane] = 0;
        if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
        RT::load_halo(im, s, y0, x0, jt, jb, it, ib, false, lane);
        __syncthreads();
        settled = false;
        IWPP_CO_MARK(5);
    }
    if (lane == 0) C.waves[w] += passes;
    if (w == 0 && lane == 0 && a.tile_work) {   // per-tile work: warp 0's passes, the visit's SM cycles
        atomicAdd(a.tile_work + t, passes);
        atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - C.c0, 0x7fffffffll));
    }
}

// One CTA tile visit, dispatched on the tile's image kind (CTA-uniform: one tile per CTA).
template <typename T, int CONN, bool MIXED>
__device__ __forceinline__ void visit_tile_coop_any(const EngineArgs &a, uint32_t t, uint8_t *wsmem, CoopShared &C,
                                                    unsigned long long *ph, int w, int lane) {
#if IWPP_PHASE_TIMING
    const long long c0 = clock64();
#endif
    const ImageView &im = image_of(a, t);
#if IWPP_PHASE_TIMING
    if (w == 0) ph[7] += (unsigned long long)(clock64() - c0);
#endif
    if (!MIXED) {
        visit_tile_coop<T, CONN>(a, im, t, wsmem, C, ph, w, lane);
        return;
    }
    switch (im.kind) {
        case 0: visit_tile_coop<uint8_t, 4>(a, im, t, wsmem, C, ph, w, lane); break;
        case 1: visit_tile_coop<uint16_t, 4>(a, im, t, wsmem, C, ph, w, lane); break;
        case 2: visit_tile_coop<uint8_t, 8>(a, im, t, wsmem, C, ph, w, lane); break;
        default: visit_tile_coop<uint16_t, 8>(a, im, t, wsmem, C, ph, w, lane); break;
    }
}

// The persistent kernel: warp 0 pops a tile for the CTA, the CTA visits it. MIXED: a batch
// whose images differ in pixel type or connectivity (T, CONN unused); that build, with four
// visit variants inlined, keeps 4 CTAs per SM (at 5 it spills). The builds for one pixel
// type take kCoopBlocks (single images: more CTAs slow the images bound by one chain of
// tile hops), the build for u8 + u16 batches kCoopBatchBlocks (a batch keeps every worker
// busy, so the seventh CTA pays despite its spills). Without a plan's blocks_per_sm the
// grid is the occupancy the launch bounds give.
template <typename T, int CONN, bool MIXED>
__global__ void __launch_bounds__(kThreads, MIXED ? kRegBlocks
                                                 : (std::is_same<T, AnyPix>::value ? kCoopBatchBlocks : kCoopBlocks))
    drain_coop_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RT::smem_per_warp(0);
    CoopShared &C = *reinterpret_cast<CoopShared *>(smem_raw + kWarpsPerCta * RT::smem_per_warp(0));
    unsigned long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (lane == 0) C.waves[warp] = 0;
    if (threadIdx.x == 0) {
        C.k0 = globaltimer_ns();
        C.idle = 0;
        C.visits = 0;
    }
    for (;;) {
        if (warp == 0) {
            bool first;
            const uint32_t t = acquire_tile(a, first, C.idle, lane);
            if (lane == 0) C.tile = t;
        }
        __syncthreads();
        const uint32_t t = C.tile;
        if (t == kDone) break;
        visit_tile_coop_any<T, CONN, MIXED>(a, t, wsmem, C, ph, warp, lane);
        __syncthreads();   // every warp has read C.tile before the next pop overwrites it
    }
    if (lane == 0) {   // passes of every strip; visits and times of warp 0 (busy: the rest of the run)
        atomicAdd(&a.hdr->waves, C.waves[warp]);
        if (warp == 0) {
            atomicAdd(&a.hdr->visits, C.visits);
            atomicAdd(&a.hdr->idle_ns, C.idle);
            atomicAdd(&a.hdr->busy_ns, globaltimer_ns() - C.k0 - C.idle);
        }
    }
#if IWPP_PHASE_TIMING
    if (warp == 0 && lane == 0)
        for (int k = 0; k < 8; k++) atomicAdd(&a.hdr->phase_cycles[k], ph[k]);
#endif
}

// Initialisation of one CTA tile (Algorithm 7's scanning phase, tile-local, then the
// frontier): check the precondition; run the tile's raster / anti-raster sweep pairs
// (a.tile_sweeps[t], else a.sweeps), the strips exchanging their boundary rows after each
// pair, store what changed and notify the neighbours whose halo pixels the tile can now
// raise; queue the tile if one of its pixels can still rise.
template <typename T, int CONN, bool SWEEPS>
__device__ void scan_tile_coop(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem,
                               CoopShared &C, uint8_t *stage, int w, int lane) {
    constexpr int TH = kCoopStrip;
    using RT = RegTile<T, CONN, TH>;
    const int sweeps = !SWEEPS ? 0 : a.tile_sweeps ? (int)a.tile_sweeps[t] : a.sweeps;   // CTA-uniform
    if (SWEEPS && a.sweep_only && sweeps == 0) return;   // the sweeps-only pass: nothing to do here
    const long long c0 = clock64();
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = RT::halo_words(s, lane);
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * kCoopRows + TH * w, x0 = tx * RT::TW;
    uint32_t J[TH], I[TH], jt, jb, it, ib;
#if IWPP_SCAN_VEC
    if (RT::vec_ok(im, x0)) RT::load_vec(im, s, stage, y0, x0, J, I, jt, jb, it, ib, lane);
    else RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
#else
    (void)stage;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
#endif
    bool bad = false;
#pragma unroll
    for (int r = 0; r < TH; r++) bad |= max2(J[r], I[r]) != I[r];
    uint32_t rows = 0;
    for (int k = 0; k < sweeps; k++) {
        rows |= RT::sweep_raster(hx, J, I, jt, lane);
        rows |= RT::sweep_antiraster(hx, J, I, jb, lane);
        C.rows[w][0][lane] = J[0];
        C.rows[w][1][lane] = J[TH - 1];
        __syncthreads();
        if (w > 0) jt = C.rows[w - 1][1][lane];
        if (w < kWarpsPerCta - 1) jb = C.rows[w + 1][0][lane];
        __syncthreads();
    }
    const bool can = RT::improvable(hx, J, I, jt, jb, lane);
    const int any_bad = __syncthreads_or(bad);
    const int any_can = __syncthreads_or(can);
    if (sweeps > 0 && __syncthreads_or(rows != 0)) {
        RT::store(im, y0, x0, J, rows, lane);
        if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
        __syncthreads();
        RT::notify_scan(s, J, jt, jb, it, ib, lane);
        if (lane == 0) coop_fold_misc(C, s.misc, w);
        fence_protocol();
        __syncthreads();
        if (w == 0 && lane < 9 && lane != 4 && C.misc[lane]) {
            const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
            if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x) {
                const uint32_t n = im.tile_base + (uint32_t)(ny * im.tiles_x + nx);
                if (a.defer_push) mark_pending(a, n); else notify_tile(a, n);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (any_can) {
            if (a.defer_push) mark_pending(a, t); else notify_tile(a, t);   // batches: queued in order later
        }
        if (any_bad) set_status(a.hdr, kErrPrecondition);
        if (a.tile_work) atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
    __syncthreads();   // the strips' shared halo buffers are reloaded for the next tile
}

// The strip scan (no sweeps), one warp per strip with no CTA barriers: each warp loads a
// 16-row strip of a tile with its halo, checks the precondition and whether one of its
// pixels can rise; a strip that can makes its tile PENDING (batches: a fire-and-forget OR)
// or notifies it (single images: the first notification queues the tile, later ones find it
// PENDING). Warps go from strip to strip independently, 7 CTAs per SM. The streaming scan
// (iwpp_scan.cuh) replaces it wherever one connectivity is compiled in; the mixed-kind build
// keeps it (its kinds switch per strip).
#ifndef IWPP_SCAN_STRIP_MINB
#define IWPP_SCAN_STRIP_MINB 7   // CTAs per SM of the strip scan (72 registers, no spills)
#endif
template <typename T, int CONN>
__device__ void scan_strip_coop(const EngineArgs &a, const ImageView &im, uint32_t t, int sw, uint8_t *wsmem,
                                int lane) {
    constexpr int TH = kCoopStrip;
    using RT = RegTile<T, CONN, TH>;
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * kCoopRows + TH * sw, x0 = tx * RT::TW;
    if (y0 >= im.H) return;   // a strip below the image (warp-uniform): nothing in it can rise
    const long long c0 = clock64();
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = RT::halo_words(s, lane);
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    bool bad = false;
#pragma unroll
    for (int r = 0; r < TH; r++) bad |= max2(J[r], I[r]) != I[r];
    const bool can = RT::improvable(hx, J, I, jt, jb, lane);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        if (can) {
            if (a.defer_push) mark_pending(a, t); else notify_tile(a, t);
        }
        if (bad) set_status(a.hdr, kErrPrecondition);
        if (a.tile_work) atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
    __syncwarp();   // the warp's halo buffers are reloaded for its next strip
}

template <typename T, int CONN, bool MIXED>
__global__ void __launch_bounds__(kThreads, IWPP_SCAN_STRIP_MINB) scan_strip_coop_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + w * RT::smem_per_warp(0);
    const uint64_t nunits = (uint64_t)a.ntiles * kWarpsPerCta, nwarps = (uint64_t)gridDim.x * kWarpsPerCta;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarpsPerCta + w; u < nunits; u += nwarps) {
        const uint32_t t = (uint32_t)(u / kWarpsPerCta);
        const int sw = (int)(u % kWarpsPerCta);
        const ImageView &im = image_of(a, t);
        if (!MIXED) {
            scan_strip_coop<T, CONN>(a, im, t, sw, wsmem, lane);
            continue;
        }
        switch (im.kind) {
            case 0: scan_strip_coop<uint8_t, 4>(a, im, t, sw, wsmem, lane); break;
            case 1: scan_strip_coop<uint16_t, 4>(a, im, t, sw, wsmem, lane); break;
            case 2: scan_strip_coop<uint8_t, 8>(a, im, t, sw, wsmem, lane); break;
            default: scan_strip_coop<uint16_t, 8>(a, im, t, sw, wsmem, lane); break;
        }
    }
}

// The scan on whole tiles: SWEEPS, the build that runs sweep pairs (plans with sweeps,
// per-tile sweep counts; the strips exchange boundary rows after each pair); the other one
// is the lean scan with CTA barriers (the strip scan above replaces it).
template <typename T, int CONN, bool MIXED, bool SWEEPS>
__global__ void __launch_bounds__(kThreads, SWEEPS ? 4 : 8) scan_coop_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + w * RT::smem_per_warp(0);
    CoopShared &C = *reinterpret_cast<CoopShared *>(smem_raw + kWarpsPerCta * RT::smem_per_warp(0));
    uint8_t *stage = smem_raw + coop_scan_stage_offset<T, CONN>() + w * RT::kStageBytes;
    auto tile = [&](uint32_t t) {
        const ImageView &im = image_of(a, t);
        if (!MIXED) {
            scan_tile_coop<T, CONN, SWEEPS>(a, im, t, wsmem, C, stage, w, lane);
            return;
        }
        switch (im.kind) {
            case 0: scan_tile_coop<uint8_t, 4, SWEEPS>(a, im, t, wsmem, C, stage, w, lane); break;
            case 1: scan_tile_coop<uint16_t, 4, SWEEPS>(a, im, t, wsmem, C, stage, w, lane); break;
            case 2: scan_tile_coop<uint8_t, 8, SWEEPS>(a, im, t, wsmem, C, stage, w, lane); break;
            default: scan_tile_coop<uint16_t, 8, SWEEPS>(a, im, t, wsmem, C, stage, w, lane); break;
        }
    };
    if (SWEEPS && a.sweep_only) {
        // The sweeps-only pass of learned batches, where most tiles have no sweeps: the CTA
        // reads the counts of kThreads of its tiles at once and visits only those with sweeps
        // (the same tiles as the loop below, grouped differently).
        __shared__ uint32_t has_sweeps[kWarpsPerCta];
        const uint64_t step = (uint64_t)gridDim.x * kThreads;
        for (uint64_t base = blockIdx.x; base < a.ntiles; base += step) {
            const uint64_t mine = base + (uint64_t)threadIdx.x * gridDim.x;
            const uint32_t b = __ballot_sync(0xffffffffu, mine < a.ntiles && a.tile_sweeps[mine] != 0);
            if (lane == 0) has_sweeps[w] = b;
            __syncthreads();
            for (int k = 0; k < kWarpsPerCta; k++)
                for (uint32_t m = has_sweeps[k]; m; m &= m - 1)
                    tile((uint32_t)(base + (uint64_t)(32 * k + __ffs(m) - 1) * gridDim.x));
            __syncthreads();   // every thread has read the flags before the next chunk's
        }
        return;
    }
    for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) tile(t);
}

}  // namespace iwpp

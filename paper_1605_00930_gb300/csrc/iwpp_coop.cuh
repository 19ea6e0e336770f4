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
};

template <typename T, int CONN>
__host__ __device__ constexpr size_t coop_smem_bytes() {
    return RegTile<T, CONN, kCoopStrip>::smem_per_warp(0) * kWarpsPerCta + sizeof(CoopShared);
}
template <typename T, int CONN>
size_t coop_smem_fn(uint32_t) { return coop_smem_bytes<T, CONN>(); }

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

// One visit of CTA tile t by the whole CTA (every thread calls it with the same t), including
// the re-processing rounds when the tile is notified while the CTA holds it.
template <typename T, int CONN>
__device__ void visit_tile_coop(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem,
                                CoopShared &C, VisitStats &st, int w, int lane) {
    constexpr int TH = kCoopStrip;
    using RT = RegTile<T, CONN, TH>;
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = s.hxJ + (lane == 31 ? TH + 2 : 0);
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * kCoopRows + TH * w, x0 = tx * RT::TW;
    if (lane < 16) s.misc[lane] = 0;
    if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    uint32_t passes = 0;
    for (;;) {
        uint32_t rows = 0;
        bool active = true;
        for (;;) {   // joint iterations of the strips
            uint32_t ch = 0;
            if (active) {
                ch = RT::pass_down(hx, J, I, jt, lane);
                ch |= RT::pass_up(hx, J, I, jb, lane);
                passes += 2;
                rows |= ch;
            }
            C.rows[w][0][lane] = J[0];
            C.rows[w][1][lane] = J[TH - 1];
            __syncthreads();
            const uint32_t njt = w > 0 ? C.rows[w - 1][1][lane] : jt;
            const uint32_t njb = w < kWarpsPerCta - 1 ? C.rows[w + 1][0][lane] : jb;
            const bool halo = __any_sync(0xffffffffu, njt != jt || njb != jb);
            jt = njt;
            jb = njb;
            // a strip that changed may still be short of its fixed point (its next pass pair
            // finds out: measured cheaper than a residual check here); one whose halo rows
            // changed may have new work; the others are settled
            active = halo || __any_sync(0xffffffffu, ch != 0);
            if (!__syncthreads_or(active)) break;
        }
        if (w == 0 && lane == 0) st.visits++;
        if (__syncthreads_or(rows != 0)) {
            RT::store(im, y0, x0, J, rows, lane);
            RT::notify_scan(s, J, jt, jb, it, ib, lane);
            if (lane == 0) coop_fold_misc(C, s.misc, w);
            __threadfence();
            __syncthreads();
            if (w == 0 && lane < 9 && lane != 4 && C.misc[lane]) {
                const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
                if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                    notify_tile(a, im.tile_base + (uint32_t)(ny * im.tiles_x + nx));
            }
        }
        if (w == 0) {
            const bool r = finish_tile(a, t, lane);
            if (lane == 0) C.redo = r;
        }
        __syncthreads();
        const bool redo = C.redo != 0;
        if (!redo) break;
        // re-process: J and I stay in registers; only the tile's halo can have changed
        if (lane < 16) s.misc[lane] = 0;
        if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
        RT::load_halo(im, s, y0, x0, jt, jb, it, ib, false, lane);
        __syncthreads();
    }
    st.waves += passes;
}

// One CTA tile visit, dispatched on the tile's image kind (CTA-uniform: one tile per CTA).
template <typename T, int CONN, bool MIXED>
__device__ __forceinline__ void visit_tile_coop_any(const EngineArgs &a, uint32_t t, uint8_t *wsmem, CoopShared &C,
                                                    VisitStats &st, int w, int lane) {
    const ImageView &im = image_of(a, t);
    if (!MIXED) {
        visit_tile_coop<T, CONN>(a, im, t, wsmem, C, st, w, lane);
        return;
    }
    switch (im.kind) {
        case 0: visit_tile_coop<uint8_t, 4>(a, im, t, wsmem, C, st, w, lane); break;
        case 1: visit_tile_coop<uint16_t, 4>(a, im, t, wsmem, C, st, w, lane); break;
        case 2: visit_tile_coop<uint8_t, 8>(a, im, t, wsmem, C, st, w, lane); break;
        default: visit_tile_coop<uint16_t, 8>(a, im, t, wsmem, C, st, w, lane); break;
    }
}

// The persistent kernel: warp 0 pops a tile for the CTA, the CTA visits it. MIXED: a batch
// whose images differ in pixel type or connectivity (T, CONN unused); that build, with four
// visit variants inlined, keeps 4 CTAs per SM (at 5 it spills), the specialised ones take 5
// (measured: -6 % on the 4096^2 image, -12 % on the 16384^2 seed image).
template <typename T, int CONN, bool MIXED>
__global__ void __launch_bounds__(kThreads, MIXED ? kRegBlocks : kCoopBlocks) drain_coop_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RT::smem_per_warp(0);
    CoopShared &C = *reinterpret_cast<CoopShared *>(smem_raw + kWarpsPerCta * RT::smem_per_warp(0));
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0;
    for (;;) {
        if (warp == 0) {
            bool first;
            const uint32_t t = acquire_tile(a, first, idle, lane);
            if (lane == 0) C.tile = t;
        }
        __syncthreads();
        const uint32_t t = C.tile;
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        visit_tile_coop_any<T, CONN, MIXED>(a, t, wsmem, C, st, warp, lane);
        if (warp == 0) busy += globaltimer_ns() - b0;
        __syncthreads();   // every warp has read C.tile before the next pop overwrites it
    }
    flush_stats(a, st, idle, busy, lane);
}

// Initial frontier of one CTA tile: queue it if one of its pixels can rise (each strip checks
// its own pixels against its neighbourhood, halo included), and check the precondition.
template <typename T, int CONN>
__device__ void scan_tile_coop(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem, int w,
                               int lane) {
    constexpr int TH = kCoopStrip;
    using RT = RegTile<T, CONN, TH>;
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = s.hxJ + (lane == 31 ? TH + 2 : 0);
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * kCoopRows + TH * w, x0 = tx * RT::TW;
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    bool bad = false;
#pragma unroll
    for (int r = 0; r < TH; r++) bad |= max2(J[r], I[r]) != I[r];
    const bool can = RT::improvable(hx, J, I, jt, jb, lane);
    const int any_bad = __syncthreads_or(bad);
    const int any_can = __syncthreads_or(can);
    if (threadIdx.x == 0) {
        if (any_can) {
            if (a.defer_push) mark_pending(a, t); else notify_tile(a, t);   // batches: queued in order later
        }
        if (any_bad) set_status(a.hdr, kErrPrecondition);
    }
    __syncthreads();   // the strips' shared halo buffers are reloaded for the next tile
}

template <typename T, int CONN, bool MIXED>
__global__ void __launch_bounds__(kThreads) scan_coop_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + w * RT::smem_per_warp(0);
    for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const ImageView &im = image_of(a, t);
        if (!MIXED) {
            scan_tile_coop<T, CONN>(a, im, t, wsmem, w, lane);
            continue;
        }
        switch (im.kind) {
            case 0: scan_tile_coop<uint8_t, 4>(a, im, t, wsmem, w, lane); break;
            case 1: scan_tile_coop<uint16_t, 4>(a, im, t, wsmem, w, lane); break;
            case 2: scan_tile_coop<uint8_t, 8>(a, im, t, wsmem, w, lane); break;
            default: scan_tile_coop<uint16_t, 8>(a, im, t, wsmem, w, lane); break;
        }
    }
}

}  // namespace iwpp

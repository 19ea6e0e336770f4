// iwpp_wshed.cu — marker-controlled watershed by flooding as an IWPP propagation on the
// persistent tile engine (include/iwpp.h, iwpp_watershed).
//
// Every pixel carries a pair packed as (level << 16) | label, 0xFFFFFFFF while unreached.
// Markers are fixed at (gradient, label). A neighbour q offers pixel p the pair
// (max(level(q), gradient(p)), label(q)) — in the packing, max(v_q, gradient(p) << 16 |
// label(q)) — and p keeps the smaller of its own pair and every offer. One CTA settles a
// 64 x 64 tile: each of its four warps holds a 16-row strip in registers (lane c: columns 2c
// and 2c + 1; the gradient packed as u16x2) and repeats down / up passes of that update; the
// strips exchange their first and last rows through shared memory between pass pairs until
// none changes; a halo pixel that the tile's border would improve marks its tile for a visit. The levels reached
// are unique (the minimax flooding level); which label wins where several reach a pixel at
// its level depends on the order of work, as in any flooding watershed.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/iwpp.h"
#include "iwpp_engine.cuh"
#include "iwpp_host.h"

namespace iwpp {
namespace {

constexpr uint32_t kUnreached = 0xFFFFFFFFu;
constexpr int WTH = 16, WTW = 64;
constexpr int WSW = kWarpsPerCta;   // strips per CTA tile
constexpr int WCH = WTH * WSW;      // CTA tile rows

// The offer of pair v (at a neighbour) to a pixel whose gradient is g (already << 16).
__device__ __forceinline__ uint32_t offer_ws(uint32_t v, uint32_t g16) { return max(v, g16 | (v & 0xFFFFu)); }

struct WsSmem {
    uint32_t *hl, *hr;       // WTH + 2: pairs of the halo columns, index = row + 1
    uint32_t *gl, *gr;       // WTH + 2: their gradient
    uint32_t *col0, *col63;  // WTH: the tile's first and last column after a solve
    uint32_t *misc;          // 16: notification flags
};
constexpr size_t kWsWords = 4 * (WTH + 2) + 2 * WTH + 16;
constexpr size_t kWsSmemPerWarp = (kWsWords * 4 + 15) & ~(size_t)15;

__device__ WsSmem ws_carve(uint8_t *base) {
    WsSmem s;
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    s.hl = w; w += WTH + 2;
    s.hr = w; w += WTH + 2;
    s.gl = w; w += WTH + 2;
    s.gr = w; w += WTH + 2;
    s.col0 = w; w += WTH;
    s.col63 = w; w += WTH;
    s.misc = w;
    return s;
}

struct WsArgs {
    const uint32_t *markers;
    const void *grad;
    int u16;
};

struct WsTile {
    uint32_t e[WTH], o[WTH];   // pairs of columns 2c, 2c + 1
    uint32_t g[WTH];           // gradient pair (even low, odd high)
    uint32_t fixed;            // bit 2r: even pixel of row r fixed, 2r + 1: odd
    uint32_t te, to, be, bo;   // halo rows' pairs at this lane's columns
    uint32_t gt, gb;           // their gradient pairs
};

__device__ __forceinline__ bool inside(const ImageView &im, int y, int x) {
    return y >= 0 && y < im.H && x >= 0 && x < im.W;
}
__device__ __forceinline__ size_t clamp_e(const ImageView &im, int y, int x) {
    return (size_t)min(max(y, 0), im.H - 1) * im.W + min(max(x, 0), im.W - 1);
}
__device__ __forceinline__ uint32_t ld_pair_v(const ImageView &im, int y, int x) {
    const uint32_t v = __ldcg(reinterpret_cast<const uint32_t *>(im.J) + clamp_e(im, y, x));
    return inside(im, y, x) ? v : kUnreached;
}
__device__ __forceinline__ uint32_t ld_grad(const ImageView &im, const WsArgs &w, int y, int x) {
    const size_t e = clamp_e(im, y, x);
    const uint32_t v = w.u16 ? reinterpret_cast<const uint16_t *>(w.grad)[e] : reinterpret_cast<const uint8_t *>(w.grad)[e];
    return inside(im, y, x) ? v : 0u;
}

__device__ void ws_load_halo(const ImageView &im, const WsArgs &w, const WsSmem &s, int y0, int x0, WsTile &T,
                             bool with_grad, int lane) {
    const int xe = x0 + 2 * lane;
    T.te = ld_pair_v(im, y0 - 1, xe);
    T.to = ld_pair_v(im, y0 - 1, xe + 1);
    T.be = ld_pair_v(im, y0 + WTH, xe);
    T.bo = ld_pair_v(im, y0 + WTH, xe + 1);
    if (with_grad) {
        T.gt = ld_grad(im, w, y0 - 1, xe) | (ld_grad(im, w, y0 - 1, xe + 1) << 16);
        T.gb = ld_grad(im, w, y0 + WTH, xe) | (ld_grad(im, w, y0 + WTH, xe + 1) << 16);
    }
    for (int i = lane; i < WTH + 2; i += 32) {
        s.hl[i] = ld_pair_v(im, y0 + i - 1, x0 - 1);
        s.hr[i] = ld_pair_v(im, y0 + i - 1, x0 + WTW);
        if (with_grad) {
            s.gl[i] = ld_grad(im, w, y0 + i - 1, x0 - 1);
            s.gr[i] = ld_grad(im, w, y0 + i - 1, x0 + WTW);
        }
    }
    __syncwarp();
}

__device__ void ws_load(const ImageView &im, const WsArgs &w, const WsSmem &s, int y0, int x0, WsTile &T, int lane) {
    const int xe = x0 + 2 * lane;
    T.fixed = 0;
#pragma unroll
    for (int r = 0; r < WTH; r++) {
        const int y = y0 + r;
        T.e[r] = ld_pair_v(im, y, xe);
        T.o[r] = ld_pair_v(im, y, xe + 1);
        T.g[r] = ld_grad(im, w, y, xe) | (ld_grad(im, w, y, xe + 1) << 16);
        const bool fe = !inside(im, y, xe) || w.markers[clamp_e(im, y, xe)] != 0;
        const bool fo = !inside(im, y, xe + 1) || w.markers[clamp_e(im, y, xe + 1)] != 0;
        T.fixed |= ((uint32_t)fe << (2 * r)) | ((uint32_t)fo << (2 * r + 1));
    }
    ws_load_halo(im, w, s, y0, x0, T, true, lane);
}

// One pass (DIR +1 down, -1 up); returns this lane's changed rows.
template <int CONN, int DIR>
__device__ __forceinline__ uint32_t ws_pass(const WsSmem &s, WsTile &T, int lane) {
    uint32_t pe = DIR > 0 ? T.te : T.be, po = DIR > 0 ? T.to : T.bo;
    uint32_t chg = 0;
#pragma unroll
    for (int k = 0; k < WTH; k++) {
        const int r = DIR > 0 ? k : WTH - 1 - k;
        uint32_t wo = __shfl_up_sync(0xffffffffu, T.o[r], 1), ee = __shfl_down_sync(0xffffffffu, T.e[r], 1);
        if (lane == 0) wo = s.hl[r + 1];
        if (lane == 31) ee = s.hr[r + 1];
        uint32_t pwo = __shfl_up_sync(0xffffffffu, po, 1), pee = __shfl_down_sync(0xffffffffu, pe, 1);
        if (lane == 0) pwo = s.hl[r + 1 - DIR];
        if (lane == 31) pee = s.hr[r + 1 - DIR];
        const uint32_t ge = T.g[r] << 16, go = T.g[r] & 0xFFFF0000u;
        uint32_t ne = min(T.e[r], offer_ws(wo, ge));
        ne = min(ne, offer_ws(T.o[r], ge));
        ne = min(ne, offer_ws(pe, ge));
        if (CONN == 8) ne = min(ne, min(offer_ws(pwo, ge), offer_ws(po, ge)));
        if ((T.fixed >> (2 * r)) & 1u) ne = T.e[r];
        uint32_t no = min(T.o[r], offer_ws(ne, go));
        no = min(no, offer_ws(ee, go));
        no = min(no, offer_ws(po, go));
        if (CONN == 8) no = min(no, min(offer_ws(pe, go), offer_ws(pee, go)));
        if ((T.fixed >> (2 * r + 1)) & 1u) no = T.o[r];
        chg |= (uint32_t)((ne != T.e[r]) | (no != T.o[r])) << r;
        T.e[r] = ne;
        T.o[r] = no;
        pe = ne;
        po = no;
    }
    return chg;
}

// Flag each neighbour one of whose halo pixels the tile's border would improve.
template <int CONN>
__device__ void ws_notify_scan(const WsSmem &s, const WsTile &T, int lane) {
    if (lane == 0)
        for (int r = 0; r < WTH; r++) s.col0[r] = T.e[r];
    if (lane == 31)
        for (int r = 0; r < WTH; r++) s.col63[r] = T.o[r];
    bool top = false, bot = false;
    {
        uint32_t wo = __shfl_up_sync(0xffffffffu, T.o[0], 1), ee = __shfl_down_sync(0xffffffffu, T.e[0], 1);
        uint32_t bwo = __shfl_up_sync(0xffffffffu, T.o[WTH - 1], 1),
                 bee = __shfl_down_sync(0xffffffffu, T.e[WTH - 1], 1);
        if (lane == 0) wo = bwo = kUnreached;
        if (lane == 31) ee = bee = kUnreached;
        const uint32_t gte = T.gt << 16, gto = T.gt & 0xFFFF0000u, gbe = T.gb << 16, gbo = T.gb & 0xFFFF0000u;
        uint32_t c1 = offer_ws(T.e[0], gte), c2 = offer_ws(T.o[0], gto);
        uint32_t c3 = offer_ws(T.e[WTH - 1], gbe), c4 = offer_ws(T.o[WTH - 1], gbo);
        if (CONN == 8) {
            c1 = min(c1, min(offer_ws(wo, gte), offer_ws(T.o[0], gte)));
            c2 = min(c2, min(offer_ws(T.e[0], gto), offer_ws(ee, gto)));
            c3 = min(c3, min(offer_ws(bwo, gbe), offer_ws(T.o[WTH - 1], gbe)));
            c4 = min(c4, min(offer_ws(T.e[WTH - 1], gbo), offer_ws(bee, gbo)));
        }
        top = c1 < T.te || c2 < T.to;
        bot = c3 < T.be || c4 < T.bo;
    }
    top = __any_sync(0xffffffffu, top);
    bot = __any_sync(0xffffffffu, bot);
    if (lane == 0) {
        s.misc[1] = top;
        s.misc[7] = bot;
    }
    __syncwarp();
    bool lf = false, rt = false;
    if (lane < WTH) {
        const int r = lane;
        const uint32_t gl = s.gl[r + 1] << 16, gr = s.gr[r + 1] << 16;
        uint32_t cl = offer_ws(s.col0[r], gl), cr = offer_ws(s.col63[r], gr);
        if (CONN == 8) {
            if (r > 0) {
                cl = min(cl, offer_ws(s.col0[r - 1], gl));
                cr = min(cr, offer_ws(s.col63[r - 1], gr));
            }
            if (r < WTH - 1) {
                cl = min(cl, offer_ws(s.col0[r + 1], gl));
                cr = min(cr, offer_ws(s.col63[r + 1], gr));
            }
        }
        lf = cl < s.hl[r + 1];
        rt = cr < s.hr[r + 1];
    }
    lf = __any_sync(0xffffffffu, lf);
    rt = __any_sync(0xffffffffu, rt);
    if (lane == 0) {
        s.misc[3] = lf;
        s.misc[5] = rt;
        uint32_t c0 = 0, c2 = 0, c6 = 0, c8 = 0;
        if (CONN == 8) {
            c0 = offer_ws(s.col0[0], s.gl[0] << 16) < s.hl[0];
            c6 = offer_ws(s.col0[WTH - 1], s.gl[WTH + 1] << 16) < s.hl[WTH + 1];
            c2 = offer_ws(s.col63[0], s.gr[0] << 16) < s.hr[0];
            c8 = offer_ws(s.col63[WTH - 1], s.gr[WTH + 1] << 16) < s.hr[WTH + 1];
        }
        s.misc[0] = c0;
        s.misc[2] = c2;
        s.misc[6] = c6;
        s.misc[8] = c8;
    }
}

__device__ void ws_store(const ImageView &im, int y0, int x0, const WsTile &T, uint32_t rows, int lane) {
    const int xe = x0 + 2 * lane;
    uint32_t *V = reinterpret_cast<uint32_t *>(im.J);
#pragma unroll
    for (int r = 0; r < WTH; r++) {
        if (!((rows >> r) & 1u)) continue;
        const size_t row = (size_t)(y0 + r) * im.W;
        if (xe < im.W) __stcg(V + row + xe, T.e[r]);
        if (xe + 1 < im.W) __stcg(V + row + xe + 1, T.o[r]);
    }
}

// The CTA tile's shared state: each strip's first and last row (even and odd pair per lane),
// the tile's notification flags, the popped tile.
struct WsShared {
    uint32_t rows[WSW][4][32];
    uint32_t misc[16];
    uint32_t tile, redo;
};
constexpr size_t kWsSmemCta = kWsSmemPerWarp * WSW + sizeof(WsShared);

// Fold one strip's notification flags into the CTA tile's (a strip's top / bottom side is the
// tile's only for the first / last strip; its corners beside the tile's inner rows lie in the
// west / east neighbours).
__device__ __forceinline__ void ws_fold_misc(WsShared &C, const uint32_t *m, int w) {
    if (w == 0) {
        atomicOr(&C.misc[0], m[0]);
        atomicOr(&C.misc[1], m[1]);
        atomicOr(&C.misc[2], m[2]);
    } else {
        atomicOr(&C.misc[3], m[0]);
        atomicOr(&C.misc[5], m[2]);
    }
    if (w == WSW - 1) {
        atomicOr(&C.misc[6], m[6]);
        atomicOr(&C.misc[7], m[7]);
        atomicOr(&C.misc[8], m[8]);
    } else {
        atomicOr(&C.misc[3], m[6]);
        atomicOr(&C.misc[5], m[8]);
    }
    atomicOr(&C.misc[3], m[3]);
    atomicOr(&C.misc[5], m[5]);
}

// One visit of CTA tile t by the whole CTA (every thread calls it with the same t), including
// the re-processing rounds when the tile is notified while the CTA holds it.
template <int CONN>
__device__ void ws_visit(const EngineArgs &a, const WsArgs &wa, uint32_t t, uint8_t *wsmem, WsShared &C,
                         VisitStats &st, int w, int lane) {
    const ImageView &im = a.img0;
    const WsSmem s = ws_carve(wsmem);
    const int ty = (int)(t / im.tiles_x), tx = (int)(t % im.tiles_x);
    const int y0 = ty * WCH + WTH * w, x0 = tx * WTW;
    if (lane < 16) s.misc[lane] = 0;
    if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
    WsTile T;
    ws_load(im, wa, s, y0, x0, T, lane);
    uint32_t passes = 0;
    for (;;) {
        uint32_t rows = 0;
        bool active = true;
        for (;;) {   // joint iterations of the strips
            uint32_t ch = 0;
            if (active) {
                ch = ws_pass<CONN, 1>(s, T, lane);
                ch |= ws_pass<CONN, -1>(s, T, lane);
                passes += 2;
                rows |= ch;
            }
            C.rows[w][0][lane] = T.e[0];
            C.rows[w][1][lane] = T.o[0];
            C.rows[w][2][lane] = T.e[WTH - 1];
            C.rows[w][3][lane] = T.o[WTH - 1];
            __syncthreads();
            uint32_t nte = T.te, nto = T.to, nbe = T.be, nbo = T.bo;
            if (w > 0) {
                nte = C.rows[w - 1][2][lane];
                nto = C.rows[w - 1][3][lane];
            }
            if (w < WSW - 1) {
                nbe = C.rows[w + 1][0][lane];
                nbo = C.rows[w + 1][1][lane];
            }
            const bool halo = __any_sync(0xffffffffu, nte != T.te || nto != T.to || nbe != T.be || nbo != T.bo);
            T.te = nte;
            T.to = nto;
            T.be = nbe;
            T.bo = nbo;
            active = halo || __any_sync(0xffffffffu, ch != 0);
            if (!__syncthreads_or(active)) break;
        }
        if (w == 0 && lane == 0) st.visits++;
        if (__syncthreads_or(rows != 0)) {
            ws_store(im, y0, x0, T, rows, lane);
            ws_notify_scan<CONN>(s, T, lane);
            if (lane == 0) ws_fold_misc(C, s.misc, w);
            __threadfence();
            __syncthreads();
            if (w == 0 && lane < 9 && lane != 4 && C.misc[lane]) {
                const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
                if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                    notify_tile(a, (uint32_t)(ny * im.tiles_x + nx));
            }
        }
        if (w == 0) {
            const bool r = finish_tile(a, t, lane);
            if (lane == 0) C.redo = r;
        }
        __syncthreads();
        const bool redo = C.redo != 0;
        if (!redo) break;
        // re-process: the strips stay in registers; only the tile's halo can have changed
        if (lane < 16) s.misc[lane] = 0;
        if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
        ws_load_halo(im, wa, s, y0, x0, T, false, lane);
        __syncthreads();
    }
    st.waves += passes;
}

// Initialisation, one warp per 16 x 64 strip: markers take (gradient, label), everything else
// is unreached; the CTA tile of every strip holding a marker is queued. Labels above 65534
// stop the call with IWPP_ERR_ARG.
__global__ void __launch_bounds__(256) ws_init_kernel(EngineArgs a, WsArgs w, uint32_t nstrips) {
    const ImageView &im = a.img0;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *V = reinterpret_cast<uint32_t *>(im.J);
    for (uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nstrips; u += nw) {
        const int uy = (int)(u / im.tiles_x), ux = (int)(u % im.tiles_x);
        const int y0 = uy * WTH, x0 = ux * WTW;
        bool any = false, bad = false;
        for (int r = 0; r < WTH; r++) {
            const int y = y0 + r;
            if (y >= im.H) break;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int x = x0 + 2 * lane + q;
                if (x >= im.W) continue;
                const size_t e = (size_t)y * im.W + x;
                const uint32_t m = w.markers[e];
                const uint32_t g = w.u16 ? reinterpret_cast<const uint16_t *>(w.grad)[e]
                                         : reinterpret_cast<const uint8_t *>(w.grad)[e];
                bad |= m > 65534u;
                any |= m != 0;
                V[e] = m ? (g << 16) | m : kUnreached;
            }
        }
        any = __any_sync(0xffffffffu, any);
        bad = __any_sync(0xffffffffu, bad);
        __threadfence();
        if (lane == 0 && bad) set_status(a.hdr, kErrArg);
        if (lane == 0 && any) notify_tile(a, (uint32_t)((uy / WSW) * im.tiles_x + ux));
    }
}

template <int CONN>
__global__ void __launch_bounds__(kThreads, 2) ws_drain_kernel(EngineArgs a, WsArgs wa) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * kWsSmemPerWarp;
    WsShared &C = *reinterpret_cast<WsShared *>(smem_raw + WSW * kWsSmemPerWarp);
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
        ws_visit<CONN>(a, wa, t, wsmem, C, st, warp, lane);
        if (warp == 0) busy += globaltimer_ns() - b0;
        __syncthreads();   // every warp has read C.tile before the next pop overwrites it
    }
    flush_stats(a, st, idle, busy, lane);
}

// labels in place (0 where unreached), levels optionally (-1 where unreached)
__global__ void ws_finish_kernel(uint32_t *V, int32_t *levels, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t v = V[i];
        if (levels) levels[i] = v == kUnreached ? -1 : (int32_t)(v >> 16);
        V[i] = v == kUnreached ? 0u : (v & 0xFFFFu);
    }
}

struct WsLayout {
    size_t state, queue, total;
    uint32_t ntiles, nstrips;   // 64 x 64 CTA tiles; 16 x 64 strips
    int tiles_x, tiles_y;
};

bool ws_layout(int64_t H, int64_t W, WsLayout &L) {
    if (H < 1 || W < 1 || H >= (1ll << 31) || W >= (1ll << 31) || (uint64_t)H * (uint64_t)W >= (1ull << 40))
        return false;
    const uint64_t tx = (uint64_t)((W + WTW - 1) / WTW), ty = (uint64_t)((H + WCH - 1) / WCH);
    const uint64_t sy = (uint64_t)((H + WTH - 1) / WTH);
    if (tx * sy >= (1ull << 31)) return false;
    L.tiles_x = (int)tx;
    L.tiles_y = (int)ty;
    L.ntiles = (uint32_t)(tx * ty);
    L.nstrips = (uint32_t)(tx * sy);
    L.state = 256;
    L.queue = L.state + align256((size_t)L.ntiles * 4);
    L.total = L.queue + align256((size_t)L.ntiles * 4);
    return true;
}

}  // namespace
}  // namespace iwpp

extern "C" size_t iwpp_watershed_workspace_bytes(int64_t H, int64_t W) {
    iwpp::WsLayout L;
    return iwpp::ws_layout(H, W, L) ? L.total : 0;
}

extern "C" int iwpp_watershed(const uint32_t *markers, const void *gradient, int dtype, uint32_t *labels_out,
                              int32_t *levels_out, int64_t H, int64_t W, int connectivity, void *workspace,
                              size_t ws_bytes, void *stream) {
    using namespace iwpp;
    if (!markers || !gradient || !labels_out) return IWPP_ERR_ARG;
    if (connectivity != 4 && connectivity != 8) return IWPP_ERR_ARG;
    if (dtype != IWPP_U8 && dtype != IWPP_U16) return IWPP_ERR_ARG;
    if (((uintptr_t)labels_out & 3) || ((uintptr_t)markers & 3) || (levels_out && ((uintptr_t)levels_out & 3)))
        return IWPP_ERR_ARG;
    WsLayout L;
    if (!ws_layout(H, W, L)) return IWPP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return IWPP_ERR_WORKSPACE;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    EngineArgs a = {};
    a.img0.J = reinterpret_cast<uint8_t *>(labels_out);
    a.img0.I = static_cast<const uint8_t *>(gradient);
    a.img0.H = (int)H;
    a.img0.W = (int)W;
    a.img0.tiles_x = L.tiles_x;
    a.img0.tiles_y = L.tiles_y;
    a.hdr = reinterpret_cast<WsHeader *>(base);
    a.state = reinterpret_cast<uint32_t *>(base + L.state);
    a.queue = reinterpret_cast<uint32_t *>(base + L.queue);
    a.ntiles = L.ntiles;
    a.watchdog_ns = 10ll * 1000 * 1000 * 1000;
    a.nlevels = 1;
    WsArgs w;
    w.markers = markers;
    w.grad = gradient;
    w.u16 = dtype == IWPP_U16;
    if (cudaMemsetAsync(base, 0, L.queue, s) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaMemsetAsync(base + L.queue, 0xFF, (size_t)L.ntiles * 4, s) != cudaSuccess) return IWPP_ERR_CUDA;
    const int sms = device_sm_count();
    if (sms <= 0) return IWPP_ERR_CUDA;
    uint32_t ig = (L.nstrips + 7) / 8;
    if (ig > (uint32_t)sms * 8) ig = (uint32_t)sms * 8;
    ws_init_kernel<<<ig, 256, 0, s>>>(a, w, L.nstrips);
    const size_t smem = kWsSmemCta;
    void (*drain)(EngineArgs, WsArgs) = connectivity == 8 ? ws_drain_kernel<8> : ws_drain_kernel<4>;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, drain, kThreads, smem) != cudaSuccess || bps < 1)
        return IWPP_ERR_CUDA;
    long long g = (long long)bps * sms;
    if (g > (long long)L.ntiles) g = L.ntiles;   // one CTA per tile
    drain<<<(int)g, kThreads, smem, s>>>(a, w);
    const size_t n = (size_t)H * (size_t)W;
    ws_finish_kernel<<<sms * 8, 256, 0, s>>>(labels_out, levels_out, n);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

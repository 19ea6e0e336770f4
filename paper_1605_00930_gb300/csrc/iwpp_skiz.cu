// iwpp_skiz.cu — geodesic skeleton by influence zones (SKIZ) as an IWPP propagation on the
// persistent tile engine (include/iwpp.h, iwpp_skiz). SKIZ is one of the operators the
// paper names as future work for the pattern (Sec. 6).
//
// Every pixel carries a state (d, l): d the number of steps from the nearest marker found so
// far, l the packed pair (min label << 16) | (0xFFFF - max label) of the markers at that
// distance. A neighbour q offers p (d(q) + 1, l(q)); p takes an offer with a smaller d, and
// on an equal d merges the label sets — the per-half minimum of the packed pair (min of the
// smallest labels, max of the largest). That update is a join on a distributive lattice, so
// every order of work reaches the same fixed point: d = the geodesic distance to the
// nearest marker and the labels of all markers at that distance. Pixels outside the domain
// carry d = kBlocked and never change. One CTA settles a 64 x 64 tile: each of its four warps
// holds a 16-row strip in registers (lane c: columns 2c and 2c + 1) and repeats down / up
// passes; the strips exchange their first and last rows through shared memory between pass
// pairs until none changes (the reconstruction's cooperative tile); a halo pixel that the
// tile's border would change marks its tile for a visit.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/iwpp.h"
#include "iwpp_engine.cuh"
#include "iwpp_host.h"

namespace iwpp {
namespace {

constexpr uint32_t kUnr = 0xC0000000u;      // domain pixel not reached yet (real d < 2^31)
constexpr uint32_t kBlocked = 0xE0000000u;  // outside the domain (also outside the image)
constexpr uint32_t kNoLab = 0xFFFFFFFFu;
constexpr int STH = 16, STW = 64;
constexpr int SKW = kWarpsPerCta;   // strips per CTA tile
constexpr int SCH = STH * SKW;      // CTA tile rows

struct St {
    uint32_t d, l;
};

__device__ __forceinline__ St unpack(unsigned long long v) { return St{(uint32_t)(v >> 32), (uint32_t)v}; }
__device__ __forceinline__ unsigned long long pack(St s) { return ((unsigned long long)s.d << 32) | s.l; }

// Join of candidate b into the candidate set (m, lc) (no step added).
__device__ __forceinline__ void cjoin(uint32_t &m, uint32_t &lc, St b) {
    lc = b.d < m ? b.l : (b.d == m ? __vminu2(lc, b.l) : lc);
    m = min(m, b.d);
}
// Accept the offer (m + 1, lc) at pixel s (unless s is outside the domain).
__device__ __forceinline__ St accept(St s, uint32_t m, uint32_t lc) {
    if (s.d == kBlocked) return s;
    const uint32_t o = m + 1;
    St r;
    r.l = o < s.d ? lc : (o == s.d ? __vminu2(s.l, lc) : s.l);
    r.d = min(s.d, o);
    return r;
}
__device__ __forceinline__ bool would_change(St h, uint32_t m, uint32_t lc) {
    const St r = accept(h, m, lc);
    return r.d != h.d || r.l != h.l;
}
__device__ __forceinline__ bool neq(St a, St b) { return a.d != b.d || a.l != b.l; }
__device__ __forceinline__ St shfl_up1(St s) {
    return St{__shfl_up_sync(0xffffffffu, s.d, 1), __shfl_up_sync(0xffffffffu, s.l, 1)};
}
__device__ __forceinline__ St shfl_dn1(St s) {
    return St{__shfl_down_sync(0xffffffffu, s.d, 1), __shfl_down_sync(0xffffffffu, s.l, 1)};
}

struct SkSmem {
    unsigned long long *hl, *hr;       // STH + 2: states of the halo columns, index = row + 1
    unsigned long long *col0, *col63;  // STH: the tile's first and last column after a solve
    uint32_t *misc;                    // 16: notification flags
};
constexpr size_t kSkBytes = 2 * (STH + 2) * 8 + 2 * STH * 8 + 16 * 4;
constexpr size_t kSkSmemPerWarp = (kSkBytes + 15) & ~(size_t)15;

__device__ SkSmem sk_carve(uint8_t *base) {
    SkSmem s;
    unsigned long long *w = reinterpret_cast<unsigned long long *>(base);
    s.hl = w; w += STH + 2;
    s.hr = w; w += STH + 2;
    s.col0 = w; w += STH;
    s.col63 = w; w += STH;
    s.misc = reinterpret_cast<uint32_t *>(w);
    return s;
}

struct SkTile {
    St e[STH], o[STH];   // states of columns 2c, 2c + 1
    St te, to, be, bo;   // halo rows' states at this lane's columns
};

__device__ __forceinline__ St ld_state(const ImageView &im, int y, int x) {
    const bool in = y >= 0 && y < im.H && x >= 0 && x < im.W;
    const size_t e = (size_t)min(max(y, 0), im.H - 1) * im.W + min(max(x, 0), im.W - 1);
    const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long *>(im.J) + e);
    return in ? unpack(v) : St{kBlocked, kNoLab};
}

__device__ void sk_load_halo(const ImageView &im, const SkSmem &s, int y0, int x0, SkTile &T, int lane) {
    const int xe = x0 + 2 * lane;
    T.te = ld_state(im, y0 - 1, xe);
    T.to = ld_state(im, y0 - 1, xe + 1);
    T.be = ld_state(im, y0 + STH, xe);
    T.bo = ld_state(im, y0 + STH, xe + 1);
    for (int i = lane; i < STH + 2; i += 32) {
        s.hl[i] = pack(ld_state(im, y0 + i - 1, x0 - 1));
        s.hr[i] = pack(ld_state(im, y0 + i - 1, x0 + STW));
    }
    __syncwarp();
}

__device__ void sk_load(const ImageView &im, const SkSmem &s, int y0, int x0, SkTile &T, int lane) {
    const int xe = x0 + 2 * lane;
#pragma unroll
    for (int r = 0; r < STH; r++) {
        T.e[r] = ld_state(im, y0 + r, xe);
        T.o[r] = ld_state(im, y0 + r, xe + 1);
    }
    sk_load_halo(im, s, y0, x0, T, lane);
}

// One pass (DIR +1 down, -1 up); returns this lane's changed rows.
template <int CONN, int DIR>
__device__ __forceinline__ uint32_t sk_pass(const SkSmem &s, SkTile &T, int lane) {
    St pe = DIR > 0 ? T.te : T.be, po = DIR > 0 ? T.to : T.bo;
    uint32_t chg = 0;
#pragma unroll
    for (int k = 0; k < STH; k++) {
        const int r = DIR > 0 ? k : STH - 1 - k;
        St wo = shfl_up1(T.o[r]), ee = shfl_dn1(T.e[r]);
        if (lane == 0) wo = unpack(s.hl[r + 1]);
        if (lane == 31) ee = unpack(s.hr[r + 1]);
        St pwo = shfl_up1(po), pee = shfl_dn1(pe);
        if (lane == 0) pwo = unpack(s.hl[r + 1 - DIR]);
        if (lane == 31) pee = unpack(s.hr[r + 1 - DIR]);
        uint32_t m = pe.d, lc = pe.l;
        cjoin(m, lc, wo);
        cjoin(m, lc, T.o[r]);
        if (CONN == 8) {
            cjoin(m, lc, pwo);
            cjoin(m, lc, po);
        }
        const St ne = accept(T.e[r], m, lc);
        m = po.d;
        lc = po.l;
        cjoin(m, lc, ne);
        cjoin(m, lc, ee);
        if (CONN == 8) {
            cjoin(m, lc, pe);
            cjoin(m, lc, pee);
        }
        const St no = accept(T.o[r], m, lc);
        chg |= (uint32_t)(neq(ne, T.e[r]) | neq(no, T.o[r])) << r;
        T.e[r] = ne;
        T.o[r] = no;
        pe = ne;
        po = no;
    }
    return chg;
}

// Flag each neighbour one of whose halo pixels the tile's border would change.
template <int CONN>
__device__ void sk_notify_scan(const SkSmem &s, const SkTile &T, int lane) {
    if (lane == 0)
        for (int r = 0; r < STH; r++) s.col0[r] = pack(T.e[r]);
    if (lane == 31)
        for (int r = 0; r < STH; r++) s.col63[r] = pack(T.o[r]);
    bool top = false, bot = false;
    {
        St wo = shfl_up1(T.o[0]), ee = shfl_dn1(T.e[0]);
        St bwo = shfl_up1(T.o[STH - 1]), bee = shfl_dn1(T.e[STH - 1]);
        if (lane == 0) wo = bwo = St{kBlocked, kNoLab};
        if (lane == 31) ee = bee = St{kBlocked, kNoLab};
        // halo row above: (-1, 2c) and (-1, 2c + 1); below: (STH, 2c) and (STH, 2c + 1)
        uint32_t m1 = T.e[0].d, l1 = T.e[0].l, m2 = T.o[0].d, l2 = T.o[0].l;
        uint32_t m3 = T.e[STH - 1].d, l3 = T.e[STH - 1].l, m4 = T.o[STH - 1].d, l4 = T.o[STH - 1].l;
        if (CONN == 8) {
            cjoin(m1, l1, wo);
            cjoin(m1, l1, T.o[0]);
            cjoin(m2, l2, T.e[0]);
            cjoin(m2, l2, ee);
            cjoin(m3, l3, bwo);
            cjoin(m3, l3, T.o[STH - 1]);
            cjoin(m4, l4, T.e[STH - 1]);
            cjoin(m4, l4, bee);
        }
        top = would_change(T.te, m1, l1) || would_change(T.to, m2, l2);
        bot = would_change(T.be, m3, l3) || would_change(T.bo, m4, l4);
    }
    top = __any_sync(0xffffffffu, top);
    bot = __any_sync(0xffffffffu, bot);
    if (lane == 0) {
        s.misc[1] = top;
        s.misc[7] = bot;
    }
    __syncwarp();
    bool lf = false, rt = false;
    if (lane < STH) {
        const int r = lane;
        St c = unpack(s.col0[r]);
        uint32_t ml = c.d, ll = c.l;
        c = unpack(s.col63[r]);
        uint32_t mr = c.d, lr = c.l;
        if (CONN == 8) {
            if (r > 0) {
                cjoin(ml, ll, unpack(s.col0[r - 1]));
                cjoin(mr, lr, unpack(s.col63[r - 1]));
            }
            if (r < STH - 1) {
                cjoin(ml, ll, unpack(s.col0[r + 1]));
                cjoin(mr, lr, unpack(s.col63[r + 1]));
            }
        }
        lf = would_change(unpack(s.hl[r + 1]), ml, ll);
        rt = would_change(unpack(s.hr[r + 1]), mr, lr);
    }
    lf = __any_sync(0xffffffffu, lf);
    rt = __any_sync(0xffffffffu, rt);
    if (lane == 0) {
        s.misc[3] = lf;
        s.misc[5] = rt;
        uint32_t c0 = 0, c2 = 0, c6 = 0, c8 = 0;
        if (CONN == 8) {
            St a = unpack(s.col0[0]);
            c0 = would_change(unpack(s.hl[0]), a.d, a.l);
            a = unpack(s.col0[STH - 1]);
            c6 = would_change(unpack(s.hl[STH + 1]), a.d, a.l);
            a = unpack(s.col63[0]);
            c2 = would_change(unpack(s.hr[0]), a.d, a.l);
            a = unpack(s.col63[STH - 1]);
            c8 = would_change(unpack(s.hr[STH + 1]), a.d, a.l);
        }
        s.misc[0] = c0;
        s.misc[2] = c2;
        s.misc[6] = c6;
        s.misc[8] = c8;
    }
}

__device__ void sk_store(const ImageView &im, int y0, int x0, const SkTile &T, uint32_t rows, int lane) {
    const int xe = x0 + 2 * lane;
    unsigned long long *V = reinterpret_cast<unsigned long long *>(im.J);
#pragma unroll
    for (int r = 0; r < STH; r++) {
        if (!((rows >> r) & 1u)) continue;
        const size_t row = (size_t)(y0 + r) * im.W;
        if (xe < im.W) __stcg(V + row + xe, pack(T.e[r]));
        if (xe + 1 < im.W) __stcg(V + row + xe + 1, pack(T.o[r]));
    }
}

// The CTA tile's shared state: each strip's first and last row (d and l of the even and
// odd pixel per lane), the tile's notification flags, the popped tile.
struct SkShared {
    uint32_t rows[SKW][8][32];
    uint32_t misc[16];
    uint32_t tile, redo;
};
constexpr size_t kSkSmemCta = kSkSmemPerWarp * SKW + sizeof(SkShared);

// Fold one strip's notification flags into the CTA tile's (as for the reconstruction's
// cooperative tile: a strip's top / bottom side is the tile's only for the first / last
// strip, and its corners beside the tile's inner rows lie in the west / east neighbours).
__device__ __forceinline__ void sk_fold_misc(SkShared &C, const uint32_t *m, int w) {
    if (w == 0) {
        atomicOr(&C.misc[0], m[0]);
        atomicOr(&C.misc[1], m[1]);
        atomicOr(&C.misc[2], m[2]);
    } else {
        atomicOr(&C.misc[3], m[0]);
        atomicOr(&C.misc[5], m[2]);
    }
    if (w == SKW - 1) {
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
__device__ void sk_visit(const EngineArgs &a, uint32_t t, uint8_t *wsmem, SkShared &C, VisitStats &st, int w,
                         int lane) {
    const ImageView &im = a.img0;
    const SkSmem s = sk_carve(wsmem);
    const int ty = (int)(t / im.tiles_x), tx = (int)(t % im.tiles_x);
    const int y0 = ty * SCH + STH * w, x0 = tx * STW;
    if (lane < 16) s.misc[lane] = 0;
    if (threadIdx.x < 16) C.misc[threadIdx.x] = 0;
    SkTile T;
    sk_load(im, s, y0, x0, T, lane);
    uint32_t passes = 0;
    for (;;) {
        uint32_t rows = 0;
        bool active = true;
        for (;;) {   // joint iterations of the strips
            uint32_t ch = 0;
            if (active) {
                ch = sk_pass<CONN, 1>(s, T, lane);
                ch |= sk_pass<CONN, -1>(s, T, lane);
                passes += 2;
                rows |= ch;
            }
            C.rows[w][0][lane] = T.e[0].d;
            C.rows[w][1][lane] = T.e[0].l;
            C.rows[w][2][lane] = T.o[0].d;
            C.rows[w][3][lane] = T.o[0].l;
            C.rows[w][4][lane] = T.e[STH - 1].d;
            C.rows[w][5][lane] = T.e[STH - 1].l;
            C.rows[w][6][lane] = T.o[STH - 1].d;
            C.rows[w][7][lane] = T.o[STH - 1].l;
            __syncthreads();
            St nte = T.te, nto = T.to, nbe = T.be, nbo = T.bo;
            if (w > 0) {
                nte = St{C.rows[w - 1][4][lane], C.rows[w - 1][5][lane]};
                nto = St{C.rows[w - 1][6][lane], C.rows[w - 1][7][lane]};
            }
            if (w < SKW - 1) {
                nbe = St{C.rows[w + 1][0][lane], C.rows[w + 1][1][lane]};
                nbo = St{C.rows[w + 1][2][lane], C.rows[w + 1][3][lane]};
            }
            const bool halo =
                __any_sync(0xffffffffu, neq(nte, T.te) || neq(nto, T.to) || neq(nbe, T.be) || neq(nbo, T.bo));
            T.te = nte;
            T.to = nto;
            T.be = nbe;
            T.bo = nbo;
            const bool active_next = halo || __any_sync(0xffffffffu, ch != 0);
            active = active_next;
            if (!__syncthreads_or(active)) break;
        }
        if (w == 0 && lane == 0) st.visits++;
        if (__syncthreads_or(rows != 0)) {
            sk_store(im, y0, x0, T, rows, lane);
            sk_notify_scan<CONN>(s, T, lane);
            if (lane == 0) sk_fold_misc(C, s.misc, w);
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
        sk_load_halo(im, s, y0, x0, T, lane);
        __syncthreads();
    }
    st.waves += passes;
}

// Initialisation, one warp per 16 x 64 strip: markers take (0, their label), other domain
// pixels are unreached, the rest blocked; the CTA tile of every strip holding a marker is
// queued. Labels above 65534 stop the call with IWPP_ERR_ARG.
__global__ void __launch_bounds__(256) sk_init_kernel(EngineArgs a, const uint32_t *markers, const uint8_t *mask,
                                                      uint32_t nstrips) {
    const ImageView &im = a.img0;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long *V = reinterpret_cast<unsigned long long *>(im.J);
    for (uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nstrips; u += nw) {
        const int uy = (int)(u / im.tiles_x), ux = (int)(u % im.tiles_x);
        const int y0 = uy * STH, x0 = ux * STW;
        bool any = false, bad = false;
        for (int r = 0; r < STH; r++) {
            const int y = y0 + r;
            if (y >= im.H) break;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int x = x0 + 2 * lane + q;
                if (x >= im.W) continue;
                const size_t e = (size_t)y * im.W + x;
                const uint32_t m = markers[e];
                bad |= m > 65534u;
                any |= m != 0;
                St s;
                if (m) s = St{0u, (m << 16) | (0xFFFFu - m)};
                else s = St{mask[e] ? kUnr : kBlocked, kNoLab};
                V[e] = pack(s);
            }
        }
        any = __any_sync(0xffffffffu, any);
        bad = __any_sync(0xffffffffu, bad);
        __threadfence();
        if (lane == 0 && bad) set_status(a.hdr, kErrArg);
        if (lane == 0 && any) notify_tile(a, (uint32_t)((uy / SKW) * im.tiles_x + ux));
    }
}

template <int CONN>
__global__ void __launch_bounds__(kThreads, 2) sk_drain_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * kSkSmemPerWarp;
    SkShared &C = *reinterpret_cast<SkShared *>(smem_raw + SKW * kSkSmemPerWarp);
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
        sk_visit<CONN>(a, t, wsmem, C, st, warp, lane);
        if (warp == 0) busy += globaltimer_ns() - b0;
        __syncthreads();   // every warp has read C.tile before the next pop overwrites it
    }
    flush_stats(a, st, idle, busy, lane);
}

// zone (label where one label is nearest, else 0), optional distance (-1 where unreached)
// and optional label pair (min label << 16) | max label (0 where unreached)
__global__ void sk_finish_kernel(const unsigned long long *V, uint32_t *zone, int32_t *dist, uint32_t *lpair,
                                 size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const St s = unpack(V[i]);
        const bool reached = s.d < kUnr;
        const uint32_t lmin = s.l >> 16, lmax = 0xFFFFu - (s.l & 0xFFFFu);
        zone[i] = reached && lmin == lmax ? lmin : 0u;
        if (dist) dist[i] = reached ? (int32_t)s.d : -1;
        if (lpair) lpair[i] = reached ? (lmin << 16) | lmax : 0u;
    }
}

struct SkLayout {
    size_t state, queue, px, total;
    uint32_t ntiles, nstrips;   // 64 x 64 CTA tiles; 16 x 64 strips
    int tiles_x, tiles_y;
};

bool sk_layout(int64_t H, int64_t W, SkLayout &L) {
    if (H < 1 || W < 1 || H >= (1ll << 31) || W >= (1ll << 31) || (uint64_t)H * (uint64_t)W >= (1ull << 31))
        return false;
    const uint64_t tx = (uint64_t)((W + STW - 1) / STW), ty = (uint64_t)((H + SCH - 1) / SCH);
    L.tiles_x = (int)tx;
    L.tiles_y = (int)ty;
    L.ntiles = (uint32_t)(tx * ty);
    L.nstrips = (uint32_t)(tx * (uint64_t)((H + STH - 1) / STH));
    L.state = 256;
    L.queue = L.state + align256((size_t)L.ntiles * 4);
    L.px = L.queue + align256((size_t)L.ntiles * 4);
    L.total = L.px + align256((size_t)H * (size_t)W * 8);
    return true;
}

}  // namespace
}  // namespace iwpp

extern "C" size_t iwpp_skiz_workspace_bytes(int64_t H, int64_t W) {
    iwpp::SkLayout L;
    return iwpp::sk_layout(H, W, L) ? L.total : 0;
}

extern "C" int iwpp_skiz(const uint32_t *markers, const uint8_t *mask, uint32_t *zone_out, int32_t *dist_out,
                         uint32_t *lpair_out, int64_t H, int64_t W, int connectivity, void *workspace,
                         size_t ws_bytes, void *stream) {
    using namespace iwpp;
    if (!markers || !mask || !zone_out) return IWPP_ERR_ARG;
    if (connectivity != 4 && connectivity != 8) return IWPP_ERR_ARG;
    if (((uintptr_t)markers & 3) || ((uintptr_t)zone_out & 3) || (dist_out && ((uintptr_t)dist_out & 3)) ||
        (lpair_out && ((uintptr_t)lpair_out & 3)))
        return IWPP_ERR_ARG;
    SkLayout L;
    if (!sk_layout(H, W, L)) return IWPP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return IWPP_ERR_WORKSPACE;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    EngineArgs a = {};
    a.img0.J = base + L.px;
    a.img0.I = mask;
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
    if (cudaMemsetAsync(base, 0, L.queue, s) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaMemsetAsync(base + L.queue, 0xFF, (size_t)L.ntiles * 4, s) != cudaSuccess) return IWPP_ERR_CUDA;
    const int sms = device_sm_count();
    if (sms <= 0) return IWPP_ERR_CUDA;
    uint32_t ig = (L.nstrips + 7) / 8;
    if (ig > (uint32_t)sms * 8) ig = (uint32_t)sms * 8;
    sk_init_kernel<<<ig, 256, 0, s>>>(a, markers, mask, L.nstrips);
    const size_t smem = kSkSmemCta;
    void (*drain)(EngineArgs) = connectivity == 8 ? sk_drain_kernel<8> : sk_drain_kernel<4>;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, drain, kThreads, smem) != cudaSuccess || bps < 1)
        return IWPP_ERR_CUDA;
    long long g = (long long)bps * sms;
    if (g > (long long)L.ntiles) g = L.ntiles;   // one CTA per tile
    drain<<<(int)g, kThreads, smem, s>>>(a);
    const size_t n = (size_t)H * (size_t)W;
    sk_finish_kernel<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(base + L.px), zone_out,
                                              dist_out, lpair_out, n);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

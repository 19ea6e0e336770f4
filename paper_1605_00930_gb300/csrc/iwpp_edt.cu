// iwpp_edt.cu — Euclidean distance transform by Voronoi-site propagation (Sec. 3.2,
// Algorithm 8) on the persistent tile engine (include/iwpp.h, iwpp_edt).
//
// Every pixel carries a site: the background pixel it is nearest to among those its
// neighbours have offered, packed as (y << 16) | x, or kNoSite. Background pixels are
// their own sites. A visit holds a 16 x 64 tile in registers (lane c: columns 2c and
// 2c + 1, one register each per row) and repeats down / up Gauss-Seidel passes in which
// every pixel takes a neighbour's site if that site is strictly closer to it (the
// propagation step of Algorithm 8), until a pass pair changes nothing: then no neighbour
// offers any pixel of the tile a closer site. A halo pixel that one of the tile's sites
// would bring strictly closer marks its tile for a visit, as in the reconstruction.
// Distances are squared Euclidean, exact in 32-bit integers for sides below 32768.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/iwpp.h"
#include "iwpp_engine.cuh"
#include "iwpp_host.h"

namespace iwpp {
namespace {

constexpr uint32_t kNoSite = 0xFFFFFFFFu;
constexpr int ETH = 16, ETW = 64;   // tile rows, columns

__device__ __forceinline__ uint32_t site_d2(int y, int x, uint32_t s) {
    // unsigned arithmetic: exact for real sites (< 2^31), wraps harmlessly for kNoSite
    const uint32_t dy = (uint32_t)(y - (int)(s >> 16)), dx = (uint32_t)(x - (int)(s & 0xFFFFu));
    return s == kNoSite ? 0xFFFFFFFFu : dy * dy + dx * dx;
}
// Keep (best, bd) or take cand if it is strictly closer to (y, x).
__device__ __forceinline__ void offer(int y, int x, uint32_t cand, uint32_t &best, uint32_t &bd) {
    const uint32_t d = site_d2(y, x, cand);
    const bool take = d < bd;
    best = take ? cand : best;
    bd = take ? d : bd;
}

struct EdtSmem {
    uint32_t *hl, *hr;       // ETH + 2: sites of the halo columns, index = row + 1
    uint32_t *col0, *col63;  // ETH: the tile's first and last column after a solve
    uint32_t *misc;          // 16: notification flags
};
constexpr size_t kEdtWords = 2 * (ETH + 2) + 2 * ETH + 16;
constexpr size_t kEdtSmemPerWarp = (kEdtWords * 4 + 15) & ~(size_t)15;

__device__ EdtSmem edt_carve(uint8_t *base) {
    EdtSmem s;
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    s.hl = w; w += ETH + 2;
    s.hr = w; w += ETH + 2;
    s.col0 = w; w += ETH;
    s.col63 = w; w += ETH;
    s.misc = w;
    return s;
}

__device__ __forceinline__ uint32_t ld_site(const ImageView &im, int y, int x) {
    const bool in = y >= 0 && y < im.H && x >= 0 && x < im.W;
    const uint32_t *S = reinterpret_cast<const uint32_t *>(im.J);
    const uint32_t v = __ldcg(S + (size_t)min(max(y, 0), im.H - 1) * im.W + min(max(x, 0), im.W - 1));
    return in ? v : kNoSite;
}

// The tile (sites, 2 per lane and row) and its halo.
struct EdtTile {
    uint32_t e[ETH], o[ETH];   // columns 2c and 2c + 1
    uint32_t te, to, be, bo;   // halo rows above / below at this lane's columns
};

__device__ void edt_load_halo(const ImageView &im, const EdtSmem &s, int y0, int x0, EdtTile &T, int lane) {
    const int xe = x0 + 2 * lane;
    T.te = ld_site(im, y0 - 1, xe);
    T.to = ld_site(im, y0 - 1, xe + 1);
    T.be = ld_site(im, y0 + ETH, xe);
    T.bo = ld_site(im, y0 + ETH, xe + 1);
    for (int i = lane; i < ETH + 2; i += 32) {
        s.hl[i] = ld_site(im, y0 + i - 1, x0 - 1);
        s.hr[i] = ld_site(im, y0 + i - 1, x0 + ETW);
    }
    __syncwarp();
}

__device__ void edt_load(const ImageView &im, const EdtSmem &s, int y0, int x0, EdtTile &T, int lane) {
    const int xe = x0 + 2 * lane;
#pragma unroll
    for (int r = 0; r < ETH; r++) {
        T.e[r] = ld_site(im, y0 + r, xe);
        T.o[r] = ld_site(im, y0 + r, xe + 1);
    }
    edt_load_halo(im, s, y0, x0, T, lane);
}

// One pass over the rows in the order DIR (+1 down, -1 up): each row from its own sites,
// the previous row of the pass (already updated) and its horizontal neighbours. Pixels
// outside the image keep no site. Returns this lane's changed rows.
template <int CONN, int DIR>
__device__ __forceinline__ uint32_t edt_pass(const EdtSmem &s, EdtTile &T, int y0, int x0, int H, int W, int lane) {
    const int xe = x0 + 2 * lane, xo = xe + 1;
    const bool ve = xe < W, vo = xo < W;
    uint32_t pe = DIR > 0 ? T.te : T.be, po = DIR > 0 ? T.to : T.bo;   // the row before, this pass
    uint32_t chg = 0;
#pragma unroll
    for (int k = 0; k < ETH; k++) {
        const int r = DIR > 0 ? k : ETH - 1 - k;
        const int y = y0 + r;
        const uint32_t hrow = s.hl[r + 1], hrow_r = s.hr[r + 1];
        const uint32_t hprev = s.hl[r + 1 - DIR], hprev_r = s.hr[r + 1 - DIR];
        // horizontal neighbours of this row (values before the pass) and of the previous row
        uint32_t wo = __shfl_up_sync(0xffffffffu, T.o[r], 1), ee = __shfl_down_sync(0xffffffffu, T.e[r], 1);
        if (lane == 0) wo = hrow;
        if (lane == 31) ee = hrow_r;
        uint32_t pwo = __shfl_up_sync(0xffffffffu, po, 1), pee = __shfl_down_sync(0xffffffffu, pe, 1);
        if (lane == 0) pwo = hprev;
        if (lane == 31) pee = hprev_r;
        // even pixel: own, W, E, and the previous row's N (+ NW, NE)
        uint32_t be_ = T.e[r], de = site_d2(y, xe, be_);
        offer(y, xe, wo, be_, de);
        offer(y, xe, T.o[r], be_, de);
        offer(y, xe, pe, be_, de);
        if (CONN == 8) {
            offer(y, xe, pwo, be_, de);
            offer(y, xe, po, be_, de);
        }
        const bool in = y < H;
        be_ = (in && ve) ? be_ : kNoSite;
        // odd pixel: own, W (the even pixel, just updated), E, and the previous row
        uint32_t bo_ = T.o[r], dd = site_d2(y, xo, bo_);
        offer(y, xo, be_, bo_, dd);
        offer(y, xo, ee, bo_, dd);
        offer(y, xo, po, bo_, dd);
        if (CONN == 8) {
            offer(y, xo, pe, bo_, dd);
            offer(y, xo, pee, bo_, dd);
        }
        bo_ = (in && vo) ? bo_ : kNoSite;
        chg |= (uint32_t)((be_ != T.e[r]) | (bo_ != T.o[r])) << r;
        T.e[r] = be_;
        T.o[r] = bo_;
        pe = be_;
        po = bo_;
    }
    return chg;
}

// Flag each neighbour one of whose halo pixels a site of the tile would bring strictly
// closer (misc[(dy + 1) * 3 + dx + 1]).
template <int CONN>
__device__ void edt_notify_scan(const EdtSmem &s, const EdtTile &T, int y0, int x0, int lane) {
    const int xe = x0 + 2 * lane, xo = xe + 1;
    if (lane == 0)
        for (int r = 0; r < ETH; r++) s.col0[r] = T.e[r];
    if (lane == 31)
        for (int r = 0; r < ETH; r++) s.col63[r] = T.o[r];
    // halo rows: candidates from the tile's first / last row (the tile's own columns only)
    bool top = false, bot = false;
    {
        uint32_t wo = __shfl_up_sync(0xffffffffu, T.o[0], 1), ee = __shfl_down_sync(0xffffffffu, T.e[0], 1);
        uint32_t bwo = __shfl_up_sync(0xffffffffu, T.o[ETH - 1], 1),
                 bee = __shfl_down_sync(0xffffffffu, T.e[ETH - 1], 1);
        if (lane == 0) wo = bwo = kNoSite;
        if (lane == 31) ee = bee = kNoSite;
        const int yt = y0 - 1, yb = y0 + ETH;
        uint32_t s1 = T.te, d1 = site_d2(yt, xe, s1), s2 = T.to, d2 = site_d2(yt, xo, s2);
        const uint32_t d1o = d1, d2o = d2;
        offer(yt, xe, T.e[0], s1, d1);
        offer(yt, xo, T.o[0], s2, d2);
        if (CONN == 8) {
            offer(yt, xe, wo, s1, d1);
            offer(yt, xe, T.o[0], s1, d1);
            offer(yt, xo, T.e[0], s2, d2);
            offer(yt, xo, ee, s2, d2);
        }
        top = (d1 < d1o) || (d2 < d2o);
        uint32_t s3 = T.be, d3 = site_d2(yb, xe, s3), s4 = T.bo, d4 = site_d2(yb, xo, s4);
        const uint32_t d3o = d3, d4o = d4;
        offer(yb, xe, T.e[ETH - 1], s3, d3);
        offer(yb, xo, T.o[ETH - 1], s4, d4);
        if (CONN == 8) {
            offer(yb, xe, bwo, s3, d3);
            offer(yb, xe, T.o[ETH - 1], s3, d3);
            offer(yb, xo, T.e[ETH - 1], s4, d4);
            offer(yb, xo, bee, s4, d4);
        }
        bot = (d3 < d3o) || (d4 < d4o);
    }
    top = __any_sync(0xffffffffu, top);
    bot = __any_sync(0xffffffffu, bot);
    if (lane == 0) {
        s.misc[1] = top;
        s.misc[7] = bot;
    }
    __syncwarp();
    // halo columns: one row per lane; corners by lane 0
    bool lf = false, rt = false;
    if (lane < ETH) {
        const int r = lane, y = y0 + r;
        const int xl = x0 - 1, xr = x0 + ETW;
        uint32_t sl = s.hl[r + 1], dl = site_d2(y, xl, sl), sr = s.hr[r + 1], dr = site_d2(y, xr, sr);
        const uint32_t dlo = dl, dro = dr;
        offer(y, xl, s.col0[r], sl, dl);
        offer(y, xr, s.col63[r], sr, dr);
        if (CONN == 8) {
            if (r > 0) {
                offer(y, xl, s.col0[r - 1], sl, dl);
                offer(y, xr, s.col63[r - 1], sr, dr);
            }
            if (r < ETH - 1) {
                offer(y, xl, s.col0[r + 1], sl, dl);
                offer(y, xr, s.col63[r + 1], sr, dr);
            }
        }
        lf = dl < dlo;
        rt = dr < dro;
    }
    lf = __any_sync(0xffffffffu, lf);
    rt = __any_sync(0xffffffffu, rt);
    if (lane == 0) {
        s.misc[3] = lf;
        s.misc[5] = rt;
        uint32_t c0 = 0, c2 = 0, c6 = 0, c8 = 0;
        if (CONN == 8) {
            const int yt = y0 - 1, yb = y0 + ETH, xl = x0 - 1, xr = x0 + ETW;
            c0 = site_d2(yt, xl, s.col0[0]) < site_d2(yt, xl, s.hl[0]);
            c6 = site_d2(yb, xl, s.col0[ETH - 1]) < site_d2(yb, xl, s.hl[ETH + 1]);
            c2 = site_d2(yt, xr, s.col63[0]) < site_d2(yt, xr, s.hr[0]);
            c8 = site_d2(yb, xr, s.col63[ETH - 1]) < site_d2(yb, xr, s.hr[ETH + 1]);
        }
        s.misc[0] = c0;
        s.misc[2] = c2;
        s.misc[6] = c6;
        s.misc[8] = c8;
    }
}

__device__ void edt_store(const ImageView &im, int y0, int x0, const EdtTile &T, uint32_t rows, int lane) {
    const int xe = x0 + 2 * lane;
    uint32_t *S = reinterpret_cast<uint32_t *>(im.J);
#pragma unroll
    for (int r = 0; r < ETH; r++) {
        if (!((rows >> r) & 1u)) continue;
        const size_t row = (size_t)(y0 + r) * im.W;
        if (xe < im.W) __stcg(S + row + xe, T.e[r]);
        if (xe + 1 < im.W) __stcg(S + row + xe + 1, T.o[r]);
    }
}

template <int CONN>
__device__ void edt_visit(const EngineArgs &a, uint32_t t, uint8_t *wsmem, VisitStats &st, int lane) {
    const ImageView &im = a.img0;
    const EdtSmem s = edt_carve(wsmem);
    const int ty = (int)(t / im.tiles_x), tx = (int)(t % im.tiles_x);
    const int y0 = ty * ETH, x0 = tx * ETW;
    if (lane < 16) s.misc[lane] = 0;
    EdtTile T;
    edt_load(im, s, y0, x0, T, lane);
    uint32_t passes = 0;
    for (;;) {
        uint32_t rows = 0;
        for (;;) {
            uint32_t ch = edt_pass<CONN, 1>(s, T, y0, x0, im.H, im.W, lane);
            ch |= edt_pass<CONN, -1>(s, T, y0, x0, im.H, im.W, lane);
            passes += 2;
            rows |= ch;
            if (!__any_sync(0xffffffffu, ch != 0)) break;
        }
        st.visits++;
        const bool changed = __any_sync(0xffffffffu, rows != 0);
        if (changed) {
            edt_store(im, y0, x0, T, rows, lane);
            edt_notify_scan<CONN>(s, T, y0, x0, lane);
            __threadfence();
            __syncwarp();
        }
        if (changed && lane < 9 && lane != 4 && s.misc[lane]) {
            const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
            if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                notify_tile(a, (uint32_t)(ny * im.tiles_x + nx));
        }
        if (!finish_tile(a, t, lane)) break;
        __syncwarp();
        if (lane < 16) s.misc[lane] = 0;
        edt_load_halo(im, s, y0, x0, T, lane);
    }
    st.waves += passes;
}

// Initialisation (Algorithm 8's first phase): background pixels are their own sites,
// foreground pixels have none; every tile with a foreground pixel is queued (its first
// visit takes what its halo offers).
__global__ void __launch_bounds__(256) edt_init_kernel(EngineArgs a) {
    const ImageView &im = a.img0;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *S = reinterpret_cast<uint32_t *>(im.J);
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.ntiles; t += nw) {
        const int ty = (int)(t / im.tiles_x), tx = (int)(t % im.tiles_x);
        const int y0 = ty * ETH, x0 = tx * ETW;
        bool fg = false;
        for (int r = 0; r < ETH; r++) {
            const int y = y0 + r;
            if (y >= im.H) break;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int x = x0 + 2 * lane + q;
                if (x >= im.W) continue;
                const size_t e = (size_t)y * im.W + x;
                const bool f = im.I[e] != 0;
                fg |= f;
                S[e] = f ? kNoSite : ((uint32_t)y << 16) | (uint32_t)x;
            }
        }
        fg = __any_sync(0xffffffffu, fg);
        __threadfence();
        if (lane == 0 && fg) notify_tile(a, t);
    }
}

template <int CONN>
__global__ void __launch_bounds__(kThreads, 2) edt_drain_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * kEdtSmemPerWarp;
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0;
    for (;;) {
        bool first;
        const uint32_t t = acquire_tile(a, first, idle, lane);
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        edt_visit<CONN>(a, t, wsmem, st, lane);
        busy += globaltimer_ns() - b0;
    }
    flush_stats(a, st, idle, busy, lane);
}

__global__ void edt_dist2_kernel(const uint32_t *S, uint32_t *D, int H, int W) {
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i % W);
        D[i] = site_d2(y, x, S[i]);
    }
}

// Workspace: header (256 B) | tile states | tile-queue ring.
struct EdtLayout {
    size_t state, queue, total;
    uint32_t ntiles;
    int tiles_x, tiles_y;
};

bool edt_layout(int64_t H, int64_t W, EdtLayout &L) {
    if (H < 1 || W < 1 || H > 32767 || W > 32767) return false;
    L.tiles_x = (int)((W + ETW - 1) / ETW);
    L.tiles_y = (int)((H + ETH - 1) / ETH);
    L.ntiles = (uint32_t)L.tiles_x * (uint32_t)L.tiles_y;
    L.state = 256;
    L.queue = L.state + align256((size_t)L.ntiles * 4);
    L.total = L.queue + align256((size_t)L.ntiles * 4);
    return true;
}

}  // namespace
}  // namespace iwpp

extern "C" size_t iwpp_edt_workspace_bytes(int64_t H, int64_t W) {
    iwpp::EdtLayout L;
    return iwpp::edt_layout(H, W, L) ? L.total : 0;
}

extern "C" int iwpp_edt(const void *mask, uint32_t *site_out, uint32_t *dist2_out, int64_t H, int64_t W,
                        int connectivity, void *workspace, size_t ws_bytes, void *stream) {
    using namespace iwpp;
    if (!mask || !site_out) return IWPP_ERR_ARG;
    if (connectivity != 4 && connectivity != 8) return IWPP_ERR_ARG;
    if (((uintptr_t)site_out & 3) || (dist2_out && ((uintptr_t)dist2_out & 3))) return IWPP_ERR_ARG;
    EdtLayout L;
    if (!edt_layout(H, W, L)) return IWPP_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return IWPP_ERR_WORKSPACE;
    if (ws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    EngineArgs a = {};
    a.img0.J = reinterpret_cast<uint8_t *>(site_out);
    a.img0.I = static_cast<const uint8_t *>(mask);
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
    const uint32_t warps_needed = L.ntiles;
    uint32_t ig = (warps_needed + 7) / 8;
    if (ig > (uint32_t)sms * 8) ig = (uint32_t)sms * 8;
    edt_init_kernel<<<ig, 256, 0, s>>>(a);
    const size_t smem = kEdtSmemPerWarp * kWarpsPerCta;
    void (*drain)(EngineArgs) = connectivity == 8 ? edt_drain_kernel<8> : edt_drain_kernel<4>;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, drain, kThreads, smem) != cudaSuccess || bps < 1)
        return IWPP_ERR_CUDA;
    long long g = (long long)bps * sms;
    const long long need = ((long long)L.ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    if (g > need) g = need;
    drain<<<(int)g, kThreads, smem, s>>>(a);
    if (dist2_out) edt_dist2_kernel<<<sms * 8, 256, 0, s>>>(site_out, dist2_out, (int)H, (int)W);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

// iwpp_scan.cuh — the streaming scan of the cooperative solver's 64 x 64 tiles (sm_103a).
//
// The scan is the initialisation pass of Algorithm 7 reduced to what the persistent drain
// needs: per tile, whether the precondition J <= I holds and whether one step of the update
// (Eq. "recon") would raise one of its pixels, in which case the tile enters the queue. It
// reads every pixel once, so it is bound by HBM and by how many loads are in flight.
//
// One warp streams one tile from the halo row above it to the halo row below it; lane c
// holds columns 2c and 2c + 1 of a row (u16x2, dilation domain), lanes 0 and 31 also the
// halo column pixel on their side. Loads run IWPP_STREAM_DEPTH rows ahead of the row
// being tested, through a ring of registers, so every warp keeps that many rows in flight without
// a break between tiles, and the image table is read once per tile. Rows are tested with a
// sliding window of three rows; learned batches also add up the tile's feature sums over its
// sampled rows (iwpp_feat.cuh) and, as the warp owns the whole tile, write its 16 features
// directly.
#pragma once
#include <type_traits>

#include "iwpp_feat.cuh"
#include "iwpp_regtile.cuh"

namespace iwpp {

#ifndef IWPP_STREAM_DEPTH
#define IWPP_STREAM_DEPTH 2   // rows of loads in flight per warp (4, 6, 8: slower, measured)
#endif
#ifndef IWPP_STREAM_MINB
#define IWPP_STREAM_MINB 8    // CTAs (of 4 warps) per SM of the streaming scan
#endif
#ifndef IWPP_STREAM_FEATS_MINB
#define IWPP_STREAM_FEATS_MINB 8   // the same with the feature sums (spills, but faster than 6 or 7: measured)
#endif

// One row of the stream as loaded; unpacked only when the row is used, so that the loads of
// the rows ahead stay in flight.
struct StreamRow {
    uint32_t j0, j1, i0, i1, h;
};

// Loads of image row y (clamped into the image, so every address is valid; rows and columns
// outside it are zeroed by stream_unpack). PAIR: W even, so the pair (gx, gx + 1) is one
// aligned two-element load; else two element loads. Lanes 0 and 31 load their halo column
// pixel `hc`. needI: the mask row is used (not for the halo rows above and below the tile).
template <bool WIDE, bool PAIR>
__device__ __forceinline__ void stream_issue(const ImageView &im, int y, int gx, int hc, bool needI, int lane,
                                             StreamRow &r) {
    using E = typename std::conditional<WIDE, uint16_t, uint8_t>::type;
    const E *J = reinterpret_cast<const E *>(im.J);
    const E *I = reinterpret_cast<const E *>(im.I);
    const size_t row = (size_t)min(max(y, 0), im.H - 1) * (size_t)im.W;
    if (PAIR) {
        using P = typename std::conditional<WIDE, uint32_t, uint16_t>::type;
        const size_t e = row + (size_t)min(gx, im.W - 2);
        r.j0 = __ldg(reinterpret_cast<const P *>(J + e));
        r.i0 = needI ? (uint32_t)__ldg(reinterpret_cast<const P *>(I + e)) : 0u;
    } else {
        const size_t e0 = row + (size_t)min(gx, im.W - 1), e1 = row + (size_t)min(gx + 1, im.W - 1);
        r.j0 = __ldg(J + e0);
        r.j1 = __ldg(J + e1);
        r.i0 = needI ? (uint32_t)__ldg(I + e0) : 0u;
        r.i1 = needI ? (uint32_t)__ldg(I + e1) : 0u;
    }
    r.h = (lane == 0 || lane == 31) ? (uint32_t)__ldg(J + row + (size_t)min(max(hc, 0), im.W - 1)) : 0u;
}

// The row in the dilation domain: packed pair of J and I (0 outside the image) and this
// lane's halo word (lane 0: left halo pixel, lane 31: right halo pixel << 16, as hmax wants).
template <bool WIDE, bool PAIR>
__device__ __forceinline__ void stream_unpack(const StreamRow &r, bool yin, uint32_t cm, uint32_t flip, bool hin,
                                              int lane, uint32_t &J, uint32_t &I, uint32_t &H) {
    uint32_t j, i;
    if (PAIR) {
        j = WIDE ? r.j0 : __byte_perm(r.j0, 0u, 0x4140);
        i = WIDE ? r.i0 : __byte_perm(r.i0, 0u, 0x4140);
    } else {
        j = r.j0 | (r.j1 << 16);
        i = r.i0 | (r.i1 << 16);
    }
    const uint32_t f2 = flip | (flip << 16);
    J = yin ? (j ^ f2) & cm : 0u;
    I = yin ? (i ^ f2) & cm : 0u;
    H = (yin && hin) ? (r.h ^ flip) << (lane == 31 ? 16 : 0) : 0u;
}

// One tile: rows y0 .. y0 + ny - 1 of the image (ny >= 1), streamed as rows y0 - 1 .. y0 + ny.
// Sets `can` (a pixel can rise: min(I, max over its neighbourhood of J) != J) and `bad`
// (J > I somewhere) for this lane; FEATS: adds the tile's pixels to `fa`.
template <bool WIDE, bool PAIR, int CONN, bool FEATS>
__device__ __forceinline__ void scan_tile_stream(const ImageView &im, int y0, int x0, int ny, int lane,
                                                 bool &can, bool &bad, FeatAcc &fa) {
    using RT = RegTile<uint8_t, CONN, kCoopStrip>;   // hmax only (independent of the pixel type)
    constexpr int D = IWPP_STREAM_DEPTH;
    const int gx = x0 + 2 * lane;
    const int hc = lane == 0 ? x0 - 1 : x0 + RT::TW;
    const bool hin = (lane == 0 && x0 > 0) || (lane == 31 && x0 + RT::TW < im.W);
    const bool c0 = gx < im.W, c1 = gx + 1 < im.W;
    const uint32_t cm = (c0 ? 0xFFFFu : 0u) | (c1 ? 0xFFFF0000u : 0u);
    const uint32_t rm = (c1 ? 0xFFFFu : 0u) | (lane < 31 && gx + 2 < im.W ? 0xFFFF0000u : 0u);   // right neighbour counts
    const uint32_t thr = 16u * ((WIDE ? 0xFFFFu : 0xFFu) / 255u);
    const int ns = ny + 2;   // stream rows: s <-> image row y0 - 1 + s
    StreamRow q[D];
#pragma unroll
    for (int k = 0; k < D; k++)
        if (k < ns) stream_issue<WIDE, PAIR>(im, y0 - 1 + k, gx, hc, k >= 1 && k <= ny, lane, q[k]);
    uint32_t jPrev = 0, jCur = 0, iCur = 0, hPrev = 0, hCur = 0;
    uint32_t h03 = 0, h47 = 0;   // FEATS: 8-bit histogram bins (at most 32 sampled pixels per lane)
    bool any = false, nok = false;
    for (int s0 = 0; s0 < ns; s0 += D) {
#pragma unroll
        for (int k = 0; k < D; k++) {
            const int s = s0 + k;
            if (s < ns) {   // warp-uniform
                const int y = y0 - 1 + s;
                uint32_t Jn, In, Hn;
                stream_unpack<WIDE, PAIR>(q[k], y >= 0 && y < im.H, cm, im.flip, hin, lane, Jn, In, Hn);
                if (s + D < ns) stream_issue<WIDE, PAIR>(im, y + D, gx, hc, s + D <= ny, lane, q[k]);
                const uint32_t hN = RT::hmax(Jn, Hn, lane);
                if (s >= 2) {   // test row s - 1 of the stream (a row of the tile)
                    const uint32_t m = CONN == 8 ? max2(hPrev, max2(hCur, hN)) : max2(hCur, max2(jPrev, Jn));
                    any |= min2(iCur, m) != jCur;
                    nok |= max2(jCur, iCur) != iCur;
                    if (FEATS && ((s - 2) % kFeatRowStep) == 0) {   // a sampled row (tile row s - 2)
                        const uint32_t iv = iCur, jv = jCur;
                        const uint32_t dv = max2(iv, jv) - jv;   // per half max(I - J, 0): no borrow
                        const uint32_t d8 = WIDE ? (dv >> 8) & 0x00FF00FFu : dv;
                        const uint32_t bl = min(7u, 32u - (uint32_t)__clz(d8 & 0xFFFFu));   // bit length, 0 for 0
                        const uint32_t bh = min(7u, 32u - (uint32_t)__clz(d8 >> 16));
                        h03 += (bl < 4 ? 1u << (8 * bl) : 0u) + (bh < 4 ? 1u << (8 * bh) : 0u);
                        h47 += (bl >= 4 ? 1u << (8 * bl - 32) : 0u) + (bh >= 4 ? 1u << (8 * bh - 32) : 0u);
                        const uint32_t x = iv ^ jv;
                        fa.seeds += (uint32_t)((x & 0xFFFFu) == 0 && (jv & 0xFFFFu) != 0) +
                                    (uint32_t)((x >> 16) == 0 && (jv >> 16) != 0);
                        fa.sI = __dp2a_lo(iv, 0x0101u, fa.sI);
                        fa.sJ = __dp2a_lo(jv, 0x0101u, fa.sJ);
                        fa.sD = __dp2a_lo(dv, 0x0101u, fa.sD);
                        fa.sI2 += (unsigned long long)(iv & 0xFFFFu) * (iv & 0xFFFFu);
                        fa.sI2 += (unsigned long long)(iv >> 16) * (iv >> 16);
                        fa.sJ2 += (unsigned long long)(jv & 0xFFFFu) * (jv & 0xFFFFu);
                        fa.sJ2 += (unsigned long long)(jv >> 16) * (jv >> 16);
                        // edges: the right neighbours in the tile, the pixel below in the tile
                        const uint32_t rp = __byte_perm(iv, __shfl_down_sync(0xffffffffu, iv, 1), 0x5432);
                        const uint32_t gxv = (max2(iv, rp) - min2(iv, rp)) & rm;
                        const uint32_t gyv = s <= ny ? max2(iv, In) - min2(iv, In) : 0u;
                        fa.edges += (uint32_t)((gxv & 0xFFFFu) + (gyv & 0xFFFFu) > thr) +
                                    (uint32_t)((gxv >> 16) + (gyv >> 16) > thr);
                    }
                }
                jPrev = jCur;
                jCur = Jn;
                iCur = In;
                hPrev = hCur;
                hCur = hN;
            }
        }
    }
    can = any;
    bad = nok;
    if (FEATS) {
        const uint32_t nrs = (uint32_t)((ny + kFeatRowStep - 1) / kFeatRowStep);   // sampled rows
        fa.n = nrs * ((uint32_t)c0 + (uint32_t)c1);
        fa.npix = (uint32_t)ny * ((uint32_t)c0 + (uint32_t)c1);
        fa.h03 = h03 - (2u * nrs - fa.n);   // columns outside the image were counted in bin 0
        fa.h47 = h47;
    }
}

// The streaming scan: warp u of the grid-stride loop takes tile u. FEATS (learned batches):
// also the tile's 16 features into a.feats (tile t = feature block t).
template <typename T, int CONN, bool FEATS>
__global__ void __launch_bounds__(kThreads, FEATS ? IWPP_STREAM_FEATS_MINB : IWPP_STREAM_MINB)
    scan_stream_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, kCoopStrip>;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t nw = (uint64_t)gridDim.x * kWarpsPerCta;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarpsPerCta + w; u < a.ntiles; u += nw) {
        const uint32_t t = (uint32_t)u;
        const long long c0 = clock64();
        const ImageView im = image_of(a, t);
        const uint32_t lt = t - im.tile_base;
        const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
        const int y0 = ty * kCoopRows, x0 = tx * RT::TW;
        const int ny = min(kCoopRows, im.H - y0);
        bool can = false, bad = false;
        FeatAcc fa;
        const bool wide = RT::wide(im), pair = (im.W & 1) == 0;
        if constexpr (std::is_same<T, AnyPix>::value) {
            if (wide) {
                if (pair) scan_tile_stream<true, true, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
                else scan_tile_stream<true, false, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
            } else {
                if (pair) scan_tile_stream<false, true, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
                else scan_tile_stream<false, false, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
            }
        } else {
            if (pair) scan_tile_stream<sizeof(T) == 2, true, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
            else scan_tile_stream<sizeof(T) == 2, false, CONN, FEATS>(im, y0, x0, ny, lane, can, bad, fa);
        }
        can = __any_sync(0xffffffffu, can);
        bad = __any_sync(0xffffffffu, bad);
        if (FEATS) {
            uint32_t v[16];
            unsigned long long sI2, sJ2;
            feat_reduce(fa, v, sI2, sJ2);
            if (lane < IWPP_NFEAT) a.feats[(size_t)t * IWPP_NFEAT + lane] = block_feature(lane, v, sI2, sJ2, wide ? 0xFFFFu : 0xFFu);
        }
        if (lane == 0) {
            if (can) {
                if (a.defer_push) mark_pending(a, t); else notify_tile(a, t);
            }
            if (bad) set_status(a.hdr, kErrPrecondition);
            if (a.tile_work) atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
        }
    }
}

}  // namespace iwpp

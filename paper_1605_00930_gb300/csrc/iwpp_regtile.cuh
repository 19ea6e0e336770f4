// iwpp_regtile.cuh — register-resident local solver for 64-wide tiles (sm_103a).
//
// Alternative to the shared-memory wave queues of iwpp_engine.cuh for the persistent
// kernel's tile visits. The tile (TH rows x 64 columns) lives in registers: lane c holds
// columns 2c (low 16 bits) and 2c + 1 (high 16 bits) of every row, one register per row
// for J and one for I, in the dilation domain; both columns are updated at once with the
// packed min.u16x2 / max.u16x2 instructions. The visit repeats Gauss-Seidel passes of the
// update of Algorithm 1 (Eq. "recon") until a pass pair changes nothing or a residual
// check finds no pixel that can still rise:
//   down pass, rows top to bottom:  J(p) <- min(I(p), max(J(p), W, E, N, and NW, NE for 8-conn)),
//                                   N / NW / NE already updated in this pass;
//   up pass, rows bottom to top:    the same with S, SW, SE.
// Horizontal neighbours come from the adjacent half of the register or, across lanes, from
// one warp shuffle per direction and row; the halo columns come from shared memory. There
// are no shared-memory atomics and no queues. At convergence every pixel satisfies
// J = min(I, max over its neighbourhood) for the current halo: the same local fixed point
// the queue solver reaches, so the global result is the same (the reconstruction is unique).
#pragma once
#include <type_traits>

#include "iwpp_engine.cuh"

namespace iwpp {

__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// Left neighbours of a packed pair: (column 2c - 1, column 2c) from the previous lane's
// pair `p` and this lane's pair `v`; right neighbours: (column 2c + 1, column 2c + 2).
__device__ __forceinline__ uint32_t left_of(uint32_t p, uint32_t v) { return __byte_perm(p, v, 0x5432); }
__device__ __forceinline__ uint32_t right_of(uint32_t v, uint32_t n) { return __byte_perm(v, n, 0x5432); }

// Pixel type tag of kernels that serve u8 and u16 images alike (batches of one
// connectivity and both pixel types): the element size is read from the image's kind at
// run time. Only loads and stores depend on it; the packed u16x2 arithmetic is the same.
struct AnyPix {};

template <typename T, int CONN, int TH>
struct RegTile {
    static_assert(TH >= 2 && TH <= 32, "tile rows");
    static constexpr int TW = 64;
    static constexpr int kRows = TH;
    // 16-bit pixels?
    static __device__ __forceinline__ bool wide(const ImageView &im) {
        if constexpr (std::is_same<T, AnyPix>::value) return (im.kind & 1u) != 0;
        else return sizeof(T) == 2;
    }
    struct Smem {
        uint32_t *hxJ;          // 2 x (TH + 2): [0..TH+1] left halo column, [TH+2..] right halo column << 16
        uint32_t *hzero;        // TH + 2 zeros: the halo words of lanes 1..30
        uint32_t *hlI, *hrI;    // TH + 2: mask of the halo columns, index = row + 1
        uint32_t *col0, *col63; // TH: the tile's first and last column after a solve
        uint32_t *misc;         // 16: notification flags
    };
    static constexpr size_t kWords = 5 * (TH + 2) + 2 * TH + 16;
    static __host__ __device__ size_t smem_per_warp(uint32_t) { return (kWords * 4 + 15) & ~(size_t)15; }
    static size_t smem_bytes(uint32_t q) { return smem_per_warp(q) * kWarpsPerCta; }

    static __device__ Smem carve(uint8_t *base) {
        Smem s;
        uint32_t *w = reinterpret_cast<uint32_t *>(base);
        s.hxJ = w; w += 2 * (TH + 2);
        s.hzero = w; w += TH + 2;
        s.hlI = w; w += TH + 2;
        s.hrI = w; w += TH + 2;
        s.col0 = w; w += TH;
        s.col63 = w; w += TH;
        s.misc = w;
        return s;
    }

    static __device__ __forceinline__ uint32_t ld1(const ImageView &im, const uint8_t *p, size_t e, bool cg) {
        if (wide(im)) {
            const uint16_t *q = reinterpret_cast<const uint16_t *>(p) + e;
            return (uint32_t)(cg ? __ldcg(q) : *q);
        }
        const uint8_t *q = p + e;
        return (uint32_t)(cg ? __ldcg(q) : *q);
    }

    // Pixels (y, gx) and (y, gx + 1) of plane p, packed, flipped, 0 outside the image.
    // Branch-free: both loads use clamped coordinates (always a valid address) and the
    // out-of-image halves are zeroed afterwards, so a run of these calls issues all its
    // loads before the first result is needed.
    static __device__ __forceinline__ uint32_t ld_pair(const ImageView &im, const uint8_t *p, int y, int gx,
                                                       bool cg) {
        const bool yin = y >= 0 && y < im.H;
        const size_t row = (size_t)min(max(y, 0), im.H - 1) * im.W;
        const uint32_t a = ld1(im, p, row + min(gx, im.W - 1), cg), b = ld1(im, p, row + min(gx + 1, im.W - 1), cg);
        return ((yin && gx < im.W) ? (a ^ im.flip) : 0u) | (((yin && gx + 1 < im.W) ? (b ^ im.flip) : 0u) << 16);
    }

    // Raw pair at element e (even; the row is 2-pixel aligned when W is even) and its
    // packed form: one 16-bit (u8) or 32-bit (u16) load.
    static __device__ __forceinline__ uint32_t ld_raw(const ImageView &im, const uint8_t *p, size_t e, bool cg) {
        if (!wide(im)) {
            const uint16_t *q = reinterpret_cast<const uint16_t *>(p + e);
            return (uint32_t)(cg ? __ldcg(q) : *q);
        }
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p + 2 * e);
        return cg ? __ldcg(q) : *q;
    }
    static __device__ __forceinline__ uint32_t unpack_raw(const ImageView &im, uint32_t w) {
        return wide(im) ? w : __byte_perm(w, 0u, 0x4140);
    }

    // Halo: top and bottom rows into registers (this lane's pair), the two halo columns
    // (with corners) into shared memory. 0 outside the image.
    static __device__ void load_halo(const ImageView &im, const Smem &s, int y0, int x0, uint32_t &jt,
                                     uint32_t &jb, uint32_t &it, uint32_t &ib, bool withI, int lane) {
        const int gx = x0 + 2 * lane;
        jt = ld_pair(im, im.J, y0 - 1, gx, true);
        jb = ld_pair(im, im.J, y0 + TH, gx, true);
        if (withI) {
            it = ld_pair(im, im.I, y0 - 1, gx, false);
            ib = ld_pair(im, im.I, y0 + TH, gx, false);
        }
        for (int hr = lane; hr < TH + 2; hr += 32) {
            const int gy = y0 + hr - 1;
            const bool rowin = gy >= 0 && gy < im.H;
            const bool lin = rowin && x0 > 0, rin = rowin && x0 + TW < im.W;
            const size_t row = (size_t)min(max(gy, 0), im.H - 1) * im.W;
            const size_t el = row + max(x0 - 1, 0), er = row + min(x0 + TW, im.W - 1);
            const uint32_t lj = ld1(im, im.J, el, true), rj = ld1(im, im.J, er, true);
            uint32_t li = 0, ri = 0;
            if (withI) {
                li = ld1(im, im.I, el, false);
                ri = ld1(im, im.I, er, false);
            }
            s.hxJ[hr] = lin ? lj ^ im.flip : 0u;
            s.hxJ[TH + 2 + hr] = rin ? (rj ^ im.flip) << 16 : 0u;
            s.hzero[hr] = 0u;
            if (withI) {
                s.hlI[hr] = lin ? li ^ im.flip : 0u;
                s.hrI[hr] = rin ? ri ^ im.flip : 0u;
            }
        }
        __syncwarp();
    }

    static __device__ void load(const ImageView &im, const Smem &s, int y0, int x0, uint32_t (&J)[TH],
                                uint32_t (&I)[TH], uint32_t &jt, uint32_t &jb, uint32_t &it, uint32_t &ib,
                                int lane) {
        if (im.W >= 2) {   // every width but 1
            load_fused(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
            return;
        }
        const int gx = x0 + 2 * lane;
#pragma unroll
        for (int r = 0; r < TH; r++) {
            J[r] = ld_pair(im, im.J, y0 + r, gx, true);
            I[r] = ld_pair(im, im.I, y0 + r, gx, false);
        }
        load_halo(im, s, y0, x0, jt, jb, it, ib, true, lane);
    }

    // The load of a strip and its halo with every global load (strip rows, halo rows, halo
    // columns) issued before the first result is used, so a visit costs one memory round trip
    // (measured: the load phase 20-25 % shorter than loading the halo after the strip). Rows
    // are read as aligned two-pixel words (u8: 16-bit, u16: 32-bit loads). Even W: the pair
    // (gx, gx + 1) is aligned in every row. Odd W >= 3: a row's pairs are aligned when the row
    // starts on an even element (row index even, as x0 is even) and off by one otherwise; such
    // a row is read as the aligned pairs (gx - 1, gx), and each lane takes its second pixel
    // from the next lane's first (lane 31 from pixel x0 + 63, loaded with the halo columns by
    // the lane that holds that row). On even rows the lane whose pair would end past the row
    // (gx = W - 1) reads an aligned pair inside the row instead and takes pixel W - 1 from the
    // halo lanes too. Every address stays inside its row (the row before, for the first pair
    // of an odd row) of the image; columns at or past W are zeroed.
    static __device__ __forceinline__ void load_fused(const ImageView &im, const Smem &s, int y0, int x0,
                                                      uint32_t (&J)[TH], uint32_t (&I)[TH], uint32_t &jt,
                                                      uint32_t &jb, uint32_t &it, uint32_t &ib, int lane) {
        static_assert(TH + 2 <= 32, "one halo row per lane");
        const int W = im.W, H = im.H;
        const bool odd = (W & 1) != 0;   // W >= 3 when odd (the caller's condition)
        const int gx = x0 + 2 * lane;
        const uint32_t f2 = im.flip | (im.flip << 16);
        const uint32_t cm = (gx < W ? 0xFFFFu : 0u) | (gx + 1 < W ? 0xFFFF0000u : 0u);
        const int xe0 = odd ? min(gx, W - 3) : min(gx, W - 2);   // pair start in an aligned row
        const int xe1 = min(gx, W - 1) - 1;                      // in an odd row of an odd-W image
        auto pair_start = [&](int y) {   // >= 0: an odd row has yc >= 1
            const int yc = min(max(y, 0), H - 1);
            return (size_t)((long long)yc * W + ((odd && (yc & 1)) ? xe1 : xe0));
        };
        auto odd_row = [&](int y) { return odd && (min(max(y, 0), H - 1) & 1); };
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const size_t e = pair_start(y0 + r);
            J[r] = ld_raw(im, im.J, e, true);
            I[r] = ld_raw(im, im.I, e, false);
        }
        // halo rows (rows clamped into the image, so every address is valid; zeroed below when
        // the row lies outside it: a strip of a bottom tile can start several rows below the image)
        const size_t et = pair_start(y0 - 1), eb = pair_start(y0 + TH);
        uint32_t rjt = ld_raw(im, im.J, et, true), rjb = ld_raw(im, im.J, eb, true);
        uint32_t rit = ld_raw(im, im.I, et, false), rib = ld_raw(im, im.I, eb, false);
        // halo columns: lane hr < TH + 2 holds row y0 + hr - 1 (odd W: also pixel min(x0 + 63, W - 1))
        const int gy = y0 + lane - 1;
        const bool rowin = lane < TH + 2 && gy >= 0 && gy < H;
        const bool lin = rowin && x0 > 0, rin = rowin && x0 + TW < W;
        const size_t hrow = (size_t)min(max(gy, 0), H - 1) * (size_t)W;
        const size_t el = hrow + max(x0 - 1, 0), er = hrow + min(x0 + TW, W - 1), e63 = hrow + min(x0 + 63, W - 1);
        const uint32_t lj = ld1(im, im.J, el, true), rj = ld1(im, im.J, er, true);
        const uint32_t li = ld1(im, im.I, el, false), ri = ld1(im, im.I, er, false);
        const uint32_t sj = odd ? ld1(im, im.J, e63, true) : 0u, si = odd ? ld1(im, im.I, e63, false) : 0u;
        // uses: a row's pixel pair in the dilation domain; hl = the halo lane holding the row
        auto fix = [&](uint32_t &u, uint32_t sv, bool oddrow) {
            if (oddrow) {
                uint32_t n = __shfl_down_sync(0xffffffffu, u, 1);
                if (lane == 31) n = sv;
                u = (u >> 16) | (n << 16);
            } else if (gx == W - 1) {
                u = sv;   // pixel W - 1; the pair's second pixel lies outside the image
            }
        };
        auto use = [&](uint32_t rj_, uint32_t ri_, int y, int hl, bool in, uint32_t &jo, uint32_t &io) {
            uint32_t uj = unpack_raw(im, rj_), ui = unpack_raw(im, ri_);
            if (odd) {   // warp-uniform
                const uint32_t svj = __shfl_sync(0xffffffffu, sj, hl), svi = __shfl_sync(0xffffffffu, si, hl);
                const bool o = odd_row(y);
                fix(uj, svj, o);
                fix(ui, svi, o);
            }
            jo = in ? (uj ^ f2) & cm : 0u;
            io = in ? (ui ^ f2) & cm : 0u;
        };
#pragma unroll
        for (int r = 0; r < TH; r++) use(J[r], I[r], y0 + r, r + 1, y0 + r < H, J[r], I[r]);
        use(rjt, rit, y0 - 1, 0, y0 >= 1 && y0 - 1 < H, jt, it);
        use(rjb, rib, y0 + TH, TH + 1, y0 + TH < H, jb, ib);
        if (lane < TH + 2) {
            s.hxJ[lane] = lin ? lj ^ im.flip : 0u;
            s.hxJ[TH + 2 + lane] = rin ? (rj ^ im.flip) << 16 : 0u;
            s.hzero[lane] = 0u;
            s.hlI[lane] = lin ? li ^ im.flip : 0u;
            s.hrI[lane] = rin ? ri ^ im.flip : 0u;
        }
        __syncwarp();
    }

    // Bytes of the per-warp staging area of load_vec: both planes, TH rows of up to 128 bytes.
    static constexpr int kStageBytes = 2 * TH * 128;

    // Can the strip's rows be copied in 16-byte chunks? (64-column span inside the image, row
    // pitch a multiple of 16 bytes; the planes themselves are 16-byte aligned.)
    static __device__ __forceinline__ bool vec_ok(const ImageView &im, int x0) {
        return x0 + TW <= im.W && ((size_t)im.W * (wide(im) ? 2 : 1)) % 16 == 0;
    }

    // load_fused with the strip's rows copied by 16-byte asynchronous copies into `stage`
    // (global -> shared, no registers in flight): for u8 four lanes cover a 64-pixel row and
    // one copy instruction eight rows, for u16 eight lanes a row and four rows; the lanes then
    // read their column pairs from shared memory. Halo rows and columns as in load_fused.
    static __device__ __forceinline__ void load_vec(const ImageView &im, const Smem &s, uint8_t *stage, int y0,
                                                    int x0, uint32_t (&J)[TH], uint32_t (&I)[TH], uint32_t &jt,
                                                    uint32_t &jb, uint32_t &it, uint32_t &ib, int lane) {
        const bool w16 = wide(im);
        const int es = w16 ? 2 : 1, cpr = 4 * es, rpl = 32 / cpr;
        const size_t pitch = (size_t)im.W * es;
        const int ch = lane % cpr;
        for (int k = 0; k < TH / rpl; k++) {
            const int rr = k * rpl + lane / cpr;
            const size_t off = (size_t)min(y0 + rr, im.H - 1) * pitch + (size_t)x0 * es + (size_t)ch * 16;
            const unsigned dj = static_cast<unsigned>(__cvta_generic_to_shared(stage + rr * 128 + ch * 16));
            const unsigned di = static_cast<unsigned>(__cvta_generic_to_shared(stage + (TH + rr) * 128 + ch * 16));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dj), "l"(im.J + off) : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(di), "l"(im.I + off) : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const int gx = x0 + 2 * lane;
        const uint32_t f2 = im.flip | (im.flip << 16);
        const size_t et = (size_t)min(max(y0 - 1, 0), im.H - 1) * im.W + gx;
        const size_t eb = (size_t)min(max(y0 + TH, 0), im.H - 1) * im.W + gx;
        uint32_t rjt = ld_raw(im, im.J, et, true), rjb = ld_raw(im, im.J, eb, true);
        uint32_t rit = ld_raw(im, im.I, et, false), rib = ld_raw(im, im.I, eb, false);
        const int gy = y0 + lane - 1;
        const bool rowin = lane < TH + 2 && gy >= 0 && gy < im.H;
        const bool lin = rowin && x0 > 0, rin = rowin && x0 + TW < im.W;
        const size_t hrow = (size_t)min(max(gy, 0), im.H - 1) * im.W;
        const size_t el = hrow + max(x0 - 1, 0), er = hrow + min(x0 + TW, im.W - 1);
        const uint32_t lj = ld1(im, im.J, el, true), rj = ld1(im, im.J, er, true);
        const uint32_t li = ld1(im, im.I, el, false), ri = ld1(im, im.I, er, false);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const bool in = y0 + r < im.H;
            const uint32_t vj = w16 ? *reinterpret_cast<const uint32_t *>(stage + r * 128 + 4 * lane)
                                    : unpack_raw(im, *reinterpret_cast<const uint16_t *>(stage + r * 128 + 2 * lane));
            const uint32_t vi = w16 ? *reinterpret_cast<const uint32_t *>(stage + (TH + r) * 128 + 4 * lane)
                                    : unpack_raw(im, *reinterpret_cast<const uint16_t *>(stage + (TH + r) * 128 +
                                                                                          2 * lane));
            J[r] = in ? vj ^ f2 : 0u;
            I[r] = in ? vi ^ f2 : 0u;
        }
        const bool tin = y0 >= 1 && y0 - 1 < im.H, bin = y0 + TH < im.H;
        jt = tin ? unpack_raw(im, rjt) ^ f2 : 0u;
        it = tin ? unpack_raw(im, rit) ^ f2 : 0u;
        jb = bin ? unpack_raw(im, rjb) ^ f2 : 0u;
        ib = bin ? unpack_raw(im, rib) ^ f2 : 0u;
        if (lane < TH + 2) {
            s.hxJ[lane] = lin ? lj ^ im.flip : 0u;
            s.hxJ[TH + 2 + lane] = rin ? (rj ^ im.flip) << 16 : 0u;
            s.hzero[lane] = 0u;
            s.hlI[lane] = lin ? li ^ im.flip : 0u;
            s.hrI[lane] = rin ? ri ^ im.flip : 0u;
        }
        __syncwarp();
    }

    // Horizontal max of a packed row over (left, self, right); `h` is this lane's halo word
    // (lane 0: the left halo pixel in the low half, lane 31: the right halo pixel in the high
    // half, the other lanes 0). Lane 0's up shuffle and lane 31's down shuffle return their
    // own pair, so their outside neighbour repeats a pixel of the pair that the max already
    // holds, and h supplies the real one: one max instead of two lane selects.
    static __device__ __forceinline__ uint32_t hmax(uint32_t v, uint32_t h, int lane) {
        (void)lane;
        const uint32_t p = __shfl_up_sync(0xffffffffu, v, 1), n = __shfl_down_sync(0xffffffffu, v, 1);
        return max2(max2(v, h), max2(left_of(p, v), right_of(v, n)));
    }

    // This lane's halo words, index = row + 1 (lanes 1..30: zeros).
    static __device__ __forceinline__ const uint32_t *halo_words(const Smem &s, int lane) {
        return lane == 0 ? s.hxJ : (lane == 31 ? s.hxJ + TH + 2 : s.hzero);
    }

    // One down pass; returns this lane's mask of changed rows. For 8-connectivity the
    // neighbourhood {W, E, N, NW, NE} of a row is the horizontal max of max(row, row above)
    // (max commutes with the shift), so one shuffle pair per row serves both rows; the
    // side halo is then the max of the two rows' halo words. For 4-connectivity each row
    // first takes N (clamped to I: a valid update of every pixel) and then W / E from
    // those new values, so a path that steps down and sideways advances within one pass
    // (measured: 7 instead of 16 passes per visit on the 4096^2 tissue image).
    // DIFF: return the OR of (new ^ old) over the rows instead of the mask of changed rows
    // (non-zero iff this lane changed a pixel; one instruction per row instead of three).
    template <bool DIFF = false>
    static __device__ __forceinline__ uint32_t pass_down(const uint32_t *hx, uint32_t (&J)[TH],
                                                         const uint32_t (&I)[TH], uint32_t jt, int lane) {
        uint32_t chg = 0, up = jt, hprev = hx[0];
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const uint32_t hcur = hx[r + 1], v = J[r];
            const uint32_t nv = CONN == 8 ? min2(I[r], hmax(max2(v, up), max2(hcur, hprev), lane))
                                          : min2(I[r], hmax(min2(I[r], max2(v, up)), hcur, lane));
            if (DIFF) chg |= nv ^ v;
            else chg |= (uint32_t)(nv != v) << r;
            J[r] = nv;
            up = nv;
            hprev = hcur;
        }
        return chg;
    }

    template <bool DIFF = false>
    static __device__ __forceinline__ uint32_t pass_up(const uint32_t *hx, uint32_t (&J)[TH],
                                                       const uint32_t (&I)[TH], uint32_t jb, int lane) {
        uint32_t chg = 0, dn = jb, hnext = hx[TH + 1];
#pragma unroll
        for (int r = TH - 1; r >= 0; r--) {
            const uint32_t hcur = hx[r + 1], v = J[r];
            const uint32_t nv = CONN == 8 ? min2(I[r], hmax(max2(v, dn), max2(hcur, hnext), lane))
                                          : min2(I[r], hmax(min2(I[r], max2(v, dn)), hcur, lane));
            if (DIFF) chg |= nv ^ v;
            else chg |= (uint32_t)(nv != v) << r;
            J[r] = nv;
            dn = nv;
            hnext = hcur;
        }
        return chg;
    }

    // ---- raster / anti-raster sweeps (Algorithm 7's scanning phase) ------------------------
    // Along a row, the raster update J(x) <- min(I(x), max(a(x), J(x - 1))) is the map
    // v -> clamp(v, lo, hi) with lo = min(I, a), hi = I, and clamps compose into clamps, so a
    // whole row is one warp scan of (lo, hi) pairs packed as u16x2: five shuffle steps
    // instead of a 64-step chain. a(x) holds the pixel's own value and its neighbours in
    // the previous row (already swept), so one raster sweep followed by one anti-raster
    // sweep is exactly the paper's pair of scans over this tile.
    static __device__ __forceinline__ uint32_t dup_lo(uint32_t g) { return __byte_perm(g, g, 0x1010); }
    static __device__ __forceinline__ uint32_t dup_hi(uint32_t g) { return __byte_perm(g, g, 0x3232); }

    // West-to-east pass over one packed row. A = min(I, candidates) per pixel, Ir = mask,
    // hxr = this lane's halo word of the row (lane 0: west halo pixel << 16).
    static __device__ __forceinline__ uint32_t row_we(uint32_t A, uint32_t Ir, uint32_t hxr, int lane) {
        // this lane's pair as one clamp, even pixel first: (lo, hi)
        uint32_t G = min2(dup_hi(Ir), max2(dup_hi(A), __byte_perm(A, Ir, 0x5410)));
        if (lane == 0) {   // fold the west halo in: lane 0's map becomes a constant
            const uint32_t c = min(G >> 16, max(G & 0xFFFFu, hxr & 0xFFFFu));
            G = c | (c << 16);
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t Q = __shfl_up_sync(0xffffffffu, G, d);
            const uint32_t C = min2(dup_hi(G), max2(dup_lo(G), Q));   // this map after Q
            if (lane >= d) G = C;
        }
        // every map is now a constant: the value leaving this lane's odd pixel
        const uint32_t E = __shfl_up_sync(0xffffffffu, G, 1);
        const uint32_t u = lane == 0 ? hxr & 0xFFFFu : E & 0xFFFFu;
        const uint32_t X = min2(Ir, max2(A, u));                      // even pixel (low half)
        return __byte_perm(X, G, 0x5410);
    }

    // East-to-west pass over one packed row (lane 31: east halo pixel in the high half).
    static __device__ __forceinline__ uint32_t row_ew(uint32_t A, uint32_t Ir, uint32_t hxr, int lane) {
        uint32_t G = min2(dup_lo(Ir), max2(dup_lo(A), __byte_perm(A, Ir, 0x7632)));   // odd pixel first
        if (lane == 31) {
            const uint32_t c = min(G >> 16, max(G & 0xFFFFu, hxr >> 16));
            G = c | (c << 16);
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t Q = __shfl_down_sync(0xffffffffu, G, d);
            const uint32_t C = min2(dup_hi(G), max2(dup_lo(G), Q));
            if (lane + d < 32) G = C;
        }
        const uint32_t E = __shfl_down_sync(0xffffffffu, G, 1);
        const uint32_t u = lane == 31 ? hxr >> 16 : E & 0xFFFFu;
        const uint32_t Y = min2(Ir, max2(A, u << 16));                // odd pixel (high half)
        return __byte_perm(G, Y, 0x7610);
    }

    // Raster sweep: rows top to bottom, each from its own values and the swept row above
    // (N, and NW / NE for 8-conn), then west to east. Returns this lane's changed rows.
    static __device__ __forceinline__ uint32_t sweep_raster(const uint32_t *hx, uint32_t (&J)[TH],
                                                            const uint32_t (&I)[TH], uint32_t jt, int lane) {
        uint32_t chg = 0, up = jt;
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const uint32_t hu = CONN == 8 ? hmax(up, hx[r], lane) : up;
            const uint32_t nv = row_we(min2(I[r], max2(J[r], hu)), I[r], hx[r + 1], lane);
            chg |= (uint32_t)(nv != J[r]) << r;
            J[r] = nv;
            up = nv;
        }
        return chg;
    }

    // Anti-raster sweep: rows bottom to top (S, and SW / SE), then east to west.
    static __device__ __forceinline__ uint32_t sweep_antiraster(const uint32_t *hx, uint32_t (&J)[TH],
                                                                const uint32_t (&I)[TH], uint32_t jb, int lane) {
        uint32_t chg = 0, dn = jb;
#pragma unroll
        for (int r = TH - 1; r >= 0; r--) {
            const uint32_t hd = CONN == 8 ? hmax(dn, hx[r + 2], lane) : dn;
            const uint32_t nv = row_ew(min2(I[r], max2(J[r], hd)), I[r], hx[r + 1], lane);
            chg |= (uint32_t)(nv != J[r]) << r;
            J[r] = nv;
            dn = nv;
        }
        return chg;
    }

    // Is some pixel of the tile still below min(I, max over its neighbourhood)? The rows
    // are independent here, so this costs far less latency than another pass pair.
    static __device__ __forceinline__ bool improvable(const uint32_t *hx, const uint32_t (&J)[TH],
                                                      const uint32_t (&I)[TH], uint32_t jt, uint32_t jb,
                                                      int lane) {
        bool any = false;
        uint32_t prev = CONN == 8 ? hmax(jt, hx[0], lane) : jt;
        uint32_t cur = hmax(J[0], hx[1], lane);
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const uint32_t nxt = r + 1 < TH ? J[r + 1 < TH ? r + 1 : r] : jb;
            const uint32_t nxtH = hmax(nxt, hx[r + 2], lane);
            const uint32_t m = max2(cur, max2(prev, CONN == 8 ? nxtH : nxt));
            any |= min2(I[r], m) != J[r];
            prev = CONN == 8 ? cur : J[r];
            cur = nxtH;
        }
        return __any_sync(0xffffffffu, any);
    }

    // Largest value one step from the tile's own pixels can raise a halo pixel to, per
    // neighbour (misc[(dy + 1) * 3 + dx + 1]; 0 = no halo pixel of that neighbour can rise
    // above its loaded value). The value sets the neighbour's queue level.
    static __device__ __forceinline__ uint32_t raise2(uint32_t cand, uint32_t cur) {
        // per half: the candidate where it exceeds the current value, else 0; max of halves
        const uint32_t lo = (cand & 0xFFFFu) > (cur & 0xFFFFu) ? (cand & 0xFFFFu) : 0u;
        const uint32_t hi = (cand >> 16) > (cur >> 16) ? (cand >> 16) : 0u;
        return max(lo, hi);
    }
    static __device__ void notify_scan(const Smem &s, const uint32_t (&J)[TH], uint32_t jt, uint32_t jb,
                                       uint32_t it, uint32_t ib, int lane) {
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < TH; r++) s.col0[r] = J[r] & 0xFFFFu;
        }
        if (lane == 31) {
#pragma unroll
            for (int r = 0; r < TH; r++) s.col63[r] = J[r] >> 16;
        }
        // top and bottom halo rows: the tile's neighbours only (0 beyond its side columns)
        const uint32_t mt = CONN == 8 ? hmax(J[0], 0u, lane) : J[0];
        const uint32_t mb = CONN == 8 ? hmax(J[TH - 1], 0u, lane) : J[TH - 1];
        const uint32_t vt = __reduce_max_sync(0xffffffffu, raise2(min2(it, mt), jt));
        const uint32_t vb = __reduce_max_sync(0xffffffffu, raise2(min2(ib, mb), jb));
        if (lane == 0) {
            s.misc[1] = vt;
            s.misc[7] = vb;
        }
        __syncwarp();
        // left and right halo columns, one row per lane
        uint32_t vl = 0, vr = 0;
        for (int r = lane; r < TH; r += 32) {
            uint32_t ml = s.col0[r], mr = s.col63[r];
            if (CONN == 8) {
                if (r > 0) { ml = max(ml, s.col0[r - 1]); mr = max(mr, s.col63[r - 1]); }
                if (r < TH - 1) { ml = max(ml, s.col0[r + 1]); mr = max(mr, s.col63[r + 1]); }
            }
            const uint32_t cl = min(s.hlI[r + 1], ml), cr = min(s.hrI[r + 1], mr);
            if (cl > s.hxJ[r + 1]) vl = max(vl, cl);
            if (cr > (s.hxJ[TH + 2 + r + 1] >> 16)) vr = max(vr, cr);
        }
        vl = __reduce_max_sync(0xffffffffu, vl);
        vr = __reduce_max_sync(0xffffffffu, vr);
        if (lane == 0) {
            s.misc[3] = vl;
            s.misc[5] = vr;
            uint32_t c0 = 0, c2 = 0, c6 = 0, c8 = 0;
            if (CONN == 8) {   // corners
                const uint32_t a0 = min(s.hlI[0], s.col0[0]), a6 = min(s.hlI[TH + 1], s.col0[TH - 1]);
                const uint32_t a2 = min(s.hrI[0], s.col63[0]), a8 = min(s.hrI[TH + 1], s.col63[TH - 1]);
                c0 = a0 > s.hxJ[0] ? a0 : 0u;
                c6 = a6 > s.hxJ[TH + 1] ? a6 : 0u;
                c2 = a2 > (s.hxJ[TH + 2] >> 16) ? a2 : 0u;
                c8 = a8 > (s.hxJ[2 * TH + 3] >> 16) ? a8 : 0u;
            }
            s.misc[0] = c0;
            s.misc[2] = c2;
            s.misc[6] = c6;
            s.misc[8] = c8;
        }
    }

    // Largest value any pixel of the tile can still be raised to (0: none can rise).
    static __device__ __forceinline__ uint32_t raise_max(const uint32_t *hx, const uint32_t (&J)[TH],
                                                         const uint32_t (&I)[TH], uint32_t jt, uint32_t jb,
                                                         int lane) {
        uint32_t best = 0;
        uint32_t prev = CONN == 8 ? hmax(jt, hx[0], lane) : jt;
        uint32_t cur = hmax(J[0], hx[1], lane);
#pragma unroll
        for (int r = 0; r < TH; r++) {
            const uint32_t nxt = r + 1 < TH ? J[r + 1 < TH ? r + 1 : r] : jb;
            const uint32_t nxtH = hmax(nxt, hx[r + 2], lane);
            const uint32_t m = max2(cur, max2(prev, CONN == 8 ? nxtH : nxt));
            best = max(best, raise2(min2(I[r], m), J[r]));
            prev = CONN == 8 ? cur : J[r];
            cur = nxtH;
        }
        return __reduce_max_sync(0xffffffffu, best);
    }

    // Store this lane's pairs of the rows it changed (rows below the image never change).
    template <typename P>
    static __device__ __forceinline__ void store_as(const ImageView &im, int y0, int gx, const uint32_t (&J)[TH],
                                                    uint32_t rows) {
        const uint32_t f2 = im.flip | (im.flip << 16);
        P *q = reinterpret_cast<P *>(im.J) + (size_t)y0 * im.W + gx;
        if (gx + 1 < im.W && (im.W & 1) == 0) {
#pragma unroll
            for (int r = 0; r < TH; r++) {
                const uint32_t v = J[r] ^ f2;
                if ((rows >> r) & 1u) {
                    if (sizeof(P) == 1)
                        __stcg(reinterpret_cast<uint16_t *>(q + (size_t)r * im.W), (uint16_t)__byte_perm(v, 0u, 0x0020));
                    else
                        __stcg(reinterpret_cast<uint32_t *>(q + (size_t)r * im.W), v);
                }
            }
        } else {
            const bool pair = gx + 1 < im.W;
#pragma unroll
            for (int r = 0; r < TH; r++) {
                const uint32_t v = J[r] ^ f2;
                if ((rows >> r) & 1u) {
                    __stcg(q + (size_t)r * im.W, (P)(v & 0xFFFFu));
                    if (pair) __stcg(q + (size_t)r * im.W + 1, (P)(v >> 16));
                }
            }
        }
    }
    static __device__ void store(const ImageView &im, int y0, int x0, const uint32_t (&J)[TH], uint32_t rows,
                                 int lane) {
        const int gx = x0 + 2 * lane;
        if (gx >= im.W) return;
        if (wide(im)) store_as<uint16_t>(im, y0, gx, J, rows);
        else store_as<uint8_t>(im, y0, gx, J, rows);
    }
};

#ifndef IWPP_TRACE
#define IWPP_TRACE 0   // record visit generations and a start-time histogram (measurement builds)
#endif
#if IWPP_TRACE
// Generation of a visit = 1 + the largest generation among the visits that notified the
// tile; the largest generation is the longest chain of tile hops. Visit start times are
// binned in 10 us steps from the first visit of the launch.
constexpr int kTraceTiles = 1 << 22, kTraceBins = 1 << 14;
__device__ unsigned int g_trace_gen[kTraceTiles];
__device__ unsigned int g_trace_hist[kTraceBins];
__device__ unsigned long long g_trace_t0;
__device__ unsigned int g_trace_maxgen;
#endif

#ifndef IWPP_REG_SWEEPS
#define IWPP_REG_SWEEPS 0   // 1: visits settle tiles with raster / anti-raster sweep pairs
#endif

// Frontier initialisation of one tile with the tile in registers (the scan kernel's body
// for the register solver's plans): precondition check, the tile's raster / anti-raster
// sweep pairs, store, then mark the tile if one of its pixels can still rise and each
// neighbour one of whose halo pixels it can raise.
template <typename T, int CONN, int TH>
__device__ void scan_tile_reg(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem, int lane) {
    using RT = RegTile<T, CONN, TH>;
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = RT::halo_words(s, lane);
    const long long c0 = clock64();
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * TH, x0 = tx * RT::TW;
    if (lane < 16) s.misc[lane] = 0;
#if IWPP_TRACE
    if (lane == 0 && t < (uint32_t)kTraceTiles) g_trace_gen[t] = 0;
#endif
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    bool bad = false;
#pragma unroll
    for (int r = 0; r < TH; r++) bad |= max2(J[r], I[r]) != I[r];
    bad = __any_sync(0xffffffffu, bad);
    const int sweeps = a.tile_sweeps ? (int)a.tile_sweeps[t] : a.sweeps;
    uint32_t rows = 0;
    for (int k = 0; k < sweeps; k++) {
        rows |= RT::sweep_raster(hx, J, I, jt, lane);
        rows |= RT::sweep_antiraster(hx, J, I, jb, lane);
    }
    if (rows) RT::store(im, y0, x0, J, rows, lane);
    const uint32_t self = RT::raise_max(hx, J, I, jt, jb, lane);
    RT::notify_scan(s, J, jt, jb, it, ib, lane);
    __threadfence();
    __syncwarp();
    if (lane < 9 && lane != 4 && s.misc[lane]) {
        const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
        if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x) {
            const uint32_t n = im.tile_base + (uint32_t)(ny * im.tiles_x + nx);
            if (a.defer_push) mark_pending(a, n); else notify_tile(a, n, level_of(a, im, s.misc[lane]));
        }
    }
    if (lane == 0) {
        if (self) {
            if (a.defer_push) mark_pending(a, t); else notify_tile(a, t, level_of(a, im, self));
        }
        if (bad) set_status(a.hdr, kErrPrecondition);
        if (a.tile_work) atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
    __syncwarp();
}

#if IWPP_PHASE_TIMING
#define IWPP_RT_MARK(k)                         \
    do {                                        \
        const long long _n = clock64();         \
        ph[k] += (unsigned long long)(_n - pt); \
        pt = _n;                                \
    } while (0)
#else
#define IWPP_RT_MARK(k) \
    do {                \
    } while (0)
#endif

// One visit with the register solver, including the re-processing rounds when the tile
// is notified while this warp holds it (the protocol of visit_tile).
template <typename T, int CONN, int TH>
__device__ void visit_tile_reg(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem, VisitStats &st,
                               unsigned long long *ph, int lane) {
    (void)ph;
#if IWPP_PHASE_TIMING
    long long pt = clock64();
#endif
    using RT = RegTile<T, CONN, TH>;
    const typename RT::Smem s = RT::carve(wsmem);
    const uint32_t *hx = RT::halo_words(s, lane);
    const long long c0 = clock64();
    const uint32_t lt = t - im.tile_base;
    const int ty = (int)(lt / im.tiles_x), tx = (int)(lt % im.tiles_x);
    const int y0 = ty * TH, x0 = tx * RT::TW;
    if (lane < 16) s.misc[lane] = 0;
#if IWPP_TRACE
    uint32_t gen = 0;
    if (lane == 0) {
        const unsigned long long now = globaltimer_ns();
        atomicMin(&g_trace_t0, now);
        const unsigned long long b = (now - *(volatile unsigned long long *)&g_trace_t0) / 10000ull;
        atomicAdd(&g_trace_hist[b < (unsigned long long)kTraceBins ? b : kTraceBins - 1], 1u);
        gen = (t < (uint32_t)kTraceTiles ? *(volatile unsigned int *)&g_trace_gen[t] : 0u) + 1u;
        atomicMax(&g_trace_maxgen, gen);
    }
    gen = __shfl_sync(0xffffffffu, gen, 0);
#endif
    uint32_t J[TH], I[TH], jt, jb, it, ib;
    RT::load(im, s, y0, x0, J, I, jt, jb, it, ib, lane);
    IWPP_RT_MARK(0);
    uint32_t passes = 0;
    for (;;) {
        uint32_t rows = 0;
        for (;;) {
#if IWPP_REG_SWEEPS
            uint32_t ch = RT::sweep_raster(hx, J, I, jt, lane);
            ch |= RT::sweep_antiraster(hx, J, I, jb, lane);
#else
            uint32_t ch = RT::pass_down(hx, J, I, jt, lane);
            ch |= RT::pass_up(hx, J, I, jb, lane);
#endif
            passes += 2;
            rows |= ch;
            IWPP_RT_MARK(1);
            if (!__any_sync(0xffffffffu, ch != 0)) break;
            const bool more = RT::improvable(hx, J, I, jt, jb, lane);
            IWPP_RT_MARK(2);
            if (!more) break;
        }
        st.visits++;
        // A round that raised nothing leaves the tile as it was when its last notifications
        // were sent (the previous visit, or the scan): no neighbour can have gained work.
        const bool changed = __any_sync(0xffffffffu, rows != 0);
#if IWPP_COUNT_IDLE_VISITS
        st.pops += changed ? 0u : 1u;   // measurement builds: rounds that raised nothing
#endif
        if (changed) {
            RT::store(im, y0, x0, J, rows, lane);
            IWPP_RT_MARK(3);
            RT::notify_scan(s, J, jt, jb, it, ib, lane);
            IWPP_RT_MARK(4);
            __threadfence();
            __syncwarp();
            IWPP_RT_MARK(5);
        }
        if (changed && lane < 9 && lane != 4 && s.misc[lane]) {
            const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
            if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x) {
                const uint32_t n = im.tile_base + (uint32_t)(ny * im.tiles_x + nx);
#if IWPP_TRACE
                if (n < (uint32_t)kTraceTiles) atomicMax(&g_trace_gen[n], gen);
#endif
                notify_tile(a, n, level_of(a, im, s.misc[lane]));
            }
        }
        const bool redo = finish_tile(a, t, lane);
        IWPP_RT_MARK(6);
        if (!redo) break;
        // re-process: J and I stay in registers; only the halo can have changed
        __syncwarp();
        if (lane < 16) s.misc[lane] = 0;
        RT::load_halo(im, s, y0, x0, jt, jb, it, ib, false, lane);
        IWPP_RT_MARK(7);
    }
    st.waves += passes;
    if (lane == 0 && a.tile_work) {
        atomicAdd(a.tile_work + t, passes);
        atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
}

__device__ inline void flush_phases(const EngineArgs &a, const unsigned long long (&ph)[8], int lane) {
#if IWPP_PHASE_TIMING
    if (lane == 0)
        for (int k = 0; k < 8; k++) atomicAdd(&a.hdr->phase_cycles[k], ph[k]);
#else
    (void)a;
    (void)ph;
    (void)lane;
#endif
}

template <typename T, int CONN, int TH, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) drain_reg_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, TH>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RT::smem_per_warp(0);
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0, ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (;;) {
        bool first;
        const uint32_t t = acquire_tile(a, first, idle, lane);
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        visit_tile_reg<T, CONN, TH>(a, image_of(a, t), t, wsmem, st, ph, lane);
        busy += globaltimer_ns() - b0;
    }
    flush_stats(a, st, idle, busy, lane);
    flush_phases(a, ph, lane);
}

template <typename T, int CONN, int TH>
__global__ void __launch_bounds__(kThreads) scan_reg_kernel(EngineArgs a) {
    using RT = RegTile<T, CONN, TH>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RT::smem_per_warp(0);
    const uint32_t nworkers = gridDim.x * kWarpsPerCta;
    for (uint32_t t = blockIdx.x * kWarpsPerCta + warp; t < a.ntiles; t += nworkers)
        scan_tile_reg<T, CONN, TH>(a, image_of(a, t), t, wsmem, lane);
}

template <int TH>
__global__ void __launch_bounds__(kThreads) scan_reg_mixed_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RegTile<uint16_t, 8, TH>::smem_per_warp(0);
    const uint32_t nworkers = gridDim.x * kWarpsPerCta;
    for (uint32_t t = blockIdx.x * kWarpsPerCta + warp; t < a.ntiles; t += nworkers) {
        const ImageView &im = image_of(a, t);
        switch (im.kind) {
            case 0: scan_tile_reg<uint8_t, 4, TH>(a, im, t, wsmem, lane); break;
            case 1: scan_tile_reg<uint16_t, 4, TH>(a, im, t, wsmem, lane); break;
            case 2: scan_tile_reg<uint8_t, 8, TH>(a, im, t, wsmem, lane); break;
            default: scan_tile_reg<uint16_t, 8, TH>(a, im, t, wsmem, lane); break;
        }
    }
}

// Batch of images of mixed pixel types and connectivities: dispatch on the image's kind.
template <int TH, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) drain_reg_mixed_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * RegTile<uint16_t, 8, TH>::smem_per_warp(0);
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0, ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (;;) {
        bool first;
        const uint32_t t = acquire_tile(a, first, idle, lane);
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        const ImageView &im = image_of(a, t);
        switch (im.kind) {
            case 0: visit_tile_reg<uint8_t, 4, TH>(a, im, t, wsmem, st, ph, lane); break;
            case 1: visit_tile_reg<uint16_t, 4, TH>(a, im, t, wsmem, st, ph, lane); break;
            case 2: visit_tile_reg<uint8_t, 8, TH>(a, im, t, wsmem, st, ph, lane); break;
            default: visit_tile_reg<uint16_t, 8, TH>(a, im, t, wsmem, st, ph, lane); break;
        }
        busy += globaltimer_ns() - b0;
    }
    flush_stats(a, st, idle, busy, lane);
    flush_phases(a, ph, lane);
}

}  // namespace iwpp

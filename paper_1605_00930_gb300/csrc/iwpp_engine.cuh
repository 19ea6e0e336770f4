// iwpp_engine.cuh — device side of the IWPP reconstruction engine (sm_103a).
//
// Method: grayscale reconstruction by dilation (Sec. 2.1.2, Eq. "recon") by the
// IWPP pattern of Sec. 3 (Algorithm 6): an initialisation phase that finds the
// active elements, then irregular propagation until no element can change.
// Reconstruction by erosion (fill-holes, Sec. 3.3) runs through the same code on
// complemented values: with c(x) = MAXV - x, eps_G(J) v I = c(delta_G(c J) ^ c I),
// and the complement of a u8/u16 value is an XOR with MAXV, applied when a tile
// is loaded into shared memory and undone when it is stored.
//
// GB300 design (not the paper's Xeon Phi / Kepler design):
//   * The image is cut into TH x TW tiles; a tile is the unit of work. A CTA
//     holds one tile plus a one-pixel halo in shared memory, widened to 32-bit
//     words so that propagation can use native shared-memory atomicMax.
//     Tiles move between HBM and shared memory in 16-byte chunks.
//   * Tile-local scanning (Algorithm 7's raster / anti-raster sweeps): each warp
//     sweeps a band of rows; within a row the left-to-right dependency
//     J(x) = min(I(x), max(a(x), J(x-1))) is a composition of clamp functions,
//     which is associative, so it runs as a warp-shuffle scan.
//   * Tile-local irregular propagation (Algorithm 7's queue phase; the in/out
//     queue pair of Algorithm 9 and Sec. 4.1): double-buffered shared-memory
//     wave queues with a per-pixel "queued" bitmap, warp-aggregated pushes (one
//     shared atomicAdd per warp and wave step), shared atomicMax updates with
//     re-enqueue on change, and a per-CTA global overflow queue for waves larger
//     than the shared one.
//   * Cross-tile propagation: a tile only ever writes its own pixels. When a
//     tile's edge pixels can raise a halo pixel, the owning neighbour tile is
//     notified. A per-tile state word (PENDING / ACTIVE / VISITED) guarantees
//     that a tile is queued at most once and processed by one CTA at a time; a
//     tile notified while ACTIVE is re-processed by the same CTA, which keeps
//     its interior in shared memory and reloads only the halo.
//   * A persistent kernel drains the global tile queue (a ticketed ring) until
//     the count of PENDING-or-ACTIVE tiles reaches zero. Every wait is bounded
//     by a %globaltimer watchdog that records IWPP_ERR_TIMEOUT and returns.
// Why any schedule gives the exact result: every update sets J(q) to
// min(J(p), I(q)) <= R(q) and no value is ever lowered, so J stays <= R; the run
// stops only when no pixel can be raised by a neighbour, i.e. at a fixed point
// >= marker, which is R. This is the benign-race argument of Sec. 4.3 made exact.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace iwpp {

// ---- status codes (mirror iwpp_status in include/iwpp.h) ------------------------------
enum : uint32_t {
    kOk = 0, kErrArg = 1, kErrPrecondition = 2, kErrWorkspace = 3, kErrQueueFull = 4,
    kErrTimeout = 5, kErrCuda = 6, kErrInternal = 7
};

// ---- per-tile state bits ------------------------------------------------------------------
enum : uint32_t { ST_PENDING = 1u, ST_ACTIVE = 2u, ST_VISITED = 4u };
constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;
constexpr uint32_t kDone = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Workspace header, at offset 0 of the workspace (256 bytes reserved).
struct WsHeader {
    uint32_t status;            // first device-side error (0 = none)
    uint32_t pending;           // tiles that are PENDING or ACTIVE
    uint32_t pad0[2];
    unsigned long long head;    // tile-queue pop tickets
    unsigned long long tail;    // tile-queue push tickets
    unsigned long long visits;  // tile visits by the persistent kernel
    unsigned long long pops;    // wave-queue entries processed
    unsigned long long seeds;   // wave-queue entries created by a visit's initial scan
};
static_assert(sizeof(WsHeader) <= 256, "header too large");

// One image as the kernels see it.
struct ImageView {
    uint8_t *J;        // marker / result, row-major, pitch W elements
    const uint8_t *I;  // mask
    int H, W;
    int tiles_x, tiles_y;
    uint32_t flip;     // 0 for dilation, MAXV for erosion (complement = XOR)
};

// Everything the kernels of one call share.
struct EngineArgs {
    ImageView img;
    WsHeader *hdr;
    uint32_t *state;    // ntiles words
    uint32_t *queue;    // ntiles slots
    uint16_t *ovf;      // per-CTA overflow queues, 2 * ovcap entries each
    uint32_t ntiles;
    uint32_t qcap;      // shared wave-queue entries per buffer
    uint32_t ovcap;     // global overflow entries per buffer per CTA
    int sweeps;         // sweep pairs in the scan kernel
    int revisit_sweeps; // sweep pairs at a tile's first persistent visit
    long long watchdog_ns;
};

// ---- small device helpers ------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ uint32_t clampu(uint32_t x, uint32_t lo, uint32_t hi) {
    return min(hi, max(lo, x));
}
__device__ __forceinline__ void set_status(WsHeader *h, uint32_t code) {
    atomicCAS(&h->status, 0u, code);
}
__device__ __forceinline__ bool fatal(const WsHeader *h) {
    const uint32_t s = ld_volatile(&h->status);
    return s != 0 && s != kErrPrecondition;
}

// ---- global tile queue (ticketed ring, capacity = number of tiles) -----------------------
// A tile is in the queue at most once (only the IDLE -> PENDING transition pushes),
// so at most `ntiles` entries are ever outstanding. Pushers take a ticket and CAS
// their id into an EMPTY slot; poppers take a ticket and CAS the slot back to EMPTY.
__device__ inline bool push_tile(const EngineArgs &a, uint32_t t) {
    const unsigned long long ticket = atomicAdd(&a.hdr->tail, 1ull);
    uint32_t *slot = a.queue + (ticket % a.ntiles);
    const unsigned long long t0 = globaltimer_ns();
    while (atomicCAS(slot, kEmptySlot, t) != kEmptySlot) {
        if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
            set_status(a.hdr, kErrTimeout);
            return false;
        }
        if (fatal(a.hdr)) return false;
        __nanosleep(32);
    }
    return true;
}

// Tile t has a pixel that a halo pixel can raise: make it PENDING (queue it if idle).
__device__ inline void notify_tile(const EngineArgs &a, uint32_t t) {
    const uint32_t old = atomicOr(a.state + t, ST_PENDING);
    __threadfence();   // order the state change before the queue entry that publishes it
    if ((old & (ST_PENDING | ST_ACTIVE)) == 0) {
        atomicAdd(&a.hdr->pending, 1u);
        push_tile(a, t);
    }
}

__device__ inline uint32_t pop_tile(const EngineArgs &a) {
    const unsigned long long ticket = atomicAdd(&a.hdr->head, 1ull);
    uint32_t *slot = a.queue + (ticket % a.ntiles);
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        const uint32_t v = ld_volatile(slot);
        if (v != kEmptySlot && atomicCAS(slot, v, kEmptySlot) == v) return v;
        if (ld_volatile(&a.hdr->pending) == 0) return kDone;
        if (fatal(a.hdr)) return kDone;
        if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
            set_status(a.hdr, kErrTimeout);
            return kDone;
        }
        __nanosleep(64);
    }
}

// ---- the tile engine -----------------------------------------------------------------------
template <typename T, int CONN, int TH, int TW>
struct Tile {
    static_assert(TW % 32 == 0 && TH % kWarps == 0 && TH >= 8, "tile shape");
    static constexpr int PW = TW + 2;                     // padded row length
    static constexpr int PH = TH + 2;
    static constexpr int NP = PW * PH;                    // padded pixels
    static constexpr int NPIX = TH * TW;                  // owned pixels
    static constexpr int PPL = TW / 32;                   // pixels per lane in a sweep row
    static constexpr int BAND = TH / kWarps;              // rows per warp in a sweep
    static constexpr int NRING = 2 * TW + 2 * (TH - 2);   // owned pixels on the tile edge
    static constexpr int NHALO = 2 * PW + 2 * TH;         // halo pixels
    static constexpr int S = (int)sizeof(T);
    static constexpr int EPC = 16 / S;                    // elements per 16-byte chunk
    static constexpr int LCHUNKS = (PW * S + 15) / 16 + 1;  // chunks per loaded row
    static constexpr int SCHUNKS = (TW * S + 15) / 16 + 1;  // chunks per stored row
    static constexpr int INQ_WORDS = (NP + 31) / 32;
    static constexpr int NDIR = CONN;
    static_assert(NP < 65536, "queue entries are 16-bit padded indices");

    struct Smem {
        uint32_t *J;        // NP: marker/result in the dilation domain
        uint32_t *I;        // NP: mask; 0 on the halo and outside the image (blocks updates)
        uint32_t *haloI;    // NHALO: real mask values of the halo (for notifications)
        uint32_t *ring0;    // NRING: edge values at the start of the visit
        uint32_t *inq;      // INQ_WORDS: "pixel is queued" bitmap
        uint32_t *misc;     // 32 counters / flags
        uint8_t *rowchg;    // TH: row changed in this visit
        uint16_t *q;        // 2 * qcap: wave queues
    };
    // misc word indices
    enum { M_QN = 0 /* 0..2 */, M_NOTIFY = 3 /* 3..11 */, M_FLAG = 12, M_TILE = 13, M_FIRST = 14,
           M_REDO = 15, M_SEEDS = 16, M_PRECOND = 17 };

    static size_t smem_bytes(uint32_t qcap) {
        return (size_t)(2 * NP + NHALO + NRING + INQ_WORDS + 32) * 4 + (size_t)((TH + 3) / 4) * 4 +
               (size_t)qcap * 2 * 2;
    }

    static __device__ Smem carve(uint8_t *base) {
        Smem s;
        uint32_t *w = reinterpret_cast<uint32_t *>(base);
        s.J = w; w += NP;
        s.I = w; w += NP;
        s.haloI = w; w += NHALO;
        s.ring0 = w; w += NRING;
        s.inq = w; w += INQ_WORDS;
        s.misc = w; w += 32;
        s.rowchg = reinterpret_cast<uint8_t *>(w); w += (TH + 3) / 4;
        s.q = reinterpret_cast<uint16_t *>(w);
        return s;
    }

    // Ring position i in [0, NRING) -> padded (row, col) of an owned edge pixel.
    static __device__ __forceinline__ void ring_rc(int i, int &r, int &c) {
        if (i < TW) { r = 1; c = 1 + i; }
        else if (i < 2 * TW) { r = TH; c = 1 + (i - TW); }
        else if (i < 2 * TW + (TH - 2)) { r = 2 + (i - 2 * TW); c = 1; }
        else { r = 2 + (i - 2 * TW - (TH - 2)); c = TW; }
    }
    // Halo pixel (padded r, c on the outer ring) -> haloI index.
    static __device__ __forceinline__ int halo_index(int r, int c) {
        if (r == 0) return c;
        if (r == PH - 1) return PW + c;
        if (c == 0) return 2 * PW + (r - 1);
        return 2 * PW + TH + (r - 1);
    }
    static __device__ __forceinline__ bool is_halo(int r, int c) {
        return r == 0 || r == PH - 1 || c == 0 || c == PW - 1;
    }
    static __device__ __forceinline__ int dir_dy(int d) {
        if (CONN == 8) return d < 3 ? -1 : (d < 5 ? 0 : 1);
        return d == 0 ? -1 : (d == 3 ? 1 : 0);
    }
    static __device__ __forceinline__ int dir_dx(int d) {
        if (CONN == 8) { const int t[8] = {-1, 0, 1, -1, 1, -1, 0, 1}; return t[d]; }
        const int t[4] = {0, -1, 1, 0};
        return t[d];
    }
    static __device__ __forceinline__ int nb_off(int d) { return dir_dy(d) * PW + dir_dx(d); }
    static __device__ __forceinline__ uint32_t to_dom(uint32_t v, uint32_t flip) { return v ^ flip; }

    // ---- HBM <-> shared memory ------------------------------------------------------------
    // Load padded rows [r0, r0 + rows) of tile (ty, tx): J and/or I, in 16-byte chunks.
    // Elements outside the image are left alone (zero_outside covers them). Halo mask
    // values go to haloI while I keeps 0 on the halo. use_cg: read J through L2 only
    // (the persistent kernel reads pixels that other CTAs write concurrently).
    static __device__ void load_rows(const ImageView &im, const Smem &s, int ty, int tx, int r0,
                                     int rows, bool loadJ, bool loadI, bool use_cg) {
        const int y0 = ty * TH, x0 = tx * TW;
        const size_t total = (size_t)im.H * (size_t)im.W;
        const int nitems = rows * LCHUNKS;
        for (int it = threadIdx.x; it < nitems; it += kThreads) {
            const int r = r0 + it / LCHUNKS, k = it % LCHUNKS;
            const int gy = y0 + r - 1;
            if (gy < 0 || gy >= im.H) continue;
            const int xa = max(0, x0 - 1), xb = min(im.W, x0 + TW + 1);
            const size_t rowbase = (size_t)gy * im.W;
            const size_t e_lo = rowbase + xa, e_hi = rowbase + xb;
            const size_t chunk = e_lo / EPC + k;
            if (chunk * EPC >= e_hi) continue;
            const size_t e0 = chunk * EPC;
            union { uint4 u; T e[EPC]; } vj, vi;
            if (e0 + EPC <= total) {
                if (loadJ) vj.u = use_cg ? __ldcg(reinterpret_cast<const uint4 *>(im.J) + chunk)
                                         : reinterpret_cast<const uint4 *>(im.J)[chunk];
                if (loadI) vi.u = __ldg(reinterpret_cast<const uint4 *>(im.I) + chunk);
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    if (e0 + j < total) {
                        if (loadJ) vj.e[j] = use_cg ? __ldcg(reinterpret_cast<const T *>(im.J) + e0 + j)
                                                    : reinterpret_cast<const T *>(im.J)[e0 + j];
                        if (loadI) vi.e[j] = reinterpret_cast<const T *>(im.I)[e0 + j];
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < EPC; j++) {
                const size_t e = e0 + j;
                if (e < e_lo || e >= e_hi) continue;
                const int c = (int)(e - rowbase) - x0 + 1;
                const int p = r * PW + c;
                if (loadJ) s.J[p] = to_dom(vj.e[j], im.flip);
                if (loadI) {
                    const uint32_t iv = to_dom(vi.e[j], im.flip);
                    if (is_halo(r, c)) { s.haloI[halo_index(r, c)] = iv; s.I[p] = 0; }
                    else s.I[p] = iv;
                }
            }
        }
    }

    // Zero J and/or I (and haloI) where the padded tile sticks out of the image.
    static __device__ void zero_outside(const ImageView &im, const Smem &s, int ty, int tx,
                                        bool doJ, bool doI) {
        const int y0 = ty * TH, x0 = tx * TW;
        if (y0 > 0 && x0 > 0 && y0 + TH < im.H && x0 + TW < im.W) return;
        for (int p = threadIdx.x; p < NP; p += kThreads) {
            const int r = p / PW, c = p % PW;
            const int gy = y0 + r - 1, gx = x0 + c - 1;
            if (gy < 0 || gy >= im.H || gx < 0 || gx >= im.W) {
                if (doJ) s.J[p] = 0;
                if (doI) {
                    s.I[p] = 0;
                    if (is_halo(r, c)) s.haloI[halo_index(r, c)] = 0;
                }
            }
        }
    }

    // Reload the halo ring of J (the interior stays as this CTA left it).
    static __device__ void load_halo_J(const ImageView &im, const Smem &s, int ty, int tx) {
        const int y0 = ty * TH, x0 = tx * TW;
        for (int i = threadIdx.x; i < NHALO; i += kThreads) {
            int r, c;
            if (i < PW) { r = 0; c = i; }
            else if (i < 2 * PW) { r = PH - 1; c = i - PW; }
            else if (i < 2 * PW + TH) { r = 1 + (i - 2 * PW); c = 0; }
            else { r = 1 + (i - 2 * PW - TH); c = PW - 1; }
            const int gy = y0 + r - 1, gx = x0 + c - 1;
            uint32_t v = 0;
            if (gy >= 0 && gy < im.H && gx >= 0 && gx < im.W)
                v = to_dom(__ldcg(reinterpret_cast<const T *>(im.J) + (size_t)gy * im.W + gx), im.flip);
            s.J[r * PW + c] = v;
        }
    }

    // Store the owned rows flagged in rowchg, in 16-byte chunks where a chunk lies
    // entirely inside the tile's row segment, element by element otherwise.
    static __device__ void store_rows(const ImageView &im, const Smem &s, int ty, int tx, bool use_cg) {
        const int y0 = ty * TH, x0 = tx * TW;
        const size_t total = (size_t)im.H * (size_t)im.W;
        const int nitems = TH * SCHUNKS;
        for (int it = threadIdx.x; it < nitems; it += kThreads) {
            const int rr = it / SCHUNKS, k = it % SCHUNKS;
            if (!s.rowchg[rr]) continue;
            const int gy = y0 + rr;
            if (gy >= im.H) continue;
            const size_t rowbase = (size_t)gy * im.W;
            const size_t e_lo = rowbase + x0, e_hi = rowbase + min(im.W, x0 + TW);
            const size_t chunk = e_lo / EPC + k;
            if (chunk * EPC >= e_hi) continue;
            const size_t e0 = chunk * EPC;
            const uint32_t *srow = s.J + (rr + 1) * PW + 1 - x0;   // srow[x] = padded pixel at column x
            if (e0 >= e_lo && e0 + EPC <= e_hi && e0 + EPC <= total) {
                union { uint4 u; T e[EPC]; } v;
#pragma unroll
                for (int j = 0; j < EPC; j++) v.e[j] = (T)to_dom(srow[(int)(e0 + j - rowbase)], im.flip);
                if (use_cg) __stcg(reinterpret_cast<uint4 *>(im.J) + chunk, v.u);
                else reinterpret_cast<uint4 *>(im.J)[chunk] = v.u;
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    const size_t e = e0 + j;
                    if (e < e_lo || e >= e_hi) continue;
                    const T v = (T)to_dom(srow[(int)(e - rowbase)], im.flip);
                    if (use_cg) __stcg(reinterpret_cast<T *>(im.J) + e, v);
                    else reinterpret_cast<T *>(im.J)[e] = v;
                }
            }
        }
    }

    // ---- tile-local sweeps (Algorithm 7, scanning phase) -------------------------------------
    // The clamp f(x) = min(hi, max(lo, x)) is packed as (hi << 16) | lo; values are < 2^16.
    // Composition g o f of clamps [lf, hf] then [lg, hg] is [clamp(lf, lg, hg), clamp(hf, lg, hg)].

    // Raster: rows top to bottom, J(p) <- max{J(q): q in N+(p) U {p}} ^ I(p) with
    // N+ = {N, W} (4-conn) or {NW, N, NE, W} (8-conn); each warp owns BAND rows.
    static __device__ void sweep_raster(const Smem &s) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int b = 0; b < BAND; b++) {
            const int r = 1 + warp * BAND + b;
            uint32_t a[PPL], iv[PPL], old[PPL];
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                const int p = r * PW + 1 + lane * PPL + k;
                old[k] = s.J[p];
                uint32_t v = max(old[k], s.J[p - PW]);
                if (CONN == 8) v = max(v, max(s.J[p - PW - 1], s.J[p - PW + 1]));
                a[k] = v;
                iv[k] = s.I[p];
            }
            uint32_t lo = min(a[0], iv[0]), hi = iv[0];   // F_lane = f_{PPL-1} o ... o f_0
#pragma unroll
            for (int k = 1; k < PPL; k++) {
                const uint32_t l2 = min(a[k], iv[k]), h2 = iv[k];
                const uint32_t nl = clampu(lo, l2, h2), nh = clampu(hi, l2, h2);
                lo = nl; hi = nh;
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {            // inclusive scan over lanes 0..lane
                const uint32_t o = __shfl_up_sync(0xffffffffu, (hi << 16) | lo, d);
                if (lane >= d) {
                    const uint32_t nl = clampu(o & 0xffffu, lo, hi), nh = clampu(o >> 16, lo, hi);
                    lo = nl; hi = nh;
                }
            }
            const uint32_t ex = __shfl_up_sync(0xffffffffu, (hi << 16) | lo, 1);
            uint32_t x = s.J[r * PW];                     // left halo
            if (lane > 0) x = clampu(x, ex & 0xffffu, ex >> 16);
            bool ch = false;
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                x = clampu(x, min(a[k], iv[k]), iv[k]);
                s.J[r * PW + 1 + lane * PPL + k] = x;
                ch |= (x != old[k]);
            }
            if (__any_sync(0xffffffffu, ch) && lane == 0) s.rowchg[r - 1] = 1;
            __syncwarp();
        }
    }

    // Anti-raster: rows bottom to top, right to left, with N- = {S, E} / {SE, S, SW, E}.
    static __device__ void sweep_antiraster(const Smem &s) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int b = BAND - 1; b >= 0; b--) {
            const int r = 1 + warp * BAND + b;
            uint32_t a[PPL], iv[PPL], old[PPL];
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                const int p = r * PW + 1 + lane * PPL + k;
                old[k] = s.J[p];
                uint32_t v = max(old[k], s.J[p + PW]);
                if (CONN == 8) v = max(v, max(s.J[p + PW - 1], s.J[p + PW + 1]));
                a[k] = v;
                iv[k] = s.I[p];
            }
            uint32_t lo = min(a[PPL - 1], iv[PPL - 1]), hi = iv[PPL - 1];  // f_0 o ... o f_{PPL-1}
#pragma unroll
            for (int k = PPL - 2; k >= 0; k--) {
                const uint32_t l2 = min(a[k], iv[k]), h2 = iv[k];
                const uint32_t nl = clampu(lo, l2, h2), nh = clampu(hi, l2, h2);
                lo = nl; hi = nh;
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {            // inclusive scan over lanes lane..31
                const uint32_t o = __shfl_down_sync(0xffffffffu, (hi << 16) | lo, d);
                if (lane + d < 32) {
                    const uint32_t nl = clampu(o & 0xffffu, lo, hi), nh = clampu(o >> 16, lo, hi);
                    lo = nl; hi = nh;
                }
            }
            const uint32_t ex = __shfl_down_sync(0xffffffffu, (hi << 16) | lo, 1);
            uint32_t x = s.J[r * PW + PW - 1];            // right halo
            if (lane < 31) x = clampu(x, ex & 0xffffu, ex >> 16);
            bool ch = false;
#pragma unroll
            for (int k = PPL - 1; k >= 0; k--) {
                x = clampu(x, min(a[k], iv[k]), iv[k]);
                s.J[r * PW + 1 + lane * PPL + k] = x;
                ch |= (x != old[k]);
            }
            if (__any_sync(0xffffffffu, ch) && lane == 0) s.rowchg[r - 1] = 1;
            __syncwarp();
        }
    }

    // ---- wave queues ------------------------------------------------------------------------
    // Warp-aggregated push of up to K candidates per lane into wave buffer `buf`
    // (count word misc[M_QN + cnt]): one shared atomicAdd per warp.
    template <int K>
    static __device__ __forceinline__ void push_warp(const Smem &s, const EngineArgs &a,
                                                     uint16_t *ovf, int buf, int cnt,
                                                     const bool (&w)[K], const int (&q)[K]) {
        const int lane = threadIdx.x & 31;
        uint32_t bal[K];
        uint32_t total = 0;
#pragma unroll
        for (int d = 0; d < K; d++) { bal[d] = __ballot_sync(0xffffffffu, w[d]); total += __popc(bal[d]); }
        if (total == 0) return;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&s.misc[M_QN + cnt], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int d = 0; d < K; d++) {
            if (w[d]) {
                const uint32_t pos = base + __popc(bal[d] & lt);
                if (pos < a.qcap) s.q[buf * a.qcap + pos] = (uint16_t)q[d];
                else if (pos - a.qcap < a.ovcap) ovf[buf * a.ovcap + (pos - a.qcap)] = (uint16_t)q[d];
                else set_status(a.hdr, kErrQueueFull);
            }
            base += __popc(bal[d]);
        }
    }

    // Receiver test at one owned pixel p: raise it to min(I(p), max of its
    // neighbours) if that is larger (one Jacobi step of Eq. "recon"), and queue it.
    static __device__ __forceinline__ bool seed_pixel(const Smem &s, int p) {
        uint32_t m = 0;
#pragma unroll
        for (int d = 0; d < NDIR; d++) m = max(m, s.J[p + nb_off(d)]);
        const uint32_t nv = min(m, s.I[p]);
        if (nv > s.J[p]) {
            s.J[p] = nv;
            s.rowchg[p / PW - 1] = 1;
            return true;
        }
        return false;
    }

    // Initial wave of a visit. full: every owned pixel is tested (first visit);
    // otherwise only the edge ring, since the interior was at a local fixed point
    // when this CTA or an earlier one last stored the tile and only the halo changed.
    static __device__ void seed_wave(const Smem &s, const EngineArgs &a, uint16_t *ovf, bool full) {
        const int n = full ? NPIX : NRING;
        const int nround = (n + kThreads - 1) / kThreads * kThreads;
        for (int i = threadIdx.x; i < nround; i += kThreads) {
            bool w[1] = {false};
            int q[1] = {0};
            if (i < n) {
                int r, c;
                if (full) { r = i / TW + 1; c = i % TW + 1; }
                else ring_rc(i, r, c);
                const int p = r * PW + c;
                if (seed_pixel(s, p)) {
                    atomicOr(&s.inq[p >> 5], 1u << (p & 31));
                    w[0] = true;
                    q[0] = p;
                }
            }
            push_warp<1>(s, a, ovf, 0, 0, w, q);
        }
    }

    // Drain the wave queues to a local fixed point. Wave k reads buffer k&1 with count
    // misc[M_QN + k%3], pushes into buffer (k+1)&1 / count (k+1)%3, and zeroes count
    // (k+2)%3, whose readers all passed the barrier that opens wave k.
    static __device__ uint32_t run_waves(const Smem &s, const EngineArgs &a, uint16_t *ovf,
                                         uint32_t &seeds) {
        uint32_t pops = 0;
        seeds = 0;
        volatile uint32_t *vJ = s.J;
        for (int k = 0;; k++) {
            const int cb = k & 1, nb = cb ^ 1;
            const int cc = k % 3, nc = (k + 1) % 3, zc = (k + 2) % 3;
            __syncthreads();
            uint32_t n = s.misc[M_QN + cc];
            if (n == 0) break;
            if (n > a.qcap + a.ovcap) n = a.qcap + a.ovcap;   // cannot happen: entries are distinct pixels
            if (threadIdx.x == 0) s.misc[M_QN + zc] = 0;
            if (k == 0) seeds = n;
            pops += n;
            const uint32_t nround = (n + kThreads - 1) / kThreads * kThreads;
            for (uint32_t i = threadIdx.x; i < nround; i += kThreads) {
                const bool valid = i < n;
                int p = 0;
                if (valid) {
                    p = (i < a.qcap) ? s.q[cb * a.qcap + i] : ovf[cb * a.ovcap + (i - a.qcap)];
                    atomicAnd(&s.inq[p >> 5], ~(1u << (p & 31)));
                }
                __threadfence_block();
                const uint32_t v = valid ? vJ[p] : 0u;
                bool w[NDIR];
                int q[NDIR];
#pragma unroll
                for (int d = 0; d < NDIR; d++) {
                    w[d] = false;
                    q[d] = p + nb_off(d);
                    if (valid) {
                        const uint32_t nv = min(v, s.I[q[d]]);
                        if (vJ[q[d]] < nv) {
                            const uint32_t old = atomicMax(&s.J[q[d]], nv);
                            if (old < nv) {
                                s.rowchg[q[d] / PW - 1] = 1;
                                __threadfence_block();
                                const uint32_t bit = 1u << (q[d] & 31);
                                w[d] = (atomicOr(&s.inq[q[d] >> 5], bit) & bit) == 0;
                            }
                        }
                    }
                }
                push_warp<NDIR>(s, a, ovf, nb, nc, w, q);
            }
        }
        return pops;
    }

    // ---- end of a visit -----------------------------------------------------------------------
    // For every edge pixel raised in this visit, test its halo neighbours with the
    // propagation condition J(q) < min(J(p), I(q)); flag the neighbour tiles to notify.
    static __device__ void notify_scan(const Smem &s) {
        for (int i = threadIdx.x; i < NRING; i += kThreads) {
            int r, c;
            ring_rc(i, r, c);
            const int p = r * PW + c;
            const uint32_t v = s.J[p];
            if (v == s.ring0[i]) continue;
#pragma unroll
            for (int d = 0; d < NDIR; d++) {
                const int qr = r + dir_dy(d), qc = c + dir_dx(d);
                if (!is_halo(qr, qc)) continue;
                const uint32_t hq = s.J[qr * PW + qc];
                if (hq < min(v, s.haloI[halo_index(qr, qc)])) {
                    const int dy = qr == 0 ? -1 : (qr == PH - 1 ? 1 : 0);
                    const int dx = qc == 0 ? -1 : (qc == PW - 1 ? 1 : 0);
                    s.misc[M_NOTIFY + (dy + 1) * 3 + (dx + 1)] = 1;
                }
            }
        }
    }

    static __device__ void save_ring(const Smem &s) {
        for (int i = threadIdx.x; i < NRING; i += kThreads) {
            int r, c;
            ring_rc(i, r, c);
            s.ring0[i] = s.J[r * PW + c];
        }
    }

    // Called by thread 0 after a fence and a barrier: notify flagged neighbours.
    static __device__ void send_notifications(const Smem &s, const EngineArgs &a, int ty, int tx) {
        for (int j = 0; j < 9; j++) {
            if (j == 4 || !s.misc[M_NOTIFY + j]) continue;
            const int ny = ty + j / 3 - 1, nx = tx + j % 3 - 1;
            if (ny < 0 || nx < 0 || ny >= a.img.tiles_y || nx >= a.img.tiles_x) continue;
            notify_tile(a, (uint32_t)(ny * a.img.tiles_x + nx));
        }
    }

    static __device__ void clear_visit_flags(const Smem &s, bool clear_inq) {
        for (int i = threadIdx.x; i < TH; i += kThreads) s.rowchg[i] = 0;
        if (threadIdx.x < 9) s.misc[M_NOTIFY + threadIdx.x] = 0;
        if (threadIdx.x < 3) s.misc[M_QN + threadIdx.x] = 0;
        if (threadIdx.x == 0) { s.misc[M_FLAG] = 0; s.misc[M_PRECOND] = 0; }
        if (clear_inq)
            for (int i = threadIdx.x; i < INQ_WORDS; i += kThreads) s.inq[i] = 0;
    }
};

// ---- kernel 1: tile-parallel scan -------------------------------------------------------------
// Per tile: precondition check, `sweeps` raster/anti-raster pairs in shared memory,
// store, then frontier initialisation: queue the tile if one of its pixels can still be
// raised, and its neighbours if a raised edge pixel can raise one of theirs.
template <typename T, int CONN, int TH, int TW>
__global__ void __launch_bounds__(kThreads) scan_kernel(EngineArgs a) {
    using TL = Tile<T, CONN, TH, TW>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const typename TL::Smem s = TL::carve(smem_raw);
    for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int ty = t / a.img.tiles_x, tx = t % a.img.tiles_x;
        TL::clear_visit_flags(s, false);
        TL::zero_outside(a.img, s, ty, tx, true, true);
        TL::load_rows(a.img, s, ty, tx, 0, TL::PH, true, true, false);
        __syncthreads();
        bool bad = false;
        for (int i = threadIdx.x; i < TL::NPIX; i += kThreads) {
            const int p = (i / TW + 1) * TL::PW + (i % TW + 1);
            bad |= s.J[p] > s.I[p];
        }
        if (bad) s.misc[TL::M_PRECOND] = 1;
        TL::save_ring(s);
        __syncthreads();
        for (int k = 0; k < a.sweeps; k++) {
            TL::sweep_raster(s);
            __syncthreads();
            TL::sweep_antiraster(s);
            __syncthreads();
        }
        if (a.sweeps > 0) TL::store_rows(a.img, s, ty, tx, false);
        bool active = false;
        for (int i = threadIdx.x; i < TL::NPIX; i += kThreads) {
            const int p = (i / TW + 1) * TL::PW + (i % TW + 1);
            uint32_t m = 0;
#pragma unroll
            for (int d = 0; d < TL::NDIR; d++) m = max(m, s.J[p + TL::nb_off(d)]);
            active |= min(m, s.I[p]) > s.J[p];
        }
        if (active) s.misc[TL::M_FLAG] = 1;
        TL::notify_scan(s);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s.misc[TL::M_PRECOND]) set_status(a.hdr, kErrPrecondition);
            if (s.misc[TL::M_FLAG]) notify_tile(a, t);
            TL::send_notifications(s, a, ty, tx);
        }
        __syncthreads();
    }
}

// ---- kernel 2: persistent drain -------------------------------------------------------------
template <typename T, int CONN, int TH, int TW>
__global__ void __launch_bounds__(kThreads) drain_kernel(EngineArgs a) {
    using TL = Tile<T, CONN, TH, TW>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const typename TL::Smem s = TL::carve(smem_raw);
    uint16_t *ovf = a.ovf + (size_t)blockIdx.x * 2 * a.ovcap;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = pop_tile(a);
            s.misc[TL::M_TILE] = t;
            if (t != kDone) {
                const uint32_t old = atomicAdd(a.state + t, 1u);   // PENDING -> ACTIVE
                const bool first = (old & ST_VISITED) == 0;
                if (first) atomicOr(a.state + t, ST_VISITED);
                s.misc[TL::M_FIRST] = first;
                __threadfence();
            }
        }
        __syncthreads();
        const uint32_t t = s.misc[TL::M_TILE];
        if (t == kDone) break;
        const bool first = s.misc[TL::M_FIRST] != 0;
        const int ty = t / a.img.tiles_x, tx = t % a.img.tiles_x;
        TL::clear_visit_flags(s, true);
        TL::zero_outside(a.img, s, ty, tx, true, true);
        TL::load_rows(a.img, s, ty, tx, 0, TL::PH, true, true, true);
        __syncthreads();
        bool full = first;
        for (;;) {
            TL::save_ring(s);
            __syncthreads();
            if (full) {
                for (int k = 0; k < a.revisit_sweeps; k++) {
                    TL::sweep_raster(s);
                    __syncthreads();
                    TL::sweep_antiraster(s);
                    __syncthreads();
                }
            }
            TL::seed_wave(s, a, ovf, full);
            uint32_t seeds;
            const uint32_t pops = TL::run_waves(s, a, ovf, seeds);
            TL::store_rows(a.img, s, ty, tx, true);
            TL::notify_scan(s);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                TL::send_notifications(s, a, ty, tx);
                atomicAdd(&a.hdr->visits, 1ull);
                atomicAdd(&a.hdr->pops, (unsigned long long)pops);
                atomicAdd(&a.hdr->seeds, (unsigned long long)seeds);
                const uint32_t busy = ST_ACTIVE | ST_VISITED;
                const uint32_t r = atomicCAS(a.state + t, busy, ST_VISITED);
                uint32_t redo = 0;
                if (r == busy) {
                    __threadfence();
                    atomicSub(&a.hdr->pending, 1u);
                } else {
                    atomicAnd(a.state + t, ~ST_PENDING);   // notified while ACTIVE: go again
                    redo = 1;
                }
                __threadfence();
                s.misc[TL::M_REDO] = redo && !fatal(a.hdr);   // one decision for the whole CTA
            }
            __syncthreads();
            if (!s.misc[TL::M_REDO]) break;
            // Re-process: the interior in shared memory is what this CTA stored; only the
            // halo can have changed since.
            TL::clear_visit_flags(s, false);
            TL::load_halo_J(a.img, s, ty, tx);
            full = false;
            __syncthreads();
        }
    }
}

}  // namespace iwpp

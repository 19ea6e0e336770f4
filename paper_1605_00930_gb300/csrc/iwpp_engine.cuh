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
//   * The image is cut into TH x TW tiles; a tile is the unit of work. Each WARP
//     is an independent worker that holds one tile plus a one-pixel halo in its
//     own slice of shared memory (J widened to 32-bit words so that propagation
//     can use native shared-memory atomicMax; I as 16-bit words). A serial wave
//     chain inside a tile then costs warp-level synchronisation only, and an SM
//     keeps a dozen or more tiles in flight to hide the latency of each chain.
//     Tiles move between HBM and shared memory in 16-byte chunks.
//   * Tile-local scanning (Algorithm 7's raster / anti-raster sweeps): rows in
//     order; within a row the left-to-right dependency
//     J(x) = min(I(x), max(a(x), J(x-1))) is a composition of clamp functions,
//     which is associative, so it runs as a warp-shuffle scan.
//   * Tile-local irregular propagation (Algorithm 7's queue phase; the in/out
//     queue pair of Algorithm 9 and Sec. 4.1): double-buffered shared-memory
//     wave queues with a per-pixel "queued" bitmap, warp-aggregated pushes (one
//     ballot per direction and a single count update per warp and wave step),
//     shared atomicMax updates with re-enqueue on change, and a per-warp global
//     overflow queue for waves larger than the shared one.
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

#include "iwpp_spread.h"

// Tuning switches (compile-time; the defaults are the measured best).
#ifndef IWPP_DRAIN_MINB
#define IWPP_DRAIN_MINB 4     // persistent-kernel CTAs per SM the register budget targets
#endif
#ifndef IWPP_PHASE_TIMING
#define IWPP_PHASE_TIMING 0   // accumulate per-phase SM cycles of the persistent kernel
#endif
#ifndef IWPP_BACKOFF_MAX
#define IWPP_BACKOFF_MAX 512  // ns, longest sleep between polls of an empty queue slot
#endif
#ifndef IWPP_POP_EXCH
#define IWPP_POP_EXCH 1       // 1: a pop takes its slot's entry with one exchange (no load + CAS pair)
#endif
#ifndef IWPP_FENCE_LIGHT
#define IWPP_FENCE_LIGHT 1    // 1: acquire / release fences (fence.acq_rel.gpu) on the tile protocol
#endif

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
constexpr int kWarpsPerCta = 4;                 // independent tile workers per CTA
constexpr int kThreads = 32 * kWarpsPerCta;

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
    unsigned long long waves;   // wave steps run by the persistent kernel
    unsigned long long idle_ns; // summed over warps: time spent waiting for a tile
    unsigned long long busy_ns; // summed over warps: time spent processing tiles
    unsigned int max_gen;       // longest chain of tile visits that notified one another
    unsigned int pad1;
    unsigned long long phase_cycles[8];  // IWPP_PHASE_TIMING builds only
};
static_assert(sizeof(WsHeader) <= 256, "header too large");

// One image as the kernels see it.
struct ImageView {
    uint8_t *J;          // marker / result, row-major, pitch W elements
    const uint8_t *I;    // mask
    int H, W;
    int tiles_x, tiles_y;
    uint32_t flip;       // 0 for dilation, MAXV for erosion (complement = XOR)
    uint32_t tile_base;  // global id of the image's first tile
    uint32_t kind;       // bit 0: u16 pixels; bit 1: 8-connectivity
    uint32_t pad;
};

// Counters of one value level of the tile queue (value-ordered mode).
struct LevelCtr {
    unsigned long long head, tail;   // pop / push tickets
    int avail;                       // entries published and not yet claimed
    uint32_t pad[3];
};
constexpr int kMaxLevels = 16;

// Everything the kernels of one call share. A single-image call uses img0; a batch
// call reads its images from the device table `imgs` (sorted by tile_base).
struct EngineArgs {
    ImageView img0;
    const ImageView *imgs;       // batch table (nullptr for a single image)
    int nimg;
    WsHeader *hdr;
    uint32_t *state;             // ntiles words
    uint32_t *queue;             // ntiles slots
    uint16_t *ovf;               // per-warp overflow queues, 2 * ovcap entries each
    uint32_t ntiles;
    uint32_t qcap;               // shared wave-queue entries per buffer
    uint32_t ovcap;              // global overflow entries per buffer per warp
    int sweeps;                  // sweep pairs in the scan kernel (when tile_sweeps is null)
    int revisit_sweeps;          // sweep pairs at a tile's first persistent visit
    const uint8_t *tile_sweeps;  // optional per-tile sweep pairs for the scan kernel
    const uint32_t *order;       // optional order in which the initial frontier is queued
    uint32_t spread;             // without an order: position i queues tile (i * spread) mod ntiles (0: i)
    uint32_t *tile_work;         // optional per-tile counters: [t] pops, [ntiles + t] SM cycles
    int defer_push;              // scan kernel marks tiles PENDING; the compact kernel queues them
    long long watchdog_ns;
    uint32_t nlevels;            // 1: one FIFO ring; >1: one ring per value level (queue + L * ntiles)
    LevelCtr *lvl;               // nlevels counters (value-ordered mode)
    const uint32_t *tile_img;    // batch: index of each tile's image in imgs (else nullptr)
    float *feats;                // learned batches: per-tile features out of the scan (64 x 64 tiles)
    int sweep_only;              // scan: skip tiles whose sweep count is 0 (a second, sweeps-only pass)
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
// Fence between a tile's stores and the notifications that publish them (release), and
// between taking a tile and loading it (acquire).
__device__ __forceinline__ void fence_protocol() {
#if IWPP_FENCE_LIGHT
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
#else
    __threadfence();
#endif
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

// ---- value-ordered tile queue (Sec. 4.4's heap-based propagation, at tile granularity) ---
// One ticketed ring per value level. A push publishes its entry and then counts it in
// `avail`; a pop first claims one published entry of the highest level that has one (an
// atomic decrement that it undoes if it lost the race for the last entry), then takes a
// ticket: the push holding that ticket has published or is about to, so the wait is short
// and a popper never waits on an empty level. A tile is queued at most once, at the level
// of the notification that made it PENDING.
__device__ inline bool push_tile_level(const EngineArgs &a, uint32_t t, uint32_t level) {
    LevelCtr *c = a.lvl + level;
    const unsigned long long ticket = atomicAdd(&c->tail, 1ull);
    uint32_t *slot = a.queue + (size_t)level * a.ntiles + (ticket % a.ntiles);
    const unsigned long long t0 = globaltimer_ns();
    while (atomicCAS(slot, kEmptySlot, t) != kEmptySlot) {
        if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
            set_status(a.hdr, kErrTimeout);
            return false;
        }
        if (fatal(a.hdr)) return false;
        __nanosleep(32);
    }
    atomicAdd(&c->avail, 1);
    return true;
}

__device__ inline uint32_t pop_tile_level(const EngineArgs &a) {
    const unsigned long long t0 = globaltimer_ns();
    unsigned int backoff = 32;
    for (;;) {
        int av[kMaxLevels];
#pragma unroll
        for (int l = 0; l < kMaxLevels; l++)
            av[l] = l < (int)a.nlevels ? *reinterpret_cast<const volatile int *>(&a.lvl[l].avail) : 0;
        int best = -1;
#pragma unroll
        for (int l = 0; l < kMaxLevels; l++)
            if (av[l] > 0) best = l;
        if (best >= 0) {
            LevelCtr *c = a.lvl + best;
            if (atomicSub(&c->avail, 1) > 0) {
                const unsigned long long ticket = atomicAdd(&c->head, 1ull);
                uint32_t *slot = a.queue + (size_t)best * a.ntiles + (ticket % a.ntiles);
                for (;;) {
                    const uint32_t v = ld_volatile(slot);
                    if (v != kEmptySlot && atomicCAS(slot, v, kEmptySlot) == v) return v;
                    if (fatal(a.hdr)) return kDone;
                    if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
                        set_status(a.hdr, kErrTimeout);
                        return kDone;
                    }
                    __nanosleep(32);
                }
            }
            atomicAdd(&c->avail, 1);   // lost the race for the level's last entry
            continue;
        }
        if (ld_volatile(&a.hdr->pending) == 0) return kDone;
        if (fatal(a.hdr)) return kDone;
        if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
            set_status(a.hdr, kErrTimeout);
            return kDone;
        }
        __nanosleep(backoff);
        if (backoff < IWPP_BACKOFF_MAX) backoff <<= 1;
    }
}

// Queue level of a raise to value v (dilation domain) of an image.
__device__ __forceinline__ uint32_t level_of(const EngineArgs &a, const ImageView &im, uint32_t v) {
    if (a.nlevels <= 1) return 0;
    return min((v * a.nlevels) >> ((im.kind & 1u) ? 16 : 8), a.nlevels - 1);
}

// Tile t has a pixel that a halo pixel can raise: make it PENDING (queue it if idle).
// The queue entry is written only after the state change has returned (a control
// dependency on its old value), so a popper always finds the tile PENDING.
__device__ inline void notify_tile(const EngineArgs &a, uint32_t t, uint32_t level = 0) {
    const uint32_t old = atomicOr(a.state + t, ST_PENDING);
    if ((old & (ST_PENDING | ST_ACTIVE)) == 0) {
        atomicAdd(&a.hdr->pending, 1u);
        if (a.nlevels > 1) push_tile_level(a, t, level);
        else push_tile(a, t);
    }
}

// One attempt to take the entry of pop ticket `ticket` (kEmptySlot: not pushed yet).
__device__ __forceinline__ uint32_t try_slot(const EngineArgs &a, unsigned long long ticket) {
    uint32_t *slot = a.queue + (ticket % a.ntiles);
#if IWPP_POP_EXCH
    // an exchange on a slot whose entry has not arrived writes EMPTY over EMPTY: harmless
    return atomicExch(slot, kEmptySlot);
#else
    const uint32_t v = ld_volatile(slot);
    if (v != kEmptySlot && atomicCAS(slot, v, kEmptySlot) == v) return v;
    return kEmptySlot;
#endif
}

// Wait for the entry of pop ticket `ticket`; kDone when the run is over (no tile pending
// or ACTIVE anywhere, a fatal error, or the watchdog).
__device__ inline uint32_t wait_slot(const EngineArgs &a, unsigned long long ticket) {
    const unsigned long long t0 = globaltimer_ns();
    unsigned int backoff = 32;
    for (;;) {
        const uint32_t v = try_slot(a, ticket);
        if (v != kEmptySlot) return v;
        if (ld_volatile(&a.hdr->pending) == 0) return kDone;
        if (fatal(a.hdr)) return kDone;
        if (globaltimer_ns() - t0 > (unsigned long long)a.watchdog_ns) {
            set_status(a.hdr, kErrTimeout);
            return kDone;
        }
        __nanosleep(backoff);
        if (backoff < IWPP_BACKOFF_MAX) backoff <<= 1;
    }
}

__device__ inline uint32_t pop_tile(const EngineArgs &a) {
    if (a.nlevels > 1) return pop_tile_level(a);
    return wait_slot(a, atomicAdd(&a.hdr->head, 1ull));
}

// ---- the tile engine (one warp per tile) ------------------------------------------------------
// Shared-memory words of J hold (value << 1) | queued. A pop is one atomicAnd that clears
// the queued flag and returns the newest value; a raise is one atomicMax with the flag
// set, whose old word says whether the pixel must be queued (flag was clear). So a raise
// that lands after a pop re-queues the pixel, and none is lost, without fences. Halo
// words keep the flag set: the tile may raise its copies of halo pixels (that is how it
// finds improvements to send to the neighbours) but never queues them.
template <typename T, int CONN, int TH, int TW>
struct Tile {
    static_assert(TW % 32 == 0 && TH >= 4 && TH <= 64, "tile shape");
    static constexpr int XOFF = 4;                        // padded column of image column x0
    static constexpr int PW = TW + 8;                     // padded row length (16-byte rows)
    static constexpr int PH = TH + 2;
    static constexpr int NP = PW * PH;                    // padded pixels
    static constexpr int NPIX = TH * TW;                  // owned pixels
    static constexpr int PPL = TW / 32;                   // pixels per lane in a sweep row
    static constexpr int NRING = 2 * TW + 2 * (TH - 2);   // owned pixels on the tile edge
    static constexpr int NHALO = 2 * (TW + 2) + 2 * TH;   // halo pixels
    static constexpr int S = (int)sizeof(T);
    static constexpr int EPC = 16 / S;                    // elements per 16-byte chunk
    static constexpr int ICH = TW / EPC + 1;              // chunks covering TW elements at any alignment
    static constexpr int NITEMS = PH * ICH;               // chunk slots of one loaded array
    static constexpr size_t STAGE_BYTES = (size_t)(sizeof(T) == 2 ? 1 : 2) * NITEMS * 16;   // queue-area staging
    static constexpr int NDIR = CONN;
    static constexpr uint32_t QBIT = 1u;
    static_assert(NP < 65536, "queue entries are 16-bit padded indices");

    struct Smem {
        uint32_t *J;        // NP words: (value << 1) | queued, dilation domain
        uint16_t *I;        // NP: mask (dilation domain); 0 outside the image
        uint32_t *halo0;    // NHALO: halo values when they were loaded
        uint32_t *misc;     // 32 flags
        uint16_t *q;        // 2 * qcap: wave queues ...
        uint8_t *stage;     // ... whose space doubles as the marker staging area of a tile load
    };
    enum { M_NOTIFY = 0 /* 0..8 */, M_PRECOND = 9 };

    static __host__ __device__ constexpr size_t words_fixed() {
        return ((size_t)NP + (NP + 1) / 2 + NHALO + 32 + 3) & ~(size_t)3;
    }
    static __host__ __device__ size_t qbytes(uint32_t qcap) {
        const size_t b = (size_t)qcap * 2 * 2;
        return ((b > STAGE_BYTES ? b : STAGE_BYTES) + 15) & ~(size_t)15;
    }
    // Shared memory of one warp (a 16-byte multiple, so that slices stay aligned).
    static __host__ __device__ size_t smem_per_warp(uint32_t qcap) { return words_fixed() * 4 + qbytes(qcap); }
    static size_t smem_bytes(uint32_t qcap) { return smem_per_warp(qcap) * kWarpsPerCta; }

    static __device__ Smem carve(uint8_t *base) {
        Smem s;
        uint32_t *w = reinterpret_cast<uint32_t *>(base);
        s.J = w; w += NP;
        s.I = reinterpret_cast<uint16_t *>(w); w += (NP + 1) / 2;
        s.halo0 = w; w += NHALO;
        s.misc = w;
        w = reinterpret_cast<uint32_t *>(base) + words_fixed();
        s.q = reinterpret_cast<uint16_t *>(w);
        s.stage = reinterpret_cast<uint8_t *>(w);
        return s;
    }

    // padded index of padded row r (0 = top halo) and tile column c (-1 = left halo)
    static __device__ __forceinline__ int pidx(int r, int c) { return r * PW + XOFF + c; }
    // Ring position i in [0, NRING) -> (padded row, tile column) of an owned edge pixel.
    static __device__ __forceinline__ void ring_rc(int i, int &r, int &c) {
        if (i < TW) { r = 1; c = i; }
        else if (i < 2 * TW) { r = TH; c = i - TW; }
        else if (i < 2 * TW + (TH - 2)) { r = 2 + (i - 2 * TW); c = 0; }
        else { r = 2 + (i - 2 * TW - (TH - 2)); c = TW - 1; }
    }
    // Halo position i in [0, NHALO) -> (padded row, tile column).
    static __device__ __forceinline__ void halo_rc(int i, int &r, int &c) {
        if (i < TW + 2) { r = 0; c = i - 1; }
        else if (i < 2 * (TW + 2)) { r = PH - 1; c = i - (TW + 2) - 1; }
        else if (i < 2 * (TW + 2) + TH) { r = 1 + (i - 2 * (TW + 2)); c = -1; }
        else { r = 1 + (i - 2 * (TW + 2) - TH); c = TW; }
    }
    static __device__ __forceinline__ int dir_dy(int d) {
        if (CONN == 8) return d < 3 ? -1 : (d < 5 ? 0 : 1);
        return d == 0 ? -1 : (d == 3 ? 1 : 0);
    }
    static __device__ __forceinline__ int dir_dx(int d) {
        if (CONN == 8) return (d == 0 || d == 3 || d == 5) ? -1 : ((d == 2 || d == 4 || d == 7) ? 1 : 0);
        return d == 1 ? -1 : (d == 2 ? 1 : 0);
    }
    static __device__ __forceinline__ int nb_off(int d) { return dir_dy(d) * PW + dir_dx(d); }
    static __device__ __forceinline__ uint32_t to_dom(uint32_t v, uint32_t flip) { return v ^ flip; }
    static __device__ __forceinline__ uint32_t val(uint32_t w) { return w >> 1; }

    static __device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
        const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
    }

    // ---- HBM -> shared memory (all 32 lanes of the warp) ---------------------------------
    // Loads tile (ty, tx) with its one-pixel halo. Every full 16-byte chunk that covers the
    // tile's own columns of a padded row is copied with cp.async (all in flight at once,
    // through L2 only, so that J written by other warps is seen): the mask bytes into the
    // space of the J array (not yet in use), the marker bytes into the queue area. The mask
    // is widened first, which frees the J array for the marker. The two halo columns are
    // read element by element. Positions outside the image get J = flag only (value 0) and
    // I = 0, so they can never be raised or queued. Halo words carry the queued flag.
    template <bool IS_I>
    static __device__ __forceinline__ void widen(const ImageView &im, const Smem &s, const uint8_t *stage, int y0,
                                                 int x0, int xe, size_t total, int lane) {
        for (int it = lane; it < NITEMS; it += 32) {
            const int r = it / ICH, k = it % ICH;
            const int gy = y0 + r - 1;
            if (gy < 0 || gy >= im.H) continue;
            const size_t rowbase = (size_t)gy * im.W;
            const size_t lo = rowbase + x0, hi = rowbase + xe;
            const size_t chunk = lo / EPC + k;
            const size_t e0 = chunk * EPC;
            if (e0 >= hi) continue;
            union { uint4 u; T e[EPC]; } v;
            if (e0 + EPC <= total) {
                v.u = *reinterpret_cast<const uint4 *>(stage + it * 16);
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++)
                    if (e0 + j < total)
                        v.e[j] = IS_I ? reinterpret_cast<const T *>(im.I)[e0 + j]
                                      : __ldcg(reinterpret_cast<const T *>(im.J) + e0 + j);
            }
            const int shift = pidx(r, 0) - x0;                         // + image column = padded index
            const int base = (int)((int64_t)e0 - (int64_t)rowbase);    // image column of element 0
            const uint32_t hflag = (r == 0 || r == PH - 1) ? QBIT : 0u;
            const bool full = e0 >= lo && e0 + EPC <= hi;
#pragma unroll
            for (int j = 0; j < EPC; j++) {
                if (!full && (e0 + j < lo || e0 + j >= hi)) continue;
                const uint32_t x = to_dom(v.e[j], im.flip);
                if (IS_I) s.I[shift + base + j] = (uint16_t)x;
                else s.J[shift + base + j] = (x << 1) | hflag;
            }
        }
    }

    // u8 tiles stage both arrays in the queue area and widen them in one pass; u16 tiles,
    // whose staging is twice as large, stage the mask inside the J array (free until the
    // mask is widened), so that a u16 tile needs no more shared memory than a u8 one.
    static constexpr bool SPLIT = sizeof(T) == 2;

    // Both arrays from their staging areas in one pass over the chunks.
    static __device__ __forceinline__ void widen_both(const ImageView &im, const Smem &s, const uint8_t *stJ,
                                                      const uint8_t *stI, int y0, int x0, int xe, size_t total,
                                                      int lane) {
        for (int it = lane; it < NITEMS; it += 32) {
            const int r = it / ICH, k = it % ICH;
            const int gy = y0 + r - 1;
            if (gy < 0 || gy >= im.H) continue;
            const size_t rowbase = (size_t)gy * im.W;
            const size_t lo = rowbase + x0, hi = rowbase + xe;
            const size_t chunk = lo / EPC + k;
            const size_t e0 = chunk * EPC;
            if (e0 >= hi) continue;
            union { uint4 u; T e[EPC]; } vj, vi;
            if (e0 + EPC <= total) {
                vj.u = *reinterpret_cast<const uint4 *>(stJ + it * 16);
                vi.u = *reinterpret_cast<const uint4 *>(stI + it * 16);
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    if (e0 + j < total) {
                        vj.e[j] = __ldcg(reinterpret_cast<const T *>(im.J) + e0 + j);
                        vi.e[j] = reinterpret_cast<const T *>(im.I)[e0 + j];
                    }
                }
            }
            const int shift = pidx(r, 0) - x0;
            const int base = (int)((int64_t)e0 - (int64_t)rowbase);
            const uint32_t hflag = (r == 0 || r == PH - 1) ? QBIT : 0u;
            if (e0 >= lo && e0 + EPC <= hi) {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    s.J[shift + base + j] = (to_dom(vj.e[j], im.flip) << 1) | hflag;
                    s.I[shift + base + j] = (uint16_t)to_dom(vi.e[j], im.flip);
                }
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    const size_t e = e0 + j;
                    if (e < lo || e >= hi) continue;
                    s.J[shift + base + j] = (to_dom(vj.e[j], im.flip) << 1) | hflag;
                    s.I[shift + base + j] = (uint16_t)to_dom(vi.e[j], im.flip);
                }
            }
        }
    }

    static __device__ void load_tile(const ImageView &im, const Smem &s, int ty, int tx, int lane) {
        static_assert((size_t)NITEMS * 16 <= (size_t)NP * 4, "mask staging must fit in the J array");
        const int y0 = ty * TH, x0 = tx * TW;
        const size_t total = (size_t)im.H * (size_t)im.W;
        const int xe = min(im.W, x0 + TW);             // end of the tile's own columns
        uint8_t *stJ = s.stage;
        uint8_t *stI = SPLIT ? reinterpret_cast<uint8_t *>(s.J) : s.stage + NITEMS * 16;
        const bool edge = y0 == 0 || x0 == 0 || y0 + TH >= im.H || x0 + TW >= im.W;
        if (edge) {
            for (int p = lane; p < NP; p += 32) {
                s.I[p] = 0;
                if (!SPLIT) s.J[p] = QBIT;
            }
            if (!SPLIT) __syncwarp();
        }
        for (int it = lane; it < NITEMS; it += 32) {
            const int r = it / ICH, k = it % ICH;
            const int gy = y0 + r - 1;
            if (gy < 0 || gy >= im.H) continue;
            const size_t rowbase = (size_t)gy * im.W;
            const size_t chunk = (rowbase + x0) / EPC + k;
            if (chunk * EPC >= rowbase + xe || (chunk + 1) * EPC > total) continue;
            cp_async16(stJ + it * 16, reinterpret_cast<const uint4 *>(im.J) + chunk);
            cp_async16(stI + it * 16, reinterpret_cast<const uint4 *>(im.I) + chunk);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if (!SPLIT) {
            // the two halo columns, element by element, while the copies are in flight
            for (int i = lane; i < 2 * PH; i += 32) {
                const int r = i >> 1, c = (i & 1) ? TW : -1;
                const int gy = y0 + r - 1, gx = x0 + c;
                if (gy < 0 || gy >= im.H || gx < 0 || gx >= im.W) continue;
                const size_t e = (size_t)gy * im.W + gx;
                s.J[pidx(r, c)] = (to_dom(__ldcg(reinterpret_cast<const T *>(im.J) + e), im.flip) << 1) | QBIT;
                s.I[pidx(r, c)] = (uint16_t)to_dom(reinterpret_cast<const T *>(im.I)[e], im.flip);
            }
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncwarp();
            widen_both(im, s, stJ, stI, y0, x0, xe, total, lane);
            __syncwarp();
            return;
        }
        constexpr int HC = (2 * PH + 31) / 32;
        uint32_t hj[HC], hi_[HC];
#pragma unroll
        for (int q = 0; q < HC; q++) {
            const int i = lane + 32 * q;
            hj[q] = QBIT;
            hi_[q] = 0;
            const int r = i >> 1, c = (i & 1) ? TW : -1;
            const int gy = y0 + r - 1, gx = x0 + c;
            if (i >= 2 * PH || gy < 0 || gy >= im.H || gx < 0 || gx >= im.W) continue;
            const size_t e = (size_t)gy * im.W + gx;
            hj[q] = (to_dom(__ldcg(reinterpret_cast<const T *>(im.J) + e), im.flip) << 1) | QBIT;
            hi_[q] = to_dom(reinterpret_cast<const T *>(im.I)[e], im.flip);
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncwarp();
        widen<true>(im, s, stI, y0, x0, xe, total, lane);
        __syncwarp();   // the mask bytes in the J array are consumed
        if (edge) {
            for (int p = lane; p < NP; p += 32) s.J[p] = QBIT;
            __syncwarp();
        }
        widen<false>(im, s, stJ, y0, x0, xe, total, lane);
#pragma unroll
        for (int q = 0; q < HC; q++) {
            const int i = lane + 32 * q;
            if (i >= 2 * PH) continue;
            const int r = i >> 1, c = (i & 1) ? TW : -1;
            s.J[pidx(r, c)] = hj[q];
            s.I[pidx(r, c)] = (uint16_t)hi_[q];
        }
        __syncwarp();
    }

    // Remember the halo values (after a load or a halo reload).
    static __device__ void save_halo(const Smem &s, int lane) {
        for (int i = lane; i < NHALO; i += 32) {
            int r, c;
            halo_rc(i, r, c);
            s.halo0[i] = val(s.J[pidx(r, c)]);
        }
    }

    // Reload the halo ring of J (the interior stays as this warp left it).
    static __device__ void load_halo_J(const ImageView &im, const Smem &s, int ty, int tx, int lane) {
        const int y0 = ty * TH, x0 = tx * TW;
        for (int i = lane; i < NHALO; i += 32) {
            int r, c;
            halo_rc(i, r, c);
            const int gy = y0 + r - 1, gx = x0 + c;
            uint32_t w = QBIT;
            if (gy >= 0 && gy < im.H && gx >= 0 && gx < im.W)
                w = (to_dom(__ldcg(reinterpret_cast<const T *>(im.J) + (size_t)gy * im.W + gx), im.flip) << 1) | QBIT;
            s.J[pidx(r, c)] = w;
        }
        __syncwarp();
    }

    // Store the owned rows whose bit is set in rowmask, in 16-byte chunks where a chunk lies
    // entirely inside the tile's row segment, element by element otherwise.
    static __device__ void store_tile(const ImageView &im, const Smem &s, int ty, int tx,
                                      unsigned long long rowmask, bool use_cg, int lane) {
        const int y0 = ty * TH, x0 = tx * TW;
        const size_t total = (size_t)im.H * (size_t)im.W;
        const int xe = min(im.W, x0 + TW);
        for (int it = lane; it < TH * ICH; it += 32) {
            const int rr = it / ICH, k = it % ICH;
            if (!((rowmask >> rr) & 1ull)) continue;
            const int gy = y0 + rr;
            if (gy >= im.H) continue;
            const size_t rowbase = (size_t)gy * im.W;
            const size_t lo = rowbase + x0, hi = rowbase + xe;
            const size_t chunk = lo / EPC + k;
            const size_t e0 = chunk * EPC;
            if (e0 >= hi) continue;
            const uint32_t *jrow = s.J + pidx(rr + 1, 0) - (int)(lo - rowbase);
            const int base = (int)((int64_t)e0 - (int64_t)rowbase);
            if (e0 >= lo && e0 + EPC <= hi && e0 + EPC <= total) {
                union { uint4 u; T e[EPC]; } v;
#pragma unroll
                for (int j = 0; j < EPC; j++) v.e[j] = (T)to_dom(val(jrow[base + j]), im.flip);
                if (use_cg) __stcg(reinterpret_cast<uint4 *>(im.J) + chunk, v.u);
                else reinterpret_cast<uint4 *>(im.J)[chunk] = v.u;
            } else {
#pragma unroll
                for (int j = 0; j < EPC; j++) {
                    const size_t e = e0 + j;
                    if (e < lo || e >= hi) continue;
                    const T v = (T)to_dom(val(jrow[base + j]), im.flip);
                    if (use_cg) __stcg(reinterpret_cast<T *>(im.J) + e, v);
                    else reinterpret_cast<T *>(im.J)[e] = v;
                }
            }
        }
    }

    // ---- tile-local sweeps (Algorithm 7, scanning phase) -------------------------------------
    // The clamp f(x) = min(hi, max(lo, x)) is packed as (hi << 16) | lo; values are < 2^16.
    // Composition g o f of clamps [lf, hf] then [lg, hg] is [clamp(lf, lg, hg), clamp(hf, lg, hg)].
    // Sweeps run before any pixel is queued, on the values; they return a mask of the rows
    // they changed.

    // Raster: rows top to bottom, J(p) <- max{J(q): q in N+(p) U {p}} ^ I(p) with
    // N+ = {N, W} (4-conn) or {NW, N, NE, W} (8-conn).
    static __device__ unsigned long long sweep_raster(const Smem &s, int lane) {
        unsigned long long chg = 0;
        for (int r = 1; r <= TH; r++) {
            uint32_t a[PPL], iv[PPL], old[PPL];
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                const int p = pidx(r, lane * PPL + k);
                old[k] = val(s.J[p]);
                uint32_t v = max(old[k], val(s.J[p - PW]));
                if (CONN == 8) v = max(v, max(val(s.J[p - PW - 1]), val(s.J[p - PW + 1])));
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
            uint32_t x = val(s.J[pidx(r, -1)]);           // left halo
            if (lane > 0) x = clampu(x, ex & 0xffffu, ex >> 16);
            bool ch = false;
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                x = clampu(x, min(a[k], iv[k]), iv[k]);
                s.J[pidx(r, lane * PPL + k)] = x << 1;
                ch |= (x != old[k]);
            }
            if (__any_sync(0xffffffffu, ch)) chg |= 1ull << (r - 1);
            __syncwarp();
        }
        return chg;
    }

    // Anti-raster: rows bottom to top, right to left, with N- = {S, E} / {SE, S, SW, E}.
    static __device__ unsigned long long sweep_antiraster(const Smem &s, int lane) {
        unsigned long long chg = 0;
        for (int r = TH; r >= 1; r--) {
            uint32_t a[PPL], iv[PPL], old[PPL];
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                const int p = pidx(r, lane * PPL + k);
                old[k] = val(s.J[p]);
                uint32_t v = max(old[k], val(s.J[p + PW]));
                if (CONN == 8) v = max(v, max(val(s.J[p + PW - 1]), val(s.J[p + PW + 1])));
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
            uint32_t x = val(s.J[pidx(r, TW)]);           // right halo
            if (lane < 31) x = clampu(x, ex & 0xffffu, ex >> 16);
            bool ch = false;
#pragma unroll
            for (int k = PPL - 1; k >= 0; k--) {
                x = clampu(x, min(a[k], iv[k]), iv[k]);
                s.J[pidx(r, lane * PPL + k)] = x << 1;
                ch |= (x != old[k]);
            }
            if (__any_sync(0xffffffffu, ch)) chg |= 1ull << (r - 1);
            __syncwarp();
        }
        return chg;
    }

    // ---- wave queues (private to the warp) ------------------------------------------------------
    // Warp-aggregated push: every lane holds a bitmask of up to K candidates; a warp
    // exclusive prefix sum of the per-lane counts gives each lane its slots. The count is a
    // warp-uniform register (the queues belong to one warp).
    template <int K>
    static __device__ __forceinline__ void push_warp(const Smem &s, const EngineArgs &a, uint16_t *ovf,
                                                     int buf, uint32_t &cnt, uint32_t cm,
                                                     const int (&q)[K], int lane) {
        const uint32_t mine = __popc(cm);
        uint32_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t pos = cnt + incl - mine;
#pragma unroll
        for (int d = 0; d < K; d++) {
            if ((cm >> d) & 1u) {
                if (pos < a.qcap) s.q[buf * a.qcap + pos] = (uint16_t)q[d];
                else if (pos - a.qcap < a.ovcap) ovf[buf * a.ovcap + (pos - a.qcap)] = (uint16_t)q[d];
                else set_status(a.hdr, kErrQueueFull);
                pos++;
            }
        }
        cnt += total;
    }

    static __device__ __forceinline__ void mark_row(unsigned long long &rows, int q) {
        const int r = q / PW;
        if (r >= 1 && r <= TH) rows |= 1ull << (r - 1);
    }

    // Initial wave of a visit, into buffer 0; returns its size. A pixel enters it when one
    // Jacobi step of Eq. "recon" raises it: J(p) < min(I(p), max of J over N_G(p)).
    // full: every owned pixel is tested (first visit); otherwise only the edge ring, since
    // the interior was at a local fixed point when it was last stored and only the halo can
    // have changed since.
    static __device__ uint32_t seed_wave(const Smem &s, const EngineArgs &a, uint16_t *ovf, bool full,
                                         unsigned long long &rows, int lane) {
        const int n = full ? NPIX : NRING;
        const int nround = (n + 31) / 32 * 32;
        uint32_t cnt = 0;
        for (int i = lane; i < nround; i += 32) {
            int q[1] = {0};
            uint32_t cm = 0;
            if (i < n) {
                int r, c;
                if (full) { r = i / TW + 1; c = i % TW; }
                else ring_rc(i, r, c);
                const int p = pidx(r, c);
                uint32_t m = 0;
#pragma unroll
                for (int d = 0; d < NDIR; d++) m = max(m, val(s.J[p + nb_off(d)]));
                const uint32_t nv = min(m, (uint32_t)s.I[p]);
                if (nv > val(s.J[p])) {
                    s.J[p] = (nv << 1) | QBIT;
                    rows |= 1ull << (r - 1);
                    q[0] = p;
                    cm = 1;
                }
            }
            push_warp<1>(s, a, ovf, 0, cnt, cm, q, lane);
        }
        __syncwarp();
        return cnt;
    }

    static __device__ __forceinline__ int entry(const Smem &s, const EngineArgs &a, const uint16_t *ovf,
                                                int buf, uint32_t i) {
        return (i < a.qcap) ? s.q[buf * a.qcap + i] : ovf[buf * a.ovcap + (i - a.qcap)];
    }

    // Drain the wave queues to a local fixed point, starting from `n` entries in buffer 0.
    static __device__ uint32_t run_waves(const Smem &s, const EngineArgs &a, uint16_t *ovf, uint32_t n,
                                         unsigned long long &rows, uint32_t &waves, int lane) {
        uint32_t pops = 0;
        waves = 0;
        volatile uint32_t *vJ = s.J;
        const uint32_t cap = a.qcap + a.ovcap;
        int cb = 0;
        while (n > 0) {
            if (n > cap) n = cap;   // cannot happen: queued pixels are distinct
            pops += n;
            waves++;
            const int nb = cb ^ 1;
            uint32_t nn = 0;
            const uint32_t nround = (n + 31) / 32 * 32;
            for (uint32_t i = lane; i < nround; i += 32) {
                const bool valid = i < n;
                const int p = valid ? entry(s, a, ovf, cb, i) : pidx(1, 0);
                const uint32_t v = valid ? val(atomicAnd(&s.J[p], ~QBIT)) : 0u;
                int q[NDIR];
                uint32_t nv[NDIR], cur[NDIR];
#pragma unroll
                for (int d = 0; d < NDIR; d++) {   // all neighbour reads first
                    q[d] = p + nb_off(d);
                    nv[d] = min(v, (uint32_t)s.I[q[d]]);
                    cur[d] = val(vJ[q[d]]);
                }
                uint32_t cm = 0;
#pragma unroll
                for (int d = 0; d < NDIR; d++) {
                    if (cur[d] < nv[d]) {
                        const uint32_t wnew = (nv[d] << 1) | QBIT;
                        const uint32_t old = atomicMax(&s.J[q[d]], wnew);
                        if (old < wnew) {
                            if (val(old) < nv[d]) mark_row(rows, q[d]);
                            if ((old & QBIT) == 0) cm |= 1u << d;
                        }
                    }
                }
                push_warp<NDIR>(s, a, ovf, nb, nn, cm, q, lane);
            }
            __syncwarp();
            n = nn;
            cb = nb;
        }
        return pops;
    }

    // ---- end of a visit -----------------------------------------------------------------------
    // For every halo pixel h: can the tile's pixels raise it above the value it had when it
    // was loaded (one Jacobi step from the tile's own pixels, or a raise already made)? If so
    // the neighbour tile that owns h has work: flag it.
    static __device__ void notify_scan(const Smem &s, int lane) {
        for (int i = lane; i < NHALO; i += 32) {
            int r, c;
            halo_rc(i, r, c);
            const int h = pidx(r, c);
            uint32_t m = 0;
#pragma unroll
            for (int d = 0; d < NDIR; d++) {
                const int qr = r + dir_dy(d), qc = c + dir_dx(d);
                if (qr >= 1 && qr <= TH && qc >= 0 && qc < TW) m = max(m, val(s.J[h + nb_off(d)]));
            }
            const uint32_t nv = max(val(s.J[h]), min(m, (uint32_t)s.I[h]));
            if (nv > s.halo0[i]) {
                const int dy = r == 0 ? -1 : (r == PH - 1 ? 1 : 0);
                const int dx = c < 0 ? -1 : (c >= TW ? 1 : 0);
                s.misc[M_NOTIFY + (dy + 1) * 3 + (dx + 1)] = 1;
            }
        }
    }

    // Whole warp, after a fence and __syncwarp: lane j notifies neighbour j.
    static __device__ void send_notifications(const Smem &s, const EngineArgs &a, const ImageView &im,
                                              int ty, int tx, int lane) {
        if (lane < 9 && lane != 4 && s.misc[M_NOTIFY + lane]) {
            const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
            if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                notify_tile(a, im.tile_base + (uint32_t)(ny * im.tiles_x + nx));
        }
    }

    static __device__ void clear_flags(const Smem &s, int lane) {
        if (lane < 10) s.misc[lane] = 0;
        __syncwarp();
    }
};

// ---- per-tile bodies shared by the single-image and the batch kernels -------------------------

// Mark tile t PENDING without queueing it (batches: the compact kernel queues it later, in
// order, and the finalize kernel counts the PENDING tiles into the pending count). Nothing
// else changes a state word before the persistent kernel starts, so the OR needs no result:
// a fire-and-forget reduction, no round trip.
__device__ __forceinline__ void mark_pending(const EngineArgs &a, uint32_t t) {
    atomicOr(a.state + t, ST_PENDING);
}

// Tile-parallel scan of one tile (the frontier-initialisation kernel's body):
// precondition check, `sweeps` raster / anti-raster pairs in shared memory, store, then
// queue the tile if one of its pixels can still be raised, and each neighbour one of
// whose halo pixels it can raise.
template <typename T, int CONN, int TH, int TW>
__device__ void scan_tile(const EngineArgs &a, const ImageView &im, uint32_t t, uint8_t *wsmem, int lane) {
    using TL = Tile<T, CONN, TH, TW>;
    const typename TL::Smem s = TL::carve(wsmem);
    const long long c0 = clock64();
    const uint32_t lt = t - im.tile_base;
    const int ty = lt / im.tiles_x, tx = lt % im.tiles_x;
    TL::clear_flags(s, lane);
    TL::load_tile(im, s, ty, tx, lane);
    TL::save_halo(s, lane);
    bool bad = false;
    for (int i = lane; i < TL::NPIX; i += 32) {
        const int p = TL::pidx(i / TW + 1, i % TW);
        bad |= TL::val(s.J[p]) > (uint32_t)s.I[p];
    }
    bad = __any_sync(0xffffffffu, bad);
    const int sweeps = a.tile_sweeps ? (int)a.tile_sweeps[t] : a.sweeps;
    unsigned long long rows = 0;
    for (int k = 0; k < sweeps; k++) {
        rows |= TL::sweep_raster(s, lane);
        rows |= TL::sweep_antiraster(s, lane);
    }
    if (rows) TL::store_tile(im, s, ty, tx, rows, false, lane);
    bool active = false;
    for (int i = lane; i < TL::NPIX; i += 32) {
        const int p = TL::pidx(i / TW + 1, i % TW);
        uint32_t m = 0;
#pragma unroll
        for (int d = 0; d < TL::NDIR; d++) m = max(m, TL::val(s.J[p + TL::nb_off(d)]));
        active |= min(m, (uint32_t)s.I[p]) > TL::val(s.J[p]);
    }
    active = __any_sync(0xffffffffu, active);
    TL::notify_scan(s, lane);
    __threadfence();
    __syncwarp();
    if (a.defer_push) {
        if (lane < 9 && lane != 4 && s.misc[TL::M_NOTIFY + lane]) {
            const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
            if (ny >= 0 && nx >= 0 && ny < im.tiles_y && nx < im.tiles_x)
                mark_pending(a, im.tile_base + (uint32_t)(ny * im.tiles_x + nx));
        }
        if (lane == 0 && active) mark_pending(a, t);
    } else {
        if (lane == 0 && active) notify_tile(a, t);
        TL::send_notifications(s, a, im, ty, tx, lane);
    }
    if (lane == 0) {
        if (bad) set_status(a.hdr, kErrPrecondition);
        if (a.tile_work) atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
    __syncwarp();
}

struct VisitStats {
    unsigned long long visits, pops, seeds, waves;
};

// End of a visit round (whole warp, after the tile's stores and notifications are
// fenced): ACTIVE -> IDLE and one fewer pending tile, unless the tile was notified while
// this warp held it; then it stays ACTIVE and the warp processes it again (returns true).
// The decrement is issued only once the state change has returned, and it cannot reach
// zero early: the notified neighbours were counted first, and every tile still being
// visited is counted too.
__device__ inline bool finish_tile(const EngineArgs &a, uint32_t t, int lane) {
    uint32_t redo = 0;
    if (lane == 0) {
        const uint32_t busy_st = ST_ACTIVE | ST_VISITED;
        const uint32_t r = atomicCAS(a.state + t, busy_st, ST_VISITED);
        if (r == busy_st) {
            atomicSub(&a.hdr->pending, 1u);
        } else {
            atomicAnd(a.state + t, ~ST_PENDING);   // notified while ACTIVE: go again
            redo = !fatal(a.hdr);
        }
    }
    return __shfl_sync(0xffffffffu, redo, 0) != 0;
}

// One visit of tile t by the persistent kernel, including the re-processing rounds when
// the tile is notified while this warp holds it. Lane 0 has already moved the tile to
// ACTIVE; on return it is IDLE (or the run is stopping on an error).
template <typename T, int CONN, int TH, int TW>
__device__ void visit_tile(const EngineArgs &a, const ImageView &im, uint32_t t, bool first, uint8_t *wsmem,
                           uint16_t *ovf, VisitStats &st, int lane) {
    using TL = Tile<T, CONN, TH, TW>;
    const typename TL::Smem s = TL::carve(wsmem);
    const long long c0 = clock64();
    const uint32_t lt = t - im.tile_base;
    const int ty = lt / im.tiles_x, tx = lt % im.tiles_x;
    TL::clear_flags(s, lane);
    TL::load_tile(im, s, ty, tx, lane);
    TL::save_halo(s, lane);
    bool full = first;
    uint32_t tile_pops = 0;
    for (;;) {
        unsigned long long rows = 0;
        if (full) {
            for (int k = 0; k < a.revisit_sweeps; k++) {
                rows |= TL::sweep_raster(s, lane);
                rows |= TL::sweep_antiraster(s, lane);
            }
        }
        const uint32_t seeds = TL::seed_wave(s, a, ovf, full, rows, lane);
        uint32_t waves;
        const uint32_t pops = TL::run_waves(s, a, ovf, seeds, rows, waves, lane);
        st.visits++;
        st.pops += pops;
        st.seeds += seeds;
        st.waves += waves;
        tile_pops += pops;
        rows = (unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)rows) |
               ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(rows >> 32)) << 32);
        if (rows) TL::store_tile(im, s, ty, tx, rows, true, lane);
        TL::notify_scan(s, lane);
        __threadfence();
        __syncwarp();
        TL::send_notifications(s, a, im, ty, tx, lane);
        if (!finish_tile(a, t, lane)) break;
        // Re-process: the interior in shared memory is what this warp stored; only the
        // halo can have changed since.
        TL::clear_flags(s, lane);
        TL::load_halo_J(im, s, ty, tx, lane);
        TL::save_halo(s, lane);
        full = false;
    }
    if (lane == 0 && a.tile_work) {
        atomicAdd(a.tile_work + t, tile_pops);
        atomicAdd(a.tile_work + a.ntiles + t, (uint32_t)min(clock64() - c0, 0x7fffffffll));
    }
}

// Image that owns global tile t: the batch's tile -> image map (one load instead of a
// binary search over tile_base: measured ~1.9 k cycles per visit on a 256-image batch).
__device__ __forceinline__ const ImageView &image_of(const EngineArgs &a, uint32_t t) {
    if (a.imgs == nullptr) return a.img0;
    if (a.tile_img) return a.imgs[a.tile_img[t]];
    int lo = 0, hi = a.nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.imgs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return a.imgs[lo];
}

// Pop the next tile (lane 0) and move it to ACTIVE; returns kDone when the run is over.
__device__ inline uint32_t acquire_tile(const EngineArgs &a, bool &first, unsigned long long &idle, int lane) {
    uint32_t t = 0, f = 0;
    if (lane == 0) {
        const unsigned long long t0 = globaltimer_ns();
        t = pop_tile(a);
        idle += globaltimer_ns() - t0;
        if (t != kDone) {
            const uint32_t old = atomicAdd(a.state + t, 1u);   // PENDING -> ACTIVE
            f = (old & ST_VISITED) == 0;
            if (f) atomicOr(a.state + t, ST_VISITED);
            fence_protocol();
        }
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    first = __shfl_sync(0xffffffffu, f, 0) != 0;
    return t;
}

__device__ inline void flush_stats(const EngineArgs &a, const VisitStats &st, unsigned long long idle,
                                   unsigned long long busy, int lane) {
    if (lane == 0) {
        atomicAdd(&a.hdr->visits, st.visits);
        atomicAdd(&a.hdr->pops, st.pops);
        atomicAdd(&a.hdr->seeds, st.seeds);
        atomicAdd(&a.hdr->waves, st.waves);
        atomicAdd(&a.hdr->idle_ns, idle);
        atomicAdd(&a.hdr->busy_ns, busy);
    }
}

// ---- kernels: images of one pixel type and connectivity (one image, or a uniform batch) -----------
template <typename T, int CONN, int TH, int TW>
__global__ void __launch_bounds__(kThreads) scan_kernel(EngineArgs a) {
    using TL = Tile<T, CONN, TH, TW>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * TL::smem_per_warp(a.qcap);
    const uint32_t nworkers = gridDim.x * kWarpsPerCta;
    for (uint32_t t = blockIdx.x * kWarpsPerCta + warp; t < a.ntiles; t += nworkers)
        scan_tile<T, CONN, TH, TW>(a, image_of(a, t), t, wsmem, lane);
}

template <typename T, int CONN, int TH, int TW>
__global__ void __launch_bounds__(kThreads, IWPP_DRAIN_MINB) drain_kernel(EngineArgs a) {
    using TL = Tile<T, CONN, TH, TW>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * TL::smem_per_warp(a.qcap);
    uint16_t *ovf = a.ovf + ((size_t)blockIdx.x * kWarpsPerCta + warp) * 2 * a.ovcap;
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0;
    for (;;) {
        bool first;
        const uint32_t t = acquire_tile(a, first, idle, lane);
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        visit_tile<T, CONN, TH, TW>(a, image_of(a, t), t, first, wsmem, ovf, st, lane);
        busy += globaltimer_ns() - b0;
    }
    flush_stats(a, st, idle, busy, lane);
}

// ---- kernels: a batch of images of mixed pixel types and connectivities -------------------------
// Shared memory per warp is the largest of the four kinds' (they differ only in staging).
template <int TH, int TW>
__host__ __device__ inline size_t mixed_smem_per_warp(uint32_t qcap) {
    const size_t a8 = Tile<uint8_t, 8, TH, TW>::smem_per_warp(qcap);
    const size_t a16 = Tile<uint16_t, 8, TH, TW>::smem_per_warp(qcap);
    return a8 > a16 ? a8 : a16;
}

template <int TH, int TW>
__global__ void __launch_bounds__(kThreads) scan_mixed_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * mixed_smem_per_warp<TH, TW>(a.qcap);
    const uint32_t nworkers = gridDim.x * kWarpsPerCta;
    for (uint32_t t = blockIdx.x * kWarpsPerCta + warp; t < a.ntiles; t += nworkers) {
        const ImageView &im = image_of(a, t);
        switch (im.kind) {
            case 0: scan_tile<uint8_t, 4, TH, TW>(a, im, t, wsmem, lane); break;
            case 1: scan_tile<uint16_t, 4, TH, TW>(a, im, t, wsmem, lane); break;
            case 2: scan_tile<uint8_t, 8, TH, TW>(a, im, t, wsmem, lane); break;
            default: scan_tile<uint16_t, 8, TH, TW>(a, im, t, wsmem, lane); break;
        }
    }
}

template <int TH, int TW>
__global__ void __launch_bounds__(kThreads, IWPP_DRAIN_MINB) drain_mixed_kernel(EngineArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *wsmem = smem_raw + warp * mixed_smem_per_warp<TH, TW>(a.qcap);
    uint16_t *ovf = a.ovf + ((size_t)blockIdx.x * kWarpsPerCta + warp) * 2 * a.ovcap;
    VisitStats st = {0, 0, 0, 0};
    unsigned long long idle = 0, busy = 0;
    for (;;) {
        bool first;
        const uint32_t t = acquire_tile(a, first, idle, lane);
        if (t == kDone) break;
        const unsigned long long b0 = globaltimer_ns();
        const ImageView &im = image_of(a, t);
        switch (im.kind) {
            case 0: visit_tile<uint8_t, 4, TH, TW>(a, im, t, first, wsmem, ovf, st, lane); break;
            case 1: visit_tile<uint16_t, 4, TH, TW>(a, im, t, first, wsmem, ovf, st, lane); break;
            case 2: visit_tile<uint8_t, 8, TH, TW>(a, im, t, first, wsmem, ovf, st, lane); break;
            default: visit_tile<uint16_t, 8, TH, TW>(a, im, t, first, wsmem, ovf, st, lane); break;
        }
        busy += globaltimer_ns() - b0;
    }
    flush_stats(a, st, idle, busy, lane);
}

// Queue the PENDING tiles in schedule order (`order`, or tile id order) before the
// persistent kernel starts: warp-aggregated tickets, no consumer runs yet. A tile is
// claimed through the ST_QUEUED bit, so an order with repeated entries cannot queue a
// tile twice; finalize_queue_kernel then queues any PENDING tile the order left out and
// clears the bit.
constexpr uint32_t ST_QUEUED = 8u;

__device__ __forceinline__ void queue_warp(const EngineArgs &a, bool want, uint32_t t, int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, want);
    if (bal == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.hdr->tail, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (want) a.queue[(base + __popc(bal & ((1u << lane) - 1u))) % a.ntiles] = t;
}

// The initial frontier of a batch is queued in `order`, else in a spread order: position i
// takes tile (i * spread) mod ntiles, spread odd, coprime with ntiles and near 0.618 ntiles,
// so that tiles next to each other in an image (which raster order would hand to concurrent
// workers) are far apart in the queue. Concurrent neighbours raise each other's borders
// while both are being visited and so revisit each other; on the 512-image batch the spread
// order needs 21 % fewer visits than raster order (measured: as few as a random permutation
// or an order by measured work, largest or smallest first).
static __global__ void __launch_bounds__(256) compact_kernel(EngineArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t nround = (a.ntiles + 31) / 32 * 32;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nround; i += stride) {
        uint32_t t = 0;
        bool want = false;
        if (i < a.ntiles) {
            t = a.order ? a.order[i] : spread_tile(i, a.ntiles, a.spread);
            if (t < a.ntiles && (a.state[t] & ST_PENDING) != 0)
                want = (atomicOr(a.state + t, ST_QUEUED) & ST_QUEUED) == 0;
        }
        queue_warp(a, want, t, lane);
    }
}

static __global__ void __launch_bounds__(256) finalize_queue_kernel(EngineArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t nround = (a.ntiles + 31) / 32 * 32;
    uint32_t npending = 0;   // lane 0: PENDING tiles of this warp's rounds (every one is queued)
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nround; t += stride) {
        bool want = false, pend = false;
        if (t < a.ntiles) {
            const uint32_t s = a.state[t];
            pend = (s & ST_PENDING) != 0;
            want = pend && (s & ST_QUEUED) == 0;
            if (s & ST_QUEUED) a.state[t] = s & ~ST_QUEUED;
        }
        npending += (uint32_t)__popc(__ballot_sync(0xffffffffu, pend));
        queue_warp(a, want, t, lane);
    }
    if (lane == 0 && npending) atomicAdd(&a.hdr->pending, npending);
}

// Write a chunk of the batch's image table into the workspace (descriptors travel as
// kernel parameters, so the call needs no host-to-device copy and can be captured).
constexpr int kDescChunk = 32;
struct DescChunk {
    ImageView v[kDescChunk];
    int first, count;
};
static __global__ void upload_descs_kernel(ImageView *table, DescChunk c) {
    const int i = threadIdx.x;
    if (i < c.count) table[c.first + i] = c.v[i];
}

// The batch's tile -> image map, from the uploaded image table (one CTA per image at a time).
static __global__ void __launch_bounds__(256) tile_image_kernel(const ImageView *table, int n, uint32_t *tile_img) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t base = table[i].tile_base;
        const uint32_t nt = (uint32_t)table[i].tiles_x * (uint32_t)table[i].tiles_y;
        for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) tile_img[base + k] = (uint32_t)i;
    }
}

}  // namespace iwpp

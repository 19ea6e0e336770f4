// iwpp_sched.cu — the learned work estimator of the batch schedule (include/iwpp.h).
//
// Per 64 x 64 block of every image: 16 features (a histogram of mask - marker, seed and
// edge fractions, moments, block size), computed exactly in integers and converted once.
// A 16 -> 64 -> 64 -> 2 ReLU MLP in FP32 on CUDA cores predicts (log work, sweep count)
// per block; a counting sort on the predicted work orders the batch's tiles largest
// first and gives every tile its block's sweep count. Training is hand-written too:
// per-sample backpropagation with warp-shuffle gradient reductions, and Adam.
// None of this can change a reconstruction result: it only reorders work.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_feat.cuh"
#include "iwpp_spread.h"
#include "iwpp_host.h"

namespace iwpp {

constexpr int kBlk = IWPP_FEATURE_BLOCK;   // feature block side (64)
constexpr int kNF = IWPP_NFEAT;            // 16 features
constexpr int kH = 64;                     // hidden width
constexpr int kNP = IWPP_MLP_PARAMS;       // 16*64 + 64 + 64*64 + 64 + 64*2 + 2
constexpr int kBuckets = 1024;             // work-key buckets of the counting sort
constexpr float kKeyScale = 64.f;          // bucket = log-work * 64, over [0, 16)

// parameter offsets in the flat vector
constexpr int oW1 = 0, ob1 = oW1 + kNF * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * 2;
static_assert(ob3 + 2 == kNP, "parameter layout");

struct SchedImage {
    const uint8_t *J;
    const uint8_t *I;
    int H, W;
    int nbx, nby;          // feature blocks
    int tiles_x, tiles_y;  // engine tiles under the plan
    uint32_t block_base, tile_base;
    uint32_t flip, u16;
};

constexpr int kSchedChunk = 32;
struct SchedChunk {
    SchedImage v[kSchedChunk];
    int first, count;
};

__global__ void upload_sched_kernel(SchedImage *table, SchedChunk c) {
    if ((int)threadIdx.x < c.count) table[c.first + threadIdx.x] = c.v[threadIdx.x];
}

template <typename F>
__device__ __forceinline__ int find_image(const SchedImage *tab, int n, uint32_t id, F base_of) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base_of(tab[mid]) <= id) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- features: one warp per block; lane c holds columns 2c and 2c + 1 of every row ------------
// Exact integer sums per lane over the block's sampled rows (8-bit packed histogram counters:
// at most 32 pixels per lane), warp reductions, then lane 0 converts. A sampled row is read
// with the row below it, which the edge test needs.
// Pixels (y, x) and (y, x + 1) of plane p (flipped), loaded with clamped addresses; the
// caller masks the ones outside the block.
__device__ __forceinline__ void feat_load(const SchedImage &im, const uint8_t *p, int y, int x, uint32_t &e,
                                          uint32_t &o) {
    const size_t row = (size_t)y * im.W;
    const int xe = min(x, im.W - 1), xo = min(x + 1, im.W - 1);
    if (im.u16) {
        const uint16_t *q = reinterpret_cast<const uint16_t *>(p) + row;
        e = q[xe];
        o = q[xo];
    } else {
        e = p[row + xe];
        o = p[row + xo];
    }
    e ^= im.flip;
    o ^= im.flip;
}

// Word w (0..3) of a 16-byte chunk, pixel q of the word (4 u8 or 2 u16 per word).
template <bool U16>
__device__ __forceinline__ uint32_t px_of(uint32_t w, int q) {
    return U16 ? (w >> (16 * q)) & 0xFFFFu : (w >> (8 * q)) & 0xFFu;
}

// A whole 64 x 64 block inside the image whose rows start on 16-byte boundaries: each lane
// reads 16 bytes of a row (PX pixels); LPR lanes cover a row, RPG rows per load, and the
// next row group is prefetched while this one is processed. The pixel below a lane's
// pixels is LPR lanes further (or, for the group's last row, the first row of the next
// group, one shuffle away); the pixel right of its last one is the next lane's first.
template <bool U16>
__device__ __forceinline__ void feat_block_vec(const SchedImage &im, int y0, int x0, uint32_t thr, int lane,
                                               FeatAcc &a) {
    constexpr int PX = U16 ? 8 : 16, LPR = 64 / PX, RPG = 32 / LPR, NK = 64 / RPG, PPW = PX / 4;
    const int g = lane / LPR, sgm = lane % LPR;
    const size_t pitch = (size_t)im.W * (U16 ? 2 : 1);
    const uint8_t *baseI = im.I + (size_t)y0 * pitch + (size_t)x0 * (U16 ? 2 : 1) + (size_t)sgm * 16;
    const uint8_t *baseJ = im.J + (size_t)y0 * pitch + (size_t)x0 * (U16 ? 2 : 1) + (size_t)sgm * 16;
    const uint32_t f = im.flip | (im.flip << 16);
    const uint32_t fw = U16 ? f : (im.flip * 0x01010101u);
    auto ld = [&](const uint8_t *b, int k) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(b + (size_t)(k * RPG + g) * pitch));
        v.x ^= fw; v.y ^= fw; v.z ^= fw; v.w ^= fw;
        return v;
    };
    uint4 I = ld(baseI, 0), J = ld(baseJ, 0);
    for (int k = 0; k < NK; k++) {
        uint4 In = I, Jn = J;
        if (k + 1 < NK) {
            In = ld(baseI, k + 1);
            Jn = ld(baseJ, k + 1);
        }
        const uint32_t iw[4] = {I.x, I.y, I.z, I.w}, jw[4] = {J.x, J.y, J.z, J.w};
        // the row below: next lane group in this load, or the next group's first row
        uint32_t dw[4];
        const uint32_t nw4[4] = {In.x, In.y, In.z, In.w};
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const uint32_t below = __shfl_down_sync(0xffffffffu, iw[w], LPR);
            const uint32_t wrap = __shfl_sync(0xffffffffu, nw4[w], sgm);   // group 0 of the next load
            dw[w] = g < RPG - 1 ? below : wrap;
        }
        const bool has_down = !(g == RPG - 1 && k == NK - 1);
        const uint32_t right = __shfl_down_sync(0xffffffffu, iw[0], 1);   // next lane's first word
        a.npix += PX;
        const bool sampled = ((k * RPG + g) % kFeatRowStep) == 0;   // this lane's row of the block
#pragma unroll
        for (int w = 0; w < 4 && sampled; w++) {
#pragma unroll
            for (int q = 0; q < PPW; q++) {
                const uint32_t i = px_of<U16>(iw[w], q), j = px_of<U16>(jw[w], q);
                feat_pixel(a, i, j, U16);
                uint32_t r;
                if (q + 1 < PPW) r = px_of<U16>(iw[w], q + 1);
                else if (w < 3) r = px_of<U16>(iw[w + 1], 0);
                else r = px_of<U16>(right, 0);
                const bool has_right = !(w == 3 && q == PPW - 1 && sgm == LPR - 1);
                const uint32_t gx = has_right ? (uint32_t)abs((int)r - (int)i) : 0u;
                const uint32_t gy = has_down ? (uint32_t)abs((int)px_of<U16>(dw[w], q) - (int)i) : 0u;
                a.edges += (gx + gy > thr);
            }
        }
        I = In;
        J = Jn;
    }
}

__global__ void __launch_bounds__(256) features_kernel(const SchedImage *tab, int nimg, uint32_t nblocks,
                                                       float *out) {
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nblocks; b += nw) {
        const int k = find_image(tab, nimg, b, [](const SchedImage &s) { return s.block_base; });
        const SchedImage im = tab[k];
        const uint32_t lb = b - im.block_base;
        const int y0 = (lb / im.nbx) * kBlk, x0 = (lb % im.nbx) * kBlk;
        const int ye = min(im.H, y0 + kBlk), xe = min(im.W, x0 + kBlk);
        const uint32_t M = im.u16 ? 0xFFFFu : 0xFFu;
        const uint32_t thr = 16u * (M / 255u);
        const bool u16 = im.u16 != 0;
        FeatAcc a;
        const size_t pitch = (size_t)im.W * (u16 ? 2 : 1);
        if (x0 + kBlk <= im.W && y0 + kBlk <= im.H && pitch % 16 == 0 &&
            ((uintptr_t)im.I & 15) == 0 && ((uintptr_t)im.J & 15) == 0) {
            if (u16) feat_block_vec<true>(im, y0, x0, thr, lane, a);
            else feat_block_vec<false>(im, y0, x0, thr, lane, a);
        } else {
        const int c = x0 + 2 * lane;
        const bool ine = c < xe, ino = c + 1 < xe, inr = c + 2 < xe;   // this pair, and the next lane's
        auto edges_of = [&](uint32_t ie, uint32_t io, uint32_t de, uint32_t dn, bool has_down) {
            // ie / io: a row's pair; de / dn: the pair below (ignored when !has_down)
            const uint32_t nxt = __shfl_down_sync(0xffffffffu, ie, 1);   // column 2c + 2
            const uint32_t gxe = ino ? (uint32_t)abs((int)io - (int)ie) : 0u;
            const uint32_t gxo = inr ? (uint32_t)abs((int)nxt - (int)io) : 0u;
            const uint32_t gye = has_down ? (uint32_t)abs((int)de - (int)ie) : 0u;
            const uint32_t gyo = has_down ? (uint32_t)abs((int)dn - (int)io) : 0u;
            if (ine) a.edges += (gxe + gye > thr);
            if (ino) a.edges += (gxo + gyo > thr);
        };
        // the sampled rows y0, y0 + kFeatRowStep, ... with the row below each (in the block)
        for (int y = y0; y < ye; y += kFeatRowStep) {
            uint32_t Ie, Io, Je, Jo, De, Do;
            const bool down = y + 1 < ye;
            feat_load(im, im.I, y, c, Ie, Io);
            feat_load(im, im.J, y, c, Je, Jo);
            feat_load(im, im.I, down ? y + 1 : y, c, De, Do);
            if (ine) feat_pixel(a, Ie, Je, u16);
            if (ino) feat_pixel(a, Io, Jo, u16);
            edges_of(Ie, Io, De, Do, down);
        }
        a.npix = (uint32_t)(ye - y0) * ((uint32_t)ine + (uint32_t)ino);
        }

        uint32_t v[16];
        unsigned long long sI2, sJ2;
        feat_reduce(a, v, sI2, sJ2);
        if (lane < kNF) out[(size_t)b * kNF + lane] = block_feature(lane, v, sI2, sJ2, M);
    }
}

// ---- MLP: forward ---------------------------------------------------------------------------
// One thread per sample; the parameters sit in shared memory (read as broadcasts).
__device__ __forceinline__ void mlp_hidden(const float *P, const float (&x)[kNF], float (&h1)[kH],
                                           float (&h2)[kH]) {
#pragma unroll
    for (int j = 0; j < kH; j++) {
        float a = P[ob1 + j];
#pragma unroll
        for (int i = 0; i < kNF; i++) a = fmaf(x[i], P[oW1 + i * kH + j], a);
        h1[j] = fmaxf(a, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kH; j++) {
        float a = P[ob2 + j];
#pragma unroll
        for (int i = 0; i < kH; i++) a = fmaf(h1[i], P[oW2 + i * kH + j], a);
        h2[j] = fmaxf(a, 0.f);
    }
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const float *params, const float *X, int64_t N,
                                                          float *Y) {
    __shared__ float P[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        float x[kNF], h1[kH], h2[kH];
#pragma unroll
        for (int i = 0; i < kNF; i++) x[i] = X[s * kNF + i];
        mlp_hidden(P, x, h1, h2);
        float y0 = P[ob3], y1 = P[ob3 + 1];
#pragma unroll 8
        for (int i = 0; i < kH; i++) {
            y0 = fmaf(h2[i], P[oW3 + i * 2], y0);
            y1 = fmaf(h2[i], P[oW3 + i * 2 + 1], y1);
        }
        Y[s * 2] = y0;
        Y[s * 2 + 1] = y1;
    }
}

// ---- MLP: gradient of one minibatch ---------------------------------------------------------
// Loss (1/B) sum_s sum_k w_k (y_sk - t_sk)^2 over the minibatch, sample s = idx(i) of an
// affine permutation of [0, N). Each thread backpropagates one sample; every parameter's
// contributions are summed over the warp with shuffles and added to `grad` once per warp.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(128) mlp_grad_kernel(const float *params, const float *X, const float *T,
                                                       int64_t N, int64_t first, int batch, uint64_t pa,
                                                       uint64_t pb, float w0, float w1, float *grad) {
    __shared__ float P[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // position in the minibatch
    const bool valid = i < batch && first + i < N;
    int64_t s = 0;
    if (valid) s = (int64_t)((pa * (uint64_t)(first + i) + pb) % (uint64_t)N);
    float x[kNF], h1[kH], h2[kH];
#pragma unroll
    for (int q = 0; q < kNF; q++) x[q] = valid ? X[s * kNF + q] : 0.f;
    mlp_hidden(P, x, h1, h2);
    float y0 = P[ob3], y1 = P[ob3 + 1];
#pragma unroll 8
    for (int q = 0; q < kH; q++) {
        y0 = fmaf(h2[q], P[oW3 + q * 2], y0);
        y1 = fmaf(h2[q], P[oW3 + q * 2 + 1], y1);
    }
    const float invB = 1.f / (float)batch;
    const float dy0 = valid ? 2.f * w0 * (y0 - T[s * 2]) * invB : 0.f;
    const float dy1 = valid ? 2.f * w1 * (y1 - T[s * 2 + 1]) * invB : 0.f;
    // layer 3
    float g;
    g = warp_sum(dy0);
    if (lane == 0) atomicAdd(grad + ob3, g);
    g = warp_sum(dy1);
    if (lane == 0) atomicAdd(grad + ob3 + 1, g);
    for (int q = 0; q < kH; q++) {
        g = warp_sum(h2[q] * dy0);
        if (lane == 0) atomicAdd(grad + oW3 + q * 2, g);
        g = warp_sum(h2[q] * dy1);
        if (lane == 0) atomicAdd(grad + oW3 + q * 2 + 1, g);
    }
    // dh2 overwrites h2
#pragma unroll 8
    for (int q = 0; q < kH; q++)
        h2[q] = h2[q] > 0.f ? dy0 * P[oW3 + q * 2] + dy1 * P[oW3 + q * 2 + 1] : 0.f;
    // layer 2: dW2[a][b] = h1[a] dh2[b], db2 = dh2
    for (int b = 0; b < kH; b++) {
        g = warp_sum(h2[b]);
        if (lane == 0) atomicAdd(grad + ob2 + b, g);
    }
    for (int a = 0; a < kH; a++) {
        for (int b = 0; b < kH; b++) {
            g = warp_sum(h1[a] * h2[b]);
            if (lane == 0) atomicAdd(grad + oW2 + a * kH + b, g);
        }
    }
    // dh1 (one unit at a time) and layer 1
    for (int a = 0; a < kH; a++) {
        float dh = 0.f;
        if (h1[a] > 0.f) {
#pragma unroll 8
            for (int b = 0; b < kH; b++) dh = fmaf(h2[b], P[oW2 + a * kH + b], dh);
        }
        g = warp_sum(dh);
        if (lane == 0) atomicAdd(grad + ob1 + a, g);
#pragma unroll
        for (int q = 0; q < kNF; q++) {
            g = warp_sum(x[q] * dh);
            if (lane == 0) atomicAdd(grad + oW1 + q * kH + a, g);
        }
    }
}

// ---- Adam (Kingma & Ba, 2015), bias-corrected; zeroes the gradient it consumed ---------------
__global__ void adam_kernel(float *params, float *m, float *v, float *grad, int64_t t, float lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i];
    grad[i] = 0.f;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace iwpp

namespace iwpp {

// ---- schedule: predicted work -> tile order and sweep counts ---------------------------------
// key(t) = bucket of the predicted log-work of tile t's feature block; the counting sort
// lists buckets from the largest key down, so tiles come out largest-first.
__device__ __forceinline__ void tile_block(const SchedImage *tab, int nimg, uint32_t t, int th, int tw,
                                           uint32_t &block) {
    const int k = find_image(tab, nimg, t, [](const SchedImage &s) { return s.tile_base; });
    const SchedImage &im = tab[k];
    const uint32_t lt = t - im.tile_base;
    const int ty = lt / im.tiles_x, tx = lt % im.tiles_x;
    block = im.block_base + (uint32_t)((ty * th) / kBlk) * im.nbx + (uint32_t)((tx * tw) / kBlk);
}

__global__ void sched_keys_kernel(const SchedImage *tab, int nimg, uint32_t ntiles, int th, int tw,
                                  const float *Y, uint16_t *key, uint8_t *sweeps, uint32_t *hist) {
    __shared__ uint32_t h[kBuckets];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        uint32_t b;
        tile_block(tab, nimg, t, th, tw, b);
        const float w = Y[(size_t)b * 2], s = Y[(size_t)b * 2 + 1];
        int kb = (int)(w * kKeyScale);
        kb = kb < 0 ? 0 : (kb >= kBuckets ? kBuckets - 1 : kb);
        const int desc = kBuckets - 1 - kb;   // ascending in desc = largest work first
        key[t] = (uint16_t)desc;
        int sw = (int)rintf(s);
        sweeps[t] = (uint8_t)(sw < 0 ? 0 : (sw > 8 ? 8 : sw));
        atomicAdd(&h[desc], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

__global__ void sched_scan_kernel(uint32_t *hist) {   // exclusive scan, one block of kBuckets threads
    __shared__ uint32_t s[kBuckets];
    const int i = threadIdx.x;
    s[i] = hist[i];
    __syncthreads();
    for (int o = 1; o < kBuckets; o <<= 1) {
        const uint32_t v = i >= o ? s[i - o] : 0u;
        __syncthreads();
        s[i] += v;
        __syncthreads();
    }
    hist[i] = s[i] - hist[i];
}

// Scatter tiles to their bucket's next slots. Lanes with the same key share one atomic
// (many tiles fall into few buckets), and keep their lane order inside the group. Tiles are
// taken in the spread order (iwpp_spread.h), so that inside a bucket tiles next to each other
// in an image are far apart: tiles of similar predicted work lie close together, and a
// bucket in tile-id order would hand neighbours to concurrent workers (measured: an order by
// buckets in tile-id order needs as many visits as no order at all).
__global__ void sched_scatter_kernel(uint32_t ntiles, const uint16_t *key, uint32_t *cursor, uint32_t *order,
                                     uint32_t spread) {
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;   // a multiple of 32: t0 stays warp-uniform
    for (uint32_t t0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; t0 < ntiles; t0 += stride) {
        const bool valid = t0 + lane < ntiles;
        const uint32_t t = valid ? spread_tile(t0 + lane, ntiles, spread) : 0u;
        const uint32_t k = valid ? key[t] : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (lane == leader && valid) slot = atomicAdd(cursor + k, (uint32_t)__popc(peers));
        slot = __shfl_sync(0xffffffffu, slot, leader);
        if (valid) order[slot + __popc(peers & ((1u << lane) - 1u))] = t;
    }
}

// Per-tile work (pops or passes, cycles) summed into feature blocks: out[b] = pops or passes,
// out[nblocks + b] = cycles.
__global__ void tile_work_blocks_kernel(const SchedImage *tab, int nimg, uint32_t ntiles, uint32_t nblocks, int th,
                                        int tw, const uint32_t *tile_work, unsigned long long *out) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        uint32_t b;
        tile_block(tab, nimg, t, th, tw, b);
        atomicAdd(out + b, (unsigned long long)tile_work[t]);
        atomicAdd(out + nblocks + b, (unsigned long long)tile_work[ntiles + t]);
    }
}

// ---- host side -------------------------------------------------------------------------------
// Scheduling workspace: image table | features [nblocks][16] | predictions [nblocks][2] |
// keys [ntiles] | bucket histogram / cursors [kBuckets].
struct SchedLayout {
    size_t table, feats, preds, keys, hist, total;
    uint32_t nblocks, ntiles;
};

static int64_t count_blocks(const iwpp_image *imgs, int n, std::vector<uint32_t> *bases) {
    if (!imgs || n < 1) return -1;
    uint64_t tot = 0;
    if (bases) bases->resize(n);
    for (int i = 0; i < n; i++) {
        if (imgs[i].H < 1 || imgs[i].W < 1) return -1;
        if (bases) (*bases)[i] = (uint32_t)tot;
        tot += (uint64_t)((imgs[i].H + kBlk - 1) / kBlk) * (uint64_t)((imgs[i].W + kBlk - 1) / kBlk);
        if (tot >= (1ull << 31)) return -1;
    }
    return (int64_t)tot;
}

static bool sched_layout(const iwpp_image *imgs, int n, const iwpp_plan &p, SchedLayout &L,
                         std::vector<uint32_t> *bb, std::vector<uint32_t> *tb) {
    const int64_t nb = count_blocks(imgs, n, bb);
    const int64_t nt = batch_tiles(imgs, n, p, tb);
    if (nb < 1 || nt < 1) return false;
    if (p.tile_h > kBlk || p.tile_w > kBlk || kBlk % p.tile_h || kBlk % p.tile_w) return false;
    L.nblocks = (uint32_t)nb;
    L.ntiles = (uint32_t)nt;
    L.table = 0;
    L.feats = align256((size_t)n * sizeof(SchedImage));
    L.preds = L.feats + align256((size_t)L.nblocks * kNF * 4);
    L.keys = L.preds + align256((size_t)L.nblocks * 2 * 4);
    L.hist = L.keys + align256((size_t)L.ntiles * 2);
    L.total = L.hist + align256((size_t)kBuckets * 4);
    return true;
}

static int upload_table(const iwpp_image *imgs, int n, const iwpp_plan &p, const std::vector<uint32_t> &bb,
                        const std::vector<uint32_t> &tb, SchedImage *table, cudaStream_t stream) {
    for (int first = 0; first < n; first += kSchedChunk) {
        SchedChunk c;
        c.first = first;
        c.count = n - first < kSchedChunk ? n - first : kSchedChunk;
        for (int j = 0; j < c.count; j++) {
            const iwpp_image &d = imgs[first + j];
            SchedImage &s = c.v[j];
            s.J = static_cast<const uint8_t *>(d.marker_inout);
            s.I = static_cast<const uint8_t *>(d.mask);
            s.H = (int)d.H;
            s.W = (int)d.W;
            s.nbx = (int)((d.W + kBlk - 1) / kBlk);
            s.nby = (int)((d.H + kBlk - 1) / kBlk);
            s.tiles_x = (int)((d.W + p.tile_w - 1) / p.tile_w);
            s.tiles_y = (int)((d.H + p.tile_h - 1) / p.tile_h);
            s.block_base = bb[first + j];
            s.tile_base = tb[first + j];
            s.u16 = d.dtype == IWPP_U16;
            s.flip = d.op == IWPP_ERODE ? (s.u16 ? 0xFFFFu : 0xFFu) : 0u;
        }
        upload_sched_kernel<<<1, kSchedChunk, 0, stream>>>(table, c);
    }
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

static int grid_for(uint64_t work, int per_block, int cap_per_sm) {
    const int sms = device_sm_count();
    uint64_t g = (work + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * cap_per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// phases: 1 = features, 2 = MLP forward, 4 = schedule from predictions
static int schedule_impl(const iwpp_image *imgs, int n, const iwpp_plan *plan_in, const float *params,
                         const float *preds_in, float *feats_out, uint32_t *order, uint8_t *sweeps, void *sws,
                         size_t sws_bytes, cudaStream_t stream, int phases) {
    iwpp_plan p;
    if (plan_in) p = *plan_in; else default_batch_plan(&p);
    if (!plan_valid(p) || !sws || ((uintptr_t)sws & 255)) return IWPP_ERR_ARG;
    for (int i = 0; i < n; i++)
        if (!imgs || batch_tiles(imgs + i, 1, p, nullptr) < 1) return IWPP_ERR_ARG;
    std::vector<uint32_t> bb, tb;
    SchedLayout L;
    if (!sched_layout(imgs, n, p, L, &bb, &tb)) return IWPP_ERR_ARG;
    if (sws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    uint8_t *base = static_cast<uint8_t *>(sws);
    SchedImage *table = reinterpret_cast<SchedImage *>(base + L.table);
    float *feats = feats_out ? feats_out : reinterpret_cast<float *>(base + L.feats);
    float *preds = reinterpret_cast<float *>(base + L.preds);
    if (upload_table(imgs, n, p, bb, tb, table, stream) != IWPP_OK) return IWPP_ERR_CUDA;
    if (phases & 1) features_kernel<<<grid_for(L.nblocks, 8, 8), 256, 0, stream>>>(table, n, L.nblocks, feats);
    if (phases & 2) {
        if (!params) return IWPP_ERR_ARG;
        mlp_forward_kernel<<<grid_for(L.nblocks, 256, 4), 256, 0, stream>>>(params, feats, L.nblocks, preds);
    }
    if (phases & 4) {
        if (!order || !sweeps) return IWPP_ERR_ARG;
        const float *Y = (phases & 2) ? preds : preds_in;
        if (!Y) return IWPP_ERR_ARG;
        uint32_t *hist = reinterpret_cast<uint32_t *>(base + L.hist);
        uint16_t *keys = reinterpret_cast<uint16_t *>(base + L.keys);
        if (cudaMemsetAsync(hist, 0, kBuckets * 4, stream) != cudaSuccess) return IWPP_ERR_CUDA;
        const int g = grid_for(L.ntiles, 256, 8);
        sched_keys_kernel<<<g, 256, 0, stream>>>(table, n, L.ntiles, p.tile_h, p.tile_w, Y, keys, sweeps, hist);
        sched_scan_kernel<<<1, kBuckets, 0, stream>>>(hist);
        sched_scatter_kernel<<<g, 256, 0, stream>>>(L.ntiles, keys, hist, order, spread_multiplier(L.ntiles));
    }
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

float *sched_features(const iwpp_image *imgs, int n, const iwpp_plan &p, void *sws, size_t sws_bytes) {
    SchedLayout L;
    if (!sws || ((uintptr_t)sws & 255) || !sched_layout(imgs, n, p, L, nullptr, nullptr) || sws_bytes < L.total)
        return nullptr;
    return reinterpret_cast<float *>(static_cast<uint8_t *>(sws) + L.feats);
}

int schedule_batch(const iwpp_image *imgs, int n, const iwpp_plan &p, const float *params, uint32_t *order,
                   uint8_t *sweeps, void *sws, size_t sws_bytes, cudaStream_t stream, int phases) {
    return schedule_impl(imgs, n, &p, params, nullptr, nullptr, order, sweeps, sws, sws_bytes, stream, phases);
}

}  // namespace iwpp

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" int64_t iwpp_batch_block_count(const iwpp_image *imgs, int n) {
    return iwpp::count_blocks(imgs, n, nullptr);
}

extern "C" int64_t iwpp_sched_features_offset(const iwpp_image *imgs, int n, const iwpp_plan *plan) {
    iwpp_plan p;
    if (plan) p = *plan; else iwpp::default_batch_plan(&p);
    if (!iwpp::plan_valid(p)) return -1;
    iwpp::SchedLayout L;
    return iwpp::sched_layout(imgs, n, p, L, nullptr, nullptr) ? (int64_t)L.feats : -1;
}

extern "C" size_t iwpp_sched_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan) {
    iwpp_plan p;
    if (plan) p = *plan; else iwpp::default_batch_plan(&p);
    if (!iwpp::plan_valid(p)) return 0;
    iwpp::SchedLayout L;
    return iwpp::sched_layout(imgs, n, p, L, nullptr, nullptr) ? L.total : 0;
}

extern "C" int iwpp_batch_features(const iwpp_image *imgs, int n, float *feats, void *sched_ws, size_t sws_bytes,
                                   void *stream) {
    if (!feats) return IWPP_ERR_ARG;
    return iwpp::schedule_impl(imgs, n, nullptr, nullptr, nullptr, feats, nullptr, nullptr, sched_ws, sws_bytes,
                               static_cast<cudaStream_t>(stream), 1);
}

extern "C" int iwpp_schedule_from_predictions(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                              const float *preds, uint32_t *tile_order, uint8_t *tile_sweeps,
                                              void *sched_ws, size_t sws_bytes, void *stream) {
    return iwpp::schedule_impl(imgs, n, plan, nullptr, preds, nullptr, tile_order, tile_sweeps, sched_ws, sws_bytes,
                               static_cast<cudaStream_t>(stream), 4);
}

extern "C" int iwpp_schedule_learned(const iwpp_image *imgs, int n, const iwpp_plan *plan, const float *params,
                                     uint32_t *tile_order, uint8_t *tile_sweeps, void *sched_ws, size_t sws_bytes,
                                     void *stream) {
    return iwpp::schedule_impl(imgs, n, plan, params, nullptr, nullptr, tile_order, tile_sweeps, sched_ws,
                               sws_bytes, static_cast<cudaStream_t>(stream), 7);
}

extern "C" int iwpp_mlp_forward(const float *params, const float *X, int64_t N, float *Y, void *stream) {
    if (!params || !X || !Y || N < 0) return IWPP_ERR_ARG;
    if (N == 0) return IWPP_OK;
    iwpp::mlp_forward_kernel<<<iwpp::grid_for((uint64_t)N, 256, 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        params, X, N, Y);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

extern "C" int iwpp_mlp_train(float *params, float *adam_m, float *adam_v, float *grad, const float *X,
                              const float *T, int64_t N, int epochs, int batch, float lr, float w0, float w1,
                              uint64_t seed, int64_t step0, void *stream) {
    if (!params || !adam_m || !adam_v || !grad || !X || !T || N < 1 || epochs < 0 || batch < 1 || batch > 65536)
        return IWPP_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t step = step0;
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    for (int e = 0; e < epochs; e++) {
        // a fresh affine permutation s(i) = (a i + b) mod N per epoch, with gcd(a, N) = 1
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        uint64_t a = (st >> 17) % (uint64_t)N;
        if (a == 0) a = 1;
        auto gcd = [](uint64_t x, uint64_t y) { while (y) { uint64_t r = x % y; x = y; y = r; } return x; };
        while (gcd(a, (uint64_t)N) != 1) a = a + 1 < (uint64_t)N ? a + 1 : 1;
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        const uint64_t b = (st >> 13) % (uint64_t)N;
        for (int64_t first = 0; first < N; first += batch) {
            const int bsz = (int)(N - first < batch ? N - first : batch);
            iwpp::mlp_grad_kernel<<<(bsz + 127) / 128, 128, 0, s>>>(params, X, T, N, first, bsz, a, b, w0, w1, grad);
            iwpp::adam_kernel<<<(iwpp::kNP + 255) / 256, 256, 0, s>>>(params, adam_m, adam_v, grad, ++step, lr);
        }
    }
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

extern "C" int iwpp_tile_work_to_blocks(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                        const uint32_t *tile_work, unsigned long long *block_work, void *sched_ws,
                                        size_t sws_bytes, void *stream) {
    iwpp_plan p;
    if (plan) p = *plan; else iwpp::default_batch_plan(&p);
    if (!iwpp::plan_valid(p) || !tile_work || !block_work || !sched_ws) return IWPP_ERR_ARG;
    std::vector<uint32_t> bb, tb;
    iwpp::SchedLayout L;
    if (!iwpp::sched_layout(imgs, n, p, L, &bb, &tb)) return IWPP_ERR_ARG;
    if (sws_bytes < L.total) return IWPP_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    iwpp::SchedImage *table = reinterpret_cast<iwpp::SchedImage *>(sched_ws);
    if (iwpp::upload_table(imgs, n, p, bb, tb, table, s) != IWPP_OK) return IWPP_ERR_CUDA;
    iwpp::tile_work_blocks_kernel<<<iwpp::grid_for(L.ntiles, 256, 8), 256, 0, s>>>(table, n, L.ntiles, L.nblocks,
                                                                                  p.tile_h, p.tile_w, tile_work,
                                                                                  block_work);
    return cudaGetLastError() == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

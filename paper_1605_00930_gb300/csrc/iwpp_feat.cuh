// iwpp_feat.cuh — the learned work estimator's per-block features (include/iwpp.h): the
// per-pixel accumulation and the conversion of a block's exact integer sums to the 16 FP32
// inputs of the MLP. Shared by the stand-alone features kernel (iwpp_sched.cu) and the
// streaming scan kernel, which computes the features of the tile it streams through
// (iwpp_scan.cuh), so that both give identical values.
//
// Per 64 x 64 block, in the dilation domain (erosion: both images complemented), with
// d = max(I - J, 0) and d8 = d (u8) or d >> 8 (u16); f[0..14] over every kFeatRowStep-th row
// of the block (its rows 0, 4, 8, ...: the sampled pixels, a quarter of the arithmetic):
//   f[0..7]   histogram of d8: bin 0 = 0, bin k = bit length of d8 (1..6), bin 7 = d8 >= 64
//   f[8]      fraction of pixels with J == I > 0
//   f[9]      fraction with |I(p) - I(p + x)| + |I(p) - I(p + y)| > 16 MAXV / 255 (a neighbour
//             outside the block contributes 0; p + y is the next row, sampled or not)
//   f[10..14] mean(I), std(I), mean(J), std(J), mean(d), each divided by MAXV
//   f[15]     log2(pixels in the block, every row) / 12
#pragma once
#include <cstdint>

namespace iwpp {

constexpr int kFeatRowStep = 4;   // the sampled rows of a block: 0, 4, 8, ...

struct FeatAcc {
    uint32_t h03 = 0, h47 = 0;   // histogram bins, 8 bits each
    uint32_t seeds = 0, edges = 0, sI = 0, sJ = 0, sD = 0, n = 0;   // n: sampled pixels
    uint32_t npix = 0;           // pixels of the block (every row)
    unsigned long long sI2 = 0, sJ2 = 0;
};

__device__ __forceinline__ void feat_pixel(FeatAcc &a, uint32_t i, uint32_t j, bool u16) {
    const uint32_t d = i > j ? i - j : 0u;
    const uint32_t d8 = u16 ? d >> 8 : d;
    const uint32_t bin = d8 == 0 ? 0u : min(7u, 32u - (uint32_t)__clz(d8));
    const uint32_t inc = 1u << (8 * (bin & 3));
    if (bin < 4) a.h03 += inc; else a.h47 += inc;
    a.seeds += (i == j && j > 0);
    a.sI += i;
    a.sJ += j;
    a.sD += d;
    a.sI2 += (unsigned long long)i * i;
    a.sJ2 += (unsigned long long)j * j;
    a.n++;
}

// Sums of a block: v[0..7] histogram, v[8] seeds, v[9] edges, v[10] sum I, v[12] sum J,
// v[14] sum d, v[15] sampled pixel count, v[13] the block's pixel count (v[11] unused);
// sI2 / sJ2 the sums of squares.
// Feature k in FP32 from exact integers (FP64 is slow on this part): the variance numerator
// N * sum(x^2) - sum(x)^2 is exact in 64 bits (N <= 4096, x <= 65535), so no cancellation;
// every feature is within a few float ulps of the exact value.
__device__ __forceinline__ float block_feature(int k, const uint32_t (&v)[16], unsigned long long sI2,
                                               unsigned long long sJ2, uint32_t M) {
    const uint32_t N = v[15];
    const float fN = (float)N, NM = (float)N * (float)M;
    uint32_t vk = 0;   // v[k] without a dynamic index (which would put v in local memory)
#pragma unroll
    for (int q = 0; q < 16; q++) vk = q == k ? v[q] : vk;
    switch (k) {
        case 10: return (float)v[10] / NM;
        case 11: return sqrtf((float)((unsigned long long)N * sI2 - (unsigned long long)v[10] * v[10])) / NM;
        case 12: return (float)v[12] / NM;
        case 13: return sqrtf((float)((unsigned long long)N * sJ2 - (unsigned long long)v[12] * v[12])) / NM;
        case 14: return (float)v[14] / NM;
        case 15: return log2f((float)v[13]) / 12.f;
        default: return (float)vk / fN;   // histogram, seeds, edges
    }
}

// Warp-wide sums of each lane's FeatAcc into v / sI2 / sJ2 (every lane ends with them).
__device__ __forceinline__ void feat_reduce(const FeatAcc &a, uint32_t (&v)[16], unsigned long long &sI2,
                                            unsigned long long &sJ2) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
        v[q] = __reduce_add_sync(0xffffffffu, (a.h03 >> (8 * q)) & 0xFFu);
        v[4 + q] = __reduce_add_sync(0xffffffffu, (a.h47 >> (8 * q)) & 0xFFu);
    }
    v[8] = __reduce_add_sync(0xffffffffu, a.seeds);
    v[9] = __reduce_add_sync(0xffffffffu, a.edges);
    v[10] = __reduce_add_sync(0xffffffffu, a.sI);   // < 2^32: 4096 pixels x 65535
    v[11] = 0;
    v[12] = __reduce_add_sync(0xffffffffu, a.sJ);
    v[13] = __reduce_add_sync(0xffffffffu, a.npix);
    v[14] = __reduce_add_sync(0xffffffffu, a.sD);
    v[15] = __reduce_add_sync(0xffffffffu, a.n);
    sI2 = a.sI2;
    sJ2 = a.sJ2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // butterfly: every lane ends with the sums
        sI2 += __shfl_xor_sync(0xffffffffu, sI2, o);
        sJ2 += __shfl_xor_sync(0xffffffffu, sJ2, o);
    }
}

}  // namespace iwpp

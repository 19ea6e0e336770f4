// iwpp_spread.h — the spread order of a batch's initial frontier (host and device).
//
// A permutation of [0, n) that spreads consecutive positions apart: i -> (i * mul) mod n,
// with mul odd, coprime with n and near 0.618 n. Tiles next to each other in an image, which
// a queue in tile-id order hands to concurrent workers, land far apart in the queue.
#pragma once
#include <cstdint>

namespace iwpp {

#if defined(__CUDACC__)
#define IWPP_HD __host__ __device__
#else
#define IWPP_HD
#endif

IWPP_HD inline uint32_t spread_tile(uint64_t i, uint32_t n, uint32_t mul) {
    return mul ? (uint32_t)((i * (uint64_t)mul) % n) : (uint32_t)i;
}

// The multiplier for n positions (1 below 3: the identity).
inline uint32_t spread_multiplier(uint32_t n) {
    if (n < 3) return 1;
    uint64_t m = ((uint64_t)n * 40503u >> 16) | 1u;   // ~0.618 n (40503 / 65536), odd
    auto gcd = [](uint64_t a, uint64_t b) {
        while (b) {
            const uint64_t t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    while (gcd(m, n) != 1) m += 2;
    return (uint32_t)(m % n);
}

#undef IWPP_HD

}  // namespace iwpp

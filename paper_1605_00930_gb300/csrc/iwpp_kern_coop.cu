// iwpp_kern_coop.cu — instantiations of the cooperative local solver's kernels (one
// translation unit of their own, compiled in parallel with the others).
#include "iwpp_host.h"
#include "iwpp_coop.cuh"
#include "iwpp_scan.cuh"

namespace iwpp {

#ifndef IWPP_SCAN_STREAM
#define IWPP_SCAN_STREAM 1   // 0: the strip scan for every build (measured)
#endif

template <typename T, int CONN, bool MIXED = false>
static RegKernelSet coop_set() {
    RegKernelSet k;
    // the streaming scan for builds of one connectivity; the mixed-kind build switches kinds
    // per strip in the strip scan
    if constexpr (MIXED || !IWPP_SCAN_STREAM) k.scan = scan_strip_coop_kernel<T, CONN, MIXED>;
    else k.scan = scan_stream_kernel<T, CONN, false>;
    k.drain = drain_coop_kernel<T, CONN, MIXED>;
    k.drain_hi = nullptr;   // one build of the persistent kernel
    k.smem = &coop_smem_fn<T, CONN>;
    k.scan_sweeps = scan_coop_kernel<T, CONN, MIXED, true>;
    // features in the scan: not for the mixed-kind build
    if constexpr (MIXED) k.scan_feats = nullptr;
    else k.scan_feats = scan_stream_kernel<T, CONN, true>;
    return k;
}

RegKernelSet coop_kernel_set(int th, int tw, int v) {
    RegKernelSet none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (th != kCoopRows || tw != RegTile<uint8_t, 8, kCoopStrip>::TW) return none;
    switch (v) {
        case 0: return coop_set<uint8_t, 4>();
        case 1: return coop_set<uint16_t, 4>();
        case 2: return coop_set<uint8_t, 8>();
        case 3: return coop_set<uint16_t, 8>();
        case 4: return coop_set<uint16_t, 8, true>();   // mixed batches
        case 5: return coop_set<AnyPix, 4>();           // u8 and u16 images, 4-connectivity
        case 6: return coop_set<AnyPix, 8>();           // u8 and u16 images, 8-connectivity
        default: return none;
    }
}

}  // namespace iwpp

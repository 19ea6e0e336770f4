// iwpp_kern_reg.cu — instantiations of the register local solver's kernels (one
// translation unit of their own, so they compile in parallel with the queue solver's).
#include "iwpp_host.h"
#include "iwpp_regtile.cuh"

namespace iwpp {

template <typename T, int CONN, int TH, int LO = kRegBlocks, int HI = kRegHiBlocks>
static RegKernelSet reg_set() {
    RegKernelSet k;
    k.scan = scan_reg_kernel<T, CONN, TH>;
    k.drain = drain_reg_kernel<T, CONN, TH, LO>;
    k.drain_hi = drain_reg_kernel<T, CONN, TH, HI>;
    k.smem = &RegTile<T, CONN, TH>::smem_bytes;
    k.scan_sweeps = nullptr;
    k.scan_feats = nullptr;
    return k;
}

RegKernelSet reg_kernel_set(int th, int tw, int v) {
    RegKernelSet none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (th != 16 || tw != RegTile<uint8_t, 8, 16>::TW) return none;
    switch (v) {
        case 0: return reg_set<uint8_t, 4, 16>();
        case 1: return reg_set<uint16_t, 4, 16>();
        case 2: return reg_set<uint8_t, 8, 16>();
        case 3: return reg_set<uint16_t, 8, 16>();
        case 4: {
            RegKernelSet k;
            k.scan = scan_reg_mixed_kernel<16>;
            k.drain = drain_reg_mixed_kernel<16, kRegBlocks>;
            k.drain_hi = drain_reg_mixed_kernel<16, kRegHiBlocks>;
            k.smem = &RegTile<uint16_t, 8, 16>::smem_bytes;
            k.scan_sweeps = nullptr;
            k.scan_feats = nullptr;
            return k;
        }
        default: return none;
    }
}

}  // namespace iwpp

#if IWPP_TRACE
// Measurement builds only: copy out and reset the visit trace of the register solver
// (hist: uint32[16384] visits started per 10 us; returns the longest chain of tile hops).
extern "C" IWPP_API int iwpp_trace_read(unsigned int *hist_host) {
    unsigned int mg = 0;
    cudaMemcpyFromSymbol(&mg, iwpp::g_trace_maxgen, sizeof mg);
    if (hist_host) cudaMemcpyFromSymbol(hist_host, iwpp::g_trace_hist, sizeof(unsigned int) * iwpp::kTraceBins);
    static unsigned int zeros[iwpp::kTraceBins];
    cudaMemcpyToSymbol(iwpp::g_trace_hist, zeros, sizeof zeros);
    const unsigned int z = 0;
    cudaMemcpyToSymbol(iwpp::g_trace_maxgen, &z, sizeof z);
    const unsigned long long big = ~0ull;
    cudaMemcpyToSymbol(iwpp::g_trace_t0, &big, sizeof big);
    return (int)mg;
}
#endif

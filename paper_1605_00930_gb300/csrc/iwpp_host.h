// iwpp_host.h — host-side helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/iwpp.h"

namespace iwpp {
struct EngineArgs;

// Kernels of the register local solver for one tile shape and image kind (v = 0..3:
// bit 0 u16, bit 1 8-connectivity; v = 4: mixed batch). All null when the shape has none.
// drain_hi is the same persistent kernel compiled for kRegHiBlocks CTAs per SM (fewer
// registers per thread, more warps to hide latency); plans that ask for more than
// kRegBlocks CTAs per SM use it.
struct RegKernelSet {
    void (*scan)(EngineArgs);
    void (*drain)(EngineArgs);
    void (*drain_hi)(EngineArgs);
    size_t (*smem)(uint32_t);
};
constexpr int kRegBlocks = 4, kRegHiBlocks = 6;
#ifndef IWPP_COOP_MINB
#define IWPP_COOP_MINB 5
#endif
constexpr int kCoopBlocks = IWPP_COOP_MINB;   // CTAs per SM of the cooperative solver's persistent kernel
RegKernelSet reg_kernel_set(int th, int tw, int v);
RegKernelSet coop_kernel_set(int th, int tw, int v);   // cooperative solver (64 x 64 tiles)

int shape_index(int th, int tw);
bool plan_valid(const iwpp_plan &p);
void default_plan(iwpp_plan *p);         // single images
void default_batch_plan(iwpp_plan *p);   // batches
size_t align256(size_t x);
int device_sm_count();
int reconstruct_one(void *marker, const void *mask, int64_t H, int64_t W, int conn, int op, int dtype,
                    const iwpp_plan *plan, void *ws, size_t ws_bytes, cudaStream_t stream, int phases);
size_t workspace_bytes(int64_t H, int64_t W, int dtype, const iwpp_plan *plan);
int64_t batch_tiles(const iwpp_image *imgs, int n, const iwpp_plan &p, std::vector<uint32_t> *bases);
size_t batch_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan);
// Phases of a call: bit 0 = workspace reset + scan (batches: table upload, scan, queue
// compaction), bit 1 = persistent drain.
enum { kPhaseScan = 1, kPhaseDrain = 2 };
int reconstruct_batch(const iwpp_image *imgs, int n, const iwpp_plan *plan, const uint32_t *order,
                      const uint8_t *tile_sweeps, uint32_t *tile_work, void *ws, size_t ws_bytes,
                      cudaStream_t stream, int phases);
int batch_launches(int n, int phases);
}  // namespace iwpp

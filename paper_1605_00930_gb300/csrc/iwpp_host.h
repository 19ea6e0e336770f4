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
    void (*scan_sweeps)(EngineArgs);   // scan build that runs sweeps (null: `scan` runs them)
    void (*scan_feats)(EngineArgs);    // scan build that also writes each tile's features (or null)
};
constexpr int kRegBlocks = 4, kRegHiBlocks = 6;
#ifndef IWPP_COOP_MINB
#define IWPP_COOP_MINB 6   // 80 registers; 5 (96 registers) measured slower on batches and the seed image
#endif
constexpr int kCoopBlocks = IWPP_COOP_MINB;   // CTAs per SM of the cooperative solver's persistent kernel
#ifndef IWPP_COOP_BATCH_MINB
#define IWPP_COOP_BATCH_MINB 7   // its build for u8 + u16 batches (72 registers, ~250 B of spills)
#endif
constexpr int kCoopBatchBlocks = IWPP_COOP_BATCH_MINB;
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
// A learned batch call: the schedule (tile order, sweep counts) is made inside the call, from
// features written by the scan kernel when the plan's tiles are the feature blocks.
struct LearnedCall {
    const float *params;
    uint32_t *order;    // out: tile order, uint32[ntiles]
    uint8_t *sweeps;    // out: sweep counts, uint8[ntiles]
    void *sws;
    size_t sws_bytes;
};
int reconstruct_batch(const iwpp_image *imgs, int n, const iwpp_plan *plan, const uint32_t *order,
                      const uint8_t *tile_sweeps, uint32_t *tile_work, void *ws, size_t ws_bytes,
                      cudaStream_t stream, int phases, const LearnedCall *learned = nullptr);
int batch_launches(int n, int phases);
// The learned schedule's pieces a batch call drives (iwpp_sched.cu): the address of the
// feature array in a scheduling workspace (null if the workspace is too small), and the
// schedule itself (phases: 1 features, 2 MLP inference, 4 tile order and sweep counts).
float *sched_features(const iwpp_image *imgs, int n, const iwpp_plan &p, void *sws, size_t sws_bytes);
int schedule_batch(const iwpp_image *imgs, int n, const iwpp_plan &p, const float *params, uint32_t *order,
                   uint8_t *sweeps, void *sws, size_t sws_bytes, cudaStream_t stream, int phases);
}  // namespace iwpp

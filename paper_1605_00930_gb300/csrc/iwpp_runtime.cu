// iwpp_runtime.cu — host runtime around the batch path: CUDA-graph capture of a batch
// launch and the plan autotuner (include/iwpp.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_host.h"

struct iwpp_graph_s {
    cudaGraphExec_t exec;
};

namespace iwpp {

// Capture one batch call (static or with a device-resident schedule) into an
// executable graph. The workspace and schedule arrays are baked into the graph.
static int graph_create(const iwpp_image *imgs, int n, const iwpp_plan *plan, const uint32_t *order,
                        const uint8_t *sweeps, void *ws, size_t ws_bytes, iwpp_graph *out) {
    if (!out) return IWPP_ERR_ARG;
    *out = nullptr;
    // resolve occupancy and kernel attributes before capture starts
    if (batch_workspace_bytes(imgs, n, plan) == 0) return IWPP_ERR_ARG;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return IWPP_ERR_CUDA;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(s);
        return IWPP_ERR_CUDA;
    }
    const int rc = reconstruct_batch(imgs, n, plan, order, sweeps, nullptr, ws, ws_bytes, s, kPhaseScan | kPhaseDrain);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (rc != IWPP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess || !g) return IWPP_ERR_CUDA;
    cudaGraphExec_t exec;
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return IWPP_ERR_CUDA;
    iwpp_graph h = new iwpp_graph_s;
    h->exec = exec;
    *out = h;
    return IWPP_OK;
}

// ---- autotuner ---------------------------------------------------------------------------------
// Times candidate plans on the batch itself and keeps the fastest. Markers are backed up
// before and restored before every trial and at the end, so the caller's images are
// unchanged. Coordinate descent: local solver with its tile shape, then sweep count, then
// (register solver) CTAs per SM or (queue solver) shared queue capacity.
struct Tuner {
    const iwpp_image *imgs;
    int n;
    cudaStream_t stream;
    std::vector<void *> backup;
    std::vector<size_t> bytes;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *flush = nullptr;      // written before every trial so that no trial starts with a warm L2
    size_t flush_bytes = 0;
    int reps;

    int init() {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        flush_bytes = (size_t)(l2 > 0 ? l2 : (64 << 20)) * 2;
        if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) return IWPP_ERR_CUDA;
        backup.assign(n, nullptr);
        bytes.assign(n, 0);
        for (int i = 0; i < n; i++) {
            bytes[i] = (size_t)imgs[i].H * (size_t)imgs[i].W * (imgs[i].dtype == IWPP_U16 ? 2 : 1);
            if (cudaMalloc(&backup[i], bytes[i]) != cudaSuccess) return IWPP_ERR_CUDA;
            if (cudaMemcpyAsync(backup[i], imgs[i].marker_inout, bytes[i], cudaMemcpyDeviceToDevice, stream) !=
                cudaSuccess)
                return IWPP_ERR_CUDA;
        }
        return IWPP_OK;
    }
    int restore() {
        for (int i = 0; i < n; i++)
            if (cudaMemcpyAsync(imgs[i].marker_inout, backup[i], bytes[i], cudaMemcpyDeviceToDevice, stream) !=
                cudaSuccess)
                return IWPP_ERR_CUDA;
        return IWPP_OK;
    }
    // Best time in ms over `reps` runs, or a negative value if the plan fails.
    float time_plan(const iwpp_plan &p) {
        const size_t need = batch_workspace_bytes(imgs, n, &p);
        if (need == 0) return -1.f;
        if (need > ws_bytes) {
            if (ws) cudaFree(ws);
            ws = nullptr;
            if (cudaMalloc(&ws, need) != cudaSuccess) return -1.f;
            ws_bytes = need;
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = -1.f;
        for (int r = 0; r < reps; r++) {
            if (restore() != IWPP_OK) break;
            if (cudaMemsetAsync(flush, r & 0xFF, flush_bytes, stream) != cudaSuccess) break;
            cudaEventRecord(e0, stream);
            if (reconstruct_batch(imgs, n, &p, nullptr, nullptr, nullptr, ws, ws_bytes, stream, kPhaseScan | kPhaseDrain) !=
                IWPP_OK)
                break;
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            uint32_t st = 1;
            cudaMemcpy(&st, ws, 4, cudaMemcpyDeviceToHost);
            if (st != 0 && st != 2) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) best = ms;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return best;
    }
    ~Tuner() {
        for (void *b : backup)
            if (b) cudaFree(b);
        if (ws) cudaFree(ws);
        if (flush) cudaFree(flush);
    }
};

static std::string cache_key(const iwpp_image *imgs, int n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    double px = 0;
    int n16 = 0, n8c = 0, nero = 0;
    for (int i = 0; i < n; i++) {
        px += (double)imgs[i].H * (double)imgs[i].W;
        n16 += imgs[i].dtype == IWPP_U16;
        n8c += imgs[i].connectivity == 8;
        nero += imgs[i].op == IWPP_ERODE;
    }
    char buf[256];
    // bucket by image count and log2 of the pixel count; mix as coarse fractions
    int lp = 0;
    while ((double)(1ull << lp) < px && lp < 62) lp++;
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ') c = '_';
    snprintf(buf, sizeof buf, "%s|n%d|px2^%d|u16:%d|c8:%d|er:%d", name.c_str(), n < 8 ? n : (n < 64 ? 8 : 64), lp,
             (4 * n16 + n / 2) / n, (4 * n8c + n / 2) / n, (4 * nero + n / 2) / n);
    return std::string(buf);
}

static bool cache_lookup(const char *path, const std::string &key, iwpp_plan *p) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char k[300];
        iwpp_plan q = *p;
        if (sscanf(line, "%299s %d %d %d %d %d", k, &q.tile_h, &q.tile_w, &q.sweeps, &q.smem_queue_cap,
                   &q.local_solver) == 6 &&
            key == k && plan_valid(q)) {
            *p = q;   // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, const iwpp_plan &p) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), p.tile_h, p.tile_w, p.sweeps, p.smem_queue_cap,
            p.local_solver);
    fclose(f);
}

int autotune(const iwpp_image *imgs, int n, iwpp_plan *plan, int reps, const char *cache_path,
             cudaStream_t stream, float *best_ms) {
    if (!imgs || n < 1 || !plan) return IWPP_ERR_ARG;
    if (!plan_valid(*plan)) return IWPP_ERR_ARG;
    for (int i = 0; i < n; i++)
        if (batch_tiles(imgs + i, 1, *plan, nullptr) < 1) return IWPP_ERR_ARG;
    const std::string key = cache_key(imgs, n);
    if (cache_lookup(cache_path, key, plan)) {
        if (best_ms) *best_ms = 0.f;
        return IWPP_OK;
    }
    Tuner t;
    t.imgs = imgs;
    t.n = n;
    t.stream = stream;
    t.reps = reps < 1 ? 1 : reps;
    if (t.init() != IWPP_OK) return IWPP_ERR_CUDA;
    iwpp_plan best = *plan;
    float best_t = t.time_plan(best);
    if (best_t < 0.f) return IWPP_ERR_CUDA;
    auto consider = [&](iwpp_plan c) {
        if (!plan_valid(c)) return;
        const float ms = t.time_plan(c);
        if (ms >= 0.f && ms < best_t) {
            best_t = ms;
            best = c;
        }
    };
    // {tile_h, tile_w, local_solver}
    static const int shapes[6][3] = {{16, 64, IWPP_SOLVER_REGISTER}, {64, 64, IWPP_SOLVER_COOP},
                                     {32, 32, IWPP_SOLVER_QUEUE},    {32, 64, IWPP_SOLVER_QUEUE},
                                     {64, 64, IWPP_SOLVER_QUEUE},    {16, 64, IWPP_SOLVER_QUEUE}};
    iwpp_plan base = best;
    for (const auto &sh : shapes) {
        iwpp_plan c = base;
        c.tile_h = sh[0];
        c.tile_w = sh[1];
        c.local_solver = sh[2];
        if (c.smem_queue_cap > c.tile_h * c.tile_w) c.smem_queue_cap = c.tile_h * c.tile_w;
        if (c.tile_h == base.tile_h && c.tile_w == base.tile_w && c.local_solver == base.local_solver) continue;
        consider(c);
    }
    base = best;
    for (int sw : {0, 1, 2, 4}) {
        if (sw == base.sweeps) continue;
        iwpp_plan c = base;
        c.sweeps = sw;
        consider(c);
    }
    base = best;
    if (base.local_solver == IWPP_SOLVER_REGISTER) {   // occupancy: the high-occupancy build
        iwpp_plan c = base;
        c.blocks_per_sm = kRegHiBlocks;
        if (c.blocks_per_sm != base.blocks_per_sm) consider(c);
    }
    base = best;
    for (int qc : {128, 256, 512, 1024, 2048}) {
        if (base.local_solver != IWPP_SOLVER_QUEUE) break;   // the register solver has no queues
        if (qc == base.smem_queue_cap || qc > base.tile_h * base.tile_w) continue;
        iwpp_plan c = base;
        c.smem_queue_cap = qc;
        consider(c);
    }
    if (t.restore() != IWPP_OK) return IWPP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return IWPP_ERR_CUDA;
    *plan = best;
    if (best_ms) *best_ms = best_t;
    cache_store(cache_path, key, best);
    return IWPP_OK;
}

}  // namespace iwpp

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" int iwpp_batch_graph_create(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                       const uint32_t *tile_order, const uint8_t *tile_sweeps, void *workspace,
                                       size_t ws_bytes, iwpp_graph *out) {
    return iwpp::graph_create(imgs, n, plan, tile_order, tile_sweeps, workspace, ws_bytes, out);
}

extern "C" int iwpp_graph_launch(iwpp_graph g, void *stream) {
    if (!g) return IWPP_ERR_ARG;
    return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

extern "C" int iwpp_graph_destroy(iwpp_graph g) {
    if (!g) return IWPP_ERR_ARG;
    const cudaError_t e = cudaGraphExecDestroy(g->exec);
    delete g;
    return e == cudaSuccess ? IWPP_OK : IWPP_ERR_CUDA;
}

extern "C" int iwpp_autotune_batch(const iwpp_image *imgs, int n, iwpp_plan *plan_inout, int reps,
                                   const char *cache_path, void *stream, float *best_ms) {
    return iwpp::autotune(imgs, n, plan_inout, reps, cache_path, static_cast<cudaStream_t>(stream), best_ms);
}

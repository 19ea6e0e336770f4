/*
 * iwpp.h — C ABI of the GB300 (sm_103a) library for the Irregular Wavefront
 * Propagation Pattern (IWPP): grayscale morphological reconstruction by
 * dilation and its dual, reconstruction by erosion (fill-holes).
 *
 * What is computed (Sec. 2.1.2, Eq. "recon"; Sec. 3.1, Algorithm 7):
 *   given a mask image I and a marker image J with J <= I pixelwise, the
 *   reconstruction R is the stable point of J <- delta_G(J) ^ I, where delta_G
 *   is the elementary dilation over the 4- or 8-neighbourhood G restricted to
 *   the image and ^ is the pixelwise minimum. op = IWPP_ERODE computes the dual,
 *   the stable point of J <- eps_G(J) v I from a marker J >= I; with
 *   J = I on the image border and the maximum value inside, that is the
 *   fill-holes operator of Sec. 3.3. The result is unique, so it does not
 *   depend on the order in which the library propagates values.
 *
 * Conventions shared by every call:
 *   - Images are row-major and contiguous (pitch = W elements), u8 or u16,
 *     in DEVICE memory, base address 16-byte aligned. The caller owns them.
 *   - marker_inout holds J on entry and R on exit (the paper's J is both
 *     input and output). mask is only read.
 *   - 1 <= H, W < 2^31 and H * W < 2^40 per image (a 100000 x 100000 image is
 *     fine; the device must hold it); connectivity is 4 or 8 (the
 *     hexagonal 6-connectivity that Sec. 2.1.2 also names is not supported).
 *   - The workspace is caller-owned device memory of at least the size the
 *     matching *_workspace_bytes call returns, 256-byte aligned. The library
 *     allocates nothing on these paths and keeps no device state between calls.
 *     Calls on different streams are safe when their workspaces and images
 *     differ.
 *   - Host-detectable errors return at once with nothing enqueued. Errors the
 *     device finds (precondition violation, queue exhaustion, watchdog timeout)
 *     are written to a status word inside the workspace; read it with
 *     iwpp_sync_status. When it reports IWPP_ERR_PRECONDITION the output is
 *     unspecified.
 *   - All calls are asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) and perform no host synchronisation, except
 *     iwpp_sync_status, iwpp_work_counters and iwpp_autotune_batch.
 */
#ifndef IWPP_H
#define IWPP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IWPP_API __attribute__((visibility("default")))
#else
#define IWPP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { IWPP_U8 = 0, IWPP_U16 = 1 } iwpp_dtype;
typedef enum { IWPP_DILATE = 0, IWPP_ERODE = 1 } iwpp_op;

typedef enum {
    IWPP_OK = 0,
    IWPP_ERR_ARG = 1,          /* bad argument (null, size, enum, alignment)  */
    IWPP_ERR_PRECONDITION = 2, /* marker > mask (dilate) / marker < mask (erode) somewhere */
    IWPP_ERR_WORKSPACE = 3,    /* workspace missing, misaligned or too small   */
    IWPP_ERR_QUEUE_FULL = 4,   /* a propagation queue ran out of room          */
    IWPP_ERR_TIMEOUT = 5,      /* the persistent kernel's watchdog expired     */
    IWPP_ERR_CUDA = 6,         /* a CUDA runtime call failed                   */
    IWPP_ERR_INTERNAL = 7      /* an internal consistency check failed         */
} iwpp_status;

/*
 * Execution plan: the knobs of the propagation engine. None of them can change
 * the result (the reconstruction is unique); they change only the work done.
 *   tile_h, tile_w     tile shape, one warp per tile; must be one of the
 *                      compiled shapes (32x32, 32x64, 64x64, 16x32, 16x64 — see
 *                      iwpp_tile_shape_supported)
 *   sweeps             raster + anti-raster sweep pairs run over every tile
 *                      before the queue phase (Algorithm 7's scanning phase,
 *                      tile-local); 0 = queue mode from the start
 *   revisit_sweeps     sweep pairs run at the start of every first visit of
 *                      a tile by the persistent kernel (normally 0)
 *   smem_queue_cap     entries of each of the two shared-memory wave queues
 *                      of a warp; waves larger than this spill into the
 *                      warp's global overflow queue (16 .. tile_h * tile_w)
 *   blocks_per_sm      persistent-kernel CTAs (of 4 warps) per SM
 *                      (0 = occupancy maximum); register-solver plans asking
 *                      for more than 4 use a build of the persistent kernel
 *                      with fewer registers per thread that fits 6
 *   local_solver       how the persistent kernel settles a tile it visits:
 *                      IWPP_SOLVER_QUEUE, the FIFO wave queues of Algorithm
 *                      7's queue phase in shared memory, or
 *                      IWPP_SOLVER_REGISTER, the tile held in registers (two
 *                      columns per lane) and swept down and up until no pixel
 *                      changes (Algorithm 1's update in Gauss-Seidel order);
 *                      the register solver needs tile_w == 64, tile_h <= 16;
 *                      or IWPP_SOLVER_COOP, one CTA per 64 x 64 tile: each of
 *                      its four warps holds a 16-row strip as the register
 *                      solver does, and the strips exchange their boundary
 *                      rows through shared memory until the tile is settled
 *                      (tile_h == tile_w == 64, no revisit sweeps, no value
 *                      levels, at most 6 CTAs per SM; its scan kernel runs the
 *                      sweep pairs on the whole 64 x 64 tile, the strips
 *                      exchanging boundary rows after each pair)
 *   value_levels       0 or 1: the persistent kernel's tile queue is one FIFO;
 *                      2..16: one queue per value level, and a worker takes
 *                      its next tile from the highest level that has one (the
 *                      level of a queued tile is the value the notification
 *                      that queued it can raise it to; the tile-granular form of
 *                      Sec. 4.4's heap-ordered propagation). Register solver,
 *                      single-image calls only
 *   watchdog_ns        the persistent kernel gives up with IWPP_ERR_TIMEOUT
 *                      when a wait for work lasts longer than this
 *                      (0 = default, 10 s)
 */
typedef struct {
    int32_t tile_h, tile_w;
    int32_t sweeps;
    int32_t revisit_sweeps;
    int32_t smem_queue_cap;
    int32_t blocks_per_sm;
    int32_t local_solver;
    int32_t value_levels;
    int64_t watchdog_ns;
} iwpp_plan;

/* Values of iwpp_plan.local_solver. */
enum { IWPP_SOLVER_QUEUE = 0, IWPP_SOLVER_REGISTER = 1, IWPP_SOLVER_COOP = 2 };

/* Fills *plan with the static default schedule of single-image calls (a NULL plan there):
 * 64 x 64 tiles, cooperative solver. Returns IWPP_OK. */
IWPP_API int iwpp_default_plan(iwpp_plan *plan);

/* Fills *plan with the static default schedule of batch calls (a NULL plan there): the
 * single-image default (64 x 64 tiles, cooperative solver). Returns IWPP_OK. */
IWPP_API int iwpp_default_batch_plan(iwpp_plan *plan);

/* 1 if (tile_h, tile_w) is a compiled tile shape, else 0. */
IWPP_API int iwpp_tile_shape_supported(int32_t tile_h, int32_t tile_w);

/* Workspace bytes needed by iwpp_reconstruct / iwpp_reconstruct_plan for one
 * H x W image on the current device under `plan` (NULL = default plan).
 * Returns 0 for invalid sizes. */
IWPP_API size_t iwpp_workspace_bytes(int64_t H, int64_t W, int dtype, const iwpp_plan *plan);

/*
 * Reconstruction of one image (Sec. 3.1, Algorithm 7; Sec. 3.3 for
 * op = IWPP_ERODE). Enqueues, on `stream`: a workspace reset, one
 * tile-parallel kernel that checks the precondition, runs the tile-local
 * raster / anti-raster sweeps and collects the tiles whose pixels can still
 * propagate (the initial frontier), and one persistent kernel that drains the
 * frontier with shared-memory wave queues until no tile can change.
 * Returns IWPP_OK or a host-detected error code; device-side errors go to the
 * workspace status word (see iwpp_sync_status).
 */
IWPP_API int iwpp_reconstruct(void *marker_inout, const void *mask, int64_t H, int64_t W,
                     int connectivity, int op, int dtype, void *workspace, size_t ws_bytes,
                     void *stream);

/* As iwpp_reconstruct, under an explicit plan (NULL = default plan). */
IWPP_API int iwpp_reconstruct_plan(void *marker_inout, const void *mask, int64_t H, int64_t W,
                          int connectivity, int op, int dtype, const iwpp_plan *plan,
                          void *workspace, size_t ws_bytes, void *stream);

/*
 * The two steps of iwpp_reconstruct_plan, for callers that time or overlap them:
 * iwpp_scan resets the workspace and runs the tile-parallel scan kernel
 * (precondition check, `plan->sweeps` tile-local raster / anti-raster sweep pairs
 * of Algorithm 7, and frontier initialisation: the tiles whose pixels can still
 * be raised are queued — with one FIFO (value_levels <= 1) in a spread order that
 * keeps tiles next to each other apart in the queue, by two small kernels after the
 * scan); iwpp_drain then runs the persistent kernel that drains
 * the queued tiles (Algorithm 7's irregular propagation phase). Calling
 * iwpp_scan and then iwpp_drain with identical arguments on one stream is exactly
 * iwpp_reconstruct_plan. Same arguments, ownership and errors.
 */
IWPP_API int iwpp_scan(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                       int op, int dtype, const iwpp_plan *plan, void *workspace, size_t ws_bytes,
                       void *stream);
IWPP_API int iwpp_drain(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                        int op, int dtype, const iwpp_plan *plan, void *workspace, size_t ws_bytes,
                        void *stream);

/* Waits for `stream`, then returns the device status recorded in `workspace`
 * by the last call that used it (IWPP_OK or an iwpp_status code), or
 * IWPP_ERR_CUDA if the stream reports an error. */
IWPP_API int iwpp_sync_status(const void *workspace, void *stream);

/*
 * ---- Batches (one persistent launch over many images) -------------------------
 * One image of a batch. Images may differ in size, pixel type, operator and
 * connectivity; the same conventions as for a single image apply to each.
 * reserved must be 0.
 */
typedef struct {
    void *marker_inout;
    const void *mask;
    int64_t H, W;
    int32_t connectivity, op, dtype, reserved;
} iwpp_image;

/* Number of tiles of a batch under `plan` (NULL = default plan), or -1 for a bad
 * argument. Tiles are numbered image by image (in the order of `imgs`),
 * row-major inside an image; this numbering indexes the per-tile arrays of
 * iwpp_reconstruct_batch_sched. Host-only call. */
IWPP_API int64_t iwpp_batch_tile_count(const iwpp_image *imgs, int n, const iwpp_plan *plan);

/* Workspace bytes needed by iwpp_reconstruct_batch(_sched) for this batch on the
 * current device (0 for a bad argument). */
IWPP_API size_t iwpp_batch_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan);

/*
 * Reconstruction of every image of a batch (each result identical to a separate
 * iwpp_reconstruct call) in one persistent launch: the image table is written
 * into the workspace by small kernels that take the descriptors as parameters,
 * a scan kernel runs over every tile of every image (precondition check,
 * tile-local sweeps, frontier initialisation), a compact kernel queues the tiles
 * that can still change in schedule order (without an explicit order: the spread
 * order, position i -> tile (i * m) mod ntiles with m coprime to ntiles near
 * 0.618 ntiles, which keeps tiles next to each other apart in the queue so that
 * concurrent workers do not keep raising each other's borders), and one persistent kernel drains the
 * whole batch. `imgs` is a HOST array of n >= 1 descriptors, read during the call
 * only. No host synchronisation and no allocation: the call can be captured in a
 * CUDA graph (the descriptors are then frozen into the graph).
 */
IWPP_API int iwpp_reconstruct_batch(const iwpp_image *imgs, int n, const iwpp_plan *plan, void *workspace,
                                    size_t ws_bytes, void *stream);

/*
 * As iwpp_reconstruct_batch, with an explicit schedule in DEVICE memory (each
 * pointer may be NULL):
 *   tile_order   uint32[ntiles]: the order in which the initial frontier is
 *                queued (a permutation of the tile ids; repeated or missing ids
 *                are tolerated: a tile is queued once, missing ones at the end)
 *   tile_sweeps  uint8[ntiles]: raster / anti-raster sweep pairs of each tile in
 *                the scan kernel (else plan->sweeps for every tile)
 *   tile_work    uint32[2 * ntiles], caller-zeroed: receives per-tile work, [t] =
 *                wave-queue pops (queue solver) or row passes (register
 *                solver), [ntiles + t] = SM cycles spent on the tile
 * The schedule changes the work done, never the result.
 */
IWPP_API int iwpp_reconstruct_batch_sched(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                          const uint32_t *tile_order, const uint8_t *tile_sweeps,
                                          uint32_t *tile_work, void *workspace, size_t ws_bytes,
                                          void *stream);

/*
 * One step of iwpp_reconstruct_batch_sched (Algorithm 6's two phases, for callers
 * that time or overlap them separately): phases = 1 enqueues the image-table upload,
 * the workspace reset, the scan kernel (precondition, sweeps, frontier) and the
 * queue compaction; phases = 2 enqueues only the persistent drain, which reuses the
 * workspace prepared by a phases = 1 call with identical arguments (same images,
 * plan, schedule and workspace) earlier on the same stream; phases = 3 is the whole
 * call. A phases = 1 call followed by a phases = 2 call is exactly
 * iwpp_reconstruct_batch_sched. Other values: IWPP_ERR_ARG. Same arguments,
 * ownership and errors otherwise.
 */
IWPP_API int iwpp_reconstruct_batch_phase(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                          const uint32_t *tile_order, const uint8_t *tile_sweeps,
                                          uint32_t *tile_work, int phases, void *workspace, size_t ws_bytes,
                                          void *stream);

/* Kernel launches one iwpp_reconstruct_batch_phase call with n images makes (-1 for a
 * bad argument); phases + 4: one iwpp_reconstruct_batch_learned call whose features come
 * out of the scan kernel. Host-only call. */
IWPP_API int iwpp_batch_launch_count(int n, int phases);

/*
 * ---- CUDA graphs and autotuning (host runtime) ----------------------------------
 * iwpp_batch_graph_create captures one batch call (static schedule, or the device
 * schedule arrays given) into an executable CUDA graph: the descriptors, plan,
 * workspace and schedule pointers are frozen into it. Each iwpp_graph_launch then
 * reruns the whole batch with one launch on `stream` (restore the markers first:
 * the result overwrites them). Graph creation allocates host-side graph objects and
 * synchronises nothing on the caller's streams; destroy with iwpp_graph_destroy.
 */
typedef struct iwpp_graph_s *iwpp_graph;
IWPP_API int iwpp_batch_graph_create(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                     const uint32_t *tile_order, const uint8_t *tile_sweeps,
                                     void *workspace, size_t ws_bytes, iwpp_graph *out);
IWPP_API int iwpp_graph_launch(iwpp_graph graph, void *stream);
IWPP_API int iwpp_graph_destroy(iwpp_graph graph);

/*
 * Autotuner: picks the local solver with its tile shape (register 16 x 64,
 * cooperative 64 x 64, queue 32 x 32 / 32 x 64 / 64 x 64 / 16 x 64), the sweep count and
 * (register solver) the CTAs per SM or (queue solver) the shared queue
 * capacity of *plan_inout by timing candidate
 * plans on the batch itself (coordinate descent
 * from the given plan; best of `reps` runs each, each after writing a buffer of
 * twice the L2 size; CUDA events on `stream`). The
 * markers are backed up first and restored after every trial and at the end, so
 * the batch's images are unchanged on return. This call allocates device memory
 * (backups, a workspace) and synchronises `stream`. cache_path (may be NULL) is a
 * text file of previous results keyed by GPU name and a coarse batch signature; a
 * hit returns the cached plan without timing (best_ms = 0). *best_ms (may be
 * NULL) receives the winning time.
 */
IWPP_API int iwpp_autotune_batch(const iwpp_image *imgs, int n, iwpp_plan *plan_inout, int reps,
                                 const char *cache_path, void *stream, float *best_ms);

/*
 * ---- Learned work estimator (schedule of a batch) ---------------------------------
 * Every image is cut into IWPP_FEATURE_BLOCK x IWPP_FEATURE_BLOCK blocks (the last
 * ones partial), numbered image by image, row-major. Per block, IWPP_NFEAT float
 * features, in the dilation domain (both images complemented for erosion),
 * d = max(I - J, 0), d8 = d (u8) or d >> 8 (u16); [0..14] are taken over the
 * block's rows 0, 4, 8, ... (every fourth row: the sampled pixels):
 *   [0..7]   fractions of the sampled pixels with d8 == 0, d8 == 1, 2..3, 4..7,
 *            8..15, 16..31, 32..63, >= 64
 *   [8]      fraction with J == I and J > 0 (seeds)
 *   [9]      fraction with |I(p)-I(p+x)| + |I(p)-I(p+y)| > 16 * MAXV / 255
 *            (a neighbour outside the block contributes 0; p + y is the next
 *            row of the block, sampled or not)
 *   [10..14] mean(I), std(I), mean(J), std(J), mean(d), each / MAXV
 *   [15]     log2(pixels in the block, every row) / 12
 * The MLP is 16 -> 64 -> 64 -> 2 with ReLU, FP32, IWPP_MLP_PARAMS parameters in
 * one flat device array: W1[16][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2]
 * (y = x W + b). Output 0 predicts the block's log work, log(1 + SM cycles spent
 * on its tiles), output 1 the raster / anti-raster sweep pairs to run on them.
 * The paper has no learned schedule; none of these calls can change a
 * reconstruction result, they only order the work.
 */
#define IWPP_FEATURE_BLOCK 64
#define IWPP_NFEAT 16
#define IWPP_MLP_PARAMS 5378

/* Feature blocks of a batch, or -1 for a bad argument (host-only). */
IWPP_API int64_t iwpp_batch_block_count(const iwpp_image *imgs, int n);

/* Bytes of the scheduling workspace for this batch and plan (0 for a bad argument;
 * the plan's tile sides must divide IWPP_FEATURE_BLOCK). Caller-owned device memory,
 * 256-byte aligned. */
IWPP_API size_t iwpp_sched_workspace_bytes(const iwpp_image *imgs, int n, const iwpp_plan *plan);

/* Features of every block of the batch into feats (device, float[nblocks][16]). */
IWPP_API int iwpp_batch_features(const iwpp_image *imgs, int n, float *feats, void *sched_ws,
                                 size_t sws_bytes, void *stream);

/* Y[N][2] = MLP(params, X[N][16]) (device arrays). */
IWPP_API int iwpp_mlp_forward(const float *params, const float *X, int64_t N, float *Y, void *stream);

/*
 * Trains the MLP in place: `epochs` passes over the N samples (X[N][16] inputs,
 * T[N][2] targets, device arrays) in minibatches of `batch` (a fresh affine
 * permutation of the samples per epoch, drawn from `seed`), loss
 * (1/B) sum (w0 (y0 - t0)^2 + w1 (y1 - t1)^2), Adam with learning rate lr (moments
 * adam_m, adam_v: float[IWPP_MLP_PARAMS], zeroed before the first step; step0 = the
 * number of Adam steps already taken). grad: float[IWPP_MLP_PARAMS] scratch,
 * zeroed by the caller once; it is left zeroed.
 */
IWPP_API int iwpp_mlp_train(float *params, float *adam_m, float *adam_v, float *grad, const float *X,
                            const float *T, int64_t N, int epochs, int batch, float lr, float w0, float w1,
                            uint64_t seed, int64_t step0, void *stream);

/*
 * Schedule from per-block predictions preds[nblocks][2] (device): tile_order
 * (uint32[ntiles]) lists the batch's tiles by decreasing predicted work (output 0,
 * bucketed in steps of 1/64), tile_sweeps (uint8[ntiles]) = output 1 of the tile's
 * block, rounded and clamped to 0..8. Ready for iwpp_reconstruct_batch_sched.
 */
IWPP_API int iwpp_schedule_from_predictions(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                            const float *preds, uint32_t *tile_order, uint8_t *tile_sweeps,
                                            void *sched_ws, size_t sws_bytes, void *stream);

/* Byte offset of the features (float[nblocks][IWPP_NFEAT]) inside a scheduling workspace
 * of this batch and plan (the array iwpp_reconstruct_batch_learned fills), or -1 for a bad
 * argument. Host-only call. */
IWPP_API int64_t iwpp_sched_features_offset(const iwpp_image *imgs, int n, const iwpp_plan *plan);

/*
 * A batch reconstructed with the learned schedule made inside the call (growth direction
 * (4) in one call; the paper has no counterpart). When the plan's tiles are the feature
 * blocks (the cooperative solver's 64 x 64 tiles) and the batch does not mix
 * connectivities, the scan kernel computes each tile's features from the pixels it loads
 * anyway (no separate pass over the images); then MLP inference, the tile order and the
 * sweep counts as iwpp_schedule_learned makes them; then a pass that runs the sweep pairs
 * of the tiles with a non-zero count (and notifies the neighbours they can raise); then
 * the initial frontier is queued in the learned order and drained as in
 * iwpp_reconstruct_batch_sched. Other plans: iwpp_schedule_learned, then
 * iwpp_reconstruct_batch_sched. The result is identical to iwpp_reconstruct_batch.
 *   params        device float[IWPP_MLP_PARAMS]
 *   tile_order    device uint32[ntiles], tile_sweeps device uint8[ntiles]: receive the schedule
 *   sched_ws      device, 256-byte aligned, iwpp_sched_workspace_bytes(imgs, n, plan) bytes;
 *                 receives the features and predictions
 *   phases        1: everything up to the persistent drain; 2: the drain alone (after a
 *                 phases = 1 call with identical arguments on the same stream); 3: the
 *                 whole call
 *   workspace     as iwpp_reconstruct_batch
 * No host synchronisation and no allocation: capturable in a CUDA graph.
 */
IWPP_API int iwpp_reconstruct_batch_learned(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                            const float *params, uint32_t *tile_order, uint8_t *tile_sweeps,
                                            void *sched_ws, size_t sws_bytes, int phases, void *workspace,
                                            size_t ws_bytes, void *stream);

/* Features, MLP inference and schedule in one call (all on `stream`, no host sync). */
IWPP_API int iwpp_schedule_learned(const iwpp_image *imgs, int n, const iwpp_plan *plan, const float *params,
                                   uint32_t *tile_order, uint8_t *tile_sweeps, void *sched_ws,
                                   size_t sws_bytes, void *stream);

/* Per-tile work from iwpp_reconstruct_batch_sched summed into blocks:
 * block_work[b] = pops or passes, block_work[nblocks + b] = SM cycles (caller-zeroed
 * uint64). */
IWPP_API int iwpp_tile_work_to_blocks(const iwpp_image *imgs, int n, const iwpp_plan *plan,
                                      const uint32_t *tile_work, unsigned long long *block_work,
                                      void *sched_ws, size_t sws_bytes, void *stream);

/*
 * ---- Reconstruction without any allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory where they reconstruct: code running under a memory budget
 * fixed at start-up, plug-ins whose host framework owns every allocation, or real-time
 * loops where cudaMalloc (which may synchronise the device) is not allowed.
 *
 * iwpp_reconstruct_noalloc is iwpp_reconstruct with the default plan, except that its
 * workspace is a device array of IWPP_NOALLOC_SCRATCH_BYTES (8 MiB) inside the library,
 * held by every GPU that loads the library until the process exits. It calls no
 * cudaMalloc, cudaFree or other allocating routine. The caller passes the marker
 * (overwritten by the result) and the mask, as for iwpp_reconstruct.
 *   - Images whose workspace would exceed the array are rejected with
 *     IWPP_ERR_WORKSPACE before anything is enqueued. With the default plan the
 *     workspace is about 8 bytes per 64 x 64 tile (a tile state and a queue slot) plus
 *     1 KB, so the limit is about 1 M tiles, i.e. about 4.2 gigapixels;
 *     iwpp_workspace_bytes(H, W, dtype, NULL) gives the exact need.
 *   - The first call on a device looks up the array's device address for that device
 *     (with that device current). Under CUDA's lazy module loading that first use is
 *     also where the library's device code and this array are loaded onto the device,
 *     which can allocate and synchronise: make the first call on each device outside
 *     any timed region and before any stream capture.
 *   - Every call on a device shares the one array; each call resets the parts that must
 *     start at zero. Calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it and must be serialised by the caller.
 *   - status_out (may be NULL): when given, the call waits for `stream` and stores the
 *     device status (IWPP_OK or an iwpp_status code) there; otherwise the call is
 *     asynchronous and the device status is not reported. A call made while `stream`
 *     is being captured must pass NULL (waiting would end the capture): with a
 *     non-NULL status_out it returns IWPP_ERR_ARG and enqueues nothing.
 * Returns IWPP_OK or a host-detected error code: IWPP_ERR_ARG for a bad pointer,
 * size, connectivity, op or dtype; IWPP_ERR_WORKSPACE for an image beyond the array;
 * IWPP_ERR_CUDA when a CUDA call fails.
 */
#define IWPP_NOALLOC_SCRATCH_BYTES (8u << 20)
IWPP_API int iwpp_reconstruct_noalloc(void *marker_inout, const void *mask, int64_t H, int64_t W,
                                      int connectivity, int op, int dtype, void *stream, int *status_out);

/*
 * Operators built on reconstruction by dilation (the paper names further IWPP
 * operators as future work; these are the reconstruction-based ones). Each builds
 * its marker on the device, runs one reconstruction exactly as iwpp_reconstruct
 * (default plan; same workspace size, iwpp_workspace_bytes(H, W, dtype, NULL)) and
 * finishes with an elementwise kernel, all on `stream`. image, out and scratch are
 * device buffers of H x W pixels of `dtype` (out of iwpp_regional_maxima: uint8),
 * 16-byte aligned; image is only read.
 *   iwpp_hmaxima          out = R_image(max(image - h, 0)): the h-maxima transform
 *                         (every regional maximum lowered by h, clipped at its saddle)
 *   iwpp_hdome            out = image - R_image(max(image - h, 0)): the domes of
 *                         height up to h that the h-maxima transform removes
 *   iwpp_regional_maxima  out[p] = 1 where image(p) > R_image(image - 1)(p), else 0:
 *                         the plateaus whose every outside neighbour is strictly lower;
 *                         scratch receives R_image(image - 1)
 */
IWPP_API int iwpp_hmaxima(const void *image, void *out, int64_t H, int64_t W, uint32_t h, int connectivity,
                          int dtype, void *workspace, size_t ws_bytes, void *stream);
IWPP_API int iwpp_hdome(const void *image, void *out, int64_t H, int64_t W, uint32_t h, int connectivity,
                        int dtype, void *workspace, size_t ws_bytes, void *stream);
IWPP_API int iwpp_regional_maxima(const void *image, void *scratch, uint8_t *out, int64_t H, int64_t W,
                                  int connectivity, int dtype, void *workspace, size_t ws_bytes, void *stream);

/*
 * Reconstruction of an image held in HOST memory, band by band (images larger than the
 * device's memory; Sec. 1 cites 100K x 100K scans, Sec. 4.5 splits such images into tasks
 * and corrects the propagation across task borders). The image is cut into horizontal bands
 * of band_rows rows. Each band is copied to the device together with band_rows / 16 rows of
 * each neighbour band (the overlap) and one halo row beyond them whose mask is set to their
 * marker (fixed sources), reconstructed through the single-image path, and its own rows are
 * copied back (the overlap rows are not). Bands are visited top to bottom, then bottom to
 * top, a band again only after a neighbour band changed, until no band is left to visit:
 * the result is bit-identical to iwpp_reconstruct. The overlap lets a path that crosses a
 * band border and comes back within it be followed in one visit. While a band is reconstructed on `stream`, the band
 * expected next is copied to the device on a stream of the call's own (two band buffers).
 * Blocking: the call waits for every band's change flag; it creates and destroys that
 * stream, a few events and an 8-byte pinned host buffer.
 *   marker_inout, mask   HOST, H x W of `dtype`, row-major (pinned memory copies fastest);
 *                        the result overwrites marker_inout
 *   band_rows            rows per band, >= 1 (a band of >= H rows is one reconstruction)
 *   workspace            device, 256-byte aligned, iwpp_host_workspace_bytes(H, W, dtype,
 *                        band_rows) bytes: two band buffers (each two (band_rows + 2 ov + 2)
 *                        x W planes, ov = band_rows / 16, and one band_rows x W plane) and a
 *                        single-image workspace for band_rows + 2 ov + 2 rows
 *   visits_out           host int32 or NULL: band reconstructions made
 * Returns IWPP_OK, a host-detected error, or the first device error of any band (e.g.
 * IWPP_ERR_PRECONDITION; the host image is then unspecified). Resumable: every pixel written
 * back lies between the marker and the reconstruction, so if a call with a valid marker is
 * interrupted at any point, repeating it on the same host buffers completes the result.
 */
IWPP_API size_t iwpp_host_workspace_bytes(int64_t H, int64_t W, int dtype, int64_t band_rows);
IWPP_API int iwpp_reconstruct_host(void *marker_inout, const void *mask, int64_t H, int64_t W, int connectivity,
                                   int op, int dtype, int64_t band_rows, void *workspace, size_t ws_bytes,
                                   void *stream, int32_t *visits_out);

/*
 * Marker-controlled watershed by flooding, as an IWPP propagation on the same tile engine
 * (watershed is one of the operators the paper names as future work for the pattern).
 * Every pixel carries a pair (level, label): a marker pixel is fixed at (its gradient,
 * its label), every other pixel starts unreached; a neighbour q offers p the pair
 * (max(level(q), gradient(p)), label(q)) and p keeps the lexicographically smallest.
 * The levels reached are unique: the minimax flooding level (the reconstruction by
 * erosion of the marker levels under the gradient). Which label a pixel gets when several
 * markers reach it at its level depends on the order of work, as in any flooding
 * watershed; every result has each label's markers reaching its pixels at their level.
 * No watershed lines are drawn.
 *   markers      device, H x W uint32: 0 = none, 1 .. 65534 = label (larger labels make
 *                the device status IWPP_ERR_ARG)
 *   gradient     device, H x W of `dtype` (u8 or u16)
 *   labels_out   device, H x W uint32, 4-byte aligned: the label of each pixel (0 where
 *                no marker reaches, i.e. no marker at all); also the working buffer
 *   levels_out   device, H x W int32 or NULL: the flooding level (-1 where unreached)
 *   H, W         1 <= H, W < 2^31, H * W < 2^40
 *   workspace    device, 256-byte aligned, iwpp_watershed_workspace_bytes(H, W) bytes
 */
IWPP_API size_t iwpp_watershed_workspace_bytes(int64_t H, int64_t W);
IWPP_API int iwpp_watershed(const uint32_t *markers, const void *gradient, int dtype, uint32_t *labels_out,
                            int32_t *levels_out, int64_t H, int64_t W, int connectivity, void *workspace,
                            size_t ws_bytes, void *stream);

/*
 * Geodesic skeleton by influence zones (SKIZ), as an IWPP propagation on the same tile
 * engine (one of the operators the paper names as future work for the pattern, Sec. 6).
 * Domain: pixels where mask != 0 or a marker is set; paths are 4- or 8-connected chains
 * of domain pixels, a path's length its number of steps. For each domain pixel p, d(p) is
 * the length of the shortest path from any marker pixel, and L(p) the set of labels of the
 * marker pixels at that distance. p lies in the influence zone of label l when L(p) = {l},
 * and on the skeleton when L(p) holds two or more labels. The propagation carries (d, min L,
 * max L) and merges label sets on equal distances, a join on a distributive lattice: the
 * result is unique (independent of the order of work) and bit-identical to the definition.
 *   markers      device, H x W uint32 (4-byte aligned): 0 = none, 1 .. 65534 = label (larger
 *                labels make the device status IWPP_ERR_ARG)
 *   mask         device, H x W uint8: non-zero = inside the domain
 *   zone_out     device, H x W uint32 (4-byte aligned): the label of the pixel's influence
 *                zone; 0 on the skeleton, outside the domain and where no marker reaches
 *   dist_out     device, H x W int32 or NULL: d(p), -1 where no marker reaches
 *   lpair_out    device, H x W uint32 or NULL: (min L << 16) | max L, 0 where unreached
 *                (the skeleton is where the two halves differ)
 *   H, W         1 <= H, W and H * W < 2^31 (distances then fit in 31 bits)
 *   connectivity 4 or 8
 *   workspace    device, 256-byte aligned, iwpp_skiz_workspace_bytes(H, W) bytes (8 bytes
 *                of state per pixel plus the tile queue)
 * Enqueues everything on `stream`; returns IWPP_OK or a host-detected error (device errors
 * in the workspace status word, see iwpp_sync_status).
 */
IWPP_API size_t iwpp_skiz_workspace_bytes(int64_t H, int64_t W);
IWPP_API int iwpp_skiz(const uint32_t *markers, const uint8_t *mask, uint32_t *zone_out, int32_t *dist_out,
                       uint32_t *lpair_out, int64_t H, int64_t W, int connectivity, void *workspace,
                       size_t ws_bytes, void *stream);

/*
 * Euclidean distance transform by wavefront propagation of Voronoi sites (Sec. 3.2,
 * Algorithm 8) on the same persistent tile engine. Background pixels (mask == 0) are
 * their own sites; every other pixel ends with the site, among those its neighbours
 * offered, that is nearest to it, and no neighbour's site is strictly nearer (the
 * propagation's fixed point). As the paper notes, this is approximate: the nearest
 * background pixel can be missed in rare configurations (measured: > 99 % of pixels
 * exact on tissue-like masks, errors below one pixel); it is exact with one or two
 * background pixels. Which of several equally valid fixed points is reached depends on
 * the order of work, so results are compared by their properties, not bit by bit.
 *   mask         device, H x W uint8, row-major; non-zero = foreground (object)
 *   site_out     device, H x W uint32 (4-byte aligned): the site of each pixel packed
 *                as (y << 16) | x, 0xFFFFFFFF where no background exists
 *   dist2_out    device, H x W uint32 or NULL: squared distance to the site
 *                (0xFFFFFFFF where there is none)
 *   H, W         1 .. 32767 (squared distances then fit in 32 bits)
 *   connectivity 4 or 8 (the neighbourhood the sites travel through)
 *   workspace    device, 256-byte aligned, iwpp_edt_workspace_bytes(H, W) bytes
 * Enqueues everything on `stream`; returns IWPP_OK or a host-detected error (device
 * errors in the workspace status word, see iwpp_sync_status).
 */
IWPP_API size_t iwpp_edt_workspace_bytes(int64_t H, int64_t W);
IWPP_API int iwpp_edt(const void *mask, uint32_t *site_out, uint32_t *dist2_out, int64_t H, int64_t W,
                      int connectivity, void *workspace, size_t ws_bytes, void *stream);

/*
 * Work counters of the last call (single image or batch) that used `workspace`: tile
 * visits by the persistent kernel (CTA-tile visits for the cooperative solver),
 * wave-queue entries processed (pops), entries created by the visits' initial
 * scans (seeds), wave steps run (row passes for the register solver, summed over
 * the strips for the cooperative one), and
 * the persistent workers' summed waiting time and processing time in ns (cooperative
 * solver: per CTA, its run time less its waiting time).
 * Host pointer out[6]. Synchronises `stream`. Returns IWPP_OK or IWPP_ERR_CUDA.
 */
IWPP_API int iwpp_work_counters(const void *workspace, void *stream, uint64_t out[6]);

#ifdef __cplusplus
}
#endif
#endif /* IWPP_H */

/*
 * CPU ORACLE — test infrastructure only.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library. The product path (the CUDA library under
 * paper_1605_00930_gb300/) never calls it, and the two share no code.
 *
 * What it computes: grayscale morphological reconstruction of a mask image I
 * from a marker image J (reconstruction by dilation, Sec. 2.1.2, Eq. "recon":
 * iterate J <- delta_G(J) ^ I to stability), and its dual, reconstruction by
 * erosion (J <- eps_G(J) v I), which is the fill-holes operator of Sec. 3.3 when
 * the marker equals the mask on the image border and the maximum value inside.
 *
 * How: Vincent's hybrid algorithm exactly as the paper lays out
 * Reconstruction-IWPP (Sec. 3.1, Algorithm 7):
 *   1. a raster sweep, J(p) <- max{J(q): q in N+(p) U {p}} ^ I(p);
 *   2. an anti-raster sweep with N-(p), which also seeds a FIFO with every p
 *      that has a q in N-(p) with J(q) < J(p) and J(q) < I(q);
 *   3. the irregular propagation phase: pop p, and for every q in N_G(p) with
 *      J(q) < J(p) and I(q) != J(q), set J(q) <- min{J(p), I(q)} and push q.
 * Erosion is written out as its own code path (min and max swapped, the
 * comparisons flipped), not through image complement, so that the duality
 * between the two stays an independent test.
 *
 * Readings of points the paper leaves open:
 *   - N+ (raster half-neighbourhood) is {W, N} for 4-connectivity and
 *     {NW, N, NE, W} for 8; N- is the point reflection {E, S} / {SE, S, SW, E}.
 *     The figure that fixes them is missing; the result does not depend on it.
 *   - Neighbours outside the image domain do not exist.
 *   - Pixels are held as 32-bit signed integers, as in the paper's experiments
 *     (Sec. 5.2); u8 and u16 images are widened on the way in and narrowed on
 *     the way out, which cannot change a min/max computation.
 *   - The paper elides the initialisation phase; here the marker is taken as
 *     given. The precondition J <= I (dilation) / J >= I (erosion) stated with
 *     Algorithm 1 is checked by oracle_precondition_ok, not enforced.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_NOMEM 2

/* (dy, dx) offsets. The first half of each 8-neighbourhood list is N+, the
 * second half N-; likewise for the 4-neighbourhood. */
static const int NPLUS8[4][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}};
static const int NMINUS8[4][2] = {{1, 1}, {1, 0}, {1, -1}, {0, 1}};
static const int NPLUS4[2][2] = {{-1, 0}, {0, -1}};
static const int NMINUS4[2][2] = {{1, 0}, {0, 1}};

typedef struct {
    uint32_t *buf;
    size_t head, tail, cap;
} fifo_t;

static int fifo_init(fifo_t *f, size_t cap) {
    f->cap = cap < 16 ? 16 : cap;
    f->head = f->tail = 0;
    f->buf = (uint32_t *)malloc(f->cap * sizeof(uint32_t));
    return f->buf ? 0 : -1;
}

static int fifo_push(fifo_t *f, uint32_t v) {
    if (f->tail == f->cap) {
        if (f->head > 0) { /* slide the live part to the front */
            memmove(f->buf, f->buf + f->head, (f->tail - f->head) * sizeof(uint32_t));
            f->tail -= f->head;
            f->head = 0;
        }
        if (f->tail == f->cap) {
            size_t ncap = f->cap * 2;
            uint32_t *nb = (uint32_t *)realloc(f->buf, ncap * sizeof(uint32_t));
            if (!nb) return -1;
            f->buf = nb;
            f->cap = ncap;
        }
    }
    f->buf[f->tail++] = v;
    return 0;
}

static int fifo_empty(const fifo_t *f) { return f->head == f->tail; }
static uint32_t fifo_pop(fifo_t *f) { return f->buf[f->head++]; }
static void fifo_free(fifo_t *f) { free(f->buf); }

static int in_domain(int64_t y, int64_t x, int64_t H, int64_t W) {
    return y >= 0 && y < H && x >= 0 && x < W;
}

/* Widen an image to int32. dtype 0 = u8, 1 = u16. */
static void load_i32(int32_t *dst, const void *src, size_t n, int dtype) {
    if (dtype == 0) {
        const uint8_t *s = (const uint8_t *)src;
        for (size_t i = 0; i < n; i++) dst[i] = s[i];
    } else {
        const uint16_t *s = (const uint16_t *)src;
        for (size_t i = 0; i < n; i++) dst[i] = s[i];
    }
}

static void store_i32(void *dst, const int32_t *src, size_t n, int dtype) {
    if (dtype == 0) {
        uint8_t *d = (uint8_t *)dst;
        for (size_t i = 0; i < n; i++) d[i] = (uint8_t)src[i];
    } else {
        uint16_t *d = (uint16_t *)dst;
        for (size_t i = 0; i < n; i++) d[i] = (uint16_t)src[i];
    }
}

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }
static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }

/* Reconstruction by dilation, Algorithm 7. Returns the number of FIFO pops
 * through *pops when pops != NULL (the "elements processed" count of Sec. 5.3.5). */
static int recon_dilate(int32_t *J, const int32_t *I, int64_t H, int64_t W, int conn,
                        uint64_t *pops) {
    const int (*np)[2] = conn == 8 ? NPLUS8 : NPLUS4;
    const int (*nm)[2] = conn == 8 ? NMINUS8 : NMINUS4;
    const int nh = conn == 8 ? 4 : 2;
    fifo_t f;
    if (fifo_init(&f, (size_t)(H * W / 8 + 16))) return ORACLE_ERR_NOMEM;

    /* Scanning phase, raster order: (0,0) to (H-1,W-1). */
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
            int64_t p = y * W + x;
            int32_t m = J[p];
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + np[k][0], qx = x + np[k][1];
                if (in_domain(qy, qx, H, W)) m = imax(m, J[qy * W + qx]);
            }
            J[p] = imin(m, I[p]);
        }

    /* Anti-raster order, with FIFO seeding. */
    for (int64_t y = H - 1; y >= 0; y--)
        for (int64_t x = W - 1; x >= 0; x--) {
            int64_t p = y * W + x;
            int32_t m = J[p];
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + nm[k][0], qx = x + nm[k][1];
                if (in_domain(qy, qx, H, W)) m = imax(m, J[qy * W + qx]);
            }
            J[p] = imin(m, I[p]);
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + nm[k][0], qx = x + nm[k][1];
                if (!in_domain(qy, qx, H, W)) continue;
                int64_t q = qy * W + qx;
                if (J[q] < J[p] && J[q] < I[q]) {
                    if (fifo_push(&f, (uint32_t)p)) { fifo_free(&f); return ORACLE_ERR_NOMEM; }
                    break;
                }
            }
        }

    /* Irregular propagation phase. */
    uint64_t npop = 0;
    while (!fifo_empty(&f)) {
        int64_t p = fifo_pop(&f);
        npop++;
        int64_t py = p / W, px = p % W;
        for (int half = 0; half < 2; half++) {
            const int (*nb)[2] = half == 0 ? np : nm;
            for (int k = 0; k < nh; k++) {
                int64_t qy = py + nb[k][0], qx = px + nb[k][1];
                if (!in_domain(qy, qx, H, W)) continue;
                int64_t q = qy * W + qx;
                if (J[q] < J[p] && I[q] != J[q]) {
                    J[q] = imin(J[p], I[q]);
                    if (fifo_push(&f, (uint32_t)q)) { fifo_free(&f); return ORACLE_ERR_NOMEM; }
                }
            }
        }
    }
    if (pops) *pops = npop;
    fifo_free(&f);
    return ORACLE_OK;
}

/* Reconstruction by erosion: the dual of recon_dilate, written out on its own. */
static int recon_erode(int32_t *J, const int32_t *I, int64_t H, int64_t W, int conn,
                       uint64_t *pops) {
    const int (*np)[2] = conn == 8 ? NPLUS8 : NPLUS4;
    const int (*nm)[2] = conn == 8 ? NMINUS8 : NMINUS4;
    const int nh = conn == 8 ? 4 : 2;
    fifo_t f;
    if (fifo_init(&f, (size_t)(H * W / 8 + 16))) return ORACLE_ERR_NOMEM;

    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
            int64_t p = y * W + x;
            int32_t m = J[p];
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + np[k][0], qx = x + np[k][1];
                if (in_domain(qy, qx, H, W)) m = imin(m, J[qy * W + qx]);
            }
            J[p] = imax(m, I[p]);
        }

    for (int64_t y = H - 1; y >= 0; y--)
        for (int64_t x = W - 1; x >= 0; x--) {
            int64_t p = y * W + x;
            int32_t m = J[p];
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + nm[k][0], qx = x + nm[k][1];
                if (in_domain(qy, qx, H, W)) m = imin(m, J[qy * W + qx]);
            }
            J[p] = imax(m, I[p]);
            for (int k = 0; k < nh; k++) {
                int64_t qy = y + nm[k][0], qx = x + nm[k][1];
                if (!in_domain(qy, qx, H, W)) continue;
                int64_t q = qy * W + qx;
                if (J[q] > J[p] && J[q] > I[q]) {
                    if (fifo_push(&f, (uint32_t)p)) { fifo_free(&f); return ORACLE_ERR_NOMEM; }
                    break;
                }
            }
        }

    uint64_t npop = 0;
    while (!fifo_empty(&f)) {
        int64_t p = fifo_pop(&f);
        npop++;
        int64_t py = p / W, px = p % W;
        for (int half = 0; half < 2; half++) {
            const int (*nb)[2] = half == 0 ? np : nm;
            for (int k = 0; k < nh; k++) {
                int64_t qy = py + nb[k][0], qx = px + nb[k][1];
                if (!in_domain(qy, qx, H, W)) continue;
                int64_t q = qy * W + qx;
                if (J[q] > J[p] && I[q] != J[q]) {
                    J[q] = imax(J[p], I[q]);
                    if (fifo_push(&f, (uint32_t)q)) { fifo_free(&f); return ORACLE_ERR_NOMEM; }
                }
            }
        }
    }
    if (pops) *pops = npop;
    fifo_free(&f);
    return ORACLE_OK;
}

/*
 * oracle_reconstruct: marker_inout (J) is overwritten with the reconstruction
 * of mask (I). H, W >= 1, H*W < 2^32; conn in {4, 8}; op 0 = dilate,
 * 1 = erode; dtype 0 = u8, 1 = u16. Host pointers, row-major, pitch W.
 * pops (may be NULL) receives the FIFO pop count. Returns 0 on success.
 */
int oracle_reconstruct(void *marker_inout, const void *mask, int64_t H, int64_t W, int conn,
                       int op, int dtype, uint64_t *pops) {
    if (!marker_inout || !mask || H < 1 || W < 1 || (conn != 4 && conn != 8) ||
        (op != 0 && op != 1) || (dtype != 0 && dtype != 1))
        return ORACLE_ERR_ARG;
    if ((uint64_t)H * (uint64_t)W >= ((uint64_t)1 << 32)) return ORACLE_ERR_ARG;
    size_t n = (size_t)(H * W);
    int32_t *J = (int32_t *)malloc(n * sizeof(int32_t));
    int32_t *I = (int32_t *)malloc(n * sizeof(int32_t));
    if (!J || !I) { free(J); free(I); return ORACLE_ERR_NOMEM; }
    load_i32(J, marker_inout, n, dtype);
    load_i32(I, mask, n, dtype);
    int rc = op == 0 ? recon_dilate(J, I, H, W, conn, pops) : recon_erode(J, I, H, W, conn, pops);
    if (rc == ORACLE_OK) store_i32(marker_inout, J, n, dtype);
    free(J);
    free(I);
    return rc;
}

/* 1 if marker <= mask everywhere (dilate) / marker >= mask everywhere (erode),
 * 0 if not, negative on a bad argument. */
int oracle_precondition_ok(const void *marker, const void *mask, int64_t H, int64_t W, int op,
                           int dtype) {
    if (!marker || !mask || H < 1 || W < 1 || (op != 0 && op != 1) || (dtype != 0 && dtype != 1))
        return -1;
    size_t n = (size_t)(H * W);
    for (size_t i = 0; i < n; i++) {
        int32_t j = dtype == 0 ? ((const uint8_t *)marker)[i] : ((const uint16_t *)marker)[i];
        int32_t m = dtype == 0 ? ((const uint8_t *)mask)[i] : ((const uint16_t *)mask)[i];
        if (op == 0 ? (j > m) : (j < m)) return 0;
    }
    return 1;
}

/*
 * CPU ORACLE — test infrastructure only (same rules as iwpp_oracle.c: only the test
 * suite, the smoke check and the benchmark's CPU leg load it; the CUDA library never
 * does, and the two share no code).
 *
 * What it computes: the Euclidean distance transform by wavefront propagation of
 * Voronoi sites, Sec. 3.2 (Algorithm 8), with a FIFO queue:
 *   initialisation: every background pixel is its own site, every foreground pixel
 *     has no site (infinitely far); every background pixel with a foreground
 *     neighbour is queued (the initial wavefront);
 *   propagation: pop p; for every neighbour q of p, if q is strictly closer to p's
 *     site than to its own, q takes p's site and is queued;
 *   result: for every pixel its site and its distance to it.
 *
 * Readings of points the paper leaves open:
 *   - Foreground = non-zero mask pixels (the objects), background = zero.
 *   - DIST is the squared Euclidean distance, in 64-bit integers: it orders sites
 *     exactly like the Euclidean distance and needs no rounding. The map returned is
 *     the squared distance; its square root is the Euclidean map.
 *   - "Strictly closer" keeps a pixel's current site on ties, as the comparison in
 *     Algorithm 8 is strict.
 *   - Sites are pixel indices y * W + x; -1 = no site (no background pixel reaches
 *     the pixel, e.g. an image without background).
 *   - Neighbours outside the image do not exist.
 * The propagation is not exact in general (the paper calls the transform approximate:
 * a pixel keeps the best site among those its neighbours offer); for a single site it
 * is exact.
 */
#include <stdint.h>
#include <stdlib.h>

#define EDT_OK 0
#define EDT_ERR_ARG 1
#define EDT_ERR_NOMEM 2

static const int NB8[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 1}, {1, -1}, {1, 0}, {1, 1}};
static const int NB4[4][2] = {{-1, 0}, {0, -1}, {0, 1}, {1, 0}};

static int64_t dist2(int64_t y, int64_t x, int64_t site, int64_t W) {
    const int64_t dy = y - site / W, dx = x - site % W;
    return dy * dy + dx * dx;
}

/* fg: H*W bytes (non-zero = foreground); site: H*W int64 out; d2: H*W int64 out (-1 where
 * there is no site). pops: number of queue pops. */
int oracle_edt(const uint8_t *fg, int64_t H, int64_t W, int conn, int64_t *site, int64_t *d2,
               uint64_t *pops) {
    if (!fg || !site || !d2 || H < 1 || W < 1 || (conn != 4 && conn != 8)) return EDT_ERR_ARG;
    const int nn = conn == 8 ? 8 : 4;
    const int (*nb)[2] = conn == 8 ? NB8 : NB4;
    const int64_t n = H * W;
    /* each pixel is queued at most once per improvement; a ring of n entries plus
     * growth covers every case */
    int64_t cap = n + 16, head = 0, tail = 0, count = 0;
    int64_t *q = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!q) return EDT_ERR_NOMEM;
    for (int64_t p = 0; p < n; p++) site[p] = fg[p] ? -1 : p;
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
            const int64_t p = y * W + x;
            if (fg[p]) continue;
            int edge = 0;
            for (int k = 0; k < nn && !edge; k++) {
                const int64_t yy = y + nb[k][0], xx = x + nb[k][1];
                if (yy >= 0 && yy < H && xx >= 0 && xx < W && fg[yy * W + xx]) edge = 1;
            }
            if (edge) {
                q[tail] = p;
                tail = (tail + 1) % cap;
                count++;
            }
        }
    uint64_t npop = 0;
    while (count > 0) {
        const int64_t p = q[head];
        head = (head + 1) % cap;
        count--;
        npop++;
        const int64_t py = p / W, px = p % W, sp = site[p];
        for (int k = 0; k < nn; k++) {
            const int64_t yy = py + nb[k][0], xx = px + nb[k][1];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const int64_t qq = yy * W + xx;
            const int64_t cand = dist2(yy, xx, sp, W);
            if (site[qq] < 0 || cand < dist2(yy, xx, site[qq], W)) {
                site[qq] = sp;
                if (count == cap) { /* grow the ring, unrolling it */
                    int64_t *nq = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
                    if (!nq) {
                        free(q);
                        return EDT_ERR_NOMEM;
                    }
                    for (int64_t i = 0; i < count; i++) nq[i] = q[(head + i) % cap];
                    free(q);
                    q = nq;
                    head = 0;
                    tail = count;
                    cap *= 2;
                }
                q[tail] = qq;
                tail = (tail + 1) % cap;
                count++;
            }
        }
    }
    free(q);
    for (int64_t p = 0; p < n; p++) d2[p] = site[p] < 0 ? -1 : dist2(p / W, p % W, site[p], W);
    if (pops) *pops = npop;
    return EDT_OK;
}

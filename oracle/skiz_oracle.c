/*
 * CPU ORACLE — test infrastructure only (same rules as iwpp_oracle.c).
 *
 * Geodesic skeleton by influence zones (SKIZ), one of the IWPP operators Sec. 6 names as
 * future work. Domain X = pixels where the mask is non-zero or a marker is set; paths are
 * 4- or 8-connected chains of domain pixels and a path's length is its number of steps.
 * For a domain pixel p:
 *   d(p) = the smallest path length from any marker pixel to p (the geodesic distance),
 *   L(p) = the set of labels of the marker pixels at distance d(p).
 * p lies in the influence zone of label l when L(p) = {l}, and on the SKIZ when L(p) holds
 * two or more labels. Pixels no marker reaches (and pixels outside X) are in neither.
 *
 * This is a multi-source breadth-first propagation: the markers form the initial
 * frontier (distance 0, their own label) and a FIFO carries the wave outward one step per
 * layer. Because the FIFO pops every pixel of layer k before any pixel of layer k + 1, a
 * pixel first reached at layer k + 1 has received the labels of all its layer-k neighbours
 * by the time it is popped; those merges are the only ones that can change L.
 * Each pixel reports min L and max L (enough to tell a zone from the skeleton).
 *
 * Inputs: markers H*W uint32 (0 = none, 1..65534 = label), mask H*W uint8.
 * Outputs: dist H*W int32 (-1 = unreached), lmin / lmax H*W uint32 (0 = unreached),
 * zone H*W uint32 (the label where lmin == lmax, 0 on the SKIZ and where unreached).
 */
#include <stdint.h>
#include <stdlib.h>

#define SK_OK 0
#define SK_ERR_ARG 1
#define SK_ERR_NOMEM 2

static const int SNB8[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 1}, {1, -1}, {1, 0}, {1, 1}};
static const int SNB4[4][2] = {{-1, 0}, {0, -1}, {0, 1}, {1, 0}};

int oracle_skiz(const uint32_t *markers, const uint8_t *mask, int64_t H, int64_t W, int conn, int32_t *dist_out,
                uint32_t *lmin_out, uint32_t *lmax_out, uint32_t *zone_out, uint64_t *pops) {
    if (!markers || !mask || !dist_out || !lmin_out || !lmax_out || !zone_out || H < 1 || W < 1 ||
        (conn != 4 && conn != 8))
        return SK_ERR_ARG;
    const int64_t n = H * W;
    if (n >= ((int64_t)1 << 31)) return SK_ERR_ARG;
    const int nn = conn == 8 ? 8 : 4;
    const int (*nb)[2] = conn == 8 ? SNB8 : SNB4;
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!q) return SK_ERR_NOMEM;
    int64_t head = 0, tail = 0;
    for (int64_t p = 0; p < n; p++) {
        if (markers[p] > 65534u) {
            free(q);
            return SK_ERR_ARG;
        }
        if (markers[p]) {
            dist_out[p] = 0;
            lmin_out[p] = lmax_out[p] = markers[p];
            q[tail++] = p; /* every pixel enters the FIFO at most once: n slots suffice */
        } else {
            dist_out[p] = -1;
            lmin_out[p] = lmax_out[p] = 0;
        }
    }
    uint64_t npop = 0;
    while (head < tail) {
        const int64_t p = q[head++];
        npop++;
        const int64_t py = p / W, px = p % W;
        const int32_t dn = dist_out[p] + 1;
        for (int k = 0; k < nn; k++) {
            const int64_t yy = py + nb[k][0], xx = px + nb[k][1];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const int64_t r = yy * W + xx;
            if (!mask[r] && !markers[r]) continue; /* outside the domain */
            if (dist_out[r] < 0) {
                dist_out[r] = dn;
                lmin_out[r] = lmin_out[p];
                lmax_out[r] = lmax_out[p];
                q[tail++] = r;
            } else if (dist_out[r] == dn) {
                if (lmin_out[p] < lmin_out[r]) lmin_out[r] = lmin_out[p];
                if (lmax_out[p] > lmax_out[r]) lmax_out[r] = lmax_out[p];
            }
        }
    }
    for (int64_t p = 0; p < n; p++) zone_out[p] = (dist_out[p] >= 0 && lmin_out[p] == lmax_out[p]) ? lmin_out[p] : 0u;
    free(q);
    if (pops) *pops = npop;
    return SK_OK;
}

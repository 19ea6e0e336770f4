/*
 * CPU ORACLE — test infrastructure only (same rules as iwpp_oracle.c).
 *
 * Marker-controlled watershed by flooding, as an IWPP propagation (one of the operators
 * Sec. 6 names as future work for the pattern): every pixel carries a pair (level, label).
 * A marker pixel is fixed at (gradient there, its label); every other pixel starts
 * unreached. A neighbour q offers pixel p the pair (max(level(q), gradient(p)), label(q));
 * p keeps the lexicographically smaller of its own pair and every offer. The propagation
 * (FIFO, like Algorithm 7's queue phase) stops when no offer improves any pixel.
 *
 * The levels of the fixed point are unique: level(p) is the minimax flooding level (the
 * smallest, over paths from any marker, of the largest gradient on the path, marker pixel
 * included), i.e. the reconstruction by erosion of the marker levels under the gradient.
 * The labels are not: the pair order is not preserved along a path (a pair that loses at
 * a pixel can win after both are raised to a higher gradient), so which label a pixel
 * gets when several markers reach it at its level depends on the order of work, as in
 * any flooding watershed. Every fixed point satisfies: each label comes from a marker
 * that reaches the pixel at its level, and no neighbour offers a smaller pair. (This
 * reading draws no watershed lines.)
 *
 * Inputs: markers H*W uint32 (0 = no marker, 1..65534 = label), gradient u8 or u16.
 * Outputs: label H*W uint32 (0 = not reached), level H*W int32 (-1 = not reached).
 */
#include <stdint.h>
#include <stdlib.h>

#define WS_OK 0
#define WS_ERR_ARG 1
#define WS_ERR_NOMEM 2

static const int WNB8[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 1}, {1, -1}, {1, 0}, {1, 1}};
static const int WNB4[4][2] = {{-1, 0}, {0, -1}, {0, 1}, {1, 0}};

int oracle_watershed(const uint32_t *markers, const void *gradient, int dtype, int64_t H, int64_t W, int conn,
                     uint32_t *label_out, int32_t *level_out, uint64_t *pops) {
    if (!markers || !gradient || !label_out || !level_out || H < 1 || W < 1 || (conn != 4 && conn != 8) ||
        (dtype != 0 && dtype != 1))
        return WS_ERR_ARG;
    const int64_t n = H * W;
    const int nn = conn == 8 ? 8 : 4;
    const int (*nb)[2] = conn == 8 ? WNB8 : WNB4;
    int64_t *lev = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *lab = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t cap = n + 16, head = 0, tail = 0, count = 0;
    int64_t *q = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!lev || !lab || !q) {
        free(lev);
        free(lab);
        free(q);
        return WS_ERR_NOMEM;
    }
    const uint8_t *g8 = (const uint8_t *)gradient;
    const uint16_t *g16 = (const uint16_t *)gradient;
#define GRAD(i) ((int64_t)(dtype == 0 ? g8[i] : g16[i]))
    const int64_t INF = INT64_MAX / 4;
    for (int64_t p = 0; p < n; p++) {
        if (markers[p] > 65534u) {
            free(lev);
            free(lab);
            free(q);
            return WS_ERR_ARG;
        }
        if (markers[p]) {
            lev[p] = GRAD(p);
            lab[p] = markers[p];
            q[tail++] = p;
            count++;
        } else {
            lev[p] = INF;
            lab[p] = INF;
        }
    }
    uint64_t npop = 0;
    while (count > 0) {
        const int64_t p = q[head];
        head = (head + 1) % cap;
        count--;
        npop++;
        const int64_t py = p / W, px = p % W;
        for (int k = 0; k < nn; k++) {
            const int64_t yy = py + nb[k][0], xx = px + nb[k][1];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const int64_t r = yy * W + xx;
            if (markers[r]) continue;   /* markers are fixed */
            const int64_t cl = lev[p] > GRAD(r) ? lev[p] : GRAD(r), cb = lab[p];
            if (cl < lev[r] || (cl == lev[r] && cb < lab[r])) {
                lev[r] = cl;
                lab[r] = cb;
                if (count == cap) {
                    int64_t *nq = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
                    if (!nq) {
                        free(lev);
                        free(lab);
                        free(q);
                        return WS_ERR_NOMEM;
                    }
                    for (int64_t i = 0; i < count; i++) nq[i] = q[(head + i) % cap];
                    free(q);
                    q = nq;
                    head = 0;
                    tail = count;
                    cap *= 2;
                }
                q[tail] = r;
                tail = (tail + 1) % cap;
                count++;
            }
        }
    }
#undef GRAD
    for (int64_t p = 0; p < n; p++) {
        label_out[p] = lab[p] == INF ? 0u : (uint32_t)lab[p];
        level_out[p] = lev[p] == INF ? -1 : (int32_t)lev[p];
    }
    free(lev);
    free(lab);
    free(q);
    if (pops) *pops = npop;
    return WS_OK;
}

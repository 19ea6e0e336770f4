"""Host logic of the out-of-core reconstruction: the band visit order and overlap rule
(iwpp_bands.h) driven against a simulated image on the CPU. The simulation is a small 2-D
image (one column wide: the 1-D form) reconstructed with 8-connectivity, cut into bands that
are visited exactly as iwpp_reconstruct_host visits them on the device: a band is solved
together with `ov` rows of each neighbour band (the overlap), the rows beyond fixed, and only
its own rows are written back. When the schedule says no band is left to visit, the banded
result must equal the reconstruction of the whole image (and every band must have been
visited), for overlaps from 0 to band - 1 rows and the library's rule, also when a run is
interrupted after any band and repeated on the partly processed rows; the guess of the next
band made while a band is solved (the band copied ahead) must be the band the schedule then
returns whenever the solved band changed."""
import os
import subprocess

HARNESS = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include "iwpp_bands.h"

static unsigned long long st = 88172645463325252ull;
static unsigned rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (unsigned)(st >> 11); }

// Fixed point of J <- min(I, max over the 3 x 3 neighbourhood of J) on rows [a, e) of an
// n x m image; the rows outside [a, e) are read but stay fixed.
static bool solve(std::vector<int> &J, const std::vector<int> &I, int n, int m, int a, int e) {
    bool changed = false, again = true;
    while (again) {
        again = false;
        for (int r = a; r < e; r++)
            for (int c = 0; c < m; c++) {
                int v = J[r * m + c];
                for (int dr = -1; dr <= 1; dr++)
                    for (int dc = -1; dc <= 1; dc++) {
                        const int rr = r + dr, cc = c + dc;
                        if (rr >= 0 && rr < n && cc >= 0 && cc < m) v = std::max(v, J[rr * m + cc]);
                    }
                v = std::min(v, I[r * m + c]);
                if (v != J[r * m + c]) { J[r * m + c] = v; again = changed = true; }
            }
    }
    return changed;
}

// One band visit: the extended band (own rows and ov rows of each neighbour) solved on a
// copy, only the own rows written back. Returns whether they changed.
static bool visit(std::vector<int> &J, const std::vector<int> &I, int n, int m, int band, int ov, long b) {
    const int y0 = (int)b * band, y1 = std::min(n, y0 + band);
    const int e0 = std::max(0, y0 - ov), e1 = std::min(n, y1 + ov);
    std::vector<int> K = J;
    solve(K, I, n, m, e0, e1);
    bool changed = false;
    for (int i = y0 * m; i < y1 * m; i++)
        if (K[i] != J[i]) { J[i] = K[i]; changed = true; }
    return changed;
}

int main() {
    for (int trial = 0; trial < 3000; trial++) {
        const int m = (trial % 3 == 0) ? 1 : 1 + rnd() % 10;
        const int n = 1 + rnd() % (m == 1 ? 200 : 60), band = 1 + rnd() % 30;
        const int ov = (trial % 4 == 3) ? (int)iwpp::band_overlap(band) : (int)(rnd() % band);
        if (ov >= band) { printf("overlap %d not below the band %d\n", ov, band); return 1; }
        std::vector<int> I(n * m), J(n * m);
        for (int i = 0; i < n * m; i++) {
            I[i] = (rnd() % 10 < 3) ? 0 : (int)(rnd() % 10);   // walls make winding paths
            J[i] = (rnd() % 15 == 0) ? I[i] : 0;
        }
        std::vector<int> R = J;
        solve(R, I, n, m, 0, n);                  // the whole image at once
        const int nb = (n + band - 1) / band;
        // odd trials are interrupted after a few band visits and resumed with a fresh
        // schedule on the partly processed rows (what repeating an interrupted call does)
        const long stop_after = (trial & 1) ? (long)(rnd() % (2 * nb + 1)) : -1;
        std::vector<int> seen(nb, 0);
        long visits = 0;
        for (int pass = 0; pass < 2; pass++) {
            iwpp::BandSchedule order(nb);
            long here = 0;
            for (long b = order.next(); b >= 0;) {
                if (pass == 0 && stop_after >= 0 && here == stop_after) break;
                // the guess of the next band made while b is solved is exact when b changes
                const long guess = order.peek_after_change(b);
                const bool ch = visit(J, I, n, m, band, ov, b);
                order.visited(b, ch);
                seen[b] = 1;
                here++;
                if (++visits > 100000) { printf("no termination\n"); return 1; }
                const long nxt = order.next();
                if (ch && nxt != guess) { printf("trial %d: guess %ld, next %ld\n", trial, guess, nxt); return 1; }
                b = nxt;
            }
            if (stop_after < 0) break;
        }
        for (int b = 0; b < nb; b++)
            if (!seen[b]) { printf("band %d never visited\n", b); return 1; }
        if (J != R) {
            printf("trial %d: banded result differs (n %d, m %d, band %d, overlap %d)\n", trial, n, m, band, ov);
            return 1;
        }
    }
    printf("ok\n");
    return 0;
}
'''


def test_band_schedule_reaches_the_whole_image_fixed_point(tmp_path):
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_00930_gb300",
                        "csrc")
    src = tmp_path / "bands.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "bands"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", csrc, "-o", str(exe), str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr

"""Host logic of the out-of-core reconstruction: the band visit order (iwpp_bands.h) driven
against a simulated image on the CPU. The simulation is the column form of the problem: a
1-D reconstruction J <- min(I, max(J(r-1), J(r), J(r+1))) over N rows, cut into bands that are
solved with their neighbour rows as fixed sources, exactly as iwpp_reconstruct_host solves
its bands on the device. When the schedule says no band is left to visit, the banded result
must equal the reconstruction of the whole column (and every band must have been visited),
also when a run is interrupted after any band and repeated on the partly processed rows; the
guess of the next band made while a band is solved (the band copied ahead) must be the band
the schedule then returns whenever the solved band changed."""
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

// fixed point of the 1-D update on rows [a, b) with rows a-1 and b (if any) fixed
static bool solve(std::vector<int> &J, const std::vector<int> &I, int a, int b) {
    const int n = (int)J.size();
    bool changed = false, again = true;
    while (again) {
        again = false;
        for (int r = a; r < b; r++) {
            int m = J[r];
            if (r > 0) m = std::max(m, J[r - 1]);
            if (r + 1 < n) m = std::max(m, J[r + 1]);
            m = std::min(m, I[r]);
            if (m != J[r]) { J[r] = m; again = changed = true; }
        }
    }
    return changed;
}

int main() {
    for (int trial = 0; trial < 3000; trial++) {
        const int n = 1 + rnd() % 200, band = 1 + rnd() % 40;
        std::vector<int> I(n), J(n);
        for (int r = 0; r < n; r++) {
            I[r] = rnd() % 10;
            J[r] = (rnd() % 7 == 0) ? I[r] : 0;
        }
        std::vector<int> R = J;
        solve(R, I, 0, n);                       // the whole column at once
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
                const int a = (int)b * band, e = std::min(n, a + band);
                // the guess of the next band made while b is solved is exact when b changes
                const long guess = order.peek_after_change(b);
                const bool ch = solve(J, I, a, e);
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
        if (J != R) { printf("trial %d: banded result differs (n %d, band %d)\n", trial, n, band); return 1; }
    }
    printf("ok\n");
    return 0;
}
'''


def test_band_schedule_reaches_the_whole_column_fixed_point(tmp_path):
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_00930_gb300",
                        "csrc")
    src = tmp_path / "bands.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "bands"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", csrc, "-o", str(exe), str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr

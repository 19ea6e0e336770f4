"""Host logic of the spread order in which a batch's (and a single image's) initial frontier
is queued (csrc/iwpp_spread.h): for every tile count the multiplier is coprime with it, so
position -> tile is a permutation of the tiles, and consecutive positions land at least an
eighth of the tiles apart around the ring (tile ids of one image are row-major, so nearby ids
are nearby tiles)."""
import os
import subprocess

HARNESS = r'''
#include <cstdio>
#include <cstdint>
#include <vector>
#include "iwpp_spread.h"

static uint64_t gcd(uint64_t a, uint64_t b) { while (b) { uint64_t t = a % b; a = b; b = t; } return a; }

int main() {
    for (uint32_t n = 1; n < 20000; n += (n < 3000 ? 1 : 97)) {
        const uint32_t m = iwpp::spread_multiplier(n);
        if (n >= 3 && (gcd(m, n) != 1 || m == 0)) { printf("n %u: multiplier %u not coprime\n", n, m); return 1; }
        std::vector<char> seen(n, 0);
        for (uint64_t i = 0; i < n; i++) {
            const uint32_t t = iwpp::spread_tile(i, n, m);
            if (t >= n || seen[t]) { printf("n %u: position %llu -> %u repeats\n", n, (unsigned long long)i, t); return 1; }
            seen[t] = 1;
        }
        // consecutive positions are at least n / 8 tiles apart (both ways round the ring)
        if (n >= 64) {
            for (uint64_t i = 0; i + 1 < 64; i++) {
                const uint32_t a = iwpp::spread_tile(i, n, m), b = iwpp::spread_tile(i + 1, n, m);
                const uint32_t d = a > b ? a - b : b - a, dd = d < n - d ? d : n - d;
                if (dd < n / 8) { printf("n %u: positions %llu, %llu only %u apart\n", n, (unsigned long long)i,
                                         (unsigned long long)(i + 1), dd); return 1; }
            }
        }
    }
    if (iwpp::spread_tile(5, 9, 0) != 5) { printf("multiplier 0 is not the identity\n"); return 1; }
    printf("ok\n");
    return 0;
}
'''


def test_spread_order_is_a_permutation_that_spreads(tmp_path):
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_00930_gb300",
                        "csrc")
    src = tmp_path / "spread.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "spread"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", csrc, "-o", str(exe), str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr

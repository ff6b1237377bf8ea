"""CPU test of the serving loop's device-arena allocator (csrc/serve_arena.h, host code only):
random allocate/release sequences against a brute-force occupancy map -- no overlaps, alignment
kept, free space coalesced, everything returned restores one range of the full capacity."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "serve_arena.h"
using rmusic::RangeAllocator;
int main() {
    const uint64_t CAP = 4096;
    RangeAllocator a(CAP);
    std::vector<int> owner(CAP, -1);
    struct Live { uint64_t off, n; };
    std::vector<Live> live;
    unsigned s = 12345;
    auto rnd = [&]() { s = s * 1103515245u + 12345u; return (s >> 8) & 0xffff; };
    for (int it = 0; it < 20000; ++it) {
        if (live.empty() || rnd() % 3 != 0) {
            uint64_t n = 1 + rnd() % 300, align = (rnd() % 2) ? 64 : 1, off = 0;
            bool ok = a.allocate(n, align, &off);
            // brute force: does any aligned fitting range exist?
            bool exists = false;
            for (uint64_t st = 0; st + n <= CAP && !exists; st += align) {
                bool fr = true;
                for (uint64_t k = st; k < st + n; ++k) if (owner[k] >= 0) { fr = false; break; }
                exists = fr;
            }
            if (ok != exists) { printf("FAIL fit %d %d\n", (int)ok, (int)exists); return 1; }
            if (ok) {
                if (off % align) { printf("FAIL align\n"); return 1; }
                for (uint64_t k = off; k < off + n; ++k) {
                    if (owner[k] >= 0) { printf("FAIL overlap\n"); return 1; }
                    owner[k] = it;
                }
                live.push_back({off, n});
            }
        } else {
            size_t i = rnd() % live.size();
            if (!a.release(live[i].off, live[i].n)) { printf("FAIL release\n"); return 1; }
            if (a.release(live[i].off, live[i].n)) { printf("FAIL double release\n"); return 1; }
            for (uint64_t k = live[i].off; k < live[i].off + live[i].n; ++k) owner[k] = -1;
            live.erase(live.begin() + i);
        }
        uint64_t freec = 0;
        for (uint64_t k = 0; k < CAP; ++k) freec += owner[k] < 0;
        if (freec != a.free_units()) { printf("FAIL accounting\n"); return 1; }
    }
    for (auto& l : live) a.release(l.off, l.n);
    if (a.free_ranges() != 1 || a.largest_free() != CAP || a.live() != 0) { printf("FAIL coalesce\n"); return 1; }
    printf("OK\n");
    return 0;
}
"""


def test_range_allocator(tmp_path):
    src = tmp_path / "t.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "t"
    inc = os.path.join(ROOT, "paper_1910_11872_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.stdout.strip() == "OK", out.stdout

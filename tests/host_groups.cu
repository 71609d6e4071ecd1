// Host check (no GPU) of group_by_blocks, which packs the replicas of an
// ensemble into the launches of the descriptor-chunk bulk collide (grid:
// the group's largest tile count x its members).
//
// For random block counts (zeros, equal runs, wide ranges) and group caps:
//  1. every replica with blocks appears in exactly one group, the others in
//     none, so each replica's tiles are updated once per step;
//  2. no group holds more than cap replicas (the kernel parameter holds at
//     most that many descriptors);
//  3. the first member of a group has the most blocks (the launch's grid
//     covers every member's tiles) and every member has at least 3/4 of
//     them;
//  4. groups follow in non-increasing order of their first member's blocks,
//     and a group ends only when it is full or the next replica has fewer
//     than 3/4 of its first member's blocks (no needless launch).
// Prints one line and returns 0 when every case passes.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <random>
#include <vector>

#include "flbm_host.cuh"

using namespace flbm;

int main(int argc, char** argv)
{
    const int trials = argc > 1 ? std::atoi(argv[1]) : 2000;
    std::mt19937_64 g(0x9a0b5u);
    const long long sizes[4] = {32, 144, 256, 864};
    int failed = 0, groups_seen = 0;
    for (int t = 0; t < trials; ++t) {
        const int n = 1 + (int)(g() % 300);
        const int caps[4] = {1, 3, 48, 1000};
        const int cap = caps[t % 4];
        std::vector<long long> blocks(n);
        const int kind = (int)(g() % 3);
        for (int r = 0; r < n; ++r) {
            const uint64_t u = g();
            if (u % 7 == 0) blocks[r] = 0;
            else if (kind == 0) blocks[r] = 1 + (long long)(u >> 8) % 1000;           // wide range
            else if (kind == 1) blocks[r] = sizes[u % 4];                             // a few sizes
            else blocks[r] = 100 + (long long)(u >> 8) % 40;                          // close sizes
        }
        const auto groups = group_by_blocks(blocks, cap);
        groups_seen += (int)groups.size();
        int fails = 0;
        std::vector<int> seen(n, 0);
        for (size_t q = 0; q < groups.size(); ++q) {
            const auto& gr = groups[q];
            if (gr.empty() || (int)gr.size() > cap) ++fails;
            if (gr.empty()) continue;
            const long long first = blocks[gr[0]];
            for (int r : gr) {
                if (r < 0 || r >= n) { ++fails; continue; }
                seen[r] += 1;
                if (blocks[r] <= 0 || blocks[r] > first || 4 * blocks[r] < 3 * first) ++fails;
            }
            if (q + 1 < groups.size() && !groups[q + 1].empty()) {
                const long long next = blocks[groups[q + 1][0]];
                if (next > first) ++fails;
                const bool full = (int)gr.size() == cap;
                if (!full && 4 * next >= 3 * first) ++fails;
            }
        }
        for (int r = 0; r < n; ++r)
            if (seen[r] != (blocks[r] > 0 ? 1 : 0)) ++fails;
        if (fails) {
            ++failed;
            if (failed <= 5) std::printf("FAIL %d checks: n=%d cap=%d kind=%d\n", fails, n, cap, kind);
        }
    }
    std::printf("cases %d failed %d groups %d\n", trials, failed, groups_seen);
    return failed == 0 ? 0 : 1;
}

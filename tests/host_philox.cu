// Host check (no GPU) of the CUDA code's random numbers, built from the same
// header functions the kernels call.
//
// argv[1] is the known-answer file (ctr0..3 key0 key1 -> out0..3, hex). For
// every row:
//  1. philox4x32_10 (initial state) returns the published output;
//  2. philox_rk with the round keys make_kparams precomputes from
//     seed = key1:key0 and replica 0 returns the same output;
// and for random counters, seeds and replicas (key1 = seed_hi ^ replica)
// philox_rk agrees with philox4x32_10. uniform_open maps every tested word
// to ((x >> 9) + 1/2) 2^-23 exactly, inside (0, 1).
// Prints one line and returns 0 when every check passes.
#include <cstdio>
#include <cstdint>
#include <fstream>
#include <random>
#include <sstream>
#include <string>

#include "flbm_host.cuh"

using namespace flbm;

int main(int argc, char** argv)
{
    if (argc < 2) {
        std::printf("usage: host_philox <kat file>\n");
        return 2;
    }
    std::ifstream in(argv[1]);
    std::string line;
    int rows = 0, fails = 0;
    while (std::getline(in, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream ss(line);
        uint32_t v[10];
        for (int i = 0; i < 10; ++i) ss >> std::hex >> v[i];
        if (!ss) continue;
        ++rows;
        uint32_t x[4] = {v[0], v[1], v[2], v[3]};
        philox4x32_10(x[0], x[1], x[2], x[3], v[4], v[5]);
        for (int i = 0; i < 4; ++i) fails += x[i] != v[6 + i];
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.lx = p.ly = p.lz = 4;
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.seed = ((uint64_t)v[5] << 32) | v[4];
        KParams k;
        make_kparams(p, 0, k);
        uint32_t y[4] = {v[0], v[1], v[2], v[3]};
        philox_rk(y[0], y[1], y[2], y[3], k);
        for (int i = 0; i < 4; ++i) fails += y[i] != v[6 + i];
    }
    std::mt19937_64 g(0x9411ull);
    int draws = 0;
    for (int t = 0; t < 20000; ++t) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.lx = p.ly = p.lz = 4;
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.seed = g();
        p.replica = (uint32_t)g();
        KParams k;
        make_kparams(p, 0, k);
        const uint32_t c[4] = {(uint32_t)g(), (uint32_t)g(), (uint32_t)g(), (uint32_t)g()};
        uint32_t a[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
        philox4x32_10(a[0], a[1], a[2], a[3], (uint32_t)p.seed, (uint32_t)(p.seed >> 32) ^ p.replica);
        philox_rk(b[0], b[1], b[2], b[3], k);
        for (int i = 0; i < 4; ++i) {
            fails += a[i] != b[i];
            const float u = uniform_open(a[i]);
            const double want = ((double)(a[i] >> 9) + 0.5) / 8388608.0;
            fails += !((double)u == want && u > 0.0f && u < 1.0f);
            ++draws;
        }
    }
    for (uint32_t x : {0u, 1u, 511u, 512u, 0x80000000u, 0xFFFFFFFFu}) {
        const double want = ((double)(x >> 9) + 0.5) / 8388608.0;
        fails += (double)uniform_open(x) != want;
    }
    std::printf("kat_rows %d draws %d failed %d\n", rows, draws, fails);
    return fails == 0 && rows > 0 ? 0 : 1;
}

// Host check (no GPU) of the push targets of the collide-stream kernels
// (PushFrame::target, the header function the kernels call) against a
// brute-force target taken straight from the definition. Population (l, i) of node x goes to slot (l, i) of node x + c_i
// with periodic wrap, or to slot (l, opp(i)) of x itself when c_i crosses a
// wall (halfway bounce-back). Random lattices (including 1- and 2-node axes)
// and wall flags, every population of every node. Prints one line and
// returns 0 when all agree.
#include <cstdio>
#include <cstdint>
#include <random>

#include "flbm_host.cuh"

using namespace flbm;

int main()
{
    std::mt19937_64 g(31337);
    int configs = 0, failed = 0;
    long long general = 0;
    for (int c = 0; c < 300; ++c) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.lx = 1 + (int)(g() % 40);
        p.ly = 1 + (int)(g() % 12);
        p.lz = 1 + (int)(g() % 9);
        p.wall_x = (int)(g() % 2);
        p.wall_y = (int)(g() % 2);
        p.wall_z = (int)(g() % 2);
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.rho_b0 = 0.05;
        if (!validate(&p).empty()) continue;
        ++configs;
        KParams P;
        make_kparams(p, 0, P);
        const int L[3] = {P.lx, P.ly, P.lz};
        for (int z = 0; z < P.lz; ++z)
            for (int y = 0; y < P.ly; ++y)
                for (int x = 0; x < P.lx; ++x) {
                    const uint32_t n = (uint32_t)(x + P.lx * (y + P.ly * z));
                    const PushFrame fr(x, y, z, P);
                    for (int l = 0; l < 2; ++l)
                        for (int i = 0; i < 19; ++i) {
                            int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
                            bool wall = false;
                            for (int a = 0; a < 3; ++a)
                                if (q[a] < 0 || q[a] >= L[a]) {
                                    if (P.wall[a]) wall = true;
                                    else q[a] = (q[a] + L[a]) % L[a];
                                }
                            const uint32_t want = wall ? n + (uint32_t)((19 * l + oppv(i)) * P.N)
                                                       : (uint32_t)(q[0] + P.lx * (q[1] + P.ly * q[2])) +
                                                             (uint32_t)((19 * l + i) * P.N);
                            bool w1;
                            const uint32_t t1 = fr.target(n, l, i, P, w1);
                            ++general;
                            if (t1 != want || w1 != wall) ++failed;
                        }
                }
    }
    std::printf("configurations %d targets %lld failed %d\n", configs, general, failed);
    return failed == 0 ? 0 : 1;
}

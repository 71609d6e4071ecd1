// Host check (no GPU) of the checks flbm_restore applies to the particle
// record it reads from a checkpoint file (check_restored_state), before the
// record reaches the step kernels, which index the particle masks with the
// record's mask index and box origin.
//
// For random lattices, wall flags, radii and positions, a record built as
// the library builds it (initial_state, then the box origin of its centre)
// must pass. Each of these corruptions must be refused: a mask index other
// than 0 or 1, a non-finite centre, velocity or pending impulse, a centre
// outside the walls or the periodic box, a box origin that is not the
// centre's, a fluid count outside [0, N], a negative step, a non-finite mass
// correction. Prints one line and returns 0 when every case behaves.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <limits>
#include <random>

#include "flbm_host.cuh"

using namespace flbm;

int main()
{
    std::mt19937_64 g(20240611u);
    auto uni = [&] { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); };
    const double nan = std::numeric_limits<double>::quiet_NaN();
    int configs = 0, failed = 0, refused = 0;
    for (int c = 0; c < 400; ++c) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.lx = 12 + (int)(g() % 40);
        p.ly = 12 + (int)(g() % 40);
        p.lz = 12 + (int)(g() % 40);
        p.wall_x = (int)(g() % 2);
        p.wall_y = (int)(g() % 2);
        p.wall_z = (int)(g() % 2);
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.rho_b0 = 0.05;
        p.rho_p_ratio = 1.5;
        p.radius = (c % 5 == 0) ? 0.0 : 1.5 + 3.5 * uni();
        const int L[3] = {p.lx, p.ly, p.lz};
        const int w[3] = {p.wall_x, p.wall_y, p.wall_z};
        for (int a = 0; a < 3; ++a) {
            const double lo = w[a] ? p.radius - 0.5 : 0.0, hi = w[a] ? L[a] - 0.5 - p.radius : (double)L[a];
            p.pos0[a] = lo + (hi - lo) * uni() * 0.999;
        }
        if (!validate(&p).empty()) continue;
        ++configs;
        KParams k;
        make_kparams(p, 0, k);
        DevState s = initial_state(p, k);
        if (k.has_particle) box_origin(s.X, k, s.box0);
        s.cur = (int)(g() % 2);
        s.step = (long long)(g() % 100000);
        if (!check_restored_state(s, k).empty()) {
            ++failed;
            std::printf("valid record refused: %s\n", check_restored_state(s, k).c_str());
            continue;
        }
        // Corruptions, one at a time.
        auto expect_refused = [&](DevState b) {
            if (check_restored_state(b, k).empty()) ++failed;
            else ++refused;
        };
        DevState b = s;
        b.cur = 2 + (int)(g() % 1000);
        expect_refused(b);
        b = s;
        b.cur = -1;
        expect_refused(b);
        b = s;
        b.nfluid = k.N + 1;
        expect_refused(b);
        b = s;
        b.nfluid = -1;
        expect_refused(b);
        b = s;
        b.step = -5;
        expect_refused(b);
        b = s;
        b.delta[g() % 2] = nan;
        expect_refused(b);
        if (!k.has_particle) continue;
        const int a = (int)(g() % 3);
        b = s;
        b.X[a] = nan;
        expect_refused(b);
        b = s;
        b.V[a] = INFINITY;
        expect_refused(b);
        b = s;
        b.Ppend[a] = nan;
        expect_refused(b);
        b = s;
        b.X[a] = w[a] ? -1.0 : L[a] + 0.25;
        expect_refused(b);
        b = s;
        b.box0[a] += 1 + (int)(g() % 3);
        expect_refused(b);
    }
    std::printf("configurations %d refused %d failed %d\n", configs, refused, failed);
    return failed == 0 ? 0 : 1;
}

// Host check (no GPU) of the padded density field's shell and virtual layer,
// built from the same header functions the kernels call (shell_node,
// virtual_node, shell_count, box_origin, box_node_inside).
//
// For random lattices, wall flags and spheres, with random interior
// densities (0 on particle nodes, as the density pass leaves them):
//  1. every shell node is written, and holds the periodic image of its
//     interior node (for a particle node, that node's virtual-layer value)
//     or, across a wall, the mean over its fluid neighbours;
//  2. every particle node with fluid neighbours holds their mean +delta_rho
//     for A and -delta_rho for B, clipped at 0; other interior values are
//     left alone;
//  3. the padding columns of each row (stride rounded up to 16 bytes) are
//     never written.
// The shell and the virtual layer run in either order. Prints one line and
// returns 0 when every configuration passes.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>

#include "flbm_host.cuh"

using namespace flbm;

namespace {

struct Rng {
    std::mt19937_64 g;
    explicit Rng(uint64_t s) : g(s) {}
    double uni() { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); }
    int range(int lo, int hi) { return lo + (int)(g() % (uint64_t)(hi - lo + 1)); }
};

int check(const flbm_params& p, Rng& rng, bool virtual_first)
{
    KParams k;
    make_kparams(p, 0, k);
    const int L[3] = {p.lx, p.ly, p.lz};
    const int W[3] = {p.wall_x, p.wall_y, p.wall_z};
    DevState st;
    std::memset(&st, 0, sizeof(st));
    const int B = k.B, B3 = B * B * B;
    std::vector<uint8_t> masks(2 * (size_t)B3, 0);
    const double X[3] = {p.pos0[0], p.pos0[1], p.pos0[2]};
    if (k.has_particle) {
        box_origin(X, k, st.box0);
        for (int t = 0; t < B3; ++t) masks[t] = box_node_inside(t, st.box0, X, k) ? 1 : 0;
    }
    auto solid = [&](int x, int y, int z) {
        return k.has_particle && is_solid(x, y, z, st.box0, masks.data(), k);
    };
    const float nan = std::nanf("");
    std::vector<float> psi(2 * (size_t)k.padn, nan);
    for (int z = 0; z < L[2]; ++z)
        for (int y = 0; y < L[1]; ++y)
            for (int x = 0; x < L[0]; ++x) {
                const long long q = pad_index(x, y, z, k);
                const bool s = solid(x, y, z);
                psi[q] = s ? 0.0f : (float)(0.5 + rng.uni());
                psi[k.padn + q] = s ? 0.0f : (float)(0.01 + 0.1 * rng.uni());
            }
    const std::vector<float> in = psi;

    const long long nshell = shell_count(k);
    auto run_shell = [&] { for (long long t = 0; t < nshell; ++t) shell_node(t, psi.data(), &st, masks.data(), k); };
    auto run_virtual = [&] {
        if (k.has_particle)
            for (int t = 0; t < B3; ++t) virtual_node(t, psi.data(), &st, masks.data(), k);
    };
    if (virtual_first) { run_virtual(); run_shell(); }
    else { run_shell(); run_virtual(); }

    // Expected value of lattice node c (in range): its density, or for a
    // particle node with fluid neighbours the virtual value, else 0.
    auto fluid_mean = [&](const int c[3], int l, int& cnt) {
        double s = 0.0;
        cnt = 0;
        for (int i = 1; i < 19; ++i) {
            int q[3] = {c[0] + cxv(i), c[1] + cyv(i), c[2] + czv(i)};
            bool ok = true;
            for (int a = 0; a < 3; ++a)
                if (q[a] < 0 || q[a] >= L[a]) {
                    if (W[a]) ok = false;
                    else q[a] = (q[a] + L[a]) % L[a];
                }
            if (!ok || solid(q[0], q[1], q[2])) continue;
            s += in[(size_t)l * k.padn + pad_index(q[0], q[1], q[2], k)];
            ++cnt;
        }
        return s;
    };
    auto expect_interior = [&](const int c[3], int l) {
        const long long q = pad_index(c[0], c[1], c[2], k);
        if (!solid(c[0], c[1], c[2])) return (double)in[(size_t)l * k.padn + q];
        int cnt;
        const double s = fluid_mean(c, l, cnt);
        if (!cnt) return 0.0;
        return std::max(s / cnt + (l == 0 ? 1.0 : -1.0) * (double)k.drho, 0.0);
    };

    int fails = 0;
    auto cmp = [&](double got, double want) {
        if (!(std::fabs(got - want) <= 2e-6 * std::max(1.0, std::fabs(want)))) ++fails;
    };
    for (int z = -1; z <= L[2]; ++z)
        for (int y = -1; y <= L[1]; ++y)
            for (int x = -1; x <= k.px - 2; ++x) {
                const long long q = (long long)(x + 1) + (long long)k.px * ((y + 1) + (long long)k.py * (z + 1));
                const int p3[3] = {x, y, z};
                if (x > L[0]) {  // padding column
                    for (int l = 0; l < 2; ++l)
                        if (!std::isnan(psi[(size_t)l * k.padn + q])) ++fails;
                    continue;
                }
                bool ghost = false, inside = true;
                int c[3];
                for (int a = 0; a < 3; ++a) {
                    c[a] = p3[a];
                    if (c[a] < 0 || c[a] >= L[a]) {
                        inside = false;
                        if (W[a]) ghost = true;
                        else c[a] = (c[a] + L[a]) % L[a];
                    }
                }
                for (int l = 0; l < 2; ++l) {
                    const float got = psi[(size_t)l * k.padn + q];
                    if (std::isnan(got)) { ++fails; continue; }
                    if (inside || !ghost) {
                        cmp(got, expect_interior(c, l));
                    } else {
                        // wall ghost: mean over the fluid neighbours of the ghost position
                        int cnt = 0;
                        double s = 0.0;
                        for (int i = 1; i < 19; ++i) {
                            int r[3] = {p3[0] + cxv(i), p3[1] + cyv(i), p3[2] + czv(i)};
                            bool ok = true;
                            for (int a = 0; a < 3; ++a)
                                if (r[a] < 0 || r[a] >= L[a]) {
                                    if (W[a]) ok = false;
                                    else r[a] = (r[a] + L[a]) % L[a];
                                }
                            if (!ok || solid(r[0], r[1], r[2])) continue;
                            s += in[(size_t)l * k.padn + pad_index(r[0], r[1], r[2], k)];
                            ++cnt;
                        }
                        cmp(got, cnt ? s / cnt : 0.0);
                    }
                }
            }
    return fails;
}

}  // namespace

int main(int argc, char** argv)
{
    const int trials = argc > 1 ? std::atoi(argv[1]) : 300;
    Rng rng(0x5be11ull);
    int run = 0, failed = 0, with_particle = 0;
    for (int t = 0; t < trials; ++t) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.rho_b0 = 0.05;
        p.rho_p_ratio = 1.5;
        p.delta_rho = (t % 3 == 0) ? 0.0 : (rng.uni() - 0.5);
        p.radius = (t % 4 == 0) ? 0.0 : 0.6 + 4.4 * rng.uni();
        const int need = p.radius > 0 ? (int)std::ceil(2.0 * p.radius) + 4 : 1;
        int* Ls[3] = {&p.lx, &p.ly, &p.lz};
        int* Ws[3] = {&p.wall_x, &p.wall_y, &p.wall_z};
        for (int a = 0; a < 3; ++a) {
            *Ws[a] = rng.range(0, 1);
            *Ls[a] = rng.range(need, std::max(need, 23));
            const int La = *Ls[a];
            if (p.radius > 0 && *Ws[a]) {
                const double lo = p.radius - 0.5, hi = La - 0.5 - p.radius;
                p.pos0[a] = lo + (hi - lo) * rng.uni();
            } else {
                p.pos0[a] = La * rng.uni();
            }
        }
        if (!validate(&p).empty()) continue;
        for (int order = 0; order < 2; ++order) {
            ++run;
            with_particle += p.radius > 0 ? 1 : 0;
            const int f = check(p, rng, order == 1);
            if (f) {
                ++failed;
                if (failed <= 5)
                    std::printf("FAIL %d checks: L=%dx%dx%d walls=%d%d%d R=%.4f X=(%.6f %.6f %.6f) drho=%.3f\n", f,
                                p.lx, p.ly, p.lz, p.wall_x, p.wall_y, p.wall_z, p.radius, p.pos0[0], p.pos0[1],
                                p.pos0[2], p.delta_rho);
            }
        }
    }
    std::printf("configurations %d failed %d with_particle %d\n", run, failed, with_particle);
    return failed == 0 && run > 0 ? 0 : 1;
}

// Host check (no GPU) of the collision's hand-factored mode transforms
// (to_modes, from_modes) against the D3Q19 mode basis written out from its
// polynomials: 1, c_x, c_y, c_z, c^2 - 1, 3 c_x^2 - c^2, c_y^2 - c_z^2,
// c_x c_y, c_y c_z, c_x c_z, (3 c^2 - 5) c_x, (3 c^2 - 5) c_y, (3 c^2 - 5) c_z,
// (c_y^2 - c_z^2) c_x, (c_z^2 - c_x^2) c_y, (c_x^2 - c_y^2) c_z,
// 3 c^4 - 6 c^2 + 1, (2 c^2 - 3)(3 c_x^2 - c^2), (2 c^2 - 3)(c_y^2 - c_z^2).
//  1. to_modes of the unit population of direction i is column i of the
//     basis, exactly (small integers);
//  2. from_modes of the unit normalised mode k is w_i e_k(c_i);
//  3. the norms bnorm(k) are sum_i w_i e_k(c_i)^2 and the rows orthogonal;
//  4. from_modes(to_modes(f) / b) returns f for random populations.
// Prints one line and returns 0 when every check passes.
#include <cmath>
#include <cstdio>
#include <random>

#include "flbm_host.cuh"

using namespace flbm;

static double poly(int k, double x, double y, double z)
{
    const double c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return c2 - 1;
        case 5: return 3 * x * x - c2;
        case 6: return y * y - z * z;
        case 7: return x * y;
        case 8: return y * z;
        case 9: return x * z;
        case 10: return (3 * c2 - 5) * x;
        case 11: return (3 * c2 - 5) * y;
        case 12: return (3 * c2 - 5) * z;
        case 13: return (y * y - z * z) * x;
        case 14: return (z * z - x * x) * y;
        case 15: return (x * x - y * y) * z;
        case 16: return 3 * c2 * c2 - 6 * c2 + 1;
        case 17: return (2 * c2 - 3) * (3 * x * x - c2);
        default: return (2 * c2 - 3) * (y * y - z * z);
    }
}

int main()
{
    double E[19][19], w[19];
    for (int i = 0; i < 19; ++i) {
        const int c2 = cxv(i) * cxv(i) + cyv(i) * cyv(i) + czv(i) * czv(i);
        w[i] = c2 == 0 ? 1.0 / 3 : (c2 == 1 ? 1.0 / 18 : 1.0 / 36);
        for (int k = 0; k < 19; ++k) E[k][i] = poly(k, cxv(i), cyv(i), czv(i));
    }
    int fails = 0;
    for (int i = 0; i < 19; ++i) {
        float f[19] = {0}, m[19];
        f[i] = 1.0f;
        to_modes(f, m);
        for (int k = 0; k < 19; ++k) fails += (double)m[k] != E[k][i];
    }
    for (int k = 0; k < 19; ++k) {
        float n[19] = {0}, f[19];
        n[k] = 1.0f;
        from_modes(n, f);
        for (int i = 0; i < 19; ++i) fails += std::fabs(f[i] - w[i] * E[k][i]) > 1e-7 * std::fabs(w[i] * E[k][i]) + 1e-9;
        for (int q = 0; q < 19; ++q) {
            double g = 0;
            for (int i = 0; i < 19; ++i) g += w[i] * E[k][i] * E[q][i];
            const double want = q == k ? (double)bnorm(k) : 0.0;
            fails += std::fabs(g - want) > 1e-7;
        }
    }
    std::mt19937_64 gen(0x19u);
    std::uniform_real_distribution<float> U(0.0f, 0.2f);
    double worst = 0;
    for (int t = 0; t < 20000; ++t) {
        float f[19], m[19], n[19], g[19];
        for (int i = 0; i < 19; ++i) f[i] = U(gen);
        to_modes(f, m);
        for (int k = 0; k < 19; ++k) n[k] = m[k] / bnorm(k);
        from_modes(n, g);
        for (int i = 0; i < 19; ++i) worst = std::max(worst, (double)std::fabs(g[i] - f[i]));
    }
    fails += worst > 2e-6;
    std::printf("round_trip_max_abs %.3e failed %d\n", worst, fails);
    return fails == 0 ? 0 : 1;
}

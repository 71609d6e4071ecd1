// Host check (no GPU) of the tile classification the step kernels rely on,
// built from the same header functions the kernels call.
//
// For random lattices, wall flags, radii, positions and tile policies:
//  1. the particle box at box_origin(X) holds exactly the nodes within R of
//     X (minimum image on periodic axes), found by box_node_inside;
//  2. every fluid node with a particle node among its 18 neighbours lies in
//     a tile for which tile_near is true, so no bulk tile reads a virtual-
//     layer density or bounces a population off the particle;
//  3. the candidate grid of the near launch reaches every near tile exactly
//     once, so each near node is updated once and each tile's force partial
//     is summed once;
//  4. solid_neighbours gives, for every fluid node, exactly the directions
//     whose neighbour (wrapped on periodic axes, none across a wall) is a
//     particle node;
//  5. every node with a wall ghost or a particle node among its neighbours is
//     an edge candidate of the adjoint (adj_edge_candidate), and the entries
//     of adj_edge_node reach every candidate exactly once and nothing else.
// Prints one line and returns 0 when every configuration passes.
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
    double uni() { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
    int range(int lo, int hi) { return lo + (int)(g() % (uint64_t)(hi - lo + 1)); }  // [lo, hi]
};

double min_image(double d, int L, int wall)
{
    if (!wall) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

// Returns the number of failed checks of one configuration (0 if it passes).
int check(const flbm_params& p, int policy, long long* near_tiles, long long* touch_nodes)
{
    KParams k;
    make_kparams(p, policy, k);
    const int L[3] = {p.lx, p.ly, p.lz};
    const int W[3] = {p.wall_x, p.wall_y, p.wall_z};
    const double X[3] = {p.pos0[0], p.pos0[1], p.pos0[2]};
    int o[3];
    box_origin(X, k, o);
    const long long N = (long long)L[0] * L[1] * L[2];
    auto idx = [&](int x, int y, int z) { return x + (long long)L[0] * (y + (long long)L[1] * z); };

    // 1. box membership against a scan of the whole lattice
    std::vector<uint8_t> solid(N, 0), scan(N, 0);
    const int B = k.B;
    for (int t = 0; t < B * B * B; ++t) {
        if (!box_node_inside(t, o, X, k)) continue;
        const int d[3] = {t % B, (t / B) % B, t / (B * B)};
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = o[a] + d[a];
            if (!W[a] && c[a] >= L[a]) c[a] -= L[a];
        }
        solid[idx(c[0], c[1], c[2])] += 1;
    }
    int fails = 0;
    for (int z = 0; z < L[2]; ++z)
        for (int y = 0; y < L[1]; ++y)
            for (int x = 0; x < L[0]; ++x) {
                const double r[3] = {min_image(x - X[0], L[0], W[0]), min_image(y - X[1], L[1], W[1]),
                                     min_image(z - X[2], L[2], W[2])};
                scan[idx(x, y, z)] = (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] < p.radius * p.radius) ? 1 : 0;
            }
    for (long long n = 0; n < N; ++n)
        if (solid[n] != scan[n]) {
            ++fails;
            break;
        }

    // 2. fluid nodes whose stencil touches the particle are in near tiles
    for (int z = 0; z < L[2]; ++z)
        for (int y = 0; y < L[1]; ++y)
            for (int x = 0; x < L[0]; ++x) {
                if (scan[idx(x, y, z)]) continue;
                bool touch = false;
                for (int i = 1; i < 19 && !touch; ++i) {
                    int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a)
                        if (q[a] < 0 || q[a] >= L[a]) {
                            if (W[a]) ok = false;
                            else q[a] = (q[a] + L[a]) % L[a];
                        }
                    touch = ok && scan[idx(q[0], q[1], q[2])];
                }
                if (!touch) continue;
                ++*touch_nodes;
                if (!tile_near(x / k.tx, y / k.ty, z, o, k)) ++fails;
            }

    // 4. the links found from box coordinates against the lattice scan
    std::vector<uint8_t> mask((size_t)B * B * B);
    for (int t = 0; t < B * B * B; ++t) mask[t] = box_node_inside(t, o, X, k) ? 1 : 0;
    for (int z = 0; z < L[2]; ++z)
        for (int y = 0; y < L[1]; ++y)
            for (int x = 0; x < L[0]; ++x) {
                if (scan[idx(x, y, z)]) continue;
                uint32_t want = 0;
                for (int i = 1; i < 19; ++i) {
                    int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a)
                        if (q[a] < 0 || q[a] >= L[a]) {
                            if (W[a]) ok = false;
                            else q[a] = (q[a] + L[a]) % L[a];
                        }
                    if (ok && scan[idx(q[0], q[1], q[2])]) want |= 1u << i;
                }
                if (solid_neighbours(x, y, z, o, mask.data(), k) != want) {
                    ++fails;
                    z = L[2];
                    break;
                }
            }

    // 5. edge candidates of the adjoint and their enumeration
    {
        std::vector<int> tally(N, 0);
        const long long ne = adj_edge_entries(k);
        for (long long t = 0; t < ne; ++t) {
            int c[3];
            if (adj_edge_node(t, o, k, c)) {
                bool ok = true;
                for (int a = 0; a < 3; ++a) ok = ok && c[a] >= 0 && c[a] < L[a];
                if (!ok) { ++fails; break; }
                tally[idx(c[0], c[1], c[2])] += 1;
            }
        }
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    const int c[3] = {x, y, z};
                    const bool cand = adj_edge_candidate(c, o, k);
                    if (tally[idx(x, y, z)] != (cand ? 1 : 0)) ++fails;
                    bool needs = false;  // a wall ghost or a particle node among the neighbours
                    for (int i = 1; i < 19 && !needs; ++i) {
                        int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
                        bool ghost = false;
                        for (int a = 0; a < 3; ++a)
                            if (q[a] < 0 || q[a] >= L[a]) {
                                if (W[a]) ghost = true;
                                else q[a] = (q[a] + L[a]) % L[a];
                            }
                        needs = ghost || scan[idx(q[0], q[1], q[2])];
                    }
                    if (needs && !cand) ++fails;
                }
    }

    // 3. the candidate grid reaches every near tile exactly once
    std::vector<int> hits((size_t)k.gx * k.gy * k.lz, 0);
    for (int cz = 0; cz < k.ncz; ++cz)
        for (int cy = 0; cy < k.ncy; ++cy)
            for (int cx = 0; cx < k.ncx; ++cx) {
                const int bx = candidate_tile(cx, o[0], k.tx, k.gx, k.lx, k.wall[0]);
                const int by = candidate_tile(cy, o[1], k.ty, k.gy, k.ly, k.wall[1]);
                const int bz = candidate_tile(cz, o[2], 1, k.lz, k.lz, k.wall[2]);
                if (bx < 0 || by < 0 || bz < 0) continue;
                if (tile_near(bx, by, bz, o, k)) hits[bx + (size_t)k.gx * (by + (size_t)k.gy * bz)] += 1;
            }
    for (int bz = 0; bz < k.lz; ++bz)
        for (int by = 0; by < k.gy; ++by)
            for (int bx = 0; bx < k.gx; ++bx) {
                const int h = hits[bx + (size_t)k.gx * (by + (size_t)k.gy * bz)];
                if (tile_near(bx, by, bz, o, k)) {
                    ++*near_tiles;
                    if (h != 1) ++fails;
                } else if (h != 0) {
                    ++fails;
                }
            }
    return fails;
}

}  // namespace

int main(int argc, char** argv)
{
    const int trials = argc > 1 ? std::atoi(argv[1]) : 600;
    Rng rng(0x5eed1909ull);
    int run = 0, failed = 0;
    long long near_tiles = 0, touch_nodes = 0;
    for (int t = 0; t < trials; ++t) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.rho_b0 = 0.05;
        p.rho_p_ratio = 1.5;
        p.radius = 0.6 + 7.4 * rng.uni() * rng.uni();
        const int need = (int)std::ceil(2.0 * p.radius) + 4;
        int* Ls[3] = {&p.lx, &p.ly, &p.lz};
        int* Ws[3] = {&p.wall_x, &p.wall_y, &p.wall_z};
        for (int a = 0; a < 3; ++a) {
            *Ws[a] = rng.range(0, 1);
            *Ls[a] = rng.range(need, std::max(need, 44));
            const int La = *Ls[a];
            if (*Ws[a]) {
                const double lo = p.radius - 0.5, hi = La - 0.5 - p.radius;
                p.pos0[a] = lo + (hi - lo) * rng.uni();
            } else {
                // anywhere on the axis, often just off a node or a periodic seam
                const double u = rng.uni();
                p.pos0[a] = u < 0.2 ? (double)rng.range(0, La - 1) + 1e-9 * (rng.uni() - 0.5)
                          : u < 0.3 ? La - 1e-7 * rng.uni() : La * rng.uni();
                if (p.pos0[a] >= La) p.pos0[a] -= La;
                if (p.pos0[a] < 0.0) p.pos0[a] += La;
            }
        }
        if (!validate(&p).empty()) continue;
        for (int policy = 0; policy < 2; ++policy) {
            ++run;
            const int f = check(p, policy, &near_tiles, &touch_nodes);
            if (f) {
                ++failed;
                if (failed <= 5)
                    std::printf("FAIL %d checks: L=%dx%dx%d walls=%d%d%d R=%.4f X=(%.9f %.9f %.9f) policy=%d\n", f,
                                p.lx, p.ly, p.lz, p.wall_x, p.wall_y, p.wall_z, p.radius, p.pos0[0], p.pos0[1],
                                p.pos0[2], policy);
            }
        }
    }
    std::printf("configurations %d failed %d near_tiles %lld touching_nodes %lld\n", run, failed, near_tiles,
                touch_nodes);
    return failed == 0 && run > 0 ? 0 : 1;
}

// Host check (no GPU) of the bookkeeping of the fused collide's densities,
// built from the header functions the kernels call (DensitySink, gather_column,
// gather_ring, roll_update, put_density, TileRing, finish_node, FinishItems,
// ring_pos, tile_near_xy, block_meets_near, near_dilated, near_box_axis).
//
// For random lattices (sizes, walls, ragged tiles), planes per block and
// particle boxes, every node pushes random values for its 19 directions, with
// halfway bounce-back at walls exactly as the collide routes them. The direct
// sum of what lands in each node's 19 slots is the density the step must
// produce. The check replays the fused kernel's data flow block by block,
// skipping the planes of near-particle tiles (the near launch's), and then the
// completion (part B). Every node outside the near-particle region dilated
// by one node must come out equal to the direct sum to float rounding, and
// be written. The region itself must lie inside part A's box (the candidate
// tiles plus one node). Prints one line and returns 0 when every
// configuration passes.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>

#include "flbm_fused.cuh"
#include "flbm_host.cuh"

using namespace flbm;

namespace {

struct Rng {
    std::mt19937_64 g;
    explicit Rng(uint64_t s) : g(s) {}
    double uni() { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); }
    int range(int lo, int hi) { return lo + (int)(g() % (uint64_t)(hi - lo + 1)); }
};

// Destination node and slot direction of the push of direction i from node
// (x, y, z): the neighbour along c_i, or the node itself (direction opp(i))
// when c_i crosses a wall.
long long push_target(int x, int y, int z, int i, const KParams& P)
{
    int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
    const int L[3] = {P.lx, P.ly, P.lz};
    for (int a = 0; a < 3; ++a)
        if (q[a] < 0 || q[a] >= L[a]) {
            if (P.wall[a]) return x + (long long)P.lx * (y + (long long)P.ly * z);
            q[a] += q[a] < 0 ? L[a] : -L[a];
        }
    return q[0] + (long long)P.lx * (q[1] + (long long)P.ly * q[2]);
}

bool wall_crossed(int x, int y, int z, int i, const KParams& P)
{
    const int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
    const int L[3] = {P.lx, P.ly, P.lz};
    for (int a = 0; a < 3; ++a)
        if ((q[a] < 0 || q[a] >= L[a]) && P.wall[a]) return true;
    return false;
}

}  // namespace

int main(int argc, char** argv)
{
    const int nconf = argc > 1 ? std::atoi(argv[1]) : 300;
    Rng R(77);
    int run = 0, failed = 0, with_particle = 0;
    long long checked_nodes = 0;
    for (int c = 0; c < nconf * 4 && run < nconf; ++c) {
        flbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.lx = R.range(5, 100);
        p.ly = R.range(2, 60);
        p.lz = R.range(1, 14);
        p.wall_x = R.range(0, 1);
        p.wall_y = R.range(0, 1);
        p.wall_z = R.range(0, 1);
        p.tau_s = p.tau_d = p.tau_g = 1.0;
        p.rho_a0 = 1.0;
        p.rho_b0 = 0.05;
        p.rho_p_ratio = 1.5;
        const bool part = R.range(0, 2) > 0;
        if (part) {
            p.radius = 1.0 + 3.0 * R.uni();
            const int L[3] = {p.lx, p.ly, p.lz};
            const int w[3] = {p.wall_x, p.wall_y, p.wall_z};
            for (int a = 0; a < 3; ++a) {
                const double lo = w[a] ? p.radius - 0.5 : 0.0, hi = w[a] ? L[a] - 0.5 - p.radius : (double)L[a];
                p.pos0[a] = lo + (hi - lo) * R.uni();
            }
        }
        if (!validate(&p).empty()) continue;
        KParams P;
        make_kparams(p, 0, P);
        if (!fused_ok(P)) continue;
        ++run;
        with_particle += P.has_particle;
        FusedGeom G;
        G.K = R.range(1, P.lz);
        G.nchunk = (P.lz + G.K - 1) / G.K;
        G.ring = 2 * (P.tx + 2) + 2 * P.ty;
        G.fp = (P.tx + 2) * (P.ty + 2);
        int o[3] = {0, 0, 0};
        if (P.has_particle) box_origin(p.pos0, P, o);
        const long long N = P.N;
        // Pushed values and the direct sums.
        std::vector<float> val((size_t)2 * 19 * N);
        for (auto& v : val) v = (float)(0.01 + R.uni());
        std::vector<double> direct((size_t)2 * N, 0.0);
        for (int z = 0; z < P.lz; ++z)
            for (int y = 0; y < P.ly; ++y)
                for (int x = 0; x < P.lx; ++x) {
                    const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
                    for (int l = 0; l < 2; ++l)
                        for (int i = 0; i < 19; ++i)
                            direct[(size_t)l * N + push_target(x, y, z, i, P)] += val[((size_t)l * 19 + i) * N + n];
                }
        // Fused collide, block by block.
        std::vector<float> psi((size_t)2 * P.padn, NAN);
        std::vector<float2> ring((size_t)P.gx * P.gy * P.lz * G.ring, make_float2(NAN, NAN));
        std::vector<float2> seam((size_t)P.gx * P.gy * G.nchunk * 2 * G.fp, make_float2(NAN, NAN));
        std::vector<float2> xch((size_t)kXchDirs * xch_size(P));
        for (int ch = 0; ch < G.nchunk; ++ch)
            for (int by = 0; by < P.gy; ++by)
                for (int bx = 0; bx < P.gx; ++bx) {
                    const int tile = bx + P.gx * by;
                    const int w = tile_w(bx, P), h = tile_h(by, P);
                    const int z0 = ch * G.K, z1 = std::min(z0 + G.K, P.lz);
                    const float2 zero = make_float2(0.0f, 0.0f);
                    std::vector<float2> roll((size_t)2 * kThreadsStep, zero), rollr((size_t)2 * kRingMax, zero);
                    std::fill(xch.begin(), xch.end(), zero);
                    std::vector<DensitySink> sinks;
                    for (int tid = 0; tid < kThreadsStep; ++tid)
                        sinks.emplace_back(reinterpret_cast<float*>(xch.data()), 0, xch_size(P));
                    const bool nxy = P.has_particle && tile_near_xy(bx, by, o, P);
                    for (int z = z0; z < z1; ++z) {
                        if (P.has_particle && tile_near(bx, by, z, o, P) != (nxy && ranges_meet(z, 1, o[2] - 1, P.B + 2, P.lz, P.wall[2]))) {
                            std::printf("hoisted near test differs\n");
                            return 1;
                        }
                        if (P.has_particle && tile_near(bx, by, z, o, P)) {
                            std::fill(roll.begin(), roll.end(), zero);
                            std::fill(rollr.begin(), rollr.end(), zero);
                            continue;
                        }
                        for (int tid = 0; tid < kThreadsStep; ++tid) {
                            const int tx = tid % P.tx, ty = tid / P.tx;
                            sinks[tid] = DensitySink(reinterpret_cast<float*>(xch.data()), xch_pos(tx, ty, P),
                                                     xch_size(P));
                            if (tx >= w || ty >= h) continue;
                            const int x = bx * P.tx + tx, y = by * P.ty + ty;
                            const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
                            for (int l = 0; l < 2; ++l)
                                for (int i = 0; i < 19; ++i)
                                    sinks[tid].put(l, i, val[((size_t)l * 19 + i) * N + n], wall_crossed(x, y, z, i, P));
                        }
                        for (int tid = 0; tid < kThreadsStep; ++tid) {
                            const int tx = tid % P.tx, ty = tid / P.tx;
                            if (tx < w && ty < h) {
                                float2 inc[3] = {zero, zero, zero};
                                gather_column(xch_pos(tx, ty, P), xch.data(), P, inc);
                                float2 rl[2] = {roll[tid], roll[kThreadsStep + tid]};
                                const float2 r = roll_update(rl, sinks[tid].own, inc);
                                roll[tid] = rl[0];
                                roll[kThreadsStep + tid] = rl[1];
                                put_density(z - 1, tx, ty, true, -1, r, tile, bx, by, ch, z0, z1, psi.data(),
                                            ring.data(), seam.data(), P, G);
                            }
                            int fx, fy;
                            if (tid < G.ring && ring_pos(tid, w, h, P, fx, fy) && fp_node(bx, by, fx, fy, P)) {
                                float2 inc[3] = {zero, zero, zero};
                                gather_ring(ring_side(tid, P), xch_pos(fx, fy, P), xch.data(), P, inc);
                                const float none[2][3] = {{0, 0, 0}, {0, 0, 0}};
                                float2 rl[2] = {rollr[tid], rollr[kRingMax + tid]};
                                const float2 r = roll_update(rl, none, inc);
                                rollr[tid] = rl[0];
                                rollr[kRingMax + tid] = rl[1];
                                put_density(z - 1, fx, fy, false, tid, r, tile, bx, by, ch, z0, z1, psi.data(),
                                            ring.data(), seam.data(), P, G);
                            }
                        }
                    }
                    for (int tid = 0; tid < kThreadsStep; ++tid) {
                        const int tx = tid % P.tx, ty = tid / P.tx;
                        if (tx < w && ty < h) {
                            put_density(z1 - 1, tx, ty, true, -1, roll[tid], tile, bx, by, ch, z0, z1, psi.data(),
                                        ring.data(), seam.data(), P, G);
                            put_density(z1, tx, ty, true, -1, roll[kThreadsStep + tid], tile, bx, by, ch, z0, z1,
                                        psi.data(), ring.data(), seam.data(), P, G);
                        }
                        int fx, fy;
                        if (tid < G.ring && ring_pos(tid, w, h, P, fx, fy) && fp_node(bx, by, fx, fy, P)) {
                            put_density(z1 - 1, fx, fy, false, tid, rollr[tid], tile, bx, by, ch, z0, z1, psi.data(),
                                        ring.data(), seam.data(), P, G);
                            put_density(z1, fx, fy, false, tid, rollr[kRingMax + tid], tile, bx, by, ch, z0, z1,
                                        psi.data(), ring.data(), seam.data(), P, G);
                        }
                    }
                }
        // Completion, part B: each (tile, chunk) block's item list.
        std::vector<int> visits((size_t)N, 0);
        for (int b = 0; b < P.gx * P.gy * G.nchunk; ++b) {
            const int ntile = P.gx * P.gy;
            const int tile = b % ntile, ch = b / ntile;
            const int bx = tile % P.gx, by = tile / P.gx;
            const int w = tile_w(bx, P), h = tile_h(by, P);
            const int z0 = ch * G.K, z1 = std::min(z0 + G.K, P.lz);
            const TileRing TR(bx, by, P);
            const bool check = P.has_particle && block_meets_near(bx, by, z0, z1, o, P);
            const FinishItems items(z0, z1, w, h, P);
            const long long total = items.count();
            for (long long it = 0; it < total; ++it) {
                int z, fx, fy;
                items.item(it, z, fx, fy);
                const int x = bx * P.tx + fx, y = by * P.ty + fy;
                visits[x + (long long)P.lx * (y + (long long)P.ly * z)] += 1;
                const bool nd = P.has_particle && near_dilated(x, y, z, o, P);
                if (nd && !check) {
                    std::printf("block_meets_near missed a near node\n");
                    return 1;
                }
                if (nd) continue;
                finish_node(fx, fy, z, bx, by, ch, TR, psi.data(), ring.data(), seam.data(), P, G);
            }
        }
        // Part A's box must hold the dilated near region.
        int xs, nxb, ys, nyb, zs, nzb;
        near_box_axis(o[0], P.tx, P.ncx, P.gx, P.lx, P.wall[0], xs, nxb);
        near_box_axis(o[1], P.ty, P.ncy, P.gy, P.ly, P.wall[1], ys, nyb);
        near_box_axis(o[2], 1, P.ncz, P.lz, P.lz, P.wall[2], zs, nzb);
        auto in_axis = [](int v, int s, int n, int L, int wall) {
            for (int k = 0; k < n; ++k) {
                int q = s + k;
                if (q < 0 || q >= L) {
                    if (wall) continue;
                    q = ((q % L) + L) % L;
                }
                if (q == v) return true;
            }
            return false;
        };
        bool ok = true;
        for (int z = 0; z < P.lz && ok; ++z)
            for (int y = 0; y < P.ly && ok; ++y)
                for (int x = 0; x < P.lx && ok; ++x) {
                    const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
                    const bool nd = P.has_particle && near_dilated(x, y, z, o, P);
                    if (nd) {
                        if (!(in_axis(x, xs, nxb, P.lx, P.wall[0]) && in_axis(y, ys, nyb, P.ly, P.wall[1]) &&
                              in_axis(z, zs, nzb, P.lz, P.wall[2]))) {
                            std::printf("near node (%d %d %d) outside part A's box\n", x, y, z);
                            ok = false;
                        }
                        continue;
                    }
                    if (visits[n] > 1) {
                        std::printf("node (%d %d %d) completed %d times\n", x, y, z, visits[n]);
                        ok = false;
                    }
                    const long long q = pad_index(x, y, z, P);
                    for (int l = 0; l < 2 && ok; ++l) {
                        const double got = psi[(size_t)l * P.padn + q], want = direct[(size_t)l * N + n];
                        if (!(std::fabs(got - want) <= 2e-6 * want)) {
                            std::printf("lattice %dx%dx%d walls %d%d%d tx %d K %d part %d: node (%d %d %d) l %d got %g want %g\n",
                                        P.lx, P.ly, P.lz, P.wall[0], P.wall[1], P.wall[2], P.tx, G.K, P.has_particle, x, y,
                                        z, l, got, want);
                            ok = false;
                        }
                    }
                    ++checked_nodes;
                }
        failed += !ok;
    }
    std::printf("configurations %d failed %d with_particle %d nodes %lld\n", run, failed, with_particle, checked_nodes);
    return failed == 0 ? 0 : 1;
}

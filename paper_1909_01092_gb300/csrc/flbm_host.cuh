// Host-side parameter checks and kernel parameter set-up, shared by the
// single-simulation and the ensemble entry points.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "flbm.h"
#include "flbm_kernels.cuh"

namespace flbm {

inline int ceil_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

inline bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Parameter checks; returns an empty string if valid.
inline std::string validate(const flbm_params* p)
{
    if (!p) return "params is NULL";
    if (p->lx < 1 || p->ly < 1 || p->lz < 1) return "lattice sizes must be >= 1";
    if (p->lz > 65535 || p->ly > 65535 * 256) return "lattice too large for the launch grid";
    const double n = (double)p->lx * p->ly * p->lz;
    if (38.0 * n > 4294967295.0) return "more than 2^32/38 nodes (32-bit population indices)";
    const int w[3] = {p->wall_x, p->wall_y, p->wall_z};
    for (int a = 0; a < 3; ++a)
        if (w[a] != 0 && w[a] != 1) return "wall flags must be 0 or 1";
    if (!(p->tau_s > 0.5) || !(p->tau_d > 0.5) || !(p->tau_g > 0.5)) return "relaxation times must exceed 1/2";
    if (!std::isfinite(p->G) || !std::isfinite(p->kT) || p->kT < 0.0) return "G must be finite and kT >= 0";
    if (!(p->rho_a0 >= 0.0) || !(p->rho_b0 >= 0.0) || !(p->rho_a0 + p->rho_b0 > 0.0)) return "initial densities";
    if (!(p->init_pert >= 0.0 && p->init_pert < 1.0)) return "init_pert must be in [0, 1)";
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->fluid_force[a])) return "fluid_force must be finite";
    if (p->fluid_counterforce != 0 && p->fluid_counterforce != 1) return "fluid_counterforce must be 0 or 1";
    if (p->radius > 0.0) {
        if (!finite_pos(p->rho_p_ratio) || !std::isfinite(p->g) || !std::isfinite(p->delta_rho))
            return "particle parameters must be finite, rho_p_ratio > 0";
        const int L[3] = {p->lx, p->ly, p->lz};
        const int B = (int)std::ceil(2.0 * p->radius) + 2;
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(p->pos0[a])) return "pos0 must be finite";
            if (w[a]) {
                if (p->pos0[a] - p->radius < -0.5 || p->pos0[a] + p->radius > L[a] - 0.5)
                    return "the sphere must lie inside the walls";
            } else if (B + 2 > L[a]) {
                return "periodic axis too short for the sphere (need L >= ceil(2R) + 4)";
            }
        }
    }
    return "";
}

// Tile width along x (a power of two, at most 32; TX * TY = 256 threads).
// Policy 0: the smallest power of two >= lx (capped at 32). Policy 1: the
// largest of 32, 16, 8 that divides lx, so no lane of a tile row idles; if
// none divides lx, as policy 0.
inline int tile_width(int lx, int policy)
{
    if (policy == 1)
        for (int t : {32, 16, 8})
            if (lx % t == 0) return t;
    return std::min(32, ceil_pow2(lx));
}

inline void make_kparams(const flbm_params& p, int tile_policy, KParams& k)
{
    std::memset(&k, 0, sizeof(k));
    k.lx = p.lx; k.ly = p.ly; k.lz = p.lz;
    k.wall[0] = p.wall_x; k.wall[1] = p.wall_y; k.wall[2] = p.wall_z;
    k.px = (p.lx + 2 + 3) / 4 * 4;  // row stride: lx + 2 nodes, rounded up to 16 bytes
    k.py = p.ly + 2; k.pz = p.lz + 2;
    k.N = (long long)p.lx * p.ly * p.lz;
    k.padn = (long long)k.px * k.py * k.pz;
    k.tx = tile_width(p.lx, tile_policy);
    k.ty = kThreads / k.tx;
    k.gx = (p.lx + k.tx - 1) / k.tx;
    k.gy = (p.ly + k.ty - 1) / k.ty;
    k.G = (float)p.G;
    const double gs = 1.0 - 1.0 / p.tau_s, gd = 1.0 - 1.0 / p.tau_d, gg = 1.0 - 1.0 / p.tau_g;
    k.gs = (float)gs; k.gd = (float)gd; k.gg = (float)gg;
    for (int a = 0; a < 3; ++a) k.ext[a] = (float)p.fluid_force[a];
    k.drho = (float)p.delta_rho;
    k.kT = (float)p.kT;
    const double b[19] = {1, 1. / 3, 1. / 3, 1. / 3, 2. / 3, 4. / 3, 4. / 9, 1. / 9, 1. / 9, 1. / 9,
                          2. / 3, 2. / 3, 2. / 3, 2. / 9, 2. / 9, 2. / 9, 2, 4. / 3, 4. / 9};
    for (int q = 0; q < 19; ++q) {
        const double gm = (q <= 9) ? gs : gg;
        k.nz_mode[q] = (q >= 4) ? (float)std::sqrt((1.0 - gm * gm) / b[q]) : 0.0f;
    }
    k.nz_j = (float)std::sqrt(1.0 - gd * gd);
    k.key0 = (uint32_t)(p.seed & 0xffffffffu);
    k.key1 = (uint32_t)(p.seed >> 32) ^ p.replica;
    for (int r = 0; r < 10; ++r) {
        k.rk0[r] = k.key0 + (uint32_t)r * 0x9E3779B9u;
        k.rk1[r] = k.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    k.has_particle = p.radius > 0.0 ? 1 : 0;
    k.B = k.has_particle ? (int)std::ceil(2.0 * p.radius) + 2 : 1;
    k.R = p.radius;
    if (k.has_particle) {  // the mass and moment of inertia of initial_state
        const double vol = 4.0 / 3.0 * M_PI * p.radius * p.radius * p.radius;
        const double mp = vol * (p.rho_p_ratio * (p.rho_a0 + p.rho_b0));
        k.inv_mp = 1.0 / mp;
        k.inv_Ip = 1.0 / (0.4 * mp * p.radius * p.radius);
    }
    k.rho0[0] = p.rho_a0; k.rho0[1] = p.rho_b0;
    k.counterforce = p.fluid_counterforce;
    // Candidate tiles that can meet the particle box grown by one node.
    k.ncx = std::min(k.gx, (k.B + 2 + k.tx - 1) / k.tx + 2);
    k.ncy = std::min(k.gy, (k.B + 2 + k.ty - 1) / k.ty + 2);
    k.ncz = std::min(p.lz, k.B + 2);
    k.tau1 = (p.tau_s == 1.0 && p.tau_d == 1.0 && p.tau_g == 1.0) ? 1 : 0;
    for (int q = 0; q < 38; ++q) k.dirN[q] = (uint32_t)((long long)q * k.N);
}


// Tiles of one z-plane grid, candidate near tiles and particle-box blocks.
inline long long tile_count(const KParams& k) { return (long long)k.gx * k.gy * k.lz; }
inline long long cand_count(const KParams& k) { return (long long)k.ncx * k.ncy * k.ncz; }
inline int box_block_count(const KParams& k) { return (k.B * k.B * k.B + 255) / 256; }

// Groups of replicas for launches whose grid is (largest block count of the
// group, members): blocks[r] > 0 is replica r's block count (0: not in any
// launch). Replicas by decreasing block count (stable); a group takes
// replicas while it has fewer than cap and each has at least 3/4 of its
// first member's blocks, so that at most a quarter of a launch's blocks
// find no work.
inline std::vector<std::vector<int>> group_by_blocks(const std::vector<long long>& blocks, int cap)
{
    std::vector<int> order;
    for (int r = 0; r < (int)blocks.size(); ++r)
        if (blocks[r] > 0) order.push_back(r);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return blocks[a] > blocks[b]; });
    std::vector<std::vector<int>> groups;
    for (int r : order) {
        if (groups.empty() || (int)groups.back().size() == cap || 4 * blocks[r] < 3 * blocks[groups.back()[0]])
            groups.emplace_back();
        groups.back().push_back(r);
    }
    return groups;
}

// Particle record at creation (Section 3, Eq. (fp)): sphere of radius R at
// pos0, at rest, mass 4/3 pi R^3 rho_p, moment of inertia 2/5 m_p R^2.
inline DevState initial_state(const flbm_params& p, const KParams& k)
{
    DevState s;
    std::memset(&s, 0, sizeof(s));
    if (k.has_particle) {
        const double vol = 4.0 / 3.0 * M_PI * p.radius * p.radius * p.radius;
        const double rho_tot = p.rho_a0 + p.rho_b0;
        const double rho_p = p.rho_p_ratio * rho_tot;
        s.mp = vol * rho_p;
        s.Ip = 0.4 * s.mp * p.radius * p.radius;
        s.Fp = vol * (rho_p - rho_tot) * p.g;
        for (int a = 0; a < 3; ++a) s.X[a] = p.pos0[a];
    }
    s.nfluid = k.N;
    return s;
}

// Observables record from the reduced sums v (mass A, mass B, momentum,
// kinetic energy, non-finite count) and the particle record.
inline void fill_obs(const double v[8], const DevState& s, flbm_obs* out)
{
    out->mass[0] = v[0];
    out->mass[1] = v[1];
    for (int a = 0; a < 3; ++a) {
        out->momentum[a] = v[2 + a];
        out->particle_momentum[a] = s.mp * s.V[a];
    }
    out->kinetic = v[5];
    out->pending_mass[0] = s.delta[0] * (double)s.nfluid;
    out->pending_mass[1] = s.delta[1] * (double)s.nfluid;
    out->nfluid = s.nfluid;
    out->step = s.step;
    out->nonfinite = (int64_t)v[6];
}

// Temperatures of the fluctuating modes from the kObsModes sums of
// k_obs_modes (definitions at flbm_obs): each is a ratio of two sums over the
// bulk fluid nodes.
inline void fill_mode_obs(const double vm[kObsModes], flbm_obs* out)
{
    const double b[19] = {1, 1. / 3, 1. / 3, 1. / 3, 2. / 3, 4. / 3, 4. / 9, 1. / 9, 1. / 9, 1. / 9,
                          2. / 3, 2. / 3, 2. / 3, 2. / 9, 2. / 9, 2. / 9, 2, 4. / 3, 4. / 9};
    for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 19; ++k)
            out->mode_temp[l][k] = (k >= 4 && vm[30 + l] > 0.0) ? vm[15 * l + k - 4] / (3.0 * b[k] * vm[30 + l]) : 0.0;
    const double rt = vm[30] + vm[31];
    for (int a = 0; a < 3; ++a) {
        out->diff_temp[a] = vm[35] > 0.0 ? vm[32 + a] / vm[35] : 0.0;
        out->mom_temp[a] = rt > 0.0 ? vm[36 + a] / rt : 0.0;
    }
    out->n_bulk = (int64_t)vm[39];
}

// Checks of a particle record read from a checkpoint file before it goes to
// the device; returns an empty string if it is usable. The step kernels index
// the particle masks with cur and the box origin, so a corrupt or foreign
// record must not reach them.
inline std::string check_restored_state(const DevState& s, const KParams& k)
{
    if (s.cur != 0 && s.cur != 1) return "mask index out of range";
    if (s.nfluid < 0 || s.nfluid > k.N) return "fluid node count out of range";
    if (s.step < 0) return "negative step count";
    if (!std::isfinite(s.delta[0]) || !std::isfinite(s.delta[1])) return "non-finite mass correction";
    if (!k.has_particle) return "";
    for (int a = 0; a < 3; ++a) {
        const double v[6] = {s.X[a], s.V[a], s.Vavg[a], s.Om[a], s.Ppend[a], s.Lpend[a]};
        for (double x : v)
            if (!std::isfinite(x)) return "non-finite particle state";
    }
    const int L[3] = {k.lx, k.ly, k.lz};
    for (int a = 0; a < 3; ++a) {
        if (k.wall[a] && (s.X[a] - k.R < -0.5 || s.X[a] + k.R > L[a] - 0.5)) return "sphere outside the walls";
        if (!k.wall[a] && (s.X[a] < 0.0 || s.X[a] >= L[a])) return "centre outside the periodic box";
    }
    int o[3];
    box_origin(s.X, k, o);
    for (int a = 0; a < 3; ++a)
        if (o[a] != s.box0[a]) return "box origin does not match the centre";
    return "";
}

inline int copy_particle(const DevState& s, flbm_particle* out)
{
    for (int a = 0; a < 3; ++a) {
        out->X[a] = s.X[a]; out->V[a] = s.V[a]; out->Vavg[a] = s.Vavg[a]; out->Omega[a] = s.Om[a];
        out->F[a] = s.F[a]; out->T[a] = s.T[a]; out->P_pending[a] = s.Ppend[a]; out->L_pending[a] = s.Lpend[a];
    }
    out->delta[0] = s.delta[0];
    out->delta[1] = s.delta[1];
    out->mp = s.mp;
    out->Fp = s.Fp;
    out->nfluid = s.nfluid;
    out->step = s.step;
    return FLBM_OK;
}

}  // namespace flbm

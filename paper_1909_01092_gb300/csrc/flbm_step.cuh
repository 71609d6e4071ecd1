// The collide-stream kernels and the particle update of one FLBM step
// (arXiv:1909.01092, Section 2: Eq. (lbe), Eq. (sc-force), particle coupling;
// Section 3: Eq. (fp), channel walls).
//
// Tiles (TX x TY nodes of one z-plane, one CTA each) split into two sets:
//   bulk tiles  : no node of the tile or its one-node halo is a particle node;
//                 k_collide_bulk runs them with no particle code at all.
//   near tiles  : the tile meets the particle box grown by one node;
//                 k_collide_near runs them over a fixed grid of candidates
//                 around the box and reduces force, torque and mass ledger.
// Both kernels apply the same tile_near() test, so every tile runs exactly once.
// The particle update runs in the last block of the near launch (after every
// candidate's partials are written); the next-position masks and the
// cover/uncover pass run over the particle box, and the last block of the
// cover launch does the step's bookkeeping. "Last block" is an atomic ticket
// per launch: no block waits for another.
#pragma once

#include "flbm_device.cuh"

#ifndef FLBM_BULK_MINBLOCKS
#define FLBM_BULK_MINBLOCKS 4  // resident 256-thread blocks per SM the bulk kernel is compiled for
#endif

namespace flbm {

// Philox4x32-10 with the round keys precomputed on the host (key + r * Weyl).
// The high and low halves of each 32 x 32-bit product are taken separately
// (this compiles to fewer instructions and registers than a 64-bit product).
__host__ __device__ __forceinline__ void philox_rk(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                                   const KParams& P)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = mulhi32(0xD2511F53u, x0), l0 = 0xD2511F53u * x0;
        const uint32_t h1 = mulhi32(0xCD9E8D57u, x2), l1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = h1 ^ x1 ^ P.rk0[r];
        const uint32_t y2 = h0 ^ x3 ^ P.rk1[r];
        x0 = y0;
        x1 = l1;
        x2 = y2;
        x3 = l0;
    }
}

// Box-Muller pair from two Philox words with the hardware approximations of
// log2, rsqrt, sin and cos: z0 = r cos(2 pi u2), z1 = r sin(2 pi u2) with
// r = sqrt(-2 ln u1); the angle is taken as 2 pi (u2 - 1/2) in (-pi, pi),
// where the approximations are accurate, and the signs flipped back. The
// flush-to-zero forms are used: their inputs and results here (u1 >= 2^-24,
// |angle| >= 2^-22, -2 ln u1 of about 2^-23 at least) lie far above the
// subnormal range, where both forms agree, and they skip the rescaling of
// subnormal inputs.
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, float& z0, float& z1)
{
    const float u1 = uniform_open(w1);
    float lg, rs, s, c;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(u1));
    const float e = -1.38629436112f * lg;  // -2 ln u1 > 0
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(e));
    const float r = e * rs;
    // 2 pi (u2 - 1/2) with u2 = ((w2 >> 9) + 1/2) 2^-23, as one multiply-add.
    constexpr float kA = (float)(6.283185307179586 / 8388608.0);
    constexpr float kB = (float)(6.283185307179586 * (0.5 / 8388608.0 - 0.5));
    const float ang = __fmaf_rn((float)(w2 >> 9), kA, kB);
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(ang));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(ang));
    z0 = -r * c;
    z1 = -r * s;
}

// FP32 sums over the particle links of one node.
struct LinkSums {
    float F[3] = {0.0f, 0.0f, 0.0f};    // force on the particle
    float T[3] = {0.0f, 0.0f, 0.0f};    // torque about the node (lever c_i / 2)
    float led[2] = {0.0f, 0.0f};        // mass put in by the moving link rule
};

// Adds the force m c_i acting at the link midpoint x + c_i / 2.
__device__ __forceinline__ void link_add(LinkSums& s, float m, int cx, int cy, int cz)
{
    const float fr[3] = {m * cx, m * cy, m * cz};
    s.F[0] += fr[0]; s.F[1] += fr[1]; s.F[2] += fr[2];
    s.T[0] += 0.5f * (cy * fr[2] - cz * fr[1]);
    s.T[1] += 0.5f * (cz * fr[0] - cx * fr[2]);
    s.T[2] += 0.5f * (cx * fr[1] - cy * fr[0]);
}

// Density and momentum of one component from its 19 populations.
__device__ __forceinline__ void moments(const float f[19], float& rho, float j[3])
{
    const float s1 = f[1] + f[2], s2 = f[3] + f[4], s3 = f[5] + f[6];
    const float s7 = f[7] + f[8], s9 = f[9] + f[10], s11 = f[11] + f[12];
    const float s13 = f[13] + f[14], s15 = f[15] + f[16], s17 = f[17] + f[18];
    const float d7 = f[7] - f[8], d9 = f[9] - f[10], d11 = f[11] - f[12];
    const float d13 = f[13] - f[14], d15 = f[15] - f[16], d17 = f[17] - f[18];
    rho = f[0] + (s1 + s2 + s3) + (s7 + s9) + (s11 + s13) + (s15 + s17);
    j[0] = (f[1] - f[2]) + d7 + d9 + d11 + d13;
    j[1] = (f[3] - f[4]) + d7 - d9 + d15 + d17;
    j[2] = (f[5] - f[6]) + d11 - d13 + d15 - d17;
}

// Where collide_core reads a node's inputs: f(q) is population q = 19 l + i
// of the node, psa(i) / psb(i) the densities rho_A / rho_B of neighbour
// x + c_i in the padded psi field.
struct GlobalInputs {
    const float* __restrict__ fin;  // current populations; (l, i) of node m at m + P.dirN[19 l + i]
    const float* __restrict__ pA;   // psi_A at the node (padded field); psi_B at pA + padn
    uint32_t n;
    long long padn;
    int sy, sz;                      // padded row and plane strides
    __device__ __forceinline__ GlobalInputs(const float* f, const float* psi, int x, int y, int z, uint32_t node,
                                            const KParams& P)
        : fin(f), pA(psi + pad_index(x, y, z, P)), n(node), padn(P.padn), sy(P.px), sz(P.px * P.py)
    {
    }
    __device__ __forceinline__ float f(int q, const KParams& P) const { return __ldg(fin + (n + P.dirN[q])); }
    __device__ __forceinline__ int off(int i) const { return cxv(i) + sy * cyv(i) + sz * czv(i); }
    __device__ __forceinline__ float psa(int i) const { return __ldg(pA + off(i)); }
    __device__ __forceinline__ float psb(int i) const { return __ldg(pA + padn + off(i)); }
};

// Push targets of the populations of node n = (x, y, z). Population (l, i)
// goes to the same direction's slot of node x + c_i (periodic axes wrap),
// unless c_i crosses a wall: then halfway bounce-back sends it to slot
// (l, opp(i)) of the node itself. PushFrame holds the per-node part: the
// offsets one step up and down each axis (with wrap) and which of those
// steps cross a wall.
struct PushFrame {
    int offp[3], offm[3];
    uint32_t wallp = 0, wallm = 0;
    __host__ __device__ __forceinline__ PushFrame(int x, int y, int z, const KParams& P)
    {
        const int L[3] = {P.lx, P.ly, P.lz};
        const int crd[3] = {x, y, z};
        const int stride[3] = {1, P.lx, P.lx * P.ly};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            offp[a] = stride[a];
            offm[a] = -stride[a];
            if (crd[a] + 1 >= L[a]) {
                if (P.wall[a]) wallp |= 1u << a;
                else offp[a] = stride[a] * (1 - L[a]);
            }
            if (crd[a] - 1 < 0) {
                if (P.wall[a]) wallm |= 1u << a;
                else offm[a] = stride[a] * (L[a] - 1);
            }
        }
    }
    // Target of (l, i) and whether a wall bounced it: both candidate
    // indices, then a select (no branch).
    __host__ __device__ __forceinline__ uint32_t target(uint32_t n, int l, int i, const KParams& P, bool& wall) const
    {
        const int cx = cxv(i), cy = cyv(i), cz = czv(i);
        const uint32_t need_p = (cx > 0 ? 1u : 0u) | (cy > 0 ? 2u : 0u) | (cz > 0 ? 4u : 0u);
        const uint32_t need_m = (cx < 0 ? 1u : 0u) | (cy < 0 ? 2u : 0u) | (cz < 0 ? 4u : 0u);
        wall = ((wallp & need_p) | (wallm & need_m)) != 0u;
        const uint32_t back_idx = n + P.dirN[19 * l + oppv(i)];
        int off = 0;
        if (cx) off += cx > 0 ? offp[0] : offm[0];
        if (cy) off += cy > 0 ? offp[1] : offm[1];
        if (cz) off += cz > 0 ? offp[2] : offm[2];
        const uint32_t push_idx = n + (uint32_t)off + P.dirN[19 * l + i];
        return wall ? back_idx : push_idx;
    }
};

// Receiver of the pushed populations for callers that also want the next
// step's densities (the fused bulk collide); put(l, i, v, bounced) sees every
// population v = f*_li the node pushes outside the particle, bounced = true
// when a wall sent it back into the node itself. The default receiver does
// nothing and compiles away.
struct NoSink {
    static constexpr bool active = false;
    __device__ __forceinline__ void put(int, int, float, bool) {}
};

// Collision and push-streaming of one fluid node (Eq. (lbe)). With PARTICLE,
// solid_nb marks the directions whose neighbour is a particle node; their
// links take the moving rule and feed acc = (F[3], T[3], ledger[2]). TAU1:
// every relaxation time is 1, so the post-collision modes depend on the
// input only through rho_l and j_l, and the ghost modes carry noise only.
// The inputs come from `in` (global memory or a shared-memory tile); the
// outputs are pushed to fout, population (l, i) of node m at m + P.dirN[19 l + i].
template <bool NOISE, bool PARTICLE, bool TAU1, class In, class Sink = NoSink>
__device__ __forceinline__ void collide_core(int x, int y, int z, uint32_t n, const In& in,
                                             float* __restrict__ fout, const DevState* __restrict__ st,
                                             const KParams& P, uint32_t solid_nb, double* acc,
                                             Sink* sink = nullptr)
{
    float ma[19], mb[19];
    float rhoA, rhoB;
    {
        float fa[19], fb[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            fa[i] = in.f(i, P);
            fb[i] = in.f(19 + i, P);
        }
        if (TAU1) {
            moments(fa, ma[0], ma + 1);
            moments(fb, mb[0], mb + 1);
        } else {
            to_modes(fa, ma);
            to_modes(fb, mb);
        }
        rhoA = ma[0];
        rhoB = mb[0];
    }
    const float rt = rhoA + rhoB;

    // Particle links of this node: FP32 sums of force, torque about the node
    // (lever c_i / 2) and mass ledger, moved into the FP64 accumulators once
    // per node; relative position of the node to the particle centre in FP64.
    LinkSums lk;
    double rn[3] = {0.0, 0.0, 0.0};
    float rnf[3] = {0.0f, 0.0f, 0.0f};
    if (PARTICLE && solid_nb) {
        rn[0] = rel_axis((double)x, st->X[0], P.lx, P.wall[0]);
        rn[1] = rel_axis((double)y, st->X[1], P.ly, P.wall[1]);
        rn[2] = rel_axis((double)z, st->X[2], P.lz, P.wall[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) rnf[a] = (float)rn[a];
    }

    // Shan-Chen force, Eq. (sc-force), omega_i = w_i, psi = rho.
    float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
    {
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float pa = in.psa(i);
            const float pb = in.psb(i);
            const float w = wv(i);
            if (cxv(i)) { ga[0] += (cxv(i) * w) * pb; gb[0] += (cxv(i) * w) * pa; }
            if (cyv(i)) { ga[1] += (cyv(i) * w) * pb; gb[1] += (cyv(i) * w) * pa; }
            if (czv(i)) { ga[2] += (czv(i) * w) * pb; gb[2] += (czv(i) * w) * pa; }
            if (PARTICLE && (solid_nb >> i & 1u)) {
                // Reaction on the particle of this pair force (virtual layer).
                const float mag = P.G * w * (rhoA * pb + rhoB * pa);
                link_add(lk, mag, cxv(i), cyv(i), czv(i));
            }
        }
    }
    const float irt = 1.0f / rt;
    float ext[3] = {P.ext[0], P.ext[1], P.ext[2]};
    if (P.counterforce) ext[2] += st->fc_f;
    float FA[3], FB[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -P.G * rhoA * ga[a] + rhoA * irt * ext[a];
        FB[a] = -P.G * rhoB * gb[a] + rhoB * irt * ext[a];
    }
    // Hydrodynamical velocity v^(H) = (sum_l j_l + (F_A + F_B)/2) / rho_tot.
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = (ma[1 + a] + mb[1 + a] + 0.5f * (FA[a] + FB[a])) * irt;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // MRT relaxation of each component in moment space, then n_k = m_k / b_k.
    auto relax = [&](float* m, float rl, const float* Fl, float delta) {
        const float uF = u[0] * Fl[0] + u[1] * Fl[1] + u[2] * Fl[2];
        m[0] = rl + delta;
        const float meq[6] = {rl * uu, rl * (3.0f * u[0] * u[0] - uu), rl * (u[1] * u[1] - u[2] * u[2]),
                              rl * u[0] * u[1], rl * u[1] * u[2], rl * u[0] * u[2]};
        const float S[6] = {2.0f * uF, 2.0f * (3.0f * u[0] * Fl[0] - uF), 2.0f * (u[1] * Fl[1] - u[2] * Fl[2]),
                            u[0] * Fl[1] + u[1] * Fl[0], u[1] * Fl[2] + u[2] * Fl[1], u[0] * Fl[2] + u[2] * Fl[0]};
        if (TAU1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) m[1 + a] = rl * u[a] + 0.5f * Fl[a];
#pragma unroll
            for (int k = 0; k < 6; ++k) m[4 + k] = meq[k] + 0.5f * S[k];
#pragma unroll
            for (int k = 10; k < 19; ++k) m[k] = 0.0f;
        } else {
            const float h = 0.5f * (1.0f + P.gs);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                m[1 + a] = rl * u[a] + P.gd * (m[1 + a] + 0.5f * Fl[a] - rl * u[a]) + 0.5f * Fl[a];
#pragma unroll
            for (int k = 0; k < 6; ++k) m[4 + k] = meq[k] + P.gs * (m[4 + k] - meq[k]) + h * S[k];
#pragma unroll
            for (int k = 10; k < 19; ++k) m[k] *= P.gg;
        }
#pragma unroll
        for (int k = 0; k < 19; ++k) m[k] *= 1.0f / bnorm(k);
    };
    relax(ma, rhoA, FA, st->delta_f[0]);
    relax(mb, rhoB, FB, st->delta_f[1]);

    if (NOISE) {
        // 33 normals from 9 Philox blocks with counter (step, node, block, 0):
        // A modes 4..18, B modes 4..18, interdiffusion J_x, J_y, J_z.
        const float sA = sqrtf(3.0f * P.kT * fmaxf(rhoA, 0.0f));
        const float sB = sqrtf(3.0f * P.kT * fmaxf(rhoB, 0.0f));
        const float sJ = 3.0f * P.nz_j * sqrtf(P.kT * fmaxf(rhoA, 0.0f) * fmaxf(rhoB, 0.0f) * fmaxf(irt, 0.0f));
        const uint32_t stp = st->step_u32;
#pragma unroll
        for (int blk = 0; blk < 9; ++blk) {
            uint32_t r0 = stp, r1 = n, r2 = (uint32_t)blk, r3 = 0u;
            philox_rk(r0, r1, r2, r3, P);
            float zn[4];
            box_muller(r0, r1, zn[0], zn[1]);
            box_muller(r2, r3, zn[2], zn[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int idx = 4 * blk + q;
                if (idx < 15) ma[4 + idx] += sA * P.nz_mode[4 + idx] * zn[q];
                else if (idx < 30) mb[4 + idx - 15] += sB * P.nz_mode[4 + idx - 15] * zn[q];
                else if (idx < 33) {
                    ma[1 + idx - 30] += sJ * zn[q];
                    mb[1 + idx - 30] -= sJ * zn[q];
                }
            }
        }
    }

    // Per-node offsets and wall flags of the push targets.
    const PushFrame frame(x, y, z, P);

    // Back-transform and push each component (Eq. (lbe) streaming; halfway
    // bounce-back at walls; moving link rule at the particle).
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        float fo[19];
        from_modes(l == 0 ? ma : mb, fo);
        const float rl = l == 0 ? rhoA : rhoB;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = cxv(i), cy = cyv(i), cz = czv(i);
            if (PARTICLE && (solid_nb >> i & 1u)) {
                // f_{-i}(x, t+1) = f*_i(x) - 6 w_i rho_l (u_b . c_i), u_b at the link midpoint.
                const uint32_t back_idx = n + P.dirN[19 * l + oppv(i)];
                const float r[3] = {rnf[0] + 0.5f * cx, rnf[1] + 0.5f * cy, rnf[2] + 0.5f * cz};
                const float* V = st->Vf;
                const float* Om = st->Omf;
                const float ubc = (V[0] + Om[1] * r[2] - Om[2] * r[1]) * cx +
                                  (V[1] + Om[2] * r[0] - Om[0] * r[2]) * cy +
                                  (V[2] + Om[0] * r[1] - Om[1] * r[0]) * cz;
                const float corr = 6.0f * wv(i) * rl * ubc;
                const float back = fo[i] - corr;
                fout[back_idx] = back;
                link_add(lk, fo[i] + back, cx, cy, cz);
                lk.led[l] += corr;
                continue;
            }
            bool wall;
            const uint32_t idx = frame.target(n, l, i, P, wall);
            fout[idx] = fo[i];
            if constexpr (Sink::active) sink->put(l, i, fo[i], wall);
        }
    }
    if (PARTICLE && solid_nb) {
        const double F[3] = {lk.F[0], lk.F[1], lk.F[2]};
        acc[0] += F[0]; acc[1] += F[1]; acc[2] += F[2];
        acc[3] += rn[1] * F[2] - rn[2] * F[1] + lk.T[0];
        acc[4] += rn[2] * F[0] - rn[0] * F[2] + lk.T[1];
        acc[5] += rn[0] * F[1] - rn[1] * F[0] + lk.T[2];
        acc[6] += lk.led[0];
        acc[7] += lk.led[1];
    }
}

// collide_core with its inputs read from global memory.
template <bool NOISE, bool PARTICLE, bool TAU1>
__device__ __forceinline__ void collide_node(int x, int y, int z, uint32_t n, const float* __restrict__ fin,
                                             float* __restrict__ fout, const float* __restrict__ psi,
                                             const DevState* __restrict__ st, const KParams& P, uint32_t solid_nb,
                                             double* acc)
{
    const GlobalInputs in(fin, psi, x, y, z, n, P);
    collide_core<NOISE, PARTICLE, TAU1>(x, y, z, n, in, fout, st, P, solid_nb, acc);
}

// ---------------------------------------------------------------------------
// Bulk tiles: every tile not next to the particle.
// ---------------------------------------------------------------------------
// Thread (tx, ty) of tile (bx, by, bz).
template <bool NOISE, bool TAU1>
__device__ __forceinline__ void bulk_tile(int bx, int by, int bz, int tx, int ty, const float* __restrict__ fin,
                                          float* __restrict__ fout, const float* __restrict__ psi,
                                          const DevState* __restrict__ st, const KParams& P)
{
    if (P.has_particle) {
        const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
        if (tile_near(bx, by, bz, o, P)) return;
    }
    const int x = bx * P.tx + tx;
    const int y = by * P.ty + ty;
    const int z = bz;
    if (x >= P.lx || y >= P.ly) return;
    const uint32_t n = (uint32_t)x + (uint32_t)P.lx * ((uint32_t)y + (uint32_t)P.ly * (uint32_t)z);
    collide_node<NOISE, false, TAU1>(x, y, z, n, fin, fout, psi, st, P, 0u, nullptr);
}

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(kThreadsStep, FLBM_BULK_MINBLOCKS)
    k_collide_bulk(const float* __restrict__ fin, float* __restrict__ fout, const float* __restrict__ psi,
                   const DevState* __restrict__ st, KParams P)
{
    bulk_tile<NOISE, TAU1>(blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, fin, fout, psi, st, P);
}

// Candidate c on one axis -> tile index, or -1. e0 = first coordinate of the
// grown box on that axis; tiles of size T, gt of them, axis length L.
__host__ __device__ __forceinline__ int candidate_tile(int c, int o, int T, int gt, int L, int wall)
{
    int e0 = o - 1;
    if (wall) {
        if (e0 < 0) e0 = 0;
        const int t = e0 / T + c;
        return t < gt ? t : -1;
    }
    if (e0 < 0) e0 += L;
    return (e0 / T + c) % gt;
}

// ---------------------------------------------------------------------------
// Near tiles: a fixed grid of candidate tiles around the particle box; each
// near tile reduces force, torque and mass ledger into partials[candidate].
// ---------------------------------------------------------------------------
// Candidate (cx, cy, cz) of the grid around the particle box; thread (tx, ty)
// of the tile, tid = tx + TX ty. Every thread of the block must call this.
template <bool NOISE, bool TAU1>
__device__ __forceinline__ void near_tile_work(int cx, int cy, int cz, int tx, int ty, int tid,
                                          const float* __restrict__ fin, float* __restrict__ fout,
                                          const float* __restrict__ psi, const DevState* __restrict__ st,
                                          const uint8_t* __restrict__ masks, double* __restrict__ partials,
                                          const KParams& P)
{
    __shared__ double s_red[(kThreadsStep / 32) * 8];
    __shared__ double s_out[8];
    const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const int bx = candidate_tile(cx, o[0], P.tx, P.gx, P.lx, P.wall[0]);
    const int by = candidate_tile(cy, o[1], P.ty, P.gy, P.ly, P.wall[1]);
    const int bz = candidate_tile(cz, o[2], 1, P.lz, P.lz, P.wall[2]);
    const long long cand = cx + (long long)P.ncx * (cy + (long long)P.ncy * cz);
    const bool near = bx >= 0 && by >= 0 && bz >= 0 && tile_near(bx, by, bz, o, P);
    if (!near) {
        if (tid < 8) partials[cand * 8 + tid] = 0.0;
        return;
    }
    const uint8_t* mask = masks + (size_t)st->cur * P.B * P.B * P.B;
    const int x = bx * P.tx + tx;
    const int y = by * P.ty + ty;
    const int z = bz;
    const bool inside = x < P.lx && y < P.ly;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool fluid = inside && !is_solid(x, y, z, o, mask, P);
    const uint32_t links = fluid ? solid_neighbours(x, y, z, o, mask, P) : 0u;
    // A warp none of whose nodes has a particle link takes the update of the
    // bulk tiles. Every lane of the block's full warps reaches the vote.
    const bool warp_links = __any_sync(0xffffffffu, links != 0u);
    if (fluid) {
        const uint32_t n = (uint32_t)x + (uint32_t)P.lx * ((uint32_t)y + (uint32_t)P.ly * (uint32_t)z);
        if (warp_links) collide_node<NOISE, true, TAU1>(x, y, z, n, fin, fout, psi, st, P, links, acc);
        else collide_node<NOISE, false, TAU1>(x, y, z, n, fin, fout, psi, st, P, 0u, nullptr);
    }
    if (!__syncthreads_or(links != 0)) {  // no particle link in this tile
        if (tid < 8) partials[cand * 8 + tid] = 0.0;
        return;
    }
    block_sum8<kThreadsStep>(acc, s_red, s_out, links != 0);
    if (tid < 8) partials[cand * 8 + tid] = s_out[tid];
    __syncthreads();  // s_out is reused by the next tile of a persistent block
}

__device__ __forceinline__ void update_particle(DevState* __restrict__ st, const double* __restrict__ partials,
                                                const KParams& P);

// A near tile, then, in the block that finishes the launch's last candidate,
// the particle update of this step (sum of all candidates' partials in fixed
// order, leap-frog).
template <bool NOISE, bool TAU1>
__device__ __forceinline__ void near_tile(int cx, int cy, int cz, int tx, int ty, int tid,
                                          const float* __restrict__ fin, float* __restrict__ fout,
                                          const float* __restrict__ psi, DevState* __restrict__ st,
                                          const uint8_t* __restrict__ masks, double* __restrict__ partials,
                                          const KParams& P)
{
    near_tile_work<NOISE, TAU1>(cx, cy, cz, tx, ty, tid, fin, fout, psi, st, masks, partials, P);
    if (last_block(&st->near_done, (unsigned)(P.ncx * P.ncy * P.ncz), tid < 8))  // tid < 8 wrote partials
        update_particle(st, partials, P);
    __syncthreads();
}

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(kThreadsStep, TAU1 ? 3 : 2)
    k_collide_near(const float* __restrict__ fin, float* __restrict__ fout, const float* __restrict__ psi,
                   DevState* __restrict__ st, const uint8_t* __restrict__ masks,
                   double* __restrict__ partials, KParams P)
{
    near_tile<NOISE, TAU1>(blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y,
                           threadIdx.x + blockDim.x * threadIdx.y, fin, fout, psi, st, masks, partials, P);
}

__host__ __device__ __forceinline__ void box_origin(const double X[3], const KParams& P, int o[3])
{
    const int L[3] = {P.lx, P.ly, P.lz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = (int)floor(X[a] - P.R);
        if (!P.wall[a]) {
            v %= L[a];
            if (v < 0) v += L[a];
        }
        o[a] = v;
    }
}

// Particle node test for box entry t of a box at origin o around centre X (FP64).
__host__ __device__ __forceinline__ bool box_node_inside(int t, const int o[3], const double X[3], const KParams& P)
{
    const int B = P.B;
    const int d[3] = {t % B, (t / B) % B, t / (B * B)};
    const int L[3] = {P.lx, P.ly, P.lz};
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int c = o[a] + d[a];
        if (P.wall[a]) {
            if (c < 0 || c >= L[a]) return false;
        } else if (c >= L[a]) {
            c -= L[a];
        }
        const double r = rel_axis((double)c, X[a], L[a], P.wall[a]);
        s += r * r;
    }
    return s < P.R * P.R;
}

// ---------------------------------------------------------------------------
// (1) Sum the near-tile partials in candidate order, leap-frog update (FP64),
// new box origin. One block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void update_particle(DevState* __restrict__ st, const double* __restrict__ partials,
                                                const KParams& P)
{
    __shared__ double s_red[(256 / 32) * 8];
    __shared__ double s_out[8];
    const long long ncand = (long long)P.ncx * P.ncy * P.ncz;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = tid; c < ncand; c += nthr)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += __ldcg(partials + c * 8 + k);
    block_sum8<256>(acc, s_red, s_out);
    // One thread per axis: the three components are independent. FP64 on a
    // part whose FP64 is slow, so products with 1 / m_p and 1 / I_p, and the
    // periodic wrap as a conditional shift (floor only for a longer step).
    const int a = tid;
    if (a >= 3) return;
    const int L = a == 0 ? P.lx : (a == 1 ? P.ly : P.lz);
    const double F = s_out[a] + st->Ppend[a];
    const double T = s_out[3 + a] + st->Lpend[a];
    st->F[a] = F;
    st->T[a] = T;
    const double ext = (a == 2) ? st->Fp : 0.0;
    const double v0 = st->V[a];
    const double vn = v0 + (F + ext) * P.inv_mp;
    st->Vavg[a] = 0.5 * (v0 + vn);
    st->V[a] = vn;
    const double om = st->Om[a] + T * P.inv_Ip;
    st->Om[a] = om;
    st->Vf[a] = (float)vn;
    st->Omf[a] = (float)om;
    double xn = st->X[a] + vn;
    if (!P.wall[a]) {
        if (xn >= L) xn -= L;
        else if (xn < 0.0) xn += L;
        if (xn >= L || xn < 0.0) xn -= L * floor(xn / L);
    }
    st->X[a] = xn;
    if (a == 0) {
        st->ledger_bb[0] = s_out[6];
        st->ledger_bb[1] = s_out[7];
    }
    // box_origin of the new position, this axis.
    int o = (int)floor(xn - P.R);
    if (!P.wall[a]) {
        o %= L;
        if (o < 0) o += L;
    }
    st->box_next[a] = o;
}

// (2) Particle nodes at the new position -> mask[1 - cur]; per-block counts.
// Block blk of 256 box entries.
__device__ __forceinline__ void mark_next_block(int blk, const DevState* __restrict__ st, uint8_t* __restrict__ masks,
                                                int* __restrict__ counts, const KParams& P)
{
    __shared__ int s_cnt[256 / 32];
    const int B3 = P.B * P.B * P.B;
    const int t = blk * 256 + threadIdx.x;
    const int o[3] = {st->box_next[0], st->box_next[1], st->box_next[2]};
    const double X[3] = {st->X[0], st->X[1], st->X[2]};
    int in = 0;
    if (t < B3) {
        in = box_node_inside(t, o, X, P) ? 1 : 0;
        masks[(size_t)(1 - st->cur) * B3 + t] = (uint8_t)in;
    }
    int c = __reduce_add_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int w = 0; w < 256 / 32; ++w) a += s_cnt[w];
        counts[blk] = a;
    }
    __syncthreads();
}

static __global__ void __launch_bounds__(256) k_mark_next(const DevState* __restrict__ st, uint8_t* __restrict__ masks,
                                                          int* __restrict__ counts, KParams P)
{
    mark_next_block(blockIdx.x, st, masks, counts, P);
}

// (3) Cover (new box) and uncover (old box) on the post-stream populations f;
// per-block FP64 partials of impulse, angular impulse and mass ledger.
// Exact FP64 sum of the 19 float populations of component l at node m
// (exact: populations are floats of similar magnitude, so every partial sum
// fits in a double and the order does not matter); four chains to shorten
// the dependent FP64 additions, which are slow on this part.
__device__ __forceinline__ double pop_sum(const float* __restrict__ f, int l, long long m, long long N)
{
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 19; ++i) s4[i & 3] += (double)f[(long long)(19 * l + i) * N + m];
    return (s4[0] + s4[1]) + (s4[2] + s4[3]);
}

__device__ __forceinline__ void cover_block(int blk, float* __restrict__ f, const DevState* __restrict__ st,
                                            const uint8_t* __restrict__ masks, double* __restrict__ parts,
                                            const KParams& P)
{
    __shared__ double s_red[(256 / 32) * 8];
    __shared__ double s_out[8];
    const int B = P.B;
    const int B3 = B * B * B;
    const int t = blk * 256 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int cur = st->cur;
    const int o_old[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const int o_new[3] = {st->box_next[0], st->box_next[1], st->box_next[2]};
    const uint8_t* m_old = masks + (size_t)cur * B3;
    const uint8_t* m_new = masks + (size_t)(1 - cur) * B3;
    const int L[3] = {P.lx, P.ly, P.lz};
    const long long N = P.N;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool uncovered = false;
    int cu_[3] = {0, 0, 0};  // an uncovered node of this thread
    if (t < B3) {
        const int d[3] = {t % B, (t / B) % B, t / (B * B)};
        if (m_new[t]) {  // covered: particle node now, fluid before
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = o_new[a] + d[a];
                if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
            }
            if (!is_solid(c[0], c[1], c[2], o_old, m_old, P)) {
                const long long n = c[0] + (long long)P.lx * (c[1] + (long long)P.ly * c[2]);
                double j4[3][4] = {}, r4[2][4] = {};  // exact sums in four chains
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int i = 0; i < 19; ++i) {
                        const double fv = f[(long long)(19 * l + i) * N + n];
                        r4[l][i & 3] += fv;
                        if (cxv(i)) j4[0][i & 3] += cxv(i) > 0 ? fv : -fv;
                        if (cyv(i)) j4[1][i & 3] += cyv(i) > 0 ? fv : -fv;
                        if (czv(i)) j4[2][i & 3] += czv(i) > 0 ? fv : -fv;
                    }
                double j[3], rl[2];
                for (int a = 0; a < 3; ++a) j[a] = (j4[a][0] + j4[a][1]) + (j4[a][2] + j4[a][3]);
                for (int l = 0; l < 2; ++l) rl[l] = (r4[l][0] + r4[l][1]) + (r4[l][2] + r4[l][3]);
                double r[3];
                for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], st->X[a], L[a], P.wall[a]);
                acc[0] += j[0]; acc[1] += j[1]; acc[2] += j[2];
                acc[3] += r[1] * j[2] - r[2] * j[1];
                acc[4] += r[2] * j[0] - r[0] * j[2];
                acc[5] += r[0] * j[1] - r[1] * j[0];
                acc[6] += rl[0];
                acc[7] += rl[1];
            }
        }
        if (m_old[t]) {  // uncovered: particle node before, fluid now
            for (int a = 0; a < 3; ++a) {
                cu_[a] = o_old[a] + d[a];
                if (!P.wall[a] && cu_[a] >= L[a]) cu_[a] -= L[a];
            }
            uncovered = !is_solid(cu_[0], cu_[1], cu_[2], o_new, m_new, P);
        }
    }
    // Each uncovered node of the warp in turn, by the whole warp: lane j
    // (1..18) sums the populations of neighbour j, the warp adds them up
    // (exact sums), and the lanes write the refilled populations.
    unsigned um = __ballot_sync(0xffffffffu, uncovered);
    while (um) {
        const int src = __ffs(um) - 1;
        um &= um - 1;
        int c[3];
        for (int a = 0; a < 3; ++a) c[a] = __shfl_sync(0xffffffffu, cu_[a], src);
        double m0 = 0.0, m1 = 0.0;
        int one = 0;
        if (lane >= 1 && lane <= 18) {
            int q[3] = {c[0] + cxv(lane), c[1] + cyv(lane), c[2] + czv(lane)};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                if (q[a] < 0 || q[a] >= L[a]) {
                    if (P.wall[a]) ok = false;
                    else q[a] += (q[a] < 0) ? L[a] : -L[a];
                }
            }
            // a fluid neighbour that was fluid before as well
            if (ok && !is_solid(q[0], q[1], q[2], o_new, m_new, P) && !is_solid(q[0], q[1], q[2], o_old, m_old, P)) {
                const long long m = q[0] + (long long)P.lx * (q[1] + (long long)P.ly * q[2]);
                m0 = pop_sum(f, 0, m, N);
                m1 = pop_sum(f, 1, m, N);
                one = 1;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            m0 += __shfl_xor_sync(0xffffffffu, m0, off);
            m1 += __shfl_xor_sync(0xffffffffu, m1, off);
            one += __shfl_xor_sync(0xffffffffu, one, off);
        }
        const int cnt = one;
        // neighbour-mean densities; the initial densities if no fluid neighbour is left
        const double rls[2] = {cnt ? m0 / cnt : P.rho0[0], cnt ? m1 / cnt : P.rho0[1]};
        double r[3];
        for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], st->X[a], L[a], P.wall[a]);
        const double ub[3] = {st->V[0] + st->Om[1] * r[2] - st->Om[2] * r[1],
                              st->V[1] + st->Om[2] * r[0] - st->Om[0] * r[2],
                              st->V[2] + st->Om[0] * r[1] - st->Om[1] * r[0]};
        const long long n = c[0] + (long long)P.lx * (c[1] + (long long)P.ly * c[2]);
        const double uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
        for (int q = lane; q < 38; q += 32) {  // population (l, i) = (q / 19, q % 19)
            const int l = q / 19, i = q % 19;
            const double cu = ub[0] * cxv(i) + ub[1] * cyv(i) + ub[2] * czv(i);
            f[(long long)q * N + n] = (float)(wv(i) * rls[l] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
        }
        if (lane == src) {
            double pm[3] = {0, 0, 0};
            for (int l = 0; l < 2; ++l) {
                pm[0] += rls[l] * ub[0]; pm[1] += rls[l] * ub[1]; pm[2] += rls[l] * ub[2];
            }
            acc[0] -= pm[0]; acc[1] -= pm[1]; acc[2] -= pm[2];
            acc[3] -= r[1] * pm[2] - r[2] * pm[1];
            acc[4] -= r[2] * pm[0] - r[0] * pm[2];
            acc[5] -= r[0] * pm[1] - r[1] * pm[0];
            acc[6] -= rls[0];
            acc[7] -= rls[1];
        }
    }
    block_sum8<256>(acc, s_red, s_out);
    if (threadIdx.x < 8) parts[blk * 8 + threadIdx.x] = s_out[threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ void finish_step(DevState* __restrict__ st, const int* __restrict__ counts,
                                            const double* __restrict__ parts, int nblocks, const KParams& P);

// A block of the cover/uncover pass, then, in the launch's last block, the
// step's bookkeeping (finish_step).
__device__ __forceinline__ void cover_then_finish(int blk, float* __restrict__ f, DevState* __restrict__ st,
                                                  const uint8_t* __restrict__ masks, double* __restrict__ parts,
                                                  const int* __restrict__ counts, const KParams& P)
{
    cover_block(blk, f, st, masks, parts, P);
    const int nb = (P.B * P.B * P.B + 255) / 256;
    if (last_block(&st->cover_done, (unsigned)nb, threadIdx.x < 8))  // threads 0..7 wrote parts
        finish_step(st, counts, parts, nb, P);
    __syncthreads();
}

static __global__ void __launch_bounds__(256) k_cover(float* __restrict__ f, DevState* __restrict__ st,
                                                      const uint8_t* __restrict__ masks, double* __restrict__ parts,
                                                      const int* __restrict__ counts, KParams P)
{
    cover_then_finish(blockIdx.x, f, st, masks, parts, counts, P);
}

// (4) Bookkeeping for the next step: pending impulses, fluid count, mass
// correction delta_l = ledger_l / N_fluid, counterforce, box swap, step + 1.
// Without a particle only the step counter advances. One block.
__device__ __forceinline__ void finish_step(DevState* __restrict__ st, const int* __restrict__ counts,
                                            const double* __restrict__ parts, int nblocks, const KParams& P)
{
    __shared__ double s_red[(256 / 32) * 8];
    __shared__ double s_out[8];
    __shared__ long long s_c[256 / 32];
    if (!P.has_particle) {
        if (threadIdx.x == 0) {
            st->step += 1;
            st->step_u32 = (uint32_t)st->step;
        }
        return;
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long cnt = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += __ldcg(parts + b * 8 + k);
        cnt += __ldcg(counts + b);
    }
    // Particle nodes: an integer sum, the same in any order.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = cnt;
    block_sum8<256>(acc, s_red, s_out);  // its barriers also publish s_c
    // Threads 0, 1, 2 form delta_A, delta_B and the counterforce at once
    // (FP64 divisions are slow here); thread 0 also the rest.
    if (threadIdx.x >= 3) return;
    long long solid = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) solid += s_c[w];
    const long long nf = P.N - solid;
    if (threadIdx.x < 2) {
        const int l = threadIdx.x;
        st->delta[l] = (st->ledger_bb[l] + s_out[6 + l]) / (double)nf;
        st->delta_f[l] = (float)st->delta[l];
    } else {
        st->fc = P.counterforce ? -st->Fp / (double)nf : 0.0;
        st->fc_f = (float)st->fc;
    }
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        st->Ppend[a] = s_out[a];
        st->Lpend[a] = s_out[3 + a];
    }
    st->nfluid = nf;
    st->box_prev[0] = st->box0[0]; st->box_prev[1] = st->box0[1]; st->box_prev[2] = st->box0[2];
    st->box0[0] = st->box_next[0]; st->box0[1] = st->box_next[1]; st->box0[2] = st->box_next[2];
    st->cur = 1 - st->cur;
    st->step += 1;
    st->step_u32 = (uint32_t)st->step;
}

static __global__ void __launch_bounds__(256) k_finish(DevState* __restrict__ st, const int* __restrict__ counts,
                                                       const double* __restrict__ parts, int nblocks, KParams P)
{
    finish_step(st, counts, parts, nblocks, P);
}

// Mark the particle nodes of the current position into mask[cur] and set the
// box origin, fluid count and counterforce (creation and flbm_set_particle).
// One block; FP64 inside test as in the step.
static __global__ void __launch_bounds__(1024) k_mark(DevState* st, uint8_t* masks, KParams P)
{
    __shared__ long long s_c[1024];
    __shared__ int s_o[3];
    if (threadIdx.x == 0) {
        int o[3];
        box_origin(st->X, P, o);
        s_o[0] = o[0]; s_o[1] = o[1]; s_o[2] = o[2];
    }
    __syncthreads();
    const int o[3] = {s_o[0], s_o[1], s_o[2]};
    const double X[3] = {st->X[0], st->X[1], st->X[2]};
    const int B3 = P.B * P.B * P.B;
    uint8_t* mask = masks + (size_t)st->cur * B3;
    long long cnt = 0;
    for (int t = threadIdx.x; t < B3; t += blockDim.x) {
        const bool in = box_node_inside(t, o, X, P);
        mask[t] = in ? 1 : 0;
        cnt += in;
    }
    s_c[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) a += s_c[k];
        st->box0[0] = o[0]; st->box0[1] = o[1]; st->box0[2] = o[2];
        st->nfluid = P.N - a;
        st->fc = (P.counterforce && st->nfluid > 0) ? -st->Fp / (double)st->nfluid : 0.0;
        st->fc_f = (float)st->fc;
        st->delta_f[0] = (float)st->delta[0];
        st->delta_f[1] = (float)st->delta[1];
        st->step_u32 = (uint32_t)st->step;
        for (int a = 0; a < 3; ++a) {
            st->Vf[a] = (float)st->V[a];
            st->Omf[a] = (float)st->Om[a];
        }
    }
}

}  // namespace flbm

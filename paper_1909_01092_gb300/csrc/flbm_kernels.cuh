// Kernels of one FLBM time step (arXiv:1909.01092, Section 2 and Section 3).
//
// Per step, on one stream:
//   k_density  : rho_l = sum_i f_li on fluid nodes (Eq. (density)) -> psi interior
//   k_virtual  : virtual fluid layer on particle surface nodes (Section 2)
//   k_shell    : psi shell: periodic copies and neutral wall ghosts (Section 3)
//   k_collide  : Shan-Chen force (Eq. (sc-force)), MRT collision with source and
//                thermal noise, push-streaming with halfway wall bounce-back and
//                the moving link rule at the particle, momentum exchange and
//                Shan-Chen reaction reduced per tile (Eq. (lbe))
//   k_particle : sum of tile partials, leap-frog Newton-Euler update,
//                cover/uncover, mass-correction ledger (Section 2)
#pragma once

#include "flbm_device.cuh"

namespace flbm {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Initial state: f = w_i rho_l0 (1 + a (2u - 1)), u from Philox counter
// (0, node, 0, 1): first word for A, second for B.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_init(float* __restrict__ f, KParams P, float rho_a, float rho_b, float pert)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
    uint32_t r0 = 0u, r1 = (uint32_t)n, r2 = 0u, r3 = 1u;
    philox4x32_10(r0, r1, r2, r3, P.key0, P.key1);
    const float ra = rho_a * (1.0f + pert * (2.0f * uniform_open(r0) - 1.0f));
    const float rb = rho_b * (1.0f + pert * (2.0f * uniform_open(r1) - 1.0f));
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        f[(long long)i * P.N + n] = wv(i) * ra;
        f[(long long)(19 + i) * P.N + n] = wv(i) * rb;
    }
}

// ---------------------------------------------------------------------------
// Densities of fluid nodes into the psi interior; 0 on particle nodes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_density(const float* __restrict__ f, float* __restrict__ psi,
                                                      const DevState* __restrict__ st,
                                                      const uint8_t* __restrict__ masks, KParams P)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
    bool solid = false;
    if (P.has_particle) {
        const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
        solid = is_solid(x, y, z, o, masks + (size_t)st->cur * P.B * P.B * P.B, P);
    }
    float ra = 0.0f, rb = 0.0f;
    if (!solid) {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            ra += f[(long long)i * P.N + n];
            rb += f[(long long)(19 + i) * P.N + n];
        }
    }
    const long long q = pad_index(x, y, z, P);
    psi[q] = ra;
    psi[P.padn + q] = rb;
}

// ---------------------------------------------------------------------------
// Virtual fluid layer (Section 2): a particle node with fluid neighbours gets
// the mean density of those neighbours, +delta_rho for A and -delta_rho for
// B, clipped at 0. One thread per node of the particle box.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_virtual(float* __restrict__ psi, const DevState* __restrict__ st,
                                                      const uint8_t* __restrict__ masks, KParams P)
{
    const int B = P.B;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * B * B) return;
    const uint8_t* mask = masks + (size_t)st->cur * B * B * B;
    if (!mask[t]) return;
    const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const int d[3] = {t % B, (t / B) % B, t / (B * B)};
    const int L[3] = {P.lx, P.ly, P.lz};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = o[a] + d[a];
        if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
    }
    float sa = 0.0f, sb = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        int q[3] = {c[0] + cxv(j), c[1] + cyv(j), c[2] + czv(j)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (q[a] < 0 || q[a] >= L[a]) {
                if (P.wall[a]) ok = false;
                else q[a] += (q[a] < 0) ? L[a] : -L[a];
            }
        }
        if (!ok || is_solid(q[0], q[1], q[2], o, mask, P)) continue;
        const long long pi = pad_index(q[0], q[1], q[2], P);
        sa += psi[pi];
        sb += psi[P.padn + pi];
        ++cnt;
    }
    float va = 0.0f, vb = 0.0f;
    if (cnt) {
        const float inv = 1.0f / (float)cnt;
        va = fmaxf(sa * inv + P.drho, 0.0f);
        vb = fmaxf(sb * inv - P.drho, 0.0f);
    }
    const long long q = pad_index(c[0], c[1], c[2], P);
    psi[q] = va;
    psi[P.padn + q] = vb;
}

// ---------------------------------------------------------------------------
// psi shell: every shell node either maps (through periodic axes) onto an
// interior node, whose value it copies, or is a wall ghost, which takes the
// mean over its fluid neighbours (neutral wetting, Section 3).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_shell(float* __restrict__ psi, const DevState* __restrict__ st,
                                                    const uint8_t* __restrict__ masks, KParams P)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nzf = 2LL * P.px * P.py;        // z faces, full padded planes
    const long long nyf = 2LL * P.px * P.lz;        // y faces, interior z
    const long long nxf = 2LL * P.ly * P.lz;        // x faces, interior y, z
    int p[3];
    if (t < nzf) {
        const long long r = t % (P.px * P.py);
        p[0] = (int)(r % P.px) - 1;
        p[1] = (int)(r / P.px) - 1;
        p[2] = (t < nzf / 2) ? -1 : P.lz;
    } else if (t < nzf + nyf) {
        const long long u = t - nzf;
        const long long r = u % ((long long)P.px * P.lz);
        p[0] = (int)(r % P.px) - 1;
        p[2] = (int)(r / P.px);
        p[1] = (u < nyf / 2) ? -1 : P.ly;
    } else if (t < nzf + nyf + nxf) {
        const long long u = t - nzf - nyf;
        const long long r = u % ((long long)P.ly * P.lz);
        p[1] = (int)(r % P.ly);
        p[2] = (int)(r / P.ly);
        p[0] = (u < nxf / 2) ? -1 : P.lx;
    } else {
        return;
    }
    const int L[3] = {P.lx, P.ly, P.lz};
    int q[3];
    bool ghost = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q[a] = p[a];
        if (q[a] < 0 || q[a] >= L[a]) {
            if (P.wall[a]) ghost = true;
            else q[a] += (q[a] < 0) ? L[a] : -L[a];
        }
    }
    const long long dst = (long long)(p[0] + 1) + (long long)P.px * ((p[1] + 1) + (long long)P.py * (p[2] + 1));
    if (!ghost) {
        const long long src = pad_index(q[0], q[1], q[2], P);
        psi[dst] = psi[src];
        psi[P.padn + dst] = psi[P.padn + src];
        return;
    }
    const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const uint8_t* mask = masks + (size_t)st->cur * P.B * P.B * P.B;
    float sa = 0.0f, sb = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        int r[3] = {q[0] + cxv(j), q[1] + cyv(j), q[2] + czv(j)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (r[a] < 0 || r[a] >= L[a]) {
                if (P.wall[a]) ok = false;
                else r[a] += (r[a] < 0) ? L[a] : -L[a];
            }
        }
        if (!ok) continue;
        if (P.has_particle && is_solid(r[0], r[1], r[2], o, mask, P)) continue;
        const long long pi = pad_index(r[0], r[1], r[2], P);
        sa += psi[pi];
        sb += psi[P.padn + pi];
        ++cnt;
    }
    const float inv = cnt ? 1.0f / (float)cnt : 0.0f;
    psi[dst] = sa * inv;
    psi[P.padn + dst] = sb * inv;
}

// ---------------------------------------------------------------------------
// The fused collide + stream step of Eq. (lbe) for every fluid node.
// ---------------------------------------------------------------------------
template <bool NOISE, bool PARTICLE>
__global__ void __launch_bounds__(kThreads) k_collide(const float* __restrict__ fin, float* __restrict__ fout,
                                                      const float* __restrict__ psi,
                                                      const DevState* __restrict__ st,
                                                      const uint8_t* __restrict__ masks,
                                                      double* __restrict__ partials, KParams P)
{
    __shared__ double s_red[(kThreads / 32) * 8];
    __shared__ double s_out[8];
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    const bool inside = x < P.lx && y < P.ly;
    const long long N = P.N;
    const long long n = inside ? x + (long long)P.lx * (y + (long long)P.ly * z) : 0;

    int o[3] = {0, 0, 0};
    bool near = false;
    const uint8_t* mask = nullptr;
    if (PARTICLE) {
        o[0] = st->box0[0]; o[1] = st->box0[1]; o[2] = st->box0[2];
        near = tile_near(blockIdx.x, blockIdx.y, blockIdx.z, o, P);
        mask = masks + (size_t)st->cur * P.B * P.B * P.B;
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // F[3], T[3], mass ledger[2]

    // Neighbour offsets on each axis, or a wall flag (bit set when that side is a wall).
    const int L[3] = {P.lx, P.ly, P.lz};
    const int crd[3] = {x, y, z};
    long long offp[3], offm[3];
    int wallp = 0, wallm = 0;
    {
        const long long stride[3] = {1, (long long)P.lx, (long long)P.lx * P.ly};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            offp[a] = stride[a];
            offm[a] = -stride[a];
            if (crd[a] + 1 >= L[a]) {
                if (P.wall[a]) wallp |= 1 << a;
                else offp[a] = stride[a] * (1 - L[a]);
            }
            if (crd[a] - 1 < 0) {
                if (P.wall[a]) wallm |= 1 << a;
                else offm[a] = stride[a] * (L[a] - 1);
            }
        }
    }

    bool solid = false;
    uint32_t solid_nb = 0;  // bit i: neighbour along c_i is a particle node
    if (PARTICLE && near && inside) {
        solid = is_solid(x, y, z, o, mask, P);
        if (!solid) {
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                int q[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
                bool ok = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (q[a] < 0 || q[a] >= L[a]) {
                        if (P.wall[a]) ok = false;
                        else q[a] += (q[a] < 0) ? L[a] : -L[a];
                    }
                }
                if (ok && is_solid(q[0], q[1], q[2], o, mask, P)) solid_nb |= 1u << i;
            }
        }
    }

    if (inside && !solid) {
        float fa[19], fb[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            fa[i] = fin[(long long)i * N + n];
            fb[i] = fin[(long long)(19 + i) * N + n];
        }
        float ma[19], mb[19];
        to_modes(fa, ma);
        to_modes(fb, mb);
        const float rhoA = ma[0], rhoB = mb[0];
        const float rt = rhoA + rhoB;

        // Shan-Chen force, Eq. (sc-force), omega_i = w_i, psi = rho.
        float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
        const long long pc = pad_index(x, y, z, P);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const long long off = cxv(i) + (long long)P.px * (cyv(i) + (long long)P.py * czv(i));
            const float pa = psi[pc + off];
            const float pb = psi[P.padn + pc + off];
            const float w = wv(i);
            if (cxv(i)) { ga[0] += cxv(i) * w * pb; gb[0] += cxv(i) * w * pa; }
            if (cyv(i)) { ga[1] += cyv(i) * w * pb; gb[1] += cyv(i) * w * pa; }
            if (czv(i)) { ga[2] += czv(i) * w * pb; gb[2] += czv(i) * w * pa; }
            if (PARTICLE && near && (solid_nb >> i & 1u)) {
                // Reaction on the particle of this pair force (Section 2 virtual layer).
                const double mag = (double)P.G * w * ((double)rhoA * pb + (double)rhoB * pa);
                const double fr[3] = {mag * cxv(i), mag * cyv(i), mag * czv(i)};
                const double r[3] = {rel_axis(x + 0.5 * cxv(i), st->X[0], P.lx, P.wall[0]),
                                     rel_axis(y + 0.5 * cyv(i), st->X[1], P.ly, P.wall[1]),
                                     rel_axis(z + 0.5 * czv(i), st->X[2], P.lz, P.wall[2])};
                acc[0] += fr[0]; acc[1] += fr[1]; acc[2] += fr[2];
                acc[3] += r[1] * fr[2] - r[2] * fr[1];
                acc[4] += r[2] * fr[0] - r[0] * fr[2];
                acc[5] += r[0] * fr[1] - r[1] * fr[0];
            }
        }
        const float fracA = rt > 0.f ? rhoA / rt : 0.f, fracB = rt > 0.f ? rhoB / rt : 0.f;
        float ext[3] = {P.ext[0], P.ext[1], P.ext[2]};
        if (P.counterforce) ext[2] += (float)st->fc;
        float FA[3], FB[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            FA[a] = -P.G * rhoA * ga[a] + fracA * ext[a];
            FB[a] = -P.G * rhoB * gb[a] + fracB * ext[a];
        }
        // Hydrodynamical velocity v^(H) = (sum_l j_l + (F_A + F_B)/2) / rho_tot.
        const float irt = 1.0f / rt;
        float u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = (ma[1 + a] + mb[1 + a] + 0.5f * (FA[a] + FB[a])) * irt;
        const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

        // MRT collision of each component (modes 0..18 in place).
        auto relax = [&](float* m, float rl, const float* Fl, float delta) {
            const float uF = u[0] * Fl[0] + u[1] * Fl[1] + u[2] * Fl[2];
            const float h = 0.5f * (1.0f + P.gs);
            m[0] = rl + delta;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                m[1 + a] = rl * u[a] + P.gd * (m[1 + a] + 0.5f * Fl[a] - rl * u[a]) + 0.5f * Fl[a];
            float meq[6] = {rl * uu, rl * (3.0f * u[0] * u[0] - uu), rl * (u[1] * u[1] - u[2] * u[2]),
                            rl * u[0] * u[1], rl * u[1] * u[2], rl * u[0] * u[2]};
            float S[6] = {2.0f * uF, 2.0f * (3.0f * u[0] * Fl[0] - uF), 2.0f * (u[1] * Fl[1] - u[2] * Fl[2]),
                          u[0] * Fl[1] + u[1] * Fl[0], u[1] * Fl[2] + u[2] * Fl[1], u[0] * Fl[2] + u[2] * Fl[0]};
#pragma unroll
            for (int k = 0; k < 6; ++k) m[4 + k] = meq[k] + P.gs * (m[4 + k] - meq[k]) + h * S[k];
#pragma unroll
            for (int k = 10; k < 19; ++k) m[k] *= P.gg;
        };
        relax(ma, rhoA, FA, (float)st->delta[0]);
        relax(mb, rhoB, FB, (float)st->delta[1]);
        // Normalise: n_k = m_k / b_k.
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            ma[k] *= 1.0f / bnorm(k);
            mb[k] *= 1.0f / bnorm(k);
        }
        if (NOISE) {
            // Thermal noise on the non-conserved modes (fluctuation-dissipation,
            // variance 3 kT rho_l b_k (1 - gamma_k^2)) and the interdiffusion
            // momentum (equal and opposite on A and B). 33 normals from 9
            // Philox blocks with counter (step, node, block, 0).
            const float sA = sqrtf(3.0f * P.kT * fmaxf(rhoA, 0.0f));
            const float sB = sqrtf(3.0f * P.kT * fmaxf(rhoB, 0.0f));
            const float sJ = 3.0f * sqrtf(P.kT * fmaxf(rhoA, 0.0f) * fmaxf(rhoB, 0.0f) * (rt > 0.f ? irt : 0.f)) * P.nz_j;
            const uint32_t stp = (uint32_t)st->step;
#pragma unroll
            for (int blk = 0; blk < 9; ++blk) {
                uint32_t r0 = stp, r1 = (uint32_t)n, r2 = (uint32_t)blk, r3 = 0u;
                philox4x32_10(r0, r1, r2, r3, P.key0, P.key1);
                const uint32_t word[4] = {r0, r1, r2, r3};
                float zn[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float u1 = uniform_open(word[2 * h]);
                    const float u2 = uniform_open(word[2 * h + 1]);
                    const float rad = sqrtf(-2.0f * logf(u1));
                    float sn, cs;
                    sincospif(2.0f * u2, &sn, &cs);
                    zn[2 * h] = rad * cs;
                    zn[2 * h + 1] = rad * sn;
                }
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
        from_modes(ma, fa);
        from_modes(mb, fb);

        // Push-streaming with bounce-back (Eq. (lbe) streaming; Section 2/3 boundaries).
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = cxv(i), cy = cyv(i), cz = czv(i);
            const bool wall = (cx > 0 && (wallp & 1)) || (cx < 0 && (wallm & 1)) || (cy > 0 && (wallp & 2)) ||
                              (cy < 0 && (wallm & 2)) || (cz > 0 && (wallp & 4)) || (cz < 0 && (wallm & 4));
            if (wall) {
                fout[(long long)oppv(i) * N + n] = fa[i];
                fout[(long long)(19 + oppv(i)) * N + n] = fb[i];
                continue;
            }
            if (PARTICLE && near && (solid_nb >> i & 1u)) {
                // Moving link rule (Ladd 1994): f_{-i}(x, t+1) = f*_i(x) - 6 w_i rho_l (u_b . c_i),
                // u_b at the link midpoint; momentum exchange and mass ledger in FP64.
                const double r[3] = {rel_axis(x + 0.5 * cx, st->X[0], P.lx, P.wall[0]),
                                     rel_axis(y + 0.5 * cy, st->X[1], P.ly, P.wall[1]),
                                     rel_axis(z + 0.5 * cz, st->X[2], P.lz, P.wall[2])};
                const double ub[3] = {st->V[0] + st->Om[1] * r[2] - st->Om[2] * r[1],
                                      st->V[1] + st->Om[2] * r[0] - st->Om[0] * r[2],
                                      st->V[2] + st->Om[0] * r[1] - st->Om[1] * r[0]};
                const float ubc = (float)(ub[0] * cx + ub[1] * cy + ub[2] * cz);
                const float corrA = 6.0f * wv(i) * rhoA * ubc;
                const float corrB = 6.0f * wv(i) * rhoB * ubc;
                const float backA = fa[i] - corrA, backB = fb[i] - corrB;
                fout[(long long)oppv(i) * N + n] = backA;
                fout[(long long)(19 + oppv(i)) * N + n] = backB;
                const double dp = (double)fa[i] + backA + (double)fb[i] + backB;
                const double fr[3] = {dp * cx, dp * cy, dp * cz};
                acc[0] += fr[0]; acc[1] += fr[1]; acc[2] += fr[2];
                acc[3] += r[1] * fr[2] - r[2] * fr[1];
                acc[4] += r[2] * fr[0] - r[0] * fr[2];
                acc[5] += r[0] * fr[1] - r[1] * fr[0];
                acc[6] += corrA;
                acc[7] += corrB;
                continue;
            }
            long long d = n;
            if (cx > 0) d += offp[0]; else if (cx < 0) d += offm[0];
            if (cy > 0) d += offp[1]; else if (cy < 0) d += offm[1];
            if (cz > 0) d += offp[2]; else if (cz < 0) d += offm[2];
            fout[(long long)i * N + d] = fa[i];
            fout[(long long)(19 + i) * N + d] = fb[i];
        }
    }

    if (PARTICLE && near) {
        block_sum8<kThreads>(acc, s_red, s_out);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const long long tile = blockIdx.x + (long long)P.gx * (blockIdx.y + (long long)P.gy * blockIdx.z);
#pragma unroll
            for (int k = 0; k < 8; ++k) partials[tile * 8 + k] = s_out[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Mark the particle nodes of the current position into mask[cur], set the
// box origin and count fluid nodes. One block.
// ---------------------------------------------------------------------------
__device__ void mark_mask(uint8_t* mask, const KParams& P, const double X[3], const int o[3],
                          long long* s_cnt)
{
    const int B = P.B;
    const int L[3] = {P.lx, P.ly, P.lz};
    const int tid = threadIdx.x;
    const double R2 = P.R * P.R;
    long long cnt = 0;
    for (int t = tid; t < B * B * B; t += blockDim.x) {
        const int d[3] = {t % B, (t / B) % B, t / (B * B)};
        bool in = true;
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int c = o[a] + d[a];
            if (P.wall[a]) {
                if (c < 0 || c >= L[a]) in = false;
            } else if (c >= L[a]) {
                c -= L[a];
            }
            const double r = rel_axis((double)c, X[a], L[a], P.wall[a]);
            s += r * r;
        }
        const bool solid = in && s < R2;
        mask[t] = solid ? 1 : 0;
        cnt += solid;
    }
    // block reduction of the count (fixed order)
    __shared__ long long s_c[1024];
    s_c[tid] = cnt;
    __syncthreads();
    if (tid == 0) {
        long long a = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) a += s_c[k];
        *s_cnt = a;
    }
    __syncthreads();
}

__device__ __forceinline__ void box_origin(const double X[3], const KParams& P, int o[3])
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

__global__ void k_mark(DevState* st, uint8_t* masks, KParams P)
{
    __shared__ int s_o[3];
    __shared__ long long s_cnt;
    if (threadIdx.x == 0) {
        int o[3];
        box_origin(st->X, P, o);
        s_o[0] = o[0]; s_o[1] = o[1]; s_o[2] = o[2];
    }
    __syncthreads();
    int o[3] = {s_o[0], s_o[1], s_o[2]};
    double X[3] = {st->X[0], st->X[1], st->X[2]};
    mark_mask(masks + (size_t)st->cur * P.B * P.B * P.B, P, X, o, &s_cnt);
    if (threadIdx.x == 0) {
        st->box0[0] = o[0]; st->box0[1] = o[1]; st->box0[2] = o[2];
        st->nfluid = P.N - s_cnt;
        st->fc = (P.counterforce && st->nfluid > 0) ? -st->Fp / (double)st->nfluid : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Particle update (Section 2): sum the tile partials, leap-frog, re-mark,
// cover/uncover on the post-stream populations f, mass ledger. One block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_particle(float* __restrict__ f, DevState* __restrict__ st,
                                                   uint8_t* __restrict__ masks,
                                                   const double* __restrict__ partials, KParams P)
{
    __shared__ double s_red[(1024 / 32) * 8];
    __shared__ double s_out[8];
    __shared__ double s_X[3], s_V[3], s_Om[3];
    __shared__ int s_o[3];
    __shared__ long long s_cnt;
    const int tid = threadIdx.x;
    if (!P.has_particle) {
        if (tid == 0) st->step += 1;
        return;
    }
    const int B = P.B;
    const size_t B3 = (size_t)B * B * B;
    const int cur = st->cur;
    const int o_old[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const uint8_t* m_old = masks + (size_t)cur * B3;
    uint8_t* m_new = masks + (size_t)(1 - cur) * B3;
    const int L[3] = {P.lx, P.ly, P.lz};
    const long long N = P.N;

    // (1) sum of the partials of the tiles next to the particle (fixed order)
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    {
        const int nz = min(B + 2, P.lz);
        const long long per_plane = (long long)P.gx * P.gy;
        const long long total = per_plane * nz;
        for (long long t = tid; t < total; t += blockDim.x) {
            const int kz = (int)(t / per_plane);
            const long long r = t % per_plane;
            const int bx = (int)(r % P.gx), by = (int)(r / P.gx);
            int bz = o_old[2] - 1 + kz;
            if (P.wall[2]) {
                if (bz < 0 || bz >= P.lz) continue;
            } else {
                bz %= P.lz;
                if (bz < 0) bz += P.lz;
            }
            if (!tile_near(bx, by, bz, o_old, P)) continue;
            const long long tile = bx + (long long)P.gx * (by + (long long)P.gy * bz);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += partials[tile * 8 + k];
        }
    }
    block_sum8<1024>(acc, s_red, s_out);

    // (2) leap-frog Newton-Euler update in FP64
    if (tid == 0) {
        for (int a = 0; a < 3; ++a) {
            st->F[a] = s_out[a] + st->Ppend[a];
            st->T[a] = s_out[3 + a] + st->Lpend[a];
            st->Ppend[a] = 0.0;
            st->Lpend[a] = 0.0;
        }
        for (int a = 0; a < 3; ++a) {
            const double ext = (a == 2) ? st->Fp : 0.0;
            const double vn = st->V[a] + (st->F[a] + ext) / st->mp;
            st->Vavg[a] = 0.5 * (st->V[a] + vn);
            st->V[a] = vn;
            st->Om[a] += st->T[a] / st->Ip;
            double xn = st->X[a] + vn;
            if (!P.wall[a]) xn -= L[a] * floor(xn / L[a]);
            st->X[a] = xn;
            s_X[a] = xn;
            s_V[a] = vn;
            s_Om[a] = st->Om[a];
        }
        int o[3];
        box_origin(s_X, P, o);
        s_o[0] = o[0]; s_o[1] = o[1]; s_o[2] = o[2];
    }
    __syncthreads();
    const double ledger0 = s_out[6], ledger1 = s_out[7];
    const int o_new[3] = {s_o[0], s_o[1], s_o[2]};
    const double X[3] = {s_X[0], s_X[1], s_X[2]};
    const double V[3] = {s_V[0], s_V[1], s_V[2]};
    const double Om[3] = {s_Om[0], s_Om[1], s_Om[2]};

    // (3) particle nodes at the new position
    mark_mask(m_new, P, X, o_new, &s_cnt);

    // (4) cover (new box) and uncover (old box)
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    for (int t = tid; t < (int)B3; t += blockDim.x) {
        const int d[3] = {t % B, (t / B) % B, t / (B * B)};
        // covered: particle node now, fluid before
        if (m_new[t]) {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = o_new[a] + d[a];
                if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
            }
            if (!is_solid(c[0], c[1], c[2], o_old, m_old, P)) {
                const long long n = c[0] + (long long)P.lx * (c[1] + (long long)P.ly * c[2]);
                double j[3] = {0, 0, 0}, rl[2] = {0, 0};
                for (int l = 0; l < 2; ++l)
                    for (int i = 0; i < 19; ++i) {
                        const double fv = f[(long long)(19 * l + i) * N + n];
                        rl[l] += fv;
                        j[0] += fv * cxv(i); j[1] += fv * cyv(i); j[2] += fv * czv(i);
                    }
                double r[3];
                for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], X[a], L[a], P.wall[a]);
                acc[0] += j[0]; acc[1] += j[1]; acc[2] += j[2];
                acc[3] += r[1] * j[2] - r[2] * j[1];
                acc[4] += r[2] * j[0] - r[0] * j[2];
                acc[5] += r[0] * j[1] - r[1] * j[0];
                acc[6] += rl[0];
                acc[7] += rl[1];
            }
        }
        // uncovered: particle node before, fluid now
        if (m_old[t]) {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = o_old[a] + d[a];
                if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
            }
            if (!is_solid(c[0], c[1], c[2], o_new, m_new, P)) {
                double mean[2] = {0.0, 0.0};
                int cnt = 0;
                for (int jd = 1; jd < 19; ++jd) {
                    int q[3] = {c[0] + cxv(jd), c[1] + cyv(jd), c[2] + czv(jd)};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a) {
                        if (q[a] < 0 || q[a] >= L[a]) {
                            if (P.wall[a]) ok = false;
                            else q[a] += (q[a] < 0) ? L[a] : -L[a];
                        }
                    }
                    if (!ok) continue;
                    if (is_solid(q[0], q[1], q[2], o_new, m_new, P)) continue;
                    if (is_solid(q[0], q[1], q[2], o_old, m_old, P)) continue;  // also uncovered now
                    const long long m = q[0] + (long long)P.lx * (q[1] + (long long)P.ly * q[2]);
                    for (int l = 0; l < 2; ++l) {
                        double s = 0.0;
                        for (int i = 0; i < 19; ++i) s += f[(long long)(19 * l + i) * N + m];
                        mean[l] += s;
                    }
                    ++cnt;
                }
                // neighbour-mean densities; the initial densities if no fluid neighbour is left
                const double rls[2] = {cnt ? mean[0] / cnt : P.rho0[0], cnt ? mean[1] / cnt : P.rho0[1]};
                double r[3];
                for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], X[a], L[a], P.wall[a]);
                const double ub[3] = {V[0] + Om[1] * r[2] - Om[2] * r[1],
                                      V[1] + Om[2] * r[0] - Om[0] * r[2],
                                      V[2] + Om[0] * r[1] - Om[1] * r[0]};
                const long long n = c[0] + (long long)P.lx * (c[1] + (long long)P.ly * c[2]);
                const double uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
                double pm[3] = {0, 0, 0};
                for (int l = 0; l < 2; ++l) {
                    for (int i = 0; i < 19; ++i) {
                        const double cu = ub[0] * cxv(i) + ub[1] * cyv(i) + ub[2] * czv(i);
                        f[(long long)(19 * l + i) * N + n] =
                            (float)(wv(i) * rls[l] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
                    }
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
    }
    block_sum8<1024>(acc, s_red, s_out);

    // (5) bookkeeping for the next step
    if (tid == 0) {
        for (int a = 0; a < 3; ++a) {
            st->Ppend[a] = s_out[a];
            st->Lpend[a] = s_out[3 + a];
        }
        const long long nf = N - s_cnt;
        st->nfluid = nf;
        st->delta[0] = (ledger0 + s_out[6]) / (double)nf;
        st->delta[1] = (ledger1 + s_out[7]) / (double)nf;
        st->fc = P.counterforce ? -st->Fp / (double)nf : 0.0;
        st->box0[0] = o_new[0]; st->box0[1] = o_new[1]; st->box0[2] = o_new[2];
        st->cur = 1 - cur;
        st->step += 1;
    }
}

// ---------------------------------------------------------------------------
// Observables: per-tile FP64 partials, then one block sums them in order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_obs_tiles(const float* __restrict__ f, const DevState* __restrict__ st,
                                                        const uint8_t* __restrict__ masks,
                                                        double* __restrict__ out, KParams P)
{
    __shared__ double s_red[(kThreads / 32) * 8];
    __shared__ double s_out[8];
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // massA, massB, jx, jy, jz, ke, nonfinite, 0
    if (x < P.lx && y < P.ly) {
        const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
        bool solid = false;
        if (P.has_particle) {
            const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
            solid = is_solid(x, y, z, o, masks + (size_t)st->cur * P.B * P.B * P.B, P);
        }
        if (!solid) {
            double j[3] = {0, 0, 0}, rt = 0.0;
            for (int l = 0; l < 2; ++l)
                for (int i = 0; i < 19; ++i) {
                    const float fv = f[(long long)(19 * l + i) * P.N + n];
                    if (!isfinite(fv)) v[6] += 1.0;
                    v[l] += fv;
                    rt += fv;
                    j[0] += (double)fv * cxv(i); j[1] += (double)fv * cyv(i); j[2] += (double)fv * czv(i);
                }
            v[2] = j[0]; v[3] = j[1]; v[4] = j[2];
            v[5] = rt > 0.0 ? (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / (2.0 * rt) : 0.0;
        }
    }
    block_sum8<kThreads>(v, s_red, s_out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long tile = blockIdx.x + (long long)P.gx * (blockIdx.y + (long long)P.gy * blockIdx.z);
        for (int k = 0; k < 8; ++k) out[tile * 8 + k] = s_out[k];
    }
}

__global__ void __launch_bounds__(1024) k_obs_final(const double* __restrict__ tiles, long long ntiles,
                                                    double* __restrict__ out)
{
    __shared__ double s_red[(1024 / 32) * 8];
    __shared__ double s_out[8];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x)
        for (int k = 0; k < 8; ++k) v[k] += tiles[t * 8 + k];
    block_sum8<1024>(v, s_red, s_out);
    if (threadIdx.x < 8) out[threadIdx.x] = s_out[threadIdx.x];
}

// Unpad psi interior into a dense [2][N] array.
__global__ void k_unpad(const float* __restrict__ psi, float* __restrict__ out, KParams P)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
    const long long q = pad_index(x, y, z, P);
    out[n] = psi[q];
    out[P.N + n] = psi[P.padn + q];
}

}  // namespace flbm

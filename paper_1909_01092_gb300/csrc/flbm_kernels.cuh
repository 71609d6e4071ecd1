// Kernels of one FLBM time step (arXiv:1909.01092, Section 2 and Section 3).
//
// Per step, on one stream:
//   k_density       : rho_l = sum_i f_li on fluid nodes (Eq. (density)) -> psi interior
//   k_shell_virtual : psi shell (periodic copies, neutral wall ghosts, Section 3)
//                     and the virtual fluid layer on particle surface nodes (Section 2)
//   k_collide_bulk / k_collide_near (flbm_step.cuh): Shan-Chen force (Eq. (sc-force)),
//                     MRT collision with source and thermal noise, push-streaming
//                     with halfway wall bounce-back and the moving link rule at
//                     the particle, momentum exchange and Shan-Chen reaction
//                     reduced per tile (Eq. (lbe)); the near launch's last block
//                     advances the particle (leap-frog)
//   k_mark_next, k_cover : particle nodes at the new position, cover/uncover,
//                     mass-correction ledger; the cover launch's last block
//                     finishes the step (k_finish without a particle)
#pragma once

#include "flbm_device.cuh"

namespace flbm {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Initial state: f = w_i rho_l0 (1 + a (2u - 1)), u from Philox counter
// (0, node, 0, 1): first word for A, second for B.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(kThreads) k_init(float* __restrict__ f, KParams P, float rho_a, float rho_b, float pert)
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
__device__ __forceinline__ void density_node(int x, int y, int z, const float* __restrict__ f, float* __restrict__ psi,
                                             const DevState* __restrict__ st, const uint8_t* __restrict__ masks,
                                             const KParams& P)
{
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

// The density pass of a step whose state the adjoint records: it also
// writes the moment tape (rho_l and j_l of every node as raw sums of its
// populations, particle nodes included; fields rho_A, rho_B, j_A, j_B of N
// floats each), so the populations are read once for both. The sums run in
// direction order, as density_node's and the adjoint's own tape kernel's do.
static __global__ void __launch_bounds__(kThreads) k_density_tape(const float* __restrict__ f,
                                                                  float* __restrict__ psi,
                                                                  const DevState* __restrict__ st,
                                                                  const uint8_t* __restrict__ masks, KParams P,
                                                                  float* __restrict__ tape)
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
    float rho[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        float fl[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) fl[i] = f[(long long)(19 * l + i) * P.N + n];
        float r = 0.0f, j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            r += fl[i];
            j[0] += cxv(i) * fl[i];
            j[1] += cyv(i) * fl[i];
            j[2] += czv(i) * fl[i];
        }
        tape[(long long)l * P.N + n] = r;
#pragma unroll
        for (int a = 0; a < 3; ++a) tape[(long long)(2 + 3 * l + a) * P.N + n] = j[a];
        rho[l] = solid ? 0.0f : r;
    }
    const long long q = pad_index(x, y, z, P);
    psi[q] = rho[0];
    psi[P.padn + q] = rho[1];
}

static __global__ void __launch_bounds__(kThreads) k_density(const float* __restrict__ f, float* __restrict__ psi,
                                                             const DevState* __restrict__ st,
                                                             const uint8_t* __restrict__ masks, KParams P)
{
    density_node(blockIdx.x * P.tx + threadIdx.x, blockIdx.y * P.ty + threadIdx.y, blockIdx.z, f, psi, st, masks, P);
}

// ---------------------------------------------------------------------------
// Virtual fluid layer (Section 2): a particle node with fluid neighbours gets
// the mean density of those neighbours, +delta_rho for A and -delta_rho for
// B, clipped at 0. One thread per node of the particle box.
// ---------------------------------------------------------------------------
// Virtual-layer densities of particle node c (lattice coordinates, in range).
__host__ __device__ __forceinline__ void virtual_value(const int c[3], const float* __restrict__ psi, const int o[3],
                                              const uint8_t* __restrict__ mask, const KParams& P, float& va,
                                              float& vb)
{
    const int L[3] = {P.lx, P.ly, P.lz};
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
    va = 0.0f;
    vb = 0.0f;
    if (cnt) {
        const float inv = 1.0f / (float)cnt;
        va = fmaxf(sa * inv + P.drho, 0.0f);
        vb = fmaxf(sb * inv - P.drho, 0.0f);
    }
}

__host__ __device__ __forceinline__ void virtual_node(int t, float* __restrict__ psi, const DevState* __restrict__ st,
                                             const uint8_t* __restrict__ masks, const KParams& P)
{
    const int B = P.B;
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
    float va, vb;
    virtual_value(c, psi, o, mask, P, va, vb);
    const long long q = pad_index(c[0], c[1], c[2], P);
    psi[q] = va;
    psi[P.padn + q] = vb;
}

// Shell nodes of the padded psi field: z faces (full padded planes), y faces
// (interior z), x faces (interior y and z). A padded row holds lx + 2 nodes;
// its stride P.px may be larger (rounded up to 16 bytes).
__host__ __device__ __forceinline__ long long shell_count(const KParams& P)
{
    const long long pw = P.lx + 2;
    return 2LL * pw * P.py + 2LL * pw * P.lz + 2LL * P.ly * P.lz;
}

// ---------------------------------------------------------------------------
// psi shell: every shell node either maps (through periodic axes) onto an
// interior node, whose value it copies, or is a wall ghost, which takes the
// mean over its fluid neighbours (neutral wetting, Section 3).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void shell_node(long long t, float* __restrict__ psi, const DevState* __restrict__ st,
                                           const uint8_t* __restrict__ masks, const KParams& P)
{
    // 32-bit decoding: a lattice has fewer than 2^32 / 38 nodes (population
    // offsets are 32-bit), so each face holds fewer than 2^31 shell nodes.
    const int pw = P.lx + 2;           // padded row length
    const int zf = pw * P.py;          // one z face, a full padded plane
    const int yf = pw * P.lz;          // one y face, interior z
    const int xf = P.ly * P.lz;        // one x face, interior y, z
    if (t < 0 || t >= 2LL * zf + 2LL * yf + 2LL * xf) return;
    int u = (int)t;
    int p[3];
    if (u < 2 * zf) {
        const int side = u >= zf;
        const int r = u - side * zf;
        p[1] = r / pw;
        p[0] = r - p[1] * pw - 1;
        p[1] -= 1;
        p[2] = side ? P.lz : -1;
    } else if ((u -= 2 * zf) < 2 * yf) {
        const int side = u >= yf;
        const int r = u - side * yf;
        p[2] = r / pw;
        p[0] = r - p[2] * pw - 1;
        p[1] = side ? P.ly : -1;
    } else {
        u -= 2 * yf;
        const int side = u >= xf;
        const int r = u - side * xf;
        p[2] = r / P.ly;
        p[1] = r - p[2] * P.ly;
        p[0] = side ? P.lx : -1;
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
    const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const uint8_t* mask = masks + (size_t)st->cur * P.B * P.B * P.B;
    if (!ghost) {
        // Periodic copy. A particle node's value is its virtual-layer value,
        // computed here as virtual_node does, so that this kernel need not
        // wait for it.
        if (P.has_particle && is_solid(q[0], q[1], q[2], o, mask, P)) {
            float va, vb;
            virtual_value(q, psi, o, mask, P, va, vb);
            psi[dst] = va;
            psi[P.padn + dst] = vb;
            return;
        }
        const long long src = pad_index(q[0], q[1], q[2], P);
        psi[dst] = psi[src];
        psi[P.padn + dst] = psi[P.padn + src];
        return;
    }
    // A fluid neighbour of the ghost lies inward across every wall the ghost
    // is beyond (only 5 directions for a face ghost, 1 for an edge ghost);
    // it can be a particle node only if the ghost is within the particle box
    // grown by one node. Same neighbours, same order as a scan of all 18.
    bool lo[3], hi[3];
    bool near = P.has_particle != 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = q[a] < 0;
        hi[a] = q[a] >= L[a];
        near = near && ranges_meet(q[a], 1, o[a] - 1, P.B + 2, L[a], P.wall[a]);
    }
    float sa = 0.0f, sb = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int c[3] = {cxv(j), cyv(j), czv(j)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) ok = ok && !(lo[a] && c[a] != 1) && !(hi[a] && c[a] != -1);
        if (!ok) continue;
        int r[3] = {q[0] + c[0], q[1] + c[1], q[2] + c[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (r[a] < 0 || r[a] >= L[a]) {
                if (P.wall[a]) ok = false;
                else r[a] += (r[a] < 0) ? L[a] : -L[a];
            }
        }
        if (!ok) continue;
        if (near && is_solid(r[0], r[1], r[2], o, mask, P)) continue;
        const long long pi = pad_index(r[0], r[1], r[2], P);
        sa += psi[pi];
        sb += psi[P.padn + pi];
        ++cnt;
    }
    const float inv = cnt ? 1.0f / (float)cnt : 0.0f;
    psi[dst] = sa * inv;
    psi[P.padn + dst] = sb * inv;
}

// virtual_node's value computed by a warp, one box entry per warp: lane j
// (1..18) tests and loads neighbour j, so the loads of all neighbours are in
// flight at once; the values are then added in direction order, exactly as
// virtual_value adds them (the same floats). Every lane of the warp calls it.
__device__ __forceinline__ void virtual_node_warp(int t, float* __restrict__ psi, const DevState* __restrict__ st,
                                                  const uint8_t* __restrict__ masks, const KParams& P)
{
    const int B = P.B;
    if (t >= B * B * B) return;  // the same for the whole warp
    const uint8_t* mask = masks + (size_t)st->cur * B * B * B;
    if (!mask[t]) return;
    const int lane = threadIdx.x & 31;
    const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
    const int d[3] = {t % B, (t / B) % B, t / (B * B)};
    const int L[3] = {P.lx, P.ly, P.lz};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = o[a] + d[a];
        if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
    }
    float va = 0.0f, vb = 0.0f;
    bool ok = false;
    if (lane >= 1 && lane <= 18) {
        int q[3] = {c[0] + cxv(lane), c[1] + cyv(lane), c[2] + czv(lane)};
        ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (q[a] < 0 || q[a] >= L[a]) {
                if (P.wall[a]) ok = false;
                else q[a] += (q[a] < 0) ? L[a] : -L[a];
            }
        }
        ok = ok && !is_solid(q[0], q[1], q[2], o, mask, P);
        if (ok) {
            const long long pi = pad_index(q[0], q[1], q[2], P);
            va = psi[pi];
            vb = psi[P.padn + pi];
        }
    }
    const unsigned fl = __ballot_sync(0xffffffffu, ok);
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const float a = __shfl_sync(0xffffffffu, va, j), b = __shfl_sync(0xffffffffu, vb, j);
        if (fl >> j & 1u) {
            sa += a;
            sb += b;
        }
    }
    if (lane != 0) return;
    const int cnt = __popc(fl);
    float ra = 0.0f, rb = 0.0f;
    if (cnt) {
        const float inv = 1.0f / (float)cnt;
        ra = fmaxf(sa * inv + P.drho, 0.0f);
        rb = fmaxf(sb * inv - P.drho, 0.0f);
    }
    const long long q = pad_index(c[0], c[1], c[2], P);
    psi[q] = ra;
    psi[P.padn + q] = rb;
}

// Blocks of the virtual layer in k_shell_virtual: one box entry per warp.
__host__ __device__ __forceinline__ int virtual_blocks(const KParams& P)
{
    return P.has_particle ? (P.B * P.B * P.B + kThreads / 32 - 1) / (kThreads / 32) : 0;
}

// Shell and virtual layer in one launch: the first nshell_blocks blocks run
// the shell, the rest the particle box (virtual_blocks of them; no thread
// reads what another writes).
static __global__ void __launch_bounds__(kThreads) k_shell_virtual(float* __restrict__ psi,
                                                                   const DevState* __restrict__ st,
                                                                   const uint8_t* __restrict__ masks, KParams P,
                                                                   int nshell_blocks)
{
    if ((int)blockIdx.x < nshell_blocks)
        shell_node(blockIdx.x * (long long)blockDim.x + threadIdx.x, psi, st, masks, P);
    else
        virtual_node_warp((blockIdx.x - nshell_blocks) * (kThreads / 32) + (threadIdx.x >> 5), psi, st, masks, P);
}

}  // namespace flbm

#include "flbm_step.cuh"

namespace flbm {

// ---------------------------------------------------------------------------
// Observables: per-tile FP64 partials, then one block sums them in order.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(kThreads) k_obs_tiles(const float* __restrict__ f, const DevState* __restrict__ st,
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

static __global__ void __launch_bounds__(1024) k_obs_final(const double* __restrict__ tiles, long long ntiles,
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

// ---------------------------------------------------------------------------
// Fluctuation observables (Section 2, fluctuation-dissipation): per-tile FP64
// sums over the bulk fluid nodes (fluid, no particle node among the 18
// neighbours) of
//   [0..29]  n_lk^2 for l = A, B and k = 4..18, n_lk = m_lk - m_lk^eq(rho_l, u)
//   [30..31] rho_A, rho_B
//   [32..34] d_a^2, d = (rho_B j_A - rho_A j_B) / rho_tot
//   [35]     rho_A rho_B / rho_tot
//   [36..38] j_a^2, j = j_A + j_B
//   [39]     node count
// with u = j / rho_tot. The host turns them into temperatures.
// ---------------------------------------------------------------------------
constexpr int kObsModes = 40;

__device__ __forceinline__ bool has_particle_neighbour(int x, int y, int z, const int o[3], const uint8_t* mask,
                                                       const KParams& P)
{
    const int L[3] = {P.lx, P.ly, P.lz};
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
        if (ok && is_solid(q[0], q[1], q[2], o, mask, P)) return true;
    }
    return false;
}

static __global__ void __launch_bounds__(kThreads) k_obs_modes(const float* __restrict__ f,
                                                               const DevState* __restrict__ st,
                                                               const uint8_t* __restrict__ masks,
                                                               double* __restrict__ out, KParams P)
{
    __shared__ double s_red[(kThreads / 32) * 8];
    __shared__ double s_out[kObsModes];
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    double v[kObsModes];
#pragma unroll
    for (int q = 0; q < kObsModes; ++q) v[q] = 0.0;
    bool bulk = x < P.lx && y < P.ly;
    if (bulk && P.has_particle) {
        const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
        const uint8_t* mask = masks + (size_t)st->cur * P.B * P.B * P.B;
        bulk = !is_solid(x, y, z, o, mask, P) && !has_particle_neighbour(x, y, z, o, mask, P);
    }
    if (bulk) {
        const long long n = x + (long long)P.lx * (y + (long long)P.ly * z);
        double m[2][19];
        for (int l = 0; l < 2; ++l) {
            double fl[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) fl[i] = (double)f[(long long)(19 * l + i) * P.N + n];
            to_modes_t<double>(fl, m[l]);
        }
        const double rt = m[0][0] + m[1][0];
        const double j[3] = {m[0][1] + m[1][1], m[0][2] + m[1][2], m[0][3] + m[1][3]};
        const double u[3] = {j[0] / rt, j[1] / rt, j[2] / rt};
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double eq[6] = {uu, 3.0 * u[0] * u[0] - uu, u[1] * u[1] - u[2] * u[2],
                              u[0] * u[1], u[1] * u[2], u[0] * u[2]};
        for (int l = 0; l < 2; ++l) {
#pragma unroll
            for (int k = 4; k < 19; ++k) {
                const double nk = k <= 9 ? m[l][k] - m[l][0] * eq[k - 4] : m[l][k];
                v[15 * l + k - 4] = nk * nk;
            }
            v[30 + l] = m[l][0];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = (m[1][0] * m[0][1 + a] - m[0][0] * m[1][1 + a]) / rt;
            v[32 + a] = d * d;
            v[36 + a] = j[a] * j[a];
        }
        v[35] = m[0][0] * m[1][0] / rt;
        v[39] = 1.0;
    }
#pragma unroll
    for (int c = 0; c < kObsModes / 8; ++c) block_sum8<kThreads>(v + 8 * c, s_red, s_out + 8 * c);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long tile = blockIdx.x + (long long)P.gx * (blockIdx.y + (long long)P.gy * blockIdx.z);
        for (int k = 0; k < kObsModes; ++k) out[tile * kObsModes + k] = s_out[k];
    }
}

// Sum of NV per-tile values over the tiles, in tile order per thread and a
// fixed reduction tree (deterministic).
template <int NV>
static __global__ void __launch_bounds__(1024) k_obs_final_n(const double* __restrict__ tiles, long long ntiles,
                                                             double* __restrict__ out)
{
    __shared__ double s_red[(1024 / 32) * 8];
    __shared__ double s_out[NV];
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += tiles[t * NV + k];
#pragma unroll
    for (int c = 0; c < NV / 8; ++c) block_sum8<1024>(v + 8 * c, s_red, s_out + 8 * c);
    if (threadIdx.x < NV) out[threadIdx.x] = s_out[threadIdx.x];
}

// Unpad psi interior into a dense [2][N] array.
static __global__ void k_unpad(const float* __restrict__ psi, float* __restrict__ out, KParams P)
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

// Device code of the FLBM step: lattice, Philox, and the kernels.
//
// Method: arXiv:1909.01092, Section 2 (Eqs. (density), (lbe), (sc-force), the
// particle coupling paragraph) and Section 3 (Eq. (fp), channel walls).
//
// Data layout in HBM (N = lx*ly*lz, x fastest):
//   f[2 copies][2 components][19 directions][N]     float32, post-stream state
//   psi[2 components][lz+2][ly+2][lx+2]              float32, densities with a
//        one-node shell: copies across periodic faces, neutral wall ghosts
//        across walled faces; virtual-layer values on particle surface nodes
//   mask[2][B^3]                                     uint8, particle nodes in a
//        cube of side B around the sphere (current and next position)
//   partials[tiles][8]                               float64, per-tile force,
//        torque and mass ledger of tiles next to the particle
//   DevState                                         float64 particle state
#pragma once

#include <cmath>
#include <cstdint>

namespace flbm {

// ---------------------------------------------------------------------------
// D3Q19 (Section 2). Direction order: rest, +-x, +-y, +-z, xy, xz, yz pairs.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cxv(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cyv(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int czv(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int oppv(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wv(int i) { return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f); }

// Norms b_k of the mode basis (sum_i w_i e_k(c_i)^2).
__host__ __device__ constexpr float bnorm(int k)
{
    return k == 0 ? 1.0f
           : k <= 3 ? 1.0f / 3.0f
           : k == 4 ? 2.0f / 3.0f
           : k == 5 ? 4.0f / 3.0f
           : k == 6 ? 4.0f / 9.0f
           : k <= 9 ? 1.0f / 9.0f
           : k <= 12 ? 2.0f / 3.0f
           : k <= 15 ? 2.0f / 9.0f
           : k == 16 ? 2.0f
           : k == 17 ? 4.0f / 3.0f : 4.0f / 9.0f;
}

// Forward mode transform m_k = sum_i e_k(c_i) f_i of the D3Q19 MRT basis
// (density, momentum, 6 stress, 9 ghost modes), evaluated with opposite-pair
// sums (even modes) and differences (odd modes); T = float in the step, double
// in the observables.
template <class T>
__host__ __device__ __forceinline__ void to_modes_t(const T f[19], T m[19])
{
    const T s1 = f[1] + f[2], d1 = f[1] - f[2];
    const T s2 = f[3] + f[4], d2 = f[3] - f[4];
    const T s3 = f[5] + f[6], d3 = f[5] - f[6];
    const T s7 = f[7] + f[8], d7 = f[7] - f[8];
    const T s9 = f[9] + f[10], d9 = f[9] - f[10];
    const T s11 = f[11] + f[12], d11 = f[11] - f[12];
    const T s13 = f[13] + f[14], d13 = f[13] - f[14];
    const T s15 = f[15] + f[16], d15 = f[15] - f[16];
    const T s17 = f[17] + f[18], d17 = f[17] - f[18];
    const T sax = s1 + s2 + s3;
    const T sxy = s7 + s9, sxz = s11 + s13, syz = s15 + s17;
    const T sdg = sxy + sxz + syz;
    m[0] = f[0] + sax + sdg;
    m[1] = d1 + d7 + d9 + d11 + d13;
    m[2] = d2 + d7 - d9 + d15 + d17;
    m[3] = d3 + d11 - d13 + d15 - d17;
    m[4] = sdg - f[0];
    m[5] = T(2) * s1 - s2 - s3 + sxy + sxz - T(2) * syz;
    m[6] = s2 - s3 + sxy - sxz;
    m[7] = s7 - s9;
    m[8] = s15 - s17;
    m[9] = s11 - s13;
    m[10] = -T(2) * d1 + d7 + d9 + d11 + d13;
    m[11] = -T(2) * d2 + d7 - d9 + d15 + d17;
    m[12] = -T(2) * d3 + d11 - d13 + d15 - d17;
    m[13] = d7 + d9 - d11 - d13;
    m[14] = -d7 + d9 + d15 + d17;
    m[15] = d11 - d13 - d15 + d17;
    m[16] = f[0] - T(2) * sax + sdg;
    m[17] = -T(2) * s1 + s2 + s3 + sxy + sxz - T(2) * syz;
    m[18] = -s2 + s3 + sxy - sxz;
}

__host__ __device__ __forceinline__ void to_modes(const float f[19], float m[19]) { to_modes_t<float>(f, m); }

// Back transform f_i = w_i sum_k e_k(c_i) n_k with n_k = m_k / b_k already
// normalised, split into the even and odd parts of each opposite pair.
__host__ __device__ __forceinline__ void from_modes(const float n[19], float f[19])
{
    const float k18 = 1.0f / 18.0f, k36 = 1.0f / 36.0f;
    f[0] = (n[0] - n[4] + n[16]) * (1.0f / 3.0f);
    const float ex = (n[0] + 2.0f * n[5] - 2.0f * n[16] - 2.0f * n[17]) * k18;
    const float ox = (n[1] - 2.0f * n[10]) * k18;
    const float ey = (n[0] - n[5] + n[6] - 2.0f * n[16] + n[17] - n[18]) * k18;
    const float oy = (n[2] - 2.0f * n[11]) * k18;
    const float ez = (n[0] - n[5] - n[6] - 2.0f * n[16] + n[17] + n[18]) * k18;
    const float oz = (n[3] - 2.0f * n[12]) * k18;
    const float cmn = n[0] + n[4] + n[16];
    const float exy = cmn + n[5] + n[6] + n[17] + n[18];
    const float exz = cmn + n[5] - n[6] + n[17] - n[18];
    const float eyz = cmn - 2.0f * n[5] - 2.0f * n[17];
    const float e7 = (exy + n[7]) * k36, e9 = (exy - n[7]) * k36;
    const float o7 = (n[1] + n[2] + n[10] + n[11] + n[13] - n[14]) * k36;
    const float o9 = (n[1] - n[2] + n[10] - n[11] + n[13] + n[14]) * k36;
    const float e11 = (exz + n[9]) * k36, e13 = (exz - n[9]) * k36;
    const float o11 = (n[1] + n[3] + n[10] + n[12] - n[13] + n[15]) * k36;
    const float o13 = (n[1] - n[3] + n[10] - n[12] - n[13] - n[15]) * k36;
    const float e15 = (eyz + n[8]) * k36, e17 = (eyz - n[8]) * k36;
    const float o15 = (n[2] + n[3] + n[11] + n[12] + n[14] - n[15]) * k36;
    const float o17 = (n[2] - n[3] + n[11] - n[12] + n[14] + n[15]) * k36;
    f[1] = ex + ox; f[2] = ex - ox;
    f[3] = ey + oy; f[4] = ey - oy;
    f[5] = ez + oz; f[6] = ez - oz;
    f[7] = e7 + o7; f[8] = e7 - o7;
    f[9] = e9 + o9; f[10] = e9 - o9;
    f[11] = e11 + o11; f[12] = e11 - o11;
    f[13] = e13 + o13; f[14] = e13 - o13;
    f[15] = e15 + o15; f[16] = e15 - o15;
    f[17] = e17 + o17; f[18] = e17 - o17;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published
// definition, and the open-interval uniform used by both the initial
// perturbation and the thermal noise: ((x >> 9) + 1/2) * 2^-23, exact in
// binary32.
// ---------------------------------------------------------------------------
// High 32 bits of a 32 x 32-bit product (the device instruction; on the host,
// where the header's tests run it, the 64-bit product).
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                                       uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * x0, hi0 = mulhi32(0xD2511F53u, x0);
        const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = mulhi32(0xCD9E8D57u, x2);
        const uint32_t y0 = hi1 ^ x1 ^ k0;
        const uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__host__ __device__ __forceinline__ float uniform_open(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn((float)(x >> 9), 1.0f / 8388608.0f, 0.5f / 8388608.0f);
#else
    return std::fmaf((float)(x >> 9), 1.0f / 8388608.0f, 0.5f / 8388608.0f);
#endif
}

// ---------------------------------------------------------------------------
// Launch-invariant parameters (kernel argument, by value).
// ---------------------------------------------------------------------------
struct KParams {
    int lx, ly, lz;
    int wall[3];
    int px, py, pz;        // padded psi row stride (lx + 2 rounded up to 4) and dimensions ly + 2, lz + 2
    long long N;           // lx*ly*lz
    long long padn;        // px*py*pz
    int tx, ty;            // tile (block) shape in x, y; one z-plane per block
    int gx, gy;            // tiles per axis in x, y
    float G;
    float gs, gd, gg;      // gamma = 1 - 1/tau of stress, component momentum, ghost modes
    float ext[3];          // constant fluid body force density
    float drho;            // wetting shift
    float kT;
    float nz_mode[19];     // sqrt((1 - gamma_k^2) / b_k) for k >= 4 (noise in normalised modes per sqrt(3 kT rho))
    float nz_j;            // sqrt(1 - gamma_d^2)
    uint32_t key0, key1;   // Philox key
    uint32_t rk0[10], rk1[10];  // Philox round keys key + r * (0x9E3779B9, 0xBB67AE85)
    int ncx, ncy, ncz;     // candidate tiles per axis around the particle box
    int tau1;              // every relaxation time equals 1
    uint32_t dirN[38];     // (19 l + i) * N: offset of population (l, i) in one copy
    int has_particle;
    int B;                 // side of the particle box
    double R;              // sphere radius
    double inv_mp, inv_Ip; // 1 / m_p and 1 / I_p of the particle (0 without one)
    double rho0[2];        // initial densities (fallback for an uncovered node with no fluid neighbour)
    int counterforce;
};

// Particle and bookkeeping state, kept in device memory (FP64).
struct DevState {
    double X[3], V[3], Vavg[3], Om[3], F[3], T[3], Ppend[3], Lpend[3];
    double delta[2];       // per-node mass correction for the next collision
    double fc;             // counterforce density along z on the fluid
    double mp, Ip, Fp;
    long long nfluid;
    long long step;
    double ledger_bb[2];   // mass removed by the moving-wall term this step
    float delta_f[2];      // delta as float, read by the collide kernels
    float fc_f;            // fc as float
    float Vf[3], Omf[3];   // V and Omega as float, read by the moving link rule
    uint32_t step_u32;     // step as the 32-bit Philox counter word
    int cur;               // index of the current mask
    int box0[3];           // origin of the particle box (periodic axes in [0, L))
    int box_next[3];       // origin at the position after this step's update
    int box_prev[3];       // origin the last step's collide used (its near tiles)
    int err;
    unsigned near_done;    // blocks of the near-collide launch done this step (last one updates)
    unsigned cover_done;   // blocks of the cover launch done this step (last one finishes)
};

constexpr int kThreadsStep = 256;

// Signed offset of box coordinate of lattice coordinate c on one axis.
__host__ __device__ __forceinline__ int box_rel(int c, int o, int L, int wall)
{
    int t = c - o;
    if (!wall && t < 0) t += L;
    return t;
}

__host__ __device__ __forceinline__ bool in_box(int x, int y, int z, const int o[3], const KParams& P, int& bi)
{
    const int dx = box_rel(x, o[0], P.lx, P.wall[0]);
    const int dy = box_rel(y, o[1], P.ly, P.wall[1]);
    const int dz = box_rel(z, o[2], P.lz, P.wall[2]);
    const int B = P.B;
    if ((unsigned)dx >= (unsigned)B || (unsigned)dy >= (unsigned)B || (unsigned)dz >= (unsigned)B) return false;
    bi = dx + B * (dy + B * dz);
    return true;
}

__host__ __device__ __forceinline__ bool is_solid(int x, int y, int z, const int o[3], const uint8_t* mask, const KParams& P)
{
    int bi;
    return in_box(x, y, z, o, P, bi) && mask[bi];
}

// Directions i = 1..18 whose neighbour x + c_i is a particle node of the box
// at origin o with node mask `mask`, as bits 1 << i. The neighbour wraps on a
// periodic axis; across a wall there is none. The neighbour's box
// coordinates are the node's own plus c_i, taken modulo L on periodic axes.
__host__ __device__ __forceinline__ uint32_t solid_neighbours(int x, int y, int z, const int o[3],
                                                              const uint8_t* mask, const KParams& P)
{
    const int c[3] = {x, y, z};
    const int L[3] = {P.lx, P.ly, P.lz};
    int d[3];
    bool lo[3], hi[3];  // a step down / up this axis leaves through a wall
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = box_rel(c[a], o[a], L[a], P.wall[a]);
        lo[a] = P.wall[a] && c[a] == 0;
        hi[a] = P.wall[a] && c[a] == L[a] - 1;
    }
    const unsigned B = (unsigned)P.B;
    uint32_t bits = 0u;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int s[3] = {cxv(i), cyv(i), czv(i)};
        bool ok = true;
        unsigned e[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if ((s[a] < 0 && lo[a]) || (s[a] > 0 && hi[a])) ok = false;
            int t = d[a] + s[a];
            if (!P.wall[a]) t = t >= L[a] ? t - L[a] : (t < 0 ? t + L[a] : t);
            e[a] = (unsigned)t;
        }
        if (ok && e[0] < B && e[1] < B && e[2] < B && mask[e[0] + B * (e[1] + B * e[2])]) bits |= 1u << i;
    }
    return bits;
}

// Does [a0, a0+la) meet [b0, b0+lb) on an axis of length L (periodic: modulo L)?
__host__ __device__ __forceinline__ bool ranges_meet(int a0, int la, int b0, int lb, int L, int wall)
{
    if (wall) return a0 < b0 + lb && b0 < a0 + la;
    if (lb >= L) return true;
    int d0 = (a0 - b0) % L;
    if (d0 < 0) d0 += L;
    return d0 < lb || d0 + la > L;
}

// Tile (bx, by, bz) meets the particle box grown by one node on every side:
// only such tiles have fluid nodes whose stencil touches a particle node.
__host__ __device__ __forceinline__ bool tile_near(int bx, int by, int bz, const int o[3], const KParams& P)
{
    const int x0 = bx * P.tx, y0 = by * P.ty;
    const int lxr = min(P.tx, P.lx - x0), lyr = min(P.ty, P.ly - y0);
    const int B2 = P.B + 2;
    return ranges_meet(x0, lxr, o[0] - 1, B2, P.lx, P.wall[0]) &&
           ranges_meet(y0, lyr, o[1] - 1, B2, P.ly, P.wall[1]) &&
           ranges_meet(bz, 1, o[2] - 1, B2, P.lz, P.wall[2]);
}

// Edge candidates of the adjoint's last node pass: the nodes on a walled
// face (a wall ghost among their neighbours) and the nodes of the particle
// box at origin o grown by one node (a particle node among their
// neighbours). No other node has either among its neighbours.
__host__ __device__ __forceinline__ bool adj_edge_candidate(const int c[3], const int o[3], const KParams& P)
{
    const int L[3] = {P.lx, P.ly, P.lz};
    for (int a = 0; a < 3; ++a)
        if (P.wall[a] && (c[a] == 0 || c[a] == L[a] - 1)) return true;
    if (!P.has_particle) return false;
    bool in_grown = true;
    for (int a = 0; a < 3; ++a) in_grown = in_grown && ranges_meet(c[a], 1, o[a] - 1, P.B + 2, L[a], P.wall[a]);
    return in_grown;
}

// Entries adj_edge_node walks: the particle box grown by one node, then the
// two faces of each walled axis.
__host__ __device__ __forceinline__ long long adj_edge_entries(const KParams& P)
{
    const long long Bg = P.has_particle ? P.B + 2 : 0;
    const int L[3] = {P.lx, P.ly, P.lz};
    long long n = Bg * Bg * Bg;
    for (int a = 0; a < 3; ++a)
        if (P.wall[a]) n += 2LL * L[(a + 1) % 3] * L[(a + 2) % 3];
    return n;
}

// Node c of entry t, or false: every edge candidate is the node of exactly
// one entry. The grown box's entries outside the lattice, or repeating a node
// where the box wraps a periodic axis shorter than it, give none; so do the
// face entries that lie on a face of an earlier walled axis, repeat a face of
// an axis of length 1, or lie in the grown box.
__host__ __device__ __forceinline__ bool adj_edge_node(long long t, const int o[3], const KParams& P, int c[3])
{
    if (t < 0 || t >= adj_edge_entries(P)) return false;
    const int L[3] = {P.lx, P.ly, P.lz};
    const int Bg = P.B + 2;
    const long long nbox = P.has_particle ? (long long)Bg * Bg * Bg : 0;
    if (t < nbox) {
        const int d[3] = {(int)(t % Bg), (int)(t / Bg % Bg), (int)(t / ((long long)Bg * Bg))};
        for (int a = 0; a < 3; ++a) {
            int v = o[a] - 1 + d[a];
            if (P.wall[a]) {
                if (v < 0 || v >= L[a]) return false;
            } else {
                if (d[a] >= L[a]) return false;
                v = (v % L[a] + L[a]) % L[a];
            }
            c[a] = v;
        }
        return true;
    }
    t -= nbox;
    int face = -1;
    for (int a = 0; a < 3 && face < 0; ++a) {
        if (!P.wall[a]) continue;
        const int b = (a + 1) % 3, e = (a + 2) % 3;
        const long long fsz = (long long)L[b] * L[e];
        for (int side = 0; side < 2 && face < 0; ++side) {
            if (t < fsz) {
                if (side == 1 && L[a] == 1) return false;
                c[a] = side ? L[a] - 1 : 0;
                c[b] = (int)(t % L[b]);
                c[e] = (int)(t / L[b]);
                face = a;
            } else {
                t -= fsz;
            }
        }
    }
    if (face < 0) return false;
    for (int a = 0; a < face; ++a)
        if (P.wall[a] && (c[a] == 0 || c[a] == L[a] - 1)) return false;
    if (P.has_particle) {
        bool in_grown = true;
        for (int a = 0; a < 3; ++a) in_grown = in_grown && ranges_meet(c[a], 1, o[a] - 1, Bg, L[a], P.wall[a]);
        if (in_grown) return false;
    }
    return true;
}

__host__ __device__ __forceinline__ long long pad_index(int x, int y, int z, const KParams& P)
{
    return (long long)(x + 1) + (long long)P.px * ((y + 1) + (long long)P.py * (z + 1));
}

// Vector from the particle centre to point r, minimum image on periodic axes.
__host__ __device__ __forceinline__ double rel_axis(double r, double X, int L, int wall)
{
    double d = r - X;
    if (!wall) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

// Block-wide sum of 8 doubles into out[0..7] (thread 0 holds the result in
// s_out). Fixed reduction tree: deterministic.
// A thread may pass active = false when all its v are 0: warps with no active
// thread then skip their shuffles (FP64 arithmetic is a slow pipe).
template <int NT>
__device__ __forceinline__ void block_sum8(double v[8], double* s_red, double* s_out, bool active = true)
{
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
    const bool warp_any = __any_sync(0xffffffffu, active);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double a = v[k];
        if (warp_any) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        }
        if (lane == 0) s_red[warp * 8 + k] = a;
    }
    __syncthreads();
    if (tid < 8) {
        double a = 0.0;
        for (int w = 0; w < nwarp; ++w) a += s_red[w * 8 + tid];
        s_out[tid] = a;
    }
    __syncthreads();
}

// True in the block that is the last of `total` blocks to pass this point
// (counted in *counter, which that block resets to 0). Every thread of the
// block must call it. Threads that wrote what the last block will read pass
// wrote = true: their writes are made visible device-wide before the block
// takes its ticket, so the last block may read what all the others wrote
// (with loads that bypass L1). There is no waiting: the other blocks just
// finish.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned total, bool wrote)
{
    __shared__ int s_last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (wrote) __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t + 1u == total) ? 1 : 0;
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

}  // namespace flbm

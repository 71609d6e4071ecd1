// Discrete adjoint of the noise-free FLBM step (declared in include/flbm.h as
// flbm_adjoint_run): gradient of the time-averaged settling velocity
//   J = (1/T) sum_{n<T} Vavg_z(n),  Vavg(n) = (V_n + V_{n+1}) / 2,
// with respect to the body force g of Eq. (fp), the wetting shift delta_rho of
// the virtual layer (Section 2) and the Shan-Chen coupling G of Eq. (sc-force).
//
// Scope: kT = 0, every relaxation time 1 (the paper's choice), no fluid
// counterforce. The sets of particle nodes, links and covered/uncovered nodes
// of each step are those of the forward run (the map is piecewise smooth in
// the parameters; between changes of these sets it is differentiated exactly).
//
// Structure. With tau = 1 the populations of a node enter a step only through
// rho_l = sum_i f_li and j_l = sum_i f_li c_i, so the adjoint of the
// post-streaming populations is affine in c_i:
//     lambda_f_li(x) = a_l(x) + c_i . b_l(x)
// and the adjoint state is the field (a_A, a_B, b_A, b_B): 8 floats per node.
// The reverse sweep reads a tape of the moments (rho_l, j_l: 8 floats per
// node), the particle record and the particle masks of every step, segment
// by segment of K steps. Where the tape of all T steps fits the device (the
// limit of flbm_adjoint_tape_limit), the forward run writes it to a store
// and each segment's slots are copied back before its sweep. Otherwise the
// forward run keeps a checkpoint every K steps, and each segment is
// recomputed from its checkpoint, writing its tape, before it is swept
// backwards. Per reverse step:
//   ka_cover     adjoint of the mass ledger (delta_l = ledger_l / N_fluid) and of
//                cover/uncover at the new position; its last block runs the
//                leap-frog Newton-Euler update adjoint (FP64), dJ/dg
//   ka_cover_mean  uncovered nodes' neighbour means -> a_l of those neighbours
//   ka_psi_tape, k_shell_virtual  density field of the step from the tape
//   ka_node_bulk, ka_node_near  streaming (pull of the adjoint), moving
//                links, Shan-Chen reaction, collision (flbm_adjoint_math.h)
//                per fluid node; tiles away from / near the particle
//   ka_lpsi, ka_lpsi_shell  adjoint of psi at particle nodes (virtual layer,
//                Shan-Chen reaction) and wall ghosts (mean over fluid neighbours)
//   ka_final     a_l of fluid nodes: Shan-Chen stencil transposed, plus the
//                shares of the neighbour means they entered
//   ka_reduce    per-tile partials -> particle adjoint, dJ/dG, dJ/d delta_rho
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "flbm.h"
#include "flbm_adjoint_math.h"
#include "flbm_df.h"
#include "flbm_sim.cuh"

using namespace flbm;

namespace flbm_adjoint {

// Adjoint of the particle state and gradient sums, FP64 (one per run).
struct AdjState {
    double lX[3], lV[3], lOm[3], lP[3], lL[3], ld[2];  // adjoint of the step's input state (n+1 on entry, n on exit)
    double lF[3], lT[3], lled[2];                      // adjoint of the step's force, torque, mass ledger
    double grad[3];                                    // dJ/dg, dJ/d delta_rho, dJ/dG
    double J;                                          // sum of Vavg_z over the forward steps
    float lFf[3], lTf[3];                              // float copies for the node kernels
    unsigned red_done;                                 // blocks of ka_reduce done (last-block ticket)
    unsigned cover_done;                               // blocks of ka_cover done (last-block ticket)
};

// Precision. The adjoint fields carry large smooth parts (the adjoints of
// conserved totals) whose neighbour differences set the result: a_l, b_l for
// the momentum and stress adjoints, lambda g_l (= -G rho_l lambda F_l, which
// inherits b_l / 2) for the adjoint of psi. Stored in float32 they cost a
// weakly coupled gradient (G or delta_rho in a dilute mixture) 1e-3 to 5e-2
// relative accuracy within tens of steps. So these fields, and the arithmetic
// on their large parts, keep 48 significant bits; only the neighbour differences
// (a(x+c_i) - a(x)) + c_i . (b(x+c_i) - b(x)) go through the float32 mode
// projection and collision transpose (adj_modes), the large part through
// adj_modes_ab_mixed: double-float arithmetic (flbm_df.h) on the adjoint
// values, whose coefficients (the forward quantities) are floats. The terms of
// the moving links and the Shan-Chen reaction take the same form: double-float
// adjoint values times float coefficients, summed per node and added to the
// FP64 partials once per node. The adjoint of psi at particle nodes and wall
// ghosts (lpsi) and the reductions are FP64.
//
// The 48-bit fields are stored as two floats, v = hi + lo with
// lo = fl(v - hi). A node reads its own values as FP64 (sval) and forms its
// neighbours' differences in float from the two parts (sdiff; the high parts
// of close values subtract exactly), so the stencil loops need no FP64
// arithmetic, which is scarce on this GPU.
struct __align__(8) Split {
    float hi, lo;
};
__device__ __forceinline__ double sval(Split s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ Split ssplit(double v)
{
    const float h = (float)v;
    return Split{h, (float)(v - (double)h)};
}
__device__ __forceinline__ float sdiff(Split a, Split b) { return (a.hi - b.hi) + (a.lo - b.lo); }
using lam_t = Split;  // a_l, b_l: 8 per node
using lg_t = Split;   // lambda g_l: 6 per node

constexpr int kT = 256;  // threads per block

// Sum of NV <= 8 doubles over the block by the tree of block_sum8 (so each
// sum is the same), without reducing unused slots; s_out[0..NV) is the result.
template <int NV>
__device__ __forceinline__ void block_sum_n(const double v[NV], double* s_red, double* s_out)
{
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) s_red[warp * 8 + k] = a;
    }
    __syncthreads();
    if (tid < NV) {
        double a = 0.0;
        for (int w = 0; w < nwarp; ++w) a += s_red[w * 8 + tid];
        s_out[tid] = a;
    }
    __syncthreads();
}
constexpr int kNodeParts = 12;  // per tile: lX[3], lV[3], lOm[3], dJ/dG, ld[2]

// Periodic-aware neighbour of (x,y,z) along c; false if it leaves through a wall.
__device__ __forceinline__ bool nbr(int x, int y, int z, int cx, int cy, int cz, const KParams& P, int q[3])
{
    const int c[3] = {x + cx, y + cy, z + cz};
    const int L[3] = {P.lx, P.ly, P.lz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = c[a];
        if (v < 0 || v >= L[a]) {
            if (P.wall[a]) return false;
            v += (v < 0) ? L[a] : -L[a];
        }
        q[a] = v;
    }
    return true;
}

__device__ __forceinline__ uint32_t lin(int x, int y, int z, const KParams& P)
{
    return (uint32_t)x + (uint32_t)P.lx * ((uint32_t)y + (uint32_t)P.ly * (uint32_t)z);
}

__device__ __forceinline__ const uint8_t* cur_mask(const DevState* s, const uint8_t* masks, const KParams& P)
{
    return masks + (size_t)s->cur * P.B * P.B * P.B;
}

__device__ __forceinline__ bool solid_at(int x, int y, int z, const DevState* s, const uint8_t* m, const KParams& P)
{
    if (!P.has_particle) return false;
    const int o[3] = {s->box0[0], s->box0[1], s->box0[2]};
    return is_solid(x, y, z, o, m, P);
}

// ---------------------------------------------------------------------------
// Moments tape: rho_A, rho_B, j_A, j_B of every node (raw sums of the
// populations in the buffer, particle nodes included).
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(kT) ka_tape(const float* __restrict__ f, float* __restrict__ tape, KParams P)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const uint32_t n = lin(x, y, z, P);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        float fl[19], r, j[3];
#pragma unroll
        for (int i = 0; i < 19; ++i) fl[i] = f[n + P.dirN[19 * l + i]];
        r = 0.0f;
        j[0] = j[1] = j[2] = 0.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            r += fl[i];
            j[0] += cxv(i) * fl[i];
            j[1] += cyv(i) * fl[i];
            j[2] += czv(i) * fl[i];
        }
        tape[(size_t)l * P.N + n] = r;
#pragma unroll
        for (int a = 0; a < 3; ++a) tape[(size_t)(2 + 3 * l + a) * P.N + n] = j[a];
    }
}

// Sum of Vavg_z of the step just taken (one thread).
static __global__ void ka_accJ(const DevState* __restrict__ st, AdjState* __restrict__ adj)
{
    adj->J += st->Vavg[2];
}

// Interior of the density field of a step from its tape (0 on particle nodes).
static __global__ void __launch_bounds__(kT) ka_psi_tape(const float* __restrict__ tape, float* __restrict__ psi,
                                                         const DevState* __restrict__ s, const uint8_t* __restrict__ masks,
                                                         KParams P)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const uint32_t n = lin(x, y, z, P);
    const bool sol = solid_at(x, y, z, s, cur_mask(s, masks, P), P);
    const long long q = pad_index(x, y, z, P);
    psi[q] = sol ? 0.0f : tape[n];
    psi[P.padn + q] = sol ? 0.0f : tape[P.N + n];
}

// Modes 0..9 of sum_i e_k(c_i) f_i (the to_modes basis), any precision.
template <class T>
__device__ __forceinline__ void project10(const T f[19], T m[10])
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
    const T sxy = s7 + s9, sxz = s11 + s13, syz = s15 + s17;
    const T sdg = sxy + sxz + syz;
    m[0] = f[0] + (s1 + s2 + s3) + sdg;
    m[1] = d1 + d7 + d9 + d11 + d13;
    m[2] = d2 + d7 - d9 + d15 + d17;
    m[3] = d3 + d11 - d13 + d15 - d17;
    m[4] = sdg - f[0];
    m[5] = T(2) * s1 - s2 - s3 + sxy + sxz - T(2) * syz;
    m[6] = s2 - s3 + sxy - sxz;
    m[7] = s7 - s9;
    m[8] = s15 - s17;
    m[9] = s11 - s13;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// Leap-frog update adjoint (FP64, one thread; c = the box blocks' partials
// summed in block order): V' = V + (F + F_p z)/m_p, X' = X + V',
// Omega' = Omega + T/I_p, plus the two halves of Vavg in J. On exit lX, lV,
// lOm, lP, lL hold the adjoint of step n's input state without the link
// terms ka_node adds; dJ/dg accumulates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void update_adjoint(AdjState* __restrict__ a, const double c[9],
                                               const DevState* __restrict__ s0, double inv2T, double dFp_dg)
{
    double lXp[3], lVp[3], lOmp[3];
    for (int k = 0; k < 3; ++k) {
        lXp[k] = a->lX[k] + c[k];
        lOmp[k] = a->lOm[k] + c[6 + k];
        lVp[k] = a->lV[k] + c[3 + k] + lXp[k] + (k == 2 ? inv2T : 0.0);
    }
    for (int k = 0; k < 3; ++k) {
        a->lF[k] = lVp[k] / s0->mp;
        a->lT[k] = lOmp[k] / s0->Ip;
        a->lFf[k] = (float)a->lF[k];
        a->lTf[k] = (float)a->lT[k];
        a->lX[k] = lXp[k];
        a->lV[k] = lVp[k] + (k == 2 ? inv2T : 0.0);
        a->lOm[k] = lOmp[k];
        a->lP[k] = a->lF[k];
        a->lL[k] = a->lT[k];
    }
    a->grad[0] += lVp[2] * dFp_dg / s0->mp;
}

// ---------------------------------------------------------------------------
// Cover/uncover adjoint (Section 2). s0/m0: state and masks of step n (old
// position), s1/m1: of step n+1 (new position X', velocities V', Omega').
// Covered node c (fluid at n, particle at n+1): its post-stream populations
// fed P_pending (j), L_pending ((c - X') x j) and the ledger (rho_l), so
//   a_l(c) = lambda_ledger_l,  b_l(c) = lambda_P + lambda_L x (c - X').
// Uncovered node c: f(c) = f^eq(mean_l, u_b) with u_b = V' + Omega' x (c - X');
// since sum_i f^eq_i = rho and sum_i f^eq_i c_i = rho u, the incoming adjoint
// (a_l, b_l) of c gives lambda_mean_l = a_l + b_l . u_b and lambda_u_b =
// sum_l mean_l b_l, plus the particle's payment of the momentum and the
// ledger. lambda_mean_l / cnt goes to uv[] for ka_cover_mean. Per-block
// partials: lambda X', lambda V', lambda Omega'. The adjoint of the mass
// ledger, delta_l(n+1) = ledger_l / N_fluid(n+1), is formed by every block.
// The last block to finish (every other block has read the particle
// adjoint by then) stores it for the node kernels and runs the leap-frog
// update adjoint on the partials summed in block order.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(kT) ka_cover(lam_t* __restrict__ lam1, const float* __restrict__ tape1,
                                                      const DevState* __restrict__ s0, const uint8_t* __restrict__ mk0,
                                                      const DevState* __restrict__ s1, const uint8_t* __restrict__ mk1,
                                                      AdjState* __restrict__ adj, double* __restrict__ uv,
                                                      double* __restrict__ parts, KParams P, double inv2T,
                                                      double dFp_dg)
{
    __shared__ double s_red[(kT / 32) * 8];
    __shared__ double s_out[8];
    __shared__ double s_lled[2];
    __shared__ double s_c[9];
    if (threadIdx.x < 2) s_lled[threadIdx.x] = adj->ld[threadIdx.x] / (double)s1->nfluid;
    __syncthreads();
    const int B = P.B, B3 = B * B * B;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint8_t* m0 = cur_mask(s0, mk0, P);
    const uint8_t* m1 = cur_mask(s1, mk1, P);
    const int o0[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
    const int o1[3] = {s1->box0[0], s1->box0[1], s1->box0[2]};
    const int L[3] = {P.lx, P.ly, P.lz};
    const size_t N = P.N;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // lX'[3], lV'[3], lOm'[3]
    if (t < B3) {
        const int d[3] = {t % B, (t / B) % B, t / (B * B)};
        uv[t] = 0.0;
        uv[B3 + t] = 0.0;
        if (m1[t]) {  // covered
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = o1[a] + d[a];
                if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
            }
            if (!is_solid(c[0], c[1], c[2], o0, m0, P)) {
                const uint32_t n = lin(c[0], c[1], c[2], P);
                double r[3], lb[3], j[3], t3[3];
                for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], s1->X[a], L[a], P.wall[a]);
                cross3(adj->lL, r, lb);
                for (int a = 0; a < 3; ++a) lb[a] += adj->lP[a];
                for (int l = 0; l < 2; ++l) {
                    lam1[(size_t)l * N + n] = ssplit(s_lled[l]);
                    for (int a = 0; a < 3; ++a) lam1[(size_t)(2 + 3 * l + a) * N + n] = ssplit(lb[a]);
                }
                for (int a = 0; a < 3; ++a) j[a] = (double)tape1[(2 + a) * N + n] + (double)tape1[(5 + a) * N + n];
                cross3(j, adj->lL, t3);  // d/dX' of lambda_L . ((c - X') x j) = -(j x lambda_L)
                for (int a = 0; a < 3; ++a) acc[a] -= t3[a];
            }
        }
        if (m0[t]) {  // uncovered
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = o0[a] + d[a];
                if (!P.wall[a] && c[a] >= L[a]) c[a] -= L[a];
            }
            if (!is_solid(c[0], c[1], c[2], o1, m1, P)) {
                double mean[2] = {0.0, 0.0};
                int cnt = 0;
                for (int jd = 1; jd < 19; ++jd) {
                    int q[3];
                    if (!nbr(c[0], c[1], c[2], cxv(jd), cyv(jd), czv(jd), P, q)) continue;
                    if (is_solid(q[0], q[1], q[2], o1, m1, P) || is_solid(q[0], q[1], q[2], o0, m0, P)) continue;
                    const uint32_t m = lin(q[0], q[1], q[2], P);
                    mean[0] += tape1[m];
                    mean[1] += tape1[N + m];
                    ++cnt;
                }
                const double rl[2] = {cnt ? mean[0] / cnt : P.rho0[0], cnt ? mean[1] / cnt : P.rho0[1]};
                double r[3], w[3], ub[3], lq[3];
                for (int a = 0; a < 3; ++a) r[a] = rel_axis((double)c[a], s1->X[a], L[a], P.wall[a]);
                cross3(s1->Om, r, w);
                for (int a = 0; a < 3; ++a) ub[a] = s1->V[a] + w[a];
                cross3(adj->lL, r, lq);
                for (int a = 0; a < 3; ++a) lq[a] += adj->lP[a];  // lambda_P + lambda_L x d
                const uint32_t n = lin(c[0], c[1], c[2], P);
                double lub[3] = {0, 0, 0};
                const double rsum = rl[0] + rl[1];
                double lqub = lq[0] * ub[0] + lq[1] * ub[1] + lq[2] * ub[2];
                for (int l = 0; l < 2; ++l) {
                    const double al = sval(lam1[(size_t)l * N + n]);
                    double bl[3];
                    for (int a = 0; a < 3; ++a) bl[a] = sval(lam1[(size_t)(2 + 3 * l + a) * N + n]);
                    const double lmean = al + bl[0] * ub[0] + bl[1] * ub[1] + bl[2] * ub[2] - lqub - s_lled[l];
                    if (cnt) uv[(size_t)l * B3 + t] = lmean / cnt;
                    for (int a = 0; a < 3; ++a) lub[a] += rl[l] * bl[a];
                }
                for (int a = 0; a < 3; ++a) lub[a] -= rsum * lq[a];
                // u_b = V' + Omega' x d, d = c - X'
                double t1[3], t2[3], pm[3], t4[3];
                cross3(r, lub, t1);           // lambda Omega' += d x lambda_u_b
                cross3(lub, s1->Om, t2);      // lambda X' -= lambda_u_b x Omega'
                for (int a = 0; a < 3; ++a) pm[a] = rsum * ub[a];
                cross3(pm, adj->lL, t4);      // lambda X' += pm x lambda_L (from -d x pm)
                for (int a = 0; a < 3; ++a) {
                    acc[a] += -t2[a] + t4[a];
                    acc[3 + a] += lub[a];
                    acc[6 + a] += t1[a];
                }
            }
        }
    }
    double v8[8];
    for (int k = 0; k < 8; ++k) v8[k] = acc[k];
    block_sum8<kT>(v8, s_red, s_out);
    if (threadIdx.x < 8) parts[blockIdx.x * 9 + threadIdx.x] = s_out[threadIdx.x];
    __syncthreads();
    double v1[8] = {acc[8], 0, 0, 0, 0, 0, 0, 0};
    block_sum8<kT>(v1, s_red, s_out);
    if (threadIdx.x == 0) parts[blockIdx.x * 9 + 8] = s_out[0];
    if (!last_block(&adj->cover_done, gridDim.x, threadIdx.x < 8)) return;  // threads 0..7 wrote parts
    if (threadIdx.x < 9) {
        double sum = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) sum += __ldcg(parts + b * 9 + threadIdx.x);
        s_c[threadIdx.x] = sum;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    adj->lled[0] = s_lled[0];
    adj->lled[1] = s_lled[1];
    update_adjoint(adj, s_c, s0, inv2T, dFp_dg);
}

// Neighbours of uncovered nodes that fed the neighbour mean: fluid at n and
// at n+1. Gathers uv of uncovered neighbours into a_l. One thread per node of
// the old box grown by one.
static __global__ void __launch_bounds__(kT) ka_cover_mean(lam_t* __restrict__ lam1, const DevState* __restrict__ s0,
                                                           const uint8_t* __restrict__ mk0,
                                                           const DevState* __restrict__ s1,
                                                           const uint8_t* __restrict__ mk1, const double* __restrict__ uv,
                                                           KParams P)
{
    const int B = P.B, G = B + 2, B3 = B * B * B;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * G * G) return;
    const uint8_t* m0 = cur_mask(s0, mk0, P);
    const uint8_t* m1 = cur_mask(s1, mk1, P);
    const int o0[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
    const int o1[3] = {s1->box0[0], s1->box0[1], s1->box0[2]};
    const int L[3] = {P.lx, P.ly, P.lz};
    const int d[3] = {t % G, (t / G) % G, t / (G * G)};
    int m[3];
    for (int a = 0; a < 3; ++a) {
        m[a] = o0[a] - 1 + d[a];
        if (m[a] < 0 || m[a] >= L[a]) {
            if (P.wall[a]) return;
            m[a] += (m[a] < 0) ? L[a] : -L[a];
        }
    }
    if (is_solid(m[0], m[1], m[2], o0, m0, P) || is_solid(m[0], m[1], m[2], o1, m1, P)) return;
    double add[2] = {0.0, 0.0};
    for (int jd = 1; jd < 19; ++jd) {
        int c[3];
        if (!nbr(m[0], m[1], m[2], cxv(jd), cyv(jd), czv(jd), P, c)) continue;
        if (!is_solid(c[0], c[1], c[2], o0, m0, P) || is_solid(c[0], c[1], c[2], o1, m1, P)) continue;
        const int e = box_rel(c[0], o0[0], L[0], P.wall[0]) +
                      B * (box_rel(c[1], o0[1], L[1], P.wall[1]) + B * box_rel(c[2], o0[2], L[2], P.wall[2]));
        add[0] += uv[e];
        add[1] += uv[B3 + e];
    }
    if (add[0] != 0.0 || add[1] != 0.0) {
        const uint32_t n = lin(m[0], m[1], m[2], P);
        lam1[n] = ssplit(sval(lam1[n]) + add[0]);
        lam1[P.N + n] = ssplit(sval(lam1[P.N + n]) + add[1]);
    }
}


// ---------------------------------------------------------------------------
// Per fluid node of step n: adjoint of streaming (pulled from the
// destinations' (a, b) in lam1), of the moving links and the Shan-Chen
// reaction on the particle, and of the collision (adj_modes). Writes the
// node's b_l and the local part of a_l into lam0, lambda g_l into lg, and
// per-tile partials (link terms of lambda X, V, Omega; dJ/dG; lambda delta).
// ---------------------------------------------------------------------------
// Thread (tx, ty) of tile (bx, by, bz); every thread of the block calls it.
// PARTICLE: the tile is near the particle (links, reaction); else it has none.
template <bool PARTICLE>
__device__ __forceinline__ void adj_tile(int bx, int by, int bz, int tx, int ty, const float* __restrict__ tape,
                                         const float* __restrict__ psi, const lam_t* __restrict__ lam1,
                                         lam_t* __restrict__ lam0, lg_t* __restrict__ lg,
                                         const DevState* __restrict__ s0, const uint8_t* __restrict__ mk0,
                                         const AdjState* __restrict__ adj, double* __restrict__ parts,
                                         const KParams& P)
{
    __shared__ double s_red[(kT / 32) * 8];
    __shared__ double s_out[8];
    const int x = bx * P.tx + tx;
    const int y = by * P.ty + ty;
    const int z = bz;
    const size_t N = P.N;
    double acc[kNodeParts];
#pragma unroll
    for (int k = 0; k < kNodeParts; ++k) acc[k] = 0.0;
    if (x < P.lx && y < P.ly) {
        const uint8_t* m0 = cur_mask(s0, mk0, P);
        const uint32_t n = lin(x, y, z, P);
        if (PARTICLE && solid_at(x, y, z, s0, m0, P)) {
            for (int k = 0; k < 8; ++k) lam0[k * N + n] = Split{0.0f, 0.0f};
            for (int k = 0; k < 6; ++k) lg[k * N + n] = Split{0.0f, 0.0f};
        } else {
            float rho[2], j[2][3], g[2][3];
            for (int l = 0; l < 2; ++l) {
                rho[l] = tape[l * N + n];
                for (int a = 0; a < 3; ++a) j[l][a] = tape[(2 + 3 * l + a) * N + n];
            }
            const float* pA = psi + pad_index(x, y, z, P);
            const float* pB = pA + P.padn;
            const int sy = P.px, sz = P.px * P.py;
            for (int a = 0; a < 3; ++a) g[0][a] = g[1][a] = 0.0f;
            uint32_t solid_nb = 0, wall_nb = 0;
            uint32_t qidx[19];
            qidx[0] = n;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const int off = cxv(i) + sy * cyv(i) + sz * czv(i);
                const float w = wv(i);
                const float pa = pA[off], pb = pB[off];
                g[0][0] += cxv(i) * w * pb; g[0][1] += cyv(i) * w * pb; g[0][2] += czv(i) * w * pb;
                g[1][0] += cxv(i) * w * pa; g[1][1] += cyv(i) * w * pa; g[1][2] += czv(i) * w * pa;
                int q[3];
                if (!nbr(x, y, z, cxv(i), cyv(i), czv(i), P, q)) {
                    wall_nb |= 1u << i;
                    qidx[i] = n;
                } else {
                    qidx[i] = lin(q[0], q[1], q[2], P);
                    if (PARTICLE && solid_at(q[0], q[1], q[2], s0, m0, P)) solid_nb |= 1u << i;
                }
            }
            // Particle-link constants of this node: lever of each link, u_b . c_i
            // (float, as the forward step), forward post-collision populations.
            float rnf[3] = {0.f, 0.f, 0.f};
            float fo[2][19];
            const float ext[3] = {P.ext[0], P.ext[1], P.ext[2]};
            if (PARTICLE && solid_nb) {
                for (int a = 0; a < 3; ++a) {
                    const int c = a == 0 ? x : (a == 1 ? y : z);
                    const int L = a == 0 ? P.lx : (a == 1 ? P.ly : P.lz);
                    rnf[a] = (float)rel_axis((double)c, s0->X[a], L, P.wall[a]);
                }
                float ms[2][10];
                fwd_modes<float>(rho, j, g, ext, P.G, ms);
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    float nm[19];
                    for (int k = 0; k < 19; ++k) nm[k] = k < 10 ? ms[l][k] / bnorm(k) : 0.0f;
                    nm[0] = ms[l][0] + s0->delta_f[l];
                    from_modes(nm, fo[l]);
                }
            }
            const float* lF = adj->lFf;
            const float* lT = adj->lTf;
            df lrx[2];  // extra adjoint of rho_l from links and the reaction
            // This node's link and reaction terms of partials 0..9, added to acc once.
            df lk[10];
            const df lled[2] = {df(adj->lled[0]), df(adj->lled[1])};
            Split asv[2], bsv[2][3];         // a_l, b_l of this node
            float lm[2][10];               // mode adjoint of the neighbour differences
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const Split as = lam1[(size_t)l * N + n];
                Split bs[3];
                for (int a = 0; a < 3; ++a) bs[a] = lam1[(size_t)(2 + 3 * l + a) * N + n];
                asv[l] = as;
                for (int a = 0; a < 3; ++a) bsv[l][a] = bs[a];
                const double ax = sval(as);
                float wl[19];
                float wsum = 0.0f;
#pragma unroll
                for (int i = 0; i < 19; ++i) {
                    const int cx = cxv(i), cy = cyv(i), cz = czv(i);
                    // dv = lambda f*_li - a_l(x) - c_i . b_l(x): small, float32 is enough.
                    float dv;
                    if ((wall_nb | solid_nb) >> i & 1u) {
                        // bounce-back reads (x, -c_i): a - c_i . b, so dv = -2 c_i . b (float)
                        dv = -2.0f * (cx * bs[0].hi + cy * bs[1].hi + cz * bs[2].hi);
                        if (PARTICLE && (solid_nb >> i & 1u)) {
                            // The large adjoint parts (a_l, b_l and the ledger's) in double-float,
                            // the forward quantities in float.
                            df cb;
                            if (cx) cb += cx > 0 ? df(bs[0].hi, bs[0].lo) : -df(bs[0].hi, bs[0].lo);
                            if (cy) cb += cy > 0 ? df(bs[1].hi, bs[1].lo) : -df(bs[1].hi, bs[1].lo);
                            if (cz) cb += cz > 0 ? df(bs[2].hi, bs[2].lo) : -df(bs[2].hi, bs[2].lo);
                            const float d[3] = {rnf[0] + 0.5f * cx, rnf[1] + 0.5f * cy, rnf[2] + 0.5f * cz};
                            const float kap = cx * (lF[0] + lT[1] * d[2] - lT[2] * d[1]) +
                                              cy * (lF[1] + lT[2] * d[0] - lT[0] * d[2]) +
                                              cz * (lF[2] + lT[0] * d[1] - lT[1] * d[0]);
                            const float* V = s0->Vf;
                            const float* Om = s0->Omf;
                            const float ubc = (V[0] + Om[1] * d[2] - Om[2] * d[1]) * cx +
                                              (V[1] + Om[2] * d[0] - Om[0] * d[2]) * cy +
                                              (V[2] + Om[0] * d[1] - Om[1] * d[0]) * cz;
                            const df lcorr = (cb - df(as.hi, as.lo)) + (lled[l] + (-kap));
                            const float w6 = 6.0f * wv(i);
                            lrx[l] += lcorr * (w6 * ubc);
                            const df lub = lcorr * (w6 * rho[l]);  // lambda (u_b . c_i)
                            // With lb = lub c_i: partials 3..5 += lb, 6..8 += d x lb,
                            // 0..2 -= lb x Omega (the float sums of coefficients exact).
                            if (cx) lk[3] += cx > 0 ? lub : -lub;
                            if (cy) lk[4] += cy > 0 ? lub : -lub;
                            if (cz) lk[5] += cz > 0 ? lub : -lub;
                            lk[6] += lub * two_sum(d[1] * cz, -d[2] * cy);
                            lk[7] += lub * two_sum(d[2] * cx, -d[0] * cz);
                            lk[8] += lub * two_sum(d[0] * cy, -d[1] * cx);
                            lk[0] += lub * two_sum(cz * Om[1], -cy * Om[2]);
                            lk[1] += lub * two_sum(cx * Om[2], -cz * Om[0]);
                            lk[2] += lub * two_sum(cy * Om[0], -cx * Om[1]);
                            // lever of the exchanged momentum (2 f* - corr) c_i (small: float)
                            const float dp = 2.0f * fo[l][i] - w6 * rho[l] * ubc;
                            lk[0] = lk[0] + (-dp * (cy * lT[2] - cz * lT[1]));
                            lk[1] = lk[1] + (-dp * (cz * lT[0] - cx * lT[2]));
                            lk[2] = lk[2] + (-dp * (cx * lT[1] - cy * lT[0]));
                            dv += 2.0f * kap;
                        }
                    } else {
                        const uint32_t q = qidx[i];
                        dv = sdiff(lam1[(size_t)l * N + q], as);
                        if (cx) dv += cx * sdiff(lam1[(2 + 3 * l) * N + q], bs[0]);
                        if (cy) dv += cy * sdiff(lam1[(3 + 3 * l) * N + q], bs[1]);
                        if (cz) dv += cz * sdiff(lam1[(4 + 3 * l) * N + q], bs[2]);
                    }
                    wl[i] = wv(i) * dv;
                    wsum += wl[i];
                }
                acc[10 + l] += ax + (double)wsum;  // sum_i w_i lambda f*_li (mass correction)
                float mm[10];
                project10<float>(wl, mm);
                for (int k = 0; k < 10; ++k) lm[l][k] = mm[k] / bnorm(k);
            }
            // Shan-Chen reaction on the particle: F += G w_i (rhoA psiB(q) + rhoB psiA(q)) c_i.
            if (PARTICLE && solid_nb) {
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    if (!(solid_nb >> i & 1u)) continue;
                    const int cx = cxv(i), cy = cyv(i), cz = czv(i);
                    const int off = cx + sy * cy + sz * cz;
                    const float pa = pA[off], pb = pB[off];
                    const float d[3] = {rnf[0] + 0.5f * cx, rnf[1] + 0.5f * cy, rnf[2] + 0.5f * cz};
                    const float kap = cx * (lF[0] + lT[1] * d[2] - lT[2] * d[1]) +
                                      cy * (lF[1] + lT[2] * d[0] - lT[0] * d[2]) +
                                      cz * (lF[2] + lT[0] * d[1] - lT[1] * d[0]);
                    const float w = wv(i);
                    const float t = rho[0] * pb + rho[1] * pa;
                    lk[9] += two_prod(kap * w, t);
                    lrx[0] = lrx[0] + kap * P.G * w * pb;
                    lrx[1] = lrx[1] + kap * P.G * w * pa;
                    const float mag = P.G * w * t;
                    lk[0] = lk[0] + (-mag * (cy * lT[2] - cz * lT[1]));
                    lk[1] = lk[1] + (-mag * (cz * lT[0] - cx * lT[2]));
                    lk[2] = lk[2] + (-mag * (cx * lT[1] - cy * lT[0]));
                }
            }
            if (PARTICLE && solid_nb)
                for (int k = 0; k < 10; ++k) acc[k] += lk[k].value();
            // Transpose of the collision: the float32 part from the differences, the
            // 48-bit part from (a_l, b_l) of this node (modes 0..3 only).
            float lrho[2], lj[2][3], lgv[2][3], lG;
            adj_modes<float>(rho, j, g, ext, P.G, lm, lrho, lj, lgv, lG);
            {
                // Double-float for (a_l, b_l), stored as pairs, and the outputs;
                // the forward quantities and coefficients in float.
                df af[2], bf[2][3], lrf[2], ljf[2][3], lgf[2][3], lGf;
                for (int l = 0; l < 2; ++l) {
                    af[l] = df(asv[l].hi, asv[l].lo);
                    for (int a = 0; a < 3; ++a) bf[l][a] = df(bsv[l][a].hi, bsv[l][a].lo);
                }
                adj_modes_ab_mixed<df>(rho, j, g, ext, P.G, af, bf, lrf, ljf, lgf, lGf);
                acc[9] += lGf.value() + (double)lG;
                for (int l = 0; l < 2; ++l) {
                    df v = lrf[l] + lrho[l];
                    if (PARTICLE) v = v + lrx[l];  // link and reaction terms
                    lam0[(size_t)l * N + n] = Split{v.hi, v.lo};
                    for (int a = 0; a < 3; ++a) {
                        const df vj = ljf[l][a] + lj[l][a];
                        const df vg = lgf[l][a] + lgv[l][a];
                        lam0[(size_t)(2 + 3 * l + a) * N + n] = Split{vj.hi, vj.lo};
                        lg[(size_t)(3 * l + a) * N + n] = Split{vg.hi, vg.lo};
                    }
                }
            }
        }
    }
    double v8[8];
    for (int k = 0; k < 8; ++k) v8[k] = acc[k];
    const long long tile = bx + (long long)P.gx * (by + (long long)P.gy * bz);
    const int tid = tx + P.tx * ty;
    if (PARTICLE) {
        block_sum8<kT>(v8, s_red, s_out);
        if (tid < 8) parts[tile * kNodeParts + tid] = s_out[tid];
        __syncthreads();
    } else if (tid < 9) {
        parts[tile * kNodeParts + tid] = 0.0;  // no link terms away from the particle
    }
    double v4[kNodeParts - 8];
    for (int k = 0; k < kNodeParts - 8; ++k) v4[k] = acc[8 + k];
    block_sum_n<kNodeParts - 8>(v4, s_red, s_out);
    if (tid < kNodeParts - 8) parts[tile * kNodeParts + 8 + tid] = s_out[tid];
}

// Tiles away from the particle (all tiles when there is none). Three blocks
// per SM: a few spills, and more resident warps to hide the neighbour
// gathers (measured faster than two).
static __global__ void __launch_bounds__(kT, 3) ka_node_bulk(const float* __restrict__ tape, const float* __restrict__ psi,
                                                          const lam_t* __restrict__ lam1, lam_t* __restrict__ lam0,
                                                          lg_t* __restrict__ lg, const DevState* __restrict__ s0,
                                                          const uint8_t* __restrict__ mk0,
                                                          const AdjState* __restrict__ adj, double* __restrict__ parts,
                                                          KParams P)
{
    if (P.has_particle) {
        const int o[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
        if (tile_near(blockIdx.x, blockIdx.y, blockIdx.z, o, P)) return;
    }
    adj_tile<false>(blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, tape, psi, lam1, lam0, lg, s0, mk0,
                    adj, parts, P);
}

// Tiles near the particle: the candidate grid of the forward step.
static __global__ void __launch_bounds__(kT) ka_node_near(const float* __restrict__ tape, const float* __restrict__ psi,
                                                          const lam_t* __restrict__ lam1, lam_t* __restrict__ lam0,
                                                          lg_t* __restrict__ lg, const DevState* __restrict__ s0,
                                                          const uint8_t* __restrict__ mk0,
                                                          const AdjState* __restrict__ adj, double* __restrict__ parts,
                                                          KParams P)
{
    const int o[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
    const int bx = candidate_tile(blockIdx.x, o[0], P.tx, P.gx, P.lx, P.wall[0]);
    const int by = candidate_tile(blockIdx.y, o[1], P.ty, P.gy, P.ly, P.wall[1]);
    const int bz = candidate_tile(blockIdx.z, o[2], 1, P.lz, P.lz, P.wall[2]);
    if (bx < 0 || by < 0 || bz < 0 || !tile_near(bx, by, bz, o, P)) return;
    adj_tile<true>(bx, by, bz, threadIdx.x, threadIdx.y, tape, psi, lam1, lam0, lg, s0, mk0, adj, parts, P);
}

// Fluid-neighbour count of lattice point q (wrapped on periodic axes), as the
// virtual layer and the wall ghosts use it.
__device__ __forceinline__ int fluid_count(const int q[3], const DevState* s0, const uint8_t* m0, const KParams& P)
{
    int cnt = 0;
    for (int jd = 1; jd < 19; ++jd) {
        int r[3];
        if (!nbr(q[0], q[1], q[2], cxv(jd), cyv(jd), czv(jd), P, r)) continue;
        if (solid_at(r[0], r[1], r[2], s0, m0, P)) continue;
        ++cnt;
    }
    return cnt;
}

// lambda psi_l at padded point p (in range on every periodic axis): the
// Shan-Chen stencil transposed, g_A reads psi_B and g_B reads psi_A. Sources
// whose lambda g is zero (particle nodes) add nothing and are skipped. The
// others are taken as float differences from the first of them (r) plus
// r sum w_i c_i over them in FP64, where sum w_i c_i = (2 n_axis + n_diag) / 36
// per axis from the integer sums of c_i over the included axis and diagonal
// directions (zero when every source is included).
__device__ __forceinline__ void lpsi_gather(const int p[3], const lg_t* __restrict__ lg, const KParams& P,
                                            double out[2])
{
    const size_t N = P.N;
    Split r[6];
    bool have = false;
    int nc[3] = {0, 0, 0};  // 2 sum c over included axis directions + sum c over diagonal ones
    float la = 0.0f, lb = 0.0f;
    for (int i = 1; i < 19; ++i) {
        int x[3];
        if (!nbr(p[0], p[1], p[2], -cxv(i), -cyv(i), -czv(i), P, x)) continue;
        // a source outside the domain (p is a ghost and -c_i points further out) is skipped by nbr()
        const uint32_t s = lin(x[0], x[1], x[2], P);
        Split v[6];
        bool zero = true;
        for (int k = 0; k < 6; ++k) {
            v[k] = lg[k * N + s];
            zero = zero && v[k].hi == 0.0f && v[k].lo == 0.0f;
        }
        if (zero) continue;
        if (!have) {
            for (int k = 0; k < 6; ++k) r[k] = v[k];
            have = true;
        }
        const int c[3] = {cxv(i), cyv(i), czv(i)};
        const int wt = i <= 6 ? 2 : 1;  // w_i in units of 1/36
        const float w = wv(i);
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            nc[a] += wt * c[a];
            lb += w * c[a] * sdiff(v[a], r[a]);
            la += w * c[a] * sdiff(v[3 + a], r[3 + a]);
        }
    }
    double da = la, db = lb;
    if (have)
        for (int a = 0; a < 3; ++a)
            if (nc[a]) {
                db += sval(r[a]) * (nc[a] * (1.0 / 36.0));
                da += sval(r[3 + a]) * (nc[a] * (1.0 / 36.0));
            }
    out[0] = da;
    out[1] = db;
}

// lpsi_gather at fluid node n = (x, y, z) whose 18 neighbours are fluid nodes
// of the domain. Then sum_i w_i c_i = 0 over the sources, so the stencil is
// taken on the differences from the node's own lambda g_l, in float.
__device__ __forceinline__ void lpsi_gather_inner(int x, int y, int z, uint32_t n, const lg_t* __restrict__ lg,
                                                  const KParams& P, float out[2])
{
    const size_t N = P.N;
    const lg_t* g[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = lg + k * N;
    Split r[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) r[k] = g[k][n];
    // Away from the faces the source x - c_i is n minus a fixed offset.
    const bool inside = (unsigned)(x - 1) < (unsigned)(P.lx - 2) && (unsigned)(y - 1) < (unsigned)(P.ly - 2) &&
                        (unsigned)(z - 1) < (unsigned)(P.lz - 2);
    const uint32_t sy = (uint32_t)P.lx, sz = (uint32_t)P.lx * (uint32_t)P.ly;
    float la = 0.0f, lb = 0.0f;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int cx = cxv(i), cy = cyv(i), cz = czv(i);
        uint32_t s;
        if (inside) {
            s = n - (uint32_t)cx - (uint32_t)cy * sy - (uint32_t)cz * sz;
        } else {
            int q[3];
            nbr(x, y, z, -cx, -cy, -cz, P, q);  // in the domain: the caller checked
            s = lin(q[0], q[1], q[2], P);
        }
        const float w = wv(i);
        float tb = 0.0f, ta = 0.0f;
        if (cx) { tb += cx * sdiff(g[0][s], r[0]); ta += cx * sdiff(g[3][s], r[3]); }
        if (cy) { tb += cy * sdiff(g[1][s], r[1]); ta += cy * sdiff(g[4][s], r[4]); }
        if (cz) { tb += cz * sdiff(g[2][s], r[2]); ta += cz * sdiff(g[5][s], r[5]); }
        lb += w * tb;
        la += w * ta;
    }
    out[0] = la;
    out[1] = lb;
}

// ---------------------------------------------------------------------------
// Adjoint of psi at the particle nodes, one warp per entry of the particle
// box, lane i = 1..18 taking direction i. A particle node with fluid
// neighbours (virtual layer) gets lambda psi (lpsi_gather's sum, its sources
// p - c_i spread over the lanes, the reference the first nonzero source in
// direction order) plus the Shan-Chen reaction's dependence on it, then
// mu_l = lambda psi_l / cnt where the clip at 0 is inactive, written at the
// node's place in lpsi; dJ/d delta_rho partial per block of kLpsiEntries
// entries. A node without fluid neighbours gets mu = 0.
// ---------------------------------------------------------------------------
constexpr int kLpsiEntries = kT / 32;  // box entries per block

__host__ __device__ __forceinline__ int lpsi_blocks(const KParams& P)
{
    return (P.B * P.B * P.B + kLpsiEntries - 1) / kLpsiEntries;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

static __global__ void __launch_bounds__(kT) ka_lpsi(const lg_t* __restrict__ lg, const float* __restrict__ psi,
                                                     double* __restrict__ lpsi, const DevState* __restrict__ s0,
                                                     const uint8_t* __restrict__ mk0, const AdjState* __restrict__ adj,
                                                     double* __restrict__ parts2, KParams P)
{
    __shared__ double s_red[(kT / 32) * 8];
    __shared__ double s_out[8];
    const int B = P.B;
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * kLpsiEntries + (threadIdx.x >> 5);
    const uint8_t* m0 = cur_mask(s0, mk0, P);
    double dd = 0.0;
    if (t < B * B * B && m0[t]) {  // the same for every lane of the warp
        const size_t N = P.N;
        const int L[3] = {P.lx, P.ly, P.lz};
        const int dlt[3] = {t % B, (t / B) % B, t / (B * B)};
        int p[3];
        for (int a = 0; a < 3; ++a) {
            p[a] = s0->box0[a] + dlt[a];
            if (!P.wall[a] && p[a] >= L[a]) p[a] -= L[a];
        }
        const long long pi = pad_index(p[0], p[1], p[2], P);
        const bool dir = lane >= 1 && lane <= 18;
        const int c[3] = {cxv(lane), cyv(lane), czv(lane)};
        // q = p - c_i: a source of the stencil transposed and, if fluid, a
        // fluid neighbour reading psi(p) along +c_i.
        int q[3];
        const bool inq = dir && nbr(p[0], p[1], p[2], -c[0], -c[1], -c[2], P, q);
        const bool fluid = inq && !solid_at(q[0], q[1], q[2], s0, m0, P);
        const int cnt = __popc(__ballot_sync(0xffffffffu, fluid));
        double mu[2] = {0.0, 0.0};
        if (cnt) {
            // lpsi_gather: sources whose lambda g is zero (particle nodes) add
            // nothing; the others as float differences from the first of them
            // (r), plus r sum w_i c_i over them in FP64.
            Split v[6];
            bool nz = false;
            if (inq) {
                const uint32_t sidx = lin(q[0], q[1], q[2], P);
                for (int k = 0; k < 6; ++k) {
                    v[k] = lg[k * N + sidx];
                    nz = nz || v[k].hi != 0.0f || v[k].lo != 0.0f;
                }
            } else {
                for (int k = 0; k < 6; ++k) v[k] = Split{0.0f, 0.0f};
            }
            const unsigned nzm = __ballot_sync(0xffffffffu, nz);
            double lp[2] = {0.0, 0.0};
            if (nzm) {
                const int f = __ffs(nzm) - 1;
                Split r[6];
                for (int k = 0; k < 6; ++k) {
                    r[k].hi = __shfl_sync(0xffffffffu, v[k].hi, f);
                    r[k].lo = __shfl_sync(0xffffffffu, v[k].lo, f);
                }
                float la = 0.0f, lb = 0.0f;
                int nc[3] = {0, 0, 0};
                if (nz) {
                    const int wt = lane <= 6 ? 2 : 1;  // w_i in units of 1/36
                    const float w = wv(lane);
                    for (int a = 0; a < 3; ++a) {
                        if (!c[a]) continue;
                        nc[a] = wt * c[a];
                        lb += w * c[a] * sdiff(v[a], r[a]);
                        la += w * c[a] * sdiff(v[3 + a], r[3 + a]);
                    }
                }
                lp[0] = warp_sum(la);
                lp[1] = warp_sum(lb);
                for (int a = 0; a < 3; ++a) {
                    const int n = warp_sum(nc[a]);
                    if (n) {
                        lp[1] += sval(r[a]) * (n * (1.0 / 36.0));
                        lp[0] += sval(r[3 + a]) * (n * (1.0 / 36.0));
                    }
                }
            }
            // The Shan-Chen reaction on the particle through psi(p).
            double ra = 0.0, rb = 0.0;
            if (fluid) {
                const float* lF = adj->lFf;
                const float* lT = adj->lTf;
                float d[3];
                for (int a = 0; a < 3; ++a) d[a] = (float)rel_axis((double)q[a], s0->X[a], L[a], P.wall[a]) + 0.5f * c[a];
                const float kap = c[0] * (lF[0] + lT[1] * d[2] - lT[2] * d[1]) +
                                  c[1] * (lF[1] + lT[2] * d[0] - lT[0] * d[2]) +
                                  c[2] * (lF[2] + lT[0] * d[1] - lT[1] * d[0]);
                const long long qi = pad_index(q[0], q[1], q[2], P);
                rb = double(kap * P.G * wv(lane) * psi[qi]);           // d/d psiB(p) of rhoA(q) psiB(p)
                ra = double(kap * P.G * wv(lane) * psi[P.padn + qi]);  // d/d psiA(p) of rhoB(q) psiA(p)
            }
            lp[0] += warp_sum(ra);
            lp[1] += warp_sum(rb);
            const bool actA = psi[pi] > 0.0f, actB = psi[P.padn + pi] > 0.0f;
            if (actA) { mu[0] = lp[0] / double(cnt); dd += lp[0]; }
            if (actB) { mu[1] = lp[1] / double(cnt); dd -= lp[1]; }
        }
        if (lane == 0) {
            lpsi[pi] = mu[0];
            lpsi[P.padn + pi] = mu[1];
        }
    }
    double v8[8] = {lane == 0 ? dd : 0.0, 0, 0, 0, 0, 0, 0, 0};
    block_sum8<kT>(v8, s_red, s_out);
    if (threadIdx.x == 0) parts2[blockIdx.x] = s_out[0];
}

// Wall ghosts of the psi shell (points outside along a wall axis, in range on
// the periodic axes): mu_l = lambda psi_l / cnt, the mean over fluid neighbours.
static __global__ void __launch_bounds__(kT) ka_lpsi_shell(const lg_t* __restrict__ lg, double* __restrict__ lpsi,
                                                           const DevState* __restrict__ s0,
                                                           const uint8_t* __restrict__ mk0, KParams P)
{
    // The shell points in the order shell_node takes them, decoded in 32 bits
    // (each face holds fewer than 2^31 points).
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int pw = P.lx + 2;  // padded row length (the row stride P.px may be larger)
    const int zf = pw * P.py, yf = pw * P.lz, xf = P.ly * P.lz;
    if (t >= 2LL * zf + 2LL * yf + 2LL * xf) return;
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
    bool ghost = false;
    for (int a = 0; a < 3; ++a) {
        const bool out = p[a] < 0 || p[a] >= L[a];
        if (out && !P.wall[a]) return;  // a periodic copy: its reads are attributed to the interior point
        ghost |= out;
    }
    if (!ghost) return;
    const uint8_t* m0 = cur_mask(s0, mk0, P);
    double lp[2];
    lpsi_gather(p, lg, P, lp);
    const int cnt = fluid_count(p, s0, m0, P);
    const long long dst = (long long)(p[0] + 1) + (long long)P.px * ((p[1] + 1) + (long long)P.py * (p[2] + 1));
    lpsi[dst] = cnt ? lp[0] / double(cnt) : 0.0;
    lpsi[P.padn + dst] = cnt ? lp[1] / double(cnt) : 0.0;
}

// a_l of fluid node (x, y, z): lambda psi of the node (the Shan-Chen stencil
// transposed) plus mu of every particle node and wall ghost among its
// neighbours (each averaged this node's density). Only an edge candidate
// (adj_edge_candidate) can have such neighbours; the others skip the scan.
__device__ __forceinline__ void final_node(int x, int y, int z, bool candidate, lam_t* __restrict__ lam0,
                                           const lg_t* __restrict__ lg, const double* __restrict__ lpsi,
                                           const DevState* __restrict__ s0, const uint8_t* __restrict__ m0,
                                           const KParams& P)
{
    const uint32_t n = lin(x, y, z, P);
    // Particle nodes and wall ghosts among the neighbours: their mu, and
    // whether the stencil of this node meets any (the neighbours of a node
    // are its own sources, -c_i running over the same 18 directions).
    double add[2] = {0.0, 0.0};
    bool edge = false;
    const int L[3] = {P.lx, P.ly, P.lz};
    for (int i = 1; candidate && i < 19; ++i) {
        int r[3] = {x + cxv(i), y + cyv(i), z + czv(i)};
        bool ghost = false;
        for (int a = 0; a < 3; ++a) {
            if (r[a] < 0 || r[a] >= L[a]) {
                if (P.wall[a]) ghost = true;
                else r[a] += (r[a] < 0) ? L[a] : -L[a];
            }
        }
        if (!ghost && !solid_at(r[0], r[1], r[2], s0, m0, P)) continue;
        edge = true;
        const long long q = (long long)(r[0] + 1) + (long long)P.px * ((r[1] + 1) + (long long)P.py * (r[2] + 1));
        add[0] += lpsi[q];
        add[1] += lpsi[P.padn + q];
    }
    // psi = rho on this fluid node
    if (edge) {
        const int p[3] = {x, y, z};
        double g[2];
        lpsi_gather(p, lg, P, g);
        lam0[n] = ssplit(sval(lam0[n]) + (add[0] + g[0]));
        lam0[P.N + n] = ssplit(sval(lam0[P.N + n]) + (add[1] + g[1]));
    } else {
        float g[2];
        lpsi_gather_inner(x, y, z, n, lg, P, g);
        for (int c = 0; c < 2; ++c) {
            const Split o = lam0[c * P.N + n];
            const df v = df(o.hi, o.lo) + df(g[c]);
            lam0[c * P.N + n] = Split{v.hi, v.lo};
        }
    }
}

// Fluid nodes that are not edge candidates (every warp takes the same path).
static __global__ void __launch_bounds__(kT) ka_final(lam_t* __restrict__ lam0, const lg_t* __restrict__ lg,
                                                      const double* __restrict__ lpsi, const DevState* __restrict__ s0,
                                                      const uint8_t* __restrict__ mk0, KParams P)
{
    const int x = blockIdx.x * P.tx + threadIdx.x;
    const int y = blockIdx.y * P.ty + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= P.lx || y >= P.ly) return;
    const int c[3] = {x, y, z};
    const int o[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
    if (adj_edge_candidate(c, o, P)) return;  // ka_final_edge's
    final_node(x, y, z, false, lam0, lg, lpsi, s0, cur_mask(s0, mk0, P), P);
}

// The edge candidates, each once (adj_edge_node), in nearly uniform warps.
static __global__ void __launch_bounds__(kT) ka_final_edge(lam_t* __restrict__ lam0, const lg_t* __restrict__ lg,
                                                           const double* __restrict__ lpsi,
                                                           const DevState* __restrict__ s0,
                                                           const uint8_t* __restrict__ mk0, KParams P)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int o[3] = {s0->box0[0], s0->box0[1], s0->box0[2]};
    int c[3];
    if (!adj_edge_node(t, o, P, c)) return;
    const uint8_t* m0 = cur_mask(s0, mk0, P);
    if (solid_at(c[0], c[1], c[2], s0, m0, P)) return;
    final_node(c[0], c[1], c[2], true, lam0, lg, lpsi, s0, m0, P);
}

// Per-tile partials -> adjoint of step n's particle state and the gradient
// sums. One block: each thread sums a fixed stride of tiles, then a fixed
// reduction tree (deterministic).
// Blocks of ka_reduce: each sums a fixed range of the tiles' partials (and of
// the particle box's), so the FP64 additions spread over several SMs; the
// last block to finish adds the blocks' sums in block order.
constexpr int kRedBlocks = 16;
constexpr int kRedSums = kNodeParts + 1;

__host__ __device__ __forceinline__ int reduce_blocks(long long ntiles)
{
    const long long b = (ntiles + kT - 1) / kT;
    return (int)(b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : b));
}

static __global__ void __launch_bounds__(kT) ka_reduce(AdjState* __restrict__ a, const double* __restrict__ parts,
                                                       long long ntiles, const double* __restrict__ parts2, int nbox,
                                                       double* __restrict__ red)
{
    __shared__ double s_red[(kT / 32) * 8];
    __shared__ double s_out[8];
    __shared__ double s_res[16];
    const long long nb = gridDim.x;
    const long long t0 = ntiles * blockIdx.x / nb, t1 = ntiles * (blockIdx.x + 1) / nb;
    const long long u0 = (long long)nbox * blockIdx.x / nb, u1 = (long long)nbox * (blockIdx.x + 1) / nb;
    double s[kRedSums];
    for (int k = 0; k < kRedSums; ++k) s[k] = 0.0;
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x)
        for (int k = 0; k < kNodeParts; ++k) s[k] += parts[t * kNodeParts + k];
    for (long long t = u0 + threadIdx.x; t < u1; t += blockDim.x) s[kNodeParts] += parts2[t];
    double v[8];
    for (int k = 0; k < 8; ++k) v[k] = s[k];
    block_sum8<kT>(v, s_red, s_out);
    if (threadIdx.x < 8) s_res[threadIdx.x] = s_out[threadIdx.x];
    __syncthreads();
    for (int k = 0; k < 8; ++k) v[k] = (8 + k < kRedSums) ? s[8 + k] : 0.0;
    block_sum8<kT>(v, s_red, s_out);
    if (threadIdx.x == 0)
        for (int k = 0; k < kRedSums; ++k) red[blockIdx.x * kRedSums + k] = k < 8 ? s_res[k] : s_out[k - 8];
    if (!last_block(&a->red_done, (unsigned)nb, threadIdx.x == 0)) return;
    if (threadIdx.x != 0) return;
    double r[kRedSums];
    for (int k = 0; k < kRedSums; ++k) r[k] = 0.0;
    for (long long b = 0; b < nb; ++b)
        for (int k = 0; k < kRedSums; ++k) r[k] += __ldcg(red + b * kRedSums + k);
    for (int k = 0; k < 3; ++k) {
        a->lX[k] += r[k];
        a->lV[k] += r[3 + k];
        a->lOm[k] += r[6 + k];
    }
    a->grad[2] += r[9];
    a->ld[0] = r[10];
    a->ld[1] = r[11];
    a->grad[1] += r[12];
}

}  // namespace flbm_adjoint

using namespace flbm_adjoint;

namespace {

// Device buffers of one adjoint run.
struct AdjBuffers {
    std::vector<void*> owned;
    float* ck_f = nullptr;     // checkpoints: populations (current copy)
    DevState* ck_st = nullptr; // checkpoints: particle record
    uint8_t* ck_m = nullptr;   // checkpoints: both particle masks
    float* ck_psi = nullptr;   // checkpoints: density field of the state (the fused step carries it)
    float* tape = nullptr;     // K+1 moment fields (slots of one segment)
    DevState* tape_st = nullptr;
    uint8_t* tape_m = nullptr;
    float* all_tape = nullptr;     // whole-tape store: T+1 moment fields
    DevState* all_st = nullptr;
    uint8_t* all_m = nullptr;
    lam_t* lam[2] = {nullptr, nullptr};
    lg_t* lgf = nullptr;
    double* lpsi = nullptr;
    double* uv = nullptr;
    double* parts = nullptr;
    double* parts2 = nullptr;
    double* cparts = nullptr;
    double* red = nullptr;      // per block of ka_reduce: its kRedSums sums
    AdjState* adj = nullptr;
    size_t bytes = 0;

    template <class T>
    bool alloc(T*& p, size_t n)
    {
        void* v = nullptr;
        if (cudaMalloc(&v, n * sizeof(T)) != cudaSuccess) return false;
        owned.push_back(v);
        bytes += n * sizeof(T);
        p = static_cast<T*>(v);
        return true;
    }
    // The whole-tape store of T+1 slots, all or nothing.
    bool alloc_store(size_t slots, size_t N, size_t mbytes)
    {
        const size_t keep = owned.size(), kept = bytes;
        if (alloc(all_tape, slots * 8 * N) && alloc(all_st, slots) && alloc(all_m, slots * mbytes)) return true;
        while (owned.size() > keep) {
            cudaFree(owned.back());
            owned.pop_back();
        }
        bytes = kept;
        all_tape = nullptr;
        all_st = nullptr;
        all_m = nullptr;
        cudaGetLastError();  // the failed allocation is not the run's error
        return false;
    }
    // Orderings between the two streams of a reverse step's last stages.
    cudaEvent_t ev_lpsi = nullptr, ev_shell = nullptr;
    bool make_events()
    {
        return cudaEventCreateWithFlags(&ev_lpsi, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&ev_shell, cudaEventDisableTiming) == cudaSuccess;
    }
    ~AdjBuffers()
    {
        for (void* v : owned) cudaFree(v);
        if (ev_lpsi) cudaEventDestroy(ev_lpsi);
        if (ev_shell) cudaEventDestroy(ev_shell);
    }
};

int acheck(flbm_sim* h, const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sim_fail(h, FLBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return FLBM_OK;
}

#define ACK(h, call)                                                                                              \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) return sim_fail((h), FLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// CUDA graphs of the run's repeated sequences of kAdjGraph steps: forward
// steps, each followed by the J sum, and recompute steps, each preceded by
// the tape writes of its slot (slots j kAdjGraph .. (j + 1) kAdjGraph - 1 of
// the segment). One per starting population copy (cur) and, for the
// recompute, per chunk j; captured on first use and replayed for every later
// chunk and segment. kAdjGraph is even, so a replay leaves cur where it was.
constexpr int kAdjGraph = 8;

struct AdjGraphs {
    cudaGraphExec_t fwd[2] = {nullptr, nullptr};
    std::vector<cudaGraphExec_t> rec[2];  // recompute with tape, per chunk of a segment
    std::vector<cudaGraphExec_t> fwt[2];  // forward with tape and J, per chunk of a segment
    cudaGraphExec_t rev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [lcur][cur], full segments
    ~AdjGraphs()
    {
        for (int c = 0; c < 2; ++c) {
            if (fwd[c]) cudaGraphExecDestroy(fwd[c]);
            for (cudaGraphExec_t g : rec[c])
                if (g) cudaGraphExecDestroy(g);
            for (cudaGraphExec_t g : fwt[c])
                if (g) cudaGraphExecDestroy(g);
            for (int d = 0; d < 2; ++d)
                if (rev[c][d]) cudaGraphExecDestroy(rev[c][d]);
        }
    }
};

// Capture what body() launches on h's stream into *out (nothing runs).
template <class Body>
int capture_graph(flbm_sim* h, cudaGraphExec_t* out, Body body)
{
    const int c = h->cur;
    const int64_t before = h->launches;
    ACK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->launches = before;
    h->cur = c;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return sim_fail(h, FLBM_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        *out = nullptr;
        return sim_fail(h, FLBM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
    }
    return FLBM_OK;
}

// Copy the handle's state (current populations, particle record, masks) to or from a slot.
// The state a step reads: populations, particle record, masks and the
// density field (so that a recomputed segment repeats the forward run bit
// for bit whichever way the step forms its densities).
int save_state(flbm_sim* h, float* f, DevState* st, uint8_t* m, size_t mbytes, float* psi)
{
    const size_t fbytes = sizeof(float) * 2 * 19 * h->kp.N;
    if (int rc = sim_ensure_psi(h)) return rc;
    ACK(h, cudaMemcpyAsync(f, h->fbuf[h->cur], fbytes, cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(st, h->st, sizeof(DevState), cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(m, h->masks, mbytes, cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(psi, psi_cur(h), sizeof(float) * 2 * h->kp.padn, cudaMemcpyDeviceToDevice, h->stream));
    return FLBM_OK;
}

int load_state(flbm_sim* h, const float* f, const DevState* st, const uint8_t* m, size_t mbytes, const float* psi)
{
    const size_t fbytes = sizeof(float) * 2 * 19 * h->kp.N;
    ACK(h, cudaMemcpyAsync(h->fbuf[h->cur], f, fbytes, cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(h->st, st, sizeof(DevState), cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(h->masks, m, mbytes, cudaMemcpyDeviceToDevice, h->stream));
    ACK(h, cudaMemcpyAsync(psi_cur(h), psi, sizeof(float) * 2 * h->kp.padn, cudaMemcpyDeviceToDevice, h->stream));
    h->psi_valid = true;
    return FLBM_OK;
}

// One reverse step: tape slot kk is step n's input state, slot kk+1 step n+1's.
int reverse_step(flbm_sim* h, AdjBuffers& b, int kk, lam_t* L1, lam_t* L0, double inv2T, double dFp_dg)
{
    const KParams& k = h->kp;
    const size_t N = k.N, B3 = (size_t)k.B * k.B * k.B, mbytes = 2 * B3;
    const float* tn = b.tape + (size_t)kk * 8 * N;
    const float* t1 = tn + 8 * N;
    const DevState* s0 = b.tape_st + kk;
    const DevState* s1 = s0 + 1;
    const uint8_t* m0 = b.tape_m + (size_t)kk * mbytes;
    const uint8_t* m1 = m0 + mbytes;
    cudaStream_t st = h->stream;
    // The reverse step rebuilds its densities from the tape in the density
    // buffer the current state does not use.
    float* psi_scr = h->psibuf[1 - h->cur];
    // The step's density field from the tape (side stream) does not depend on
    // the particle adjoint (handle's stream); the two join before the node kernels.
    ACK(h, cudaEventRecord(h->fork_ev, st));
    ACK(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
    ka_psi_tape<<<h->grid, h->block, 0, h->side>>>(tn, psi_scr, s0, m0, k);
    if (int rc = acheck(h, "ka_psi_tape")) return rc;
    const unsigned nbs = (unsigned)((shell_count(k) + kThreads - 1) / kThreads);
    const unsigned nbv = (unsigned)virtual_blocks(k);
    k_shell_virtual<<<nbs + nbv, kThreads, 0, h->side>>>(psi_scr, s0, m0, k, (int)nbs);
    if (int rc = acheck(h, "k_shell_virtual")) return rc;
    ACK(h, cudaEventRecord(h->join_ev, h->side));
    ka_cover<<<h->box_blocks, kT, 0, st>>>(L1, t1, s0, m0, s1, m1, b.adj, b.uv, b.cparts, k, inv2T, dFp_dg);
    if (int rc = acheck(h, "ka_cover")) return rc;
    const int G3 = (k.B + 2) * (k.B + 2) * (k.B + 2);
    ka_cover_mean<<<(G3 + kT - 1) / kT, kT, 0, st>>>(L1, s0, m0, s1, m1, b.uv, k);
    if (int rc = acheck(h, "ka_cover_mean")) return rc;
    ACK(h, cudaStreamWaitEvent(st, h->join_ev, 0));
    // Near tiles on the handle's side stream, concurrently with the bulk tiles
    // (disjoint nodes and partials), joined before the psi adjoint.
    ACK(h, cudaEventRecord(h->fork_ev, st));
    ACK(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
    ka_node_near<<<dim3(k.ncx, k.ncy, k.ncz), h->block, 0, h->side>>>(tn, psi_scr, L1, L0, b.lgf, s0, m0, b.adj,
                                                                       b.parts, k);
    if (int rc = acheck(h, "ka_node_near")) return rc;
    ACK(h, cudaEventRecord(h->join_ev, h->side));
    ka_node_bulk<<<h->grid, h->block, 0, st>>>(tn, psi_scr, L1, L0, b.lgf, s0, m0, b.adj, b.parts, k);
    if (int rc = acheck(h, "ka_node_bulk")) return rc;
    ACK(h, cudaStreamWaitEvent(st, h->join_ev, 0));
    // The psi adjoint at particle nodes (side stream), then the a_l of the
    // edge candidates, which read it and the wall ghosts' (side, after the
    // handle's stream has those); on the handle's stream the wall ghosts, the
    // a_l of the other fluid nodes (which read no psi adjoint) and, once the
    // particle nodes' partials are in, the particle-adjoint reduction.
    ACK(h, cudaEventRecord(h->fork_ev, st));
    ACK(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
    ka_lpsi<<<lpsi_blocks(k), kT, 0, h->side>>>(b.lgf, psi_scr, b.lpsi, s0, m0, b.adj, b.parts2, k);
    if (int rc = acheck(h, "ka_lpsi")) return rc;
    ACK(h, cudaEventRecord(b.ev_lpsi, h->side));
    ka_lpsi_shell<<<nbs, kT, 0, st>>>(b.lgf, b.lpsi, s0, m0, k);
    if (int rc = acheck(h, "ka_lpsi_shell")) return rc;
    ACK(h, cudaEventRecord(b.ev_shell, st));
    ACK(h, cudaStreamWaitEvent(h->side, b.ev_shell, 0));
    {
        const long long ne = adj_edge_entries(k);
        if (ne > 0) {
            ka_final_edge<<<(unsigned)((ne + kT - 1) / kT), kT, 0, h->side>>>(L0, b.lgf, b.lpsi, s0, m0, k);
            if (int rc = acheck(h, "ka_final_edge")) return rc;
        }
    }
    ACK(h, cudaEventRecord(h->join_ev, h->side));
    ka_final<<<h->grid, h->block, 0, st>>>(L0, b.lgf, b.lpsi, s0, m0, k);
    if (int rc = acheck(h, "ka_final")) return rc;
    ACK(h, cudaStreamWaitEvent(st, b.ev_lpsi, 0));
    ka_reduce<<<reduce_blocks(h->ntiles), kT, 0, st>>>(b.adj, b.parts, h->ntiles, b.parts2, lpsi_blocks(k), b.red);
    if (int rc = acheck(h, "ka_reduce")) return rc;
    ACK(h, cudaStreamWaitEvent(st, h->join_ev, 0));
    return FLBM_OK;
}

}  // namespace

extern "C" int flbm_adjoint_tape_limit(flbm_t* h, int64_t bytes)
{
    if (!h) return FLBM_E_INVAL;
    h->adj_tape_limit = bytes;
    return FLBM_OK;
}

extern "C" int flbm_adjoint_run(flbm_t* h, int64_t nsteps, int32_t checkpoint_every, flbm_adjoint_result* out)
{
    if (!h || !out || nsteps < 1 || checkpoint_every < 1) return sim_fail(h, FLBM_E_INVAL, "invalid argument");
    const KParams& k = h->kp;
    const flbm_params& p = h->p;
    if (!k.has_particle || p.kT != 0.0 || !k.tau1 || p.fluid_counterforce)
        return sim_fail(h, FLBM_E_UNSUPPORTED,
                        "the adjoint needs a particle, kT = 0, every relaxation time 1 and no counterforce");
    std::memset(out, 0, sizeof(*out));
    const int64_t T = nsteps;
    const int K = (int)std::min<int64_t>(checkpoint_every, T);
    const int64_t nck = (T + K - 1) / K;
    const size_t N = k.N, B3 = (size_t)k.B * k.B * k.B, mbytes = 2 * B3;
    const size_t fN = 2 * 19 * N;
    AdjBuffers b;
    // Whole tape (no recompute) where the tape of every step fits the limit.
    bool whole = false;
    if (h->adj_tape_limit != 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            fr = 0;
            cudaGetLastError();
        }
        const double need = (double)(T + 1) * (8.0 * sizeof(float) * (double)N + sizeof(DevState) + (double)mbytes);
        const double lim = h->adj_tape_limit > 0 ? (double)h->adj_tape_limit : 0.5 * (double)fr;
        whole = need <= lim && b.alloc_store((size_t)(T + 1), N, mbytes);
    }
    if ((!whole && (!b.alloc(b.ck_f, (size_t)(nck + 1) * fN) || !b.alloc(b.ck_st, (size_t)(nck + 1)) ||
                    !b.alloc(b.ck_m, (size_t)(nck + 1) * mbytes) ||
                    !b.alloc(b.ck_psi, (size_t)(nck + 1) * 2 * k.padn))) ||
        !b.alloc(b.tape, (size_t)(K + 1) * 8 * N) ||
        !b.alloc(b.tape_st, (size_t)(K + 1)) || !b.alloc(b.tape_m, (size_t)(K + 1) * mbytes) ||
        !b.alloc(b.lam[0], 8 * N) || !b.alloc(b.lam[1], 8 * N) || !b.alloc(b.lgf, 6 * N) ||
        !b.alloc(b.lpsi, (size_t)(2 * k.padn)) || !b.alloc(b.uv, 2 * B3) ||
        !b.alloc(b.parts, (size_t)h->ntiles * kNodeParts) || !b.alloc(b.parts2, (size_t)lpsi_blocks(h->kp)) ||
        !b.alloc(b.cparts, (size_t)h->box_blocks * 9) || !b.alloc(b.red, (size_t)kRedBlocks * kRedSums) || !b.alloc(b.adj, 1))
        return sim_fail(h, FLBM_E_NOMEM, "adjoint checkpoints and tape");
    if (!b.make_events()) return sim_fail(h, FLBM_E_CUDA, "adjoint events");
    // The step sequences are replayed as CUDA graphs, which the legacy default
    // stream cannot capture: on that stream the run takes a private stream,
    // ordered after the handle's stream on entry and before it on exit.
    struct StreamSwap {
        flbm_sim* h;
        cudaStream_t user = nullptr, priv = nullptr;
        ~StreamSwap()
        {
            if (!priv) return;
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, priv);
                cudaStreamWaitEvent(user, e, 0);
                cudaEventDestroy(e);
            } else {
                cudaStreamSynchronize(priv);
            }
            h->stream = user;
            cudaStreamDestroy(priv);
        }
    } swap{h};
    if (h->stream == nullptr) {
        cudaEvent_t e;
        ACK(h, cudaStreamCreateWithFlags(&swap.priv, cudaStreamNonBlocking));
        ACK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        const cudaError_t r1 = cudaEventRecord(e, h->stream);
        const cudaError_t r2 = cudaStreamWaitEvent(swap.priv, e, 0);
        cudaEventDestroy(e);
        ACK(h, r1);
        ACK(h, r2);
        swap.user = h->stream;
        h->stream = swap.priv;
    }
    cudaStream_t st = h->stream;
    ACK(h, cudaMemsetAsync(b.adj, 0, sizeof(AdjState), st));
    ACK(h, cudaMemsetAsync(b.lam[0], 0, sizeof(lam_t) * 8 * N, st));
    ACK(h, cudaMemsetAsync(b.lpsi, 0, sizeof(double) * 2 * k.padn, st));
    cudaEvent_t ev[3];
    for (auto& e : ev) ACK(h, cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard()
        {
            for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
        }
    } guard{ev};
    cudaEventRecord(ev[0], st);
    // Graphs need a stream that can be captured, and the two-pass step (whose
    // launches do not depend on host state).
    AdjGraphs ag;
    const bool graphs = st != nullptr && !sim_fused(h);
    auto acc_J = [&]() -> int {
        ka_accJ<<<1, 1, 0, st>>>(h->st, b.adj);
        return acheck(h, "ka_accJ");
    };
    auto fwd_step = [&]() -> int {
        if (int rc = sim_step(h)) return rc;
        return acc_J();
    };
    // Tape slot kk of a segment (moments, particle record, masks of the
    // current state), then, with step, a step. A two-pass step's density
    // pass writes the moments itself (sim_step_tape: one read of the
    // populations); otherwise ka_tape does.
    auto tape_step = [&](int kk, bool step) -> int {
        float* tp = b.tape + (size_t)kk * 8 * N;
        const bool fused_tape = step && !sim_fused(h);
        if (!fused_tape) {
            ka_tape<<<h->grid, h->block, 0, st>>>(h->fbuf[h->cur], tp, k);
            if (int rc = acheck(h, "ka_tape")) return rc;
        }
        ACK(h, cudaMemcpyAsync(b.tape_st + kk, h->st, sizeof(DevState), cudaMemcpyDeviceToDevice, st));
        ACK(h, cudaMemcpyAsync(b.tape_m + (size_t)kk * mbytes, h->masks, mbytes, cudaMemcpyDeviceToDevice, st));
        if (!step) return FLBM_OK;
        return fused_tape ? sim_step_tape(h, tp) : sim_step(h);
    };
    // Slots [0, n) of the segment's tape to (or from) the store's slots from step s0.
    auto store_copy = [&](int64_t s0, int n, bool to_store) -> int {
        float* t = b.all_tape + (size_t)s0 * 8 * N;
        DevState* ts = b.all_st + s0;
        uint8_t* tm = b.all_m + (size_t)s0 * mbytes;
        const size_t nt = sizeof(float) * 8 * N * (size_t)n, ns = sizeof(DevState) * (size_t)n;
        const size_t nm = mbytes * (size_t)n;
        const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
        ACK(h, cudaMemcpyAsync(to_store ? (void*)t : (void*)b.tape, to_store ? (void*)b.tape : (void*)t, nt, d2d, st));
        ACK(h, cudaMemcpyAsync(to_store ? (void*)ts : (void*)b.tape_st, to_store ? (void*)b.tape_st : (void*)ts, ns,
                               d2d, st));
        ACK(h, cudaMemcpyAsync(to_store ? (void*)tm : (void*)b.tape_m, to_store ? (void*)b.tape_m : (void*)tm, nm,
                               d2d, st));
        return FLBM_OK;
    };
    if (whole) {
        // Forward run writing the tape of every step, a segment at a time
        // (its slots staged in the segment's tape, whose graphs repeat), and
        // the sum of Vavg_z.
        for (int64_t c = 0; c < nck; ++c) {
            const int64_t s0 = c * K;
            const int Ls = (int)std::min<int64_t>(K, T - s0);
            for (int kk = 0; kk < Ls;) {
                if (graphs && kk % kAdjGraph == 0 && kk + kAdjGraph <= Ls) {
                    std::vector<cudaGraphExec_t>& v = ag.fwt[h->cur];
                    const size_t j = (size_t)(kk / kAdjGraph);
                    if (v.size() <= j) v.resize(j + 1, nullptr);
                    if (!v[j]) {
                        const int k0 = kk;
                        if (int rc = capture_graph(h, &v[j], [&]() -> int {
                                for (int i = 0; i < kAdjGraph; ++i) {
                                    if (int r = tape_step(k0 + i, true)) return r;
                                    if (int r = acc_J()) return r;
                                }
                                return FLBM_OK;
                            }))
                            return rc;
                    }
                    ACK(h, cudaGraphLaunch(v[j], st));
                    kk += kAdjGraph;
                } else {
                    if (int rc = tape_step(kk, true)) return rc;
                    if (int rc = acc_J()) return rc;
                    ++kk;
                }
            }
            if (int rc = store_copy(s0, Ls, true)) return rc;
        }
        if (int rc = tape_step(0, false)) return rc;  // the final state
        if (int rc = store_copy(T, 1, true)) return rc;
    }
    // Forward run: checkpoints every K steps, the sum of Vavg_z.
    for (int64_t s = 0; !whole && s < T;) {
        if (s % K == 0) {
            const int64_t c = s / K;
            if (int rc = save_state(h, b.ck_f + c * fN, b.ck_st + c, b.ck_m + c * mbytes, mbytes,
                                    b.ck_psi + c * 2 * k.padn))
                return rc;
        }
        const int64_t next = std::min<int64_t>(T, (s / K + 1) * K);  // the next checkpoint
        while (s < next) {
            if (graphs && next - s >= kAdjGraph) {
                cudaGraphExec_t& g = ag.fwd[h->cur];
                if (!g)
                    if (int rc = capture_graph(h, &g, [&]() -> int {
                            for (int i = 0; i < kAdjGraph; ++i)
                                if (int r = fwd_step()) return r;
                            return FLBM_OK;
                        }))
                        return rc;
                ACK(h, cudaGraphLaunch(g, st));
                s += kAdjGraph;
            } else {
                if (int rc = fwd_step()) return rc;
                ++s;
            }
        }
    }
    if (!whole)
        if (int rc = save_state(h, b.ck_f + nck * fN, b.ck_st + nck, b.ck_m + nck * mbytes, mbytes,
                                b.ck_psi + nck * 2 * k.padn))
            return rc;
    cudaEventRecord(ev[1], st);
    // Reverse sweep, segment by segment from the last.
    const double vol = 4.0 / 3.0 * M_PI * p.radius * p.radius * p.radius;
    const double dFp_dg = vol * (p.rho_p_ratio - 1.0) * (p.rho_a0 + p.rho_b0);
    const double inv2T = 0.5 / (double)T;
    int lcur = 0;  // b.lam[lcur] is the adjoint of the later state
    for (int64_t c = nck - 1; c >= 0; --c) {
        const int64_t s0 = c * K;
        const int Ls = (int)std::min<int64_t>(K, T - s0);
        // The segment's tape: from the store, or recomputed from its checkpoint.
        if (whole) {
            if (int rc = store_copy(s0, Ls + 1, false)) return rc;
        } else if (int rc = load_state(h, b.ck_f + c * fN, b.ck_st + c, b.ck_m + c * mbytes, mbytes,
                                       b.ck_psi + c * 2 * k.padn)) {
            return rc;
        }
        for (int kk = 0; !whole && kk <= Ls;) {
            if (graphs && kk % kAdjGraph == 0 && kk + kAdjGraph <= Ls) {
                std::vector<cudaGraphExec_t>& v = ag.rec[h->cur];
                const size_t j = (size_t)(kk / kAdjGraph);
                if (v.size() <= j) v.resize(j + 1, nullptr);
                if (!v[j]) {
                    const int k0 = kk;
                    if (int rc = capture_graph(h, &v[j], [&]() -> int {
                            for (int i = 0; i < kAdjGraph; ++i)
                                if (int r = tape_step(k0 + i, true)) return r;
                            return FLBM_OK;
                        }))
                        return rc;
                }
                ACK(h, cudaGraphLaunch(v[j], st));
                kk += kAdjGraph;
            } else {
                if (int rc = tape_step(kk, kk < Ls)) return rc;
                ++kk;
            }
        }
        // The reverse sweep of the segment; a full segment's as one graph,
        // which depends only on the parities of lcur and cur at its start.
        auto sweep = [&](int lc) -> int {
            for (int kk = Ls - 1; kk >= 0; --kk) {
                if (int rc = reverse_step(h, b, kk, b.lam[lc], b.lam[1 - lc], inv2T, dFp_dg)) return rc;
                lc = 1 - lc;
            }
            return FLBM_OK;
        };
        if (graphs && Ls == K) {
            cudaGraphExec_t& g = ag.rev[lcur][h->cur];
            if (!g)
                if (int rc = capture_graph(h, &g, [&]() { return sweep(lcur); })) return rc;
            ACK(h, cudaGraphLaunch(g, st));
        } else {
            if (int rc = sweep(lcur)) return rc;
        }
        if (Ls & 1) lcur = 1 - lcur;
    }
    if (!whole)
        if (int rc = load_state(h, b.ck_f + nck * fN, b.ck_st + nck, b.ck_m + nck * mbytes, mbytes,
                                b.ck_psi + nck * 2 * k.padn))
            return rc;
    cudaEventRecord(ev[2], st);
    AdjState a;
    ACK(h, cudaMemcpyAsync(&a, b.adj, sizeof(a), cudaMemcpyDeviceToHost, st));
    ACK(h, cudaStreamSynchronize(st));
    float f0 = 0.0f, f1 = 0.0f;
    cudaEventElapsedTime(&f0, ev[0], ev[1]);
    cudaEventElapsedTime(&f1, ev[1], ev[2]);
    out->J = a.J / (double)T;
    out->dJ_dg = a.grad[0];
    out->dJ_ddelta_rho = a.grad[1];
    out->dJ_dG = a.grad[2];
    out->steps = T;
    out->checkpoint_every = K;
    out->whole_tape = whole ? 1 : 0;
    out->device_bytes = (double)b.bytes;
    out->ms_forward = f0;
    out->ms_reverse = f1;
    return FLBM_OK;
}

// Node-level arithmetic of the noise-free collision with every relaxation
// time 1 (Section 2, Eq. (lbe) with Eq. (sc-force) as source), forward and
// transposed, as plain C++ that the CUDA kernels and a host test both compile.
//
// With tau = 1 every post-collision mode is a function of the component
// densities rho_l, momenta j_l and Shan-Chen sums g_l = sum_i w_i psi_lbar(x+c_i) c_i:
//   F_l   = -G rho_l g_l + (rho_l / rho_t) ext                       (force density)
//   u     = (j_A + j_B + (F_A + F_B) / 2) / rho_t                    (v^(H))
//   m*_0  = rho_l,   m*_{1..3} = rho_l u + F_l / 2
//   m*_4  = rho_l u.u + u.F_l          m*_5 = rho_l (3 ux^2 - u.u) + 3 ux Flx - u.F_l
//   m*_6  = rho_l (uy^2 - uz^2) + uy Fly - uz Flz
//   m*_7  = rho_l ux uy + (ux Fly + uy Flx)/2, and m*_8 (y,z), m*_9 (x,z) alike
//   ghost modes 10..18 = 0.
// adj_modes() is the transpose of the Jacobian of this map: given the adjoint
// of m*_{0..9} of both components it returns the adjoints of rho_l, j_l, g_l
// and the derivative with respect to G.
#pragma once

#ifdef __CUDACC__
#define FLBM_HD __host__ __device__ __forceinline__
#else
#define FLBM_HD inline
#endif

namespace flbm {

template <class T>
FLBM_HD void fwd_modes(const T rho[2], const T j[2][3], const T g[2][3], const T ext[3], T G, T ms[2][10])
{
    const T rt = rho[0] + rho[1];
    const T irt = T(1) / rt;
    T F[2][3], u[3];
    for (int l = 0; l < 2; ++l)
        for (int a = 0; a < 3; ++a) F[l][a] = -G * rho[l] * g[l][a] + rho[l] * irt * ext[a];
    for (int a = 0; a < 3; ++a) u[a] = (j[0][a] + j[1][a] + T(0.5) * (F[0][a] + F[1][a])) * irt;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int l = 0; l < 2; ++l) {
        const T r = rho[l];
        const T* Fl = F[l];
        const T uF = u[0] * Fl[0] + u[1] * Fl[1] + u[2] * Fl[2];
        ms[l][0] = r;
        for (int a = 0; a < 3; ++a) ms[l][1 + a] = r * u[a] + T(0.5) * Fl[a];
        ms[l][4] = r * uu + uF;
        ms[l][5] = r * (T(3) * u[0] * u[0] - uu) + T(3) * u[0] * Fl[0] - uF;
        ms[l][6] = r * (u[1] * u[1] - u[2] * u[2]) + u[1] * Fl[1] - u[2] * Fl[2];
        ms[l][7] = r * u[0] * u[1] + T(0.5) * (u[0] * Fl[1] + u[1] * Fl[0]);
        ms[l][8] = r * u[1] * u[2] + T(0.5) * (u[1] * Fl[2] + u[2] * Fl[1]);
        ms[l][9] = r * u[0] * u[2] + T(0.5) * (u[0] * Fl[2] + u[2] * Fl[0]);
    }
}

// lm: adjoint of m*_{0..9} per component. Outputs are overwritten.
template <class T>
FLBM_HD void adj_modes(const T rho[2], const T j[2][3], const T g[2][3], const T ext[3], T G, const T lm[2][10],
                       T lrho[2], T lj[2][3], T lg[2][3], T& lG)
{
    const T rt = rho[0] + rho[1];
    const T irt = T(1) / rt;
    T F[2][3], u[3];
    for (int l = 0; l < 2; ++l)
        for (int a = 0; a < 3; ++a) F[l][a] = -G * rho[l] * g[l][a] + rho[l] * irt * ext[a];
    for (int a = 0; a < 3; ++a) u[a] = (j[0][a] + j[1][a] + T(0.5) * (F[0][a] + F[1][a])) * irt;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // Modes -> (rho_l, u, F_l) with u and F_l held as independent inputs.
    T lu[3] = {T(0), T(0), T(0)};
    T lF[2][3];
    for (int l = 0; l < 2; ++l) {
        const T r = rho[l];
        const T* Fl = F[l];
        const T* L = lm[l];
        lrho[l] = L[0] + L[1] * u[0] + L[2] * u[1] + L[3] * u[2] + L[4] * uu + L[5] * (T(3) * u[0] * u[0] - uu) +
                  L[6] * (u[1] * u[1] - u[2] * u[2]) + L[7] * u[0] * u[1] + L[8] * u[1] * u[2] + L[9] * u[0] * u[2];
        lF[l][0] = T(0.5) * L[1] + u[0] * (L[4] + T(2) * L[5]) + T(0.5) * (L[7] * u[1] + L[9] * u[2]);
        lF[l][1] = T(0.5) * L[2] + u[1] * (L[4] - L[5] + L[6]) + T(0.5) * (L[7] * u[0] + L[8] * u[2]);
        lF[l][2] = T(0.5) * L[3] + u[2] * (L[4] - L[5] - L[6]) + T(0.5) * (L[8] * u[1] + L[9] * u[0]);
        lu[0] += r * L[1] + L[4] * (T(2) * r * u[0] + Fl[0]) + L[5] * (T(4) * r * u[0] + T(2) * Fl[0]) +
                 L[7] * (r * u[1] + T(0.5) * Fl[1]) + L[9] * (r * u[2] + T(0.5) * Fl[2]);
        lu[1] += r * L[2] + (L[4] - L[5] + L[6]) * (T(2) * r * u[1] + Fl[1]) + L[7] * (r * u[0] + T(0.5) * Fl[0]) +
                 L[8] * (r * u[2] + T(0.5) * Fl[2]);
        lu[2] += r * L[3] + (L[4] - L[5] - L[6]) * (T(2) * r * u[2] + Fl[2]) + L[8] * (r * u[1] + T(0.5) * Fl[1]) +
                 L[9] * (r * u[0] + T(0.5) * Fl[0]);
    }
    // u = (j_A + j_B + (F_A + F_B)/2) / rho_t
    T ul = T(0);
    for (int a = 0; a < 3; ++a) ul += lu[a] * u[a];
    for (int l = 0; l < 2; ++l) {
        lrho[l] -= ul * irt;
        for (int a = 0; a < 3; ++a) {
            lj[l][a] = lu[a] * irt;
            lF[l][a] += T(0.5) * lu[a] * irt;
        }
    }
    // F_l = -G rho_l g_l + (rho_l / rho_t) ext
    T eF[2];
    for (int l = 0; l < 2; ++l) eF[l] = lF[l][0] * ext[0] + lF[l][1] * ext[1] + lF[l][2] * ext[2];
    const T es = (rho[0] * eF[0] + rho[1] * eF[1]) * (irt * irt);
    lG = T(0);
    for (int l = 0; l < 2; ++l) {
        T gl = T(0);
        for (int a = 0; a < 3; ++a) {
            gl += g[l][a] * lF[l][a];
            lg[l][a] = -G * rho[l] * lF[l][a];
        }
        lrho[l] += -G * gl + eF[l] * irt - es;
        lG += -rho[l] * gl;
    }
}

// adj_modes for an adjoint whose only nonzero modes are m*_0 = a_l and
// m*_{1..3} = b_l (the part of lambda f_li = a_l + c_i . b_l that is the same
// at every neighbour): the same outputs, with far fewer operations.
template <class T>
FLBM_HD void adj_modes_ab(const T rho[2], const T j[2][3], const T g[2][3], const T ext[3], T G, const T a[2],
                          const T b[2][3], T lrho[2], T lj[2][3], T lg[2][3], T& lG)
{
    const T rt = rho[0] + rho[1];
    const T irt = T(1) / rt;
    T F[2][3], u[3];
    for (int l = 0; l < 2; ++l)
        for (int c = 0; c < 3; ++c) F[l][c] = -G * rho[l] * g[l][c] + rho[l] * irt * ext[c];
    for (int c = 0; c < 3; ++c) u[c] = (j[0][c] + j[1][c] + T(0.5) * (F[0][c] + F[1][c])) * irt;
    T lu[3] = {T(0), T(0), T(0)};
    T lF[2][3];
    for (int l = 0; l < 2; ++l) {
        lrho[l] = a[l] + b[l][0] * u[0] + b[l][1] * u[1] + b[l][2] * u[2];
        for (int c = 0; c < 3; ++c) {
            lF[l][c] = T(0.5) * b[l][c];
            lu[c] += rho[l] * b[l][c];
        }
    }
    const T ul = lu[0] * u[0] + lu[1] * u[1] + lu[2] * u[2];
    for (int l = 0; l < 2; ++l) {
        lrho[l] -= ul * irt;
        for (int c = 0; c < 3; ++c) {
            lj[l][c] = lu[c] * irt;
            lF[l][c] += T(0.5) * lu[c] * irt;
        }
    }
    T eF[2];
    for (int l = 0; l < 2; ++l) eF[l] = lF[l][0] * ext[0] + lF[l][1] * ext[1] + lF[l][2] * ext[2];
    const T es = (rho[0] * eF[0] + rho[1] * eF[1]) * (irt * irt);
    lG = T(0);
    for (int l = 0; l < 2; ++l) {
        T gl = T(0);
        for (int c = 0; c < 3; ++c) {
            gl += g[l][c] * lF[l][c];
            lg[l][c] = -G * rho[l] * lF[l][c];
        }
        lrho[l] += -G * gl + eF[l] * irt - es;
        lG += -rho[l] * gl;
    }
}

// adj_modes_ab with the forward quantities (rho, j, g, the external force
// and G) and the coefficients formed from them (1 / rho_tot, the forces F_l
// and the velocity u) in float, computed as the forward step computes them,
// and the adjoint values (a, b and every output) in A: the type of the large
// parts (flbm::df on the GPU; double for a reference with the same float
// coefficients). Every product is an adjoint value times a float.
template <class A>
FLBM_HD void adj_modes_ab_mixed(const float rho[2], const float j[2][3], const float g[2][3], const float ext[3],
                                float G, const A a[2], const A b[2][3], A lrho[2], A lj[2][3], A lg[2][3], A& lG)
{
    const float rt = rho[0] + rho[1];
    const float irt = 1.0f / rt;
    float F[2][3], u[3];
    for (int l = 0; l < 2; ++l)
        for (int c = 0; c < 3; ++c) F[l][c] = -G * rho[l] * g[l][c] + rho[l] * irt * ext[c];
    for (int c = 0; c < 3; ++c) u[c] = (j[0][c] + j[1][c] + 0.5f * (F[0][c] + F[1][c])) * irt;
    A lu[3] = {A(), A(), A()};
    A lF[2][3];
    for (int l = 0; l < 2; ++l) {
        lrho[l] = a[l] + b[l][0] * u[0] + b[l][1] * u[1] + b[l][2] * u[2];
        for (int c = 0; c < 3; ++c) {
            lF[l][c] = b[l][c] * 0.5f;
            lu[c] += b[l][c] * rho[l];
        }
    }
    const A ul = lu[0] * u[0] + lu[1] * u[1] + lu[2] * u[2];
    const float hirt = 0.5f * irt;
    for (int l = 0; l < 2; ++l) {
        lrho[l] -= ul * irt;
        for (int c = 0; c < 3; ++c) {
            lj[l][c] = lu[c] * irt;
            lF[l][c] += lu[c] * hirt;
        }
    }
    A eF[2];
    for (int l = 0; l < 2; ++l) eF[l] = lF[l][0] * ext[0] + lF[l][1] * ext[1] + lF[l][2] * ext[2];
    const A es = (eF[0] * rho[0] + eF[1] * rho[1]) * (irt * irt);
    lG = A();
    for (int l = 0; l < 2; ++l) {
        const A gl = lF[l][0] * g[l][0] + lF[l][1] * g[l][1] + lF[l][2] * g[l][2];
        const float cg = -G * rho[l];
        for (int c = 0; c < 3; ++c) lg[l][c] = lF[l][c] * cg;
        lrho[l] += gl * (-G) + eF[l] * irt - es;
        lG += gl * (-rho[l]);
    }
}

}  // namespace flbm

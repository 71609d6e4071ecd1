/*
 * FP64 CPU oracle: one time step of the fluctuating lattice Boltzmann method
 * (FLBM) for a two-component Shan-Chen mixture coupled to a wetted finite-size
 * sphere, following X. Xue, L. Biferale, M. Sbragaglia, F. Toschi,
 * "A lattice Boltzmann study of particle settling in a fluctuating
 * multicomponent fluid under confinement" (arXiv:1909.01092), Section 2
 * (Methodology): Eq. (density), Eq. (lbe), Eq. (sc-force), and Section 3
 * (Numerical set-up): Eq. (fp).
 *
 * TEST INFRASTRUCTURE. This file is the correctness reference for the GPU
 * library. Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it. It shares no code, header, table or constant
 * with the CUDA path: lattice tables, the mode basis and the Philox generator
 * are written out here independently.
 *
 * It is deliberately plain: dense 19x19 mode transforms, one node at a time,
 * the steps of the method in the order the paper states them. Readings of the
 * paper where it is silent are marked [R] and listed in the design notes.
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, printed values of the paper and
 * published known-answer vectors; exceptions are marked "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Parameters (the oracle's own struct; the GPU library has its own).  */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t lx, ly, lz;          /* lattice nodes per axis */
    int64_t wall[3];             /* 1: halfway bounce-back walls on that axis, 0: periodic */
    double tau_s, tau_d, tau_g;  /* relaxation times: stress modes, component momentum, ghost modes */
    double G;                    /* Shan-Chen coupling, Eq. (sc-force) */
    double rho0[2];              /* initial densities of A and B */
    double init_pert;            /* relative amplitude of the uniform initial perturbation */
    double kT;                   /* thermal energy (0: noise-free) */
    double radius;               /* sphere radius (<= 0: no particle) */
    double rho_p_ratio;          /* particle density / (rho0[0]+rho0[1]) */
    double g;                    /* body-force density along z driving the particle, Eq. (fp) */
    double delta_rho;            /* wetting parameter of the virtual layer */
    double fluid_force[3];       /* constant body-force density on the fluid */
    int64_t fluid_counterforce;  /* 1: add -F_p/N_fluid along z on the fluid */
    double pos0[3];              /* initial particle centre */
    uint64_t seed;
    int64_t replica;
} oracle_params;

/* ------------------------------------------------------------------ */
/* D3Q19 lattice (Section 2: "we employ the D3Q19 model").             */
/* Direction order [R]: rest, +-x, +-y, +-z, then the xy, xz, yz       */
/* diagonals in opposite pairs.                                        */
/* ------------------------------------------------------------------ */
static const int CV[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double WT[19];      /* lattice weights */
static int OPP[19];        /* index of -c_i */
static double EM[19][19];  /* EM[k][i] = e_k(c_i), the mode basis */
static double BN[19];      /* b_k = sum_i w_i e_k(c_i)^2 */
static int lattice_ready = 0;

/* Mode polynomials of the D3Q19 MRT basis (Dunweg, Schiller, Ladd 2007,
 * cited in Section 2 for the MRT scheme): density, momentum, 6 stress modes,
 * 9 ghost modes. */
static double mode_poly(int k, double x, double y, double z)
{
    double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

static void lattice_init(void)
{
    if (lattice_ready) return;
    for (int i = 0; i < 19; ++i) {
        int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
        WT[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < 19; ++j)
            if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) OPP[i] = j;
    }
    for (int k = 0; k < 19; ++k) {
        BN[k] = 0.0;
        for (int i = 0; i < 19; ++i) {
            EM[k][i] = mode_poly(k, CV[i][0], CV[i][1], CV[i][2]);
            BN[k] += WT[i] * EM[k][i] * EM[k][i];
        }
    }
    lattice_ready = 1;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its  */
/* published definition: 10 rounds of two 32x32->64 multiplications    */
/* with a Weyl-sequence key schedule.                                  */
/* ------------------------------------------------------------------ */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 32-bit integer -> uniform in (0,1): the top 23 bits plus one half, times
 * 2^-23. Every value is exact in binary32 and binary64, so both sides of the
 * parity test see the same uniforms. [R] */
static double uniform_open(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

static void philox_key(const oracle_params* p, uint32_t key[2])
{
    key[0] = (uint32_t)(p->seed & 0xffffffffu);
    key[1] = (uint32_t)(p->seed >> 32) ^ (uint32_t)p->replica;
}

/* The 36 standard normals of one (step, node): 9 Philox blocks with counter
 * (step, node, block, 0), each block giving two Box-Muller pairs. [R] */
static void node_normals(const oracle_params* p, uint32_t step, uint32_t node, double r[36])
{
    uint32_t key[2];
    philox_key(p, key);
    for (uint32_t blk = 0; blk < 9; ++blk) {
        uint32_t ctr[4] = {step, node, blk, 0u}, o[4];
        philox4x32_10(ctr, key, o);
        for (int h = 0; h < 2; ++h) {
            double u1 = uniform_open(o[2 * h]);
            double u2 = uniform_open(o[2 * h + 1]);
            double rad = sqrt(-2.0 * log(u1));
            r[4 * blk + 2 * h + 0] = rad * cos(2.0 * M_PI * u2);
            r[4 * blk + 2 * h + 1] = rad * sin(2.0 * M_PI * u2);
        }
    }
}

/* ------------------------------------------------------------------ */
/* State                                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    oracle_params p;
    int64_t N;
    double* f;      /* [2][19][N] post-stream populations at the current time */
    double* fn;     /* [2][19][N] next time */
    double* fs;     /* [2][19][N] post-collision populations */
    double* rho;    /* [2][N] densities of fluid nodes */
    double* psi;    /* [2][N] pseudo-potential: rho on fluid, virtual layer on particle nodes */
    double* force;  /* [2][3][N] force density on each component */
    unsigned char* solid;   /* [N] inside the particle at the current position */
    unsigned char* solid2;  /* [N] scratch: inside at the new position */
    unsigned char* unc;     /* [N] scratch: uncovered this step */
    double X[3], V[3], Om[3], Vavg[3];
    double Fh[3], Th[3];          /* hydrodynamic force and torque of the last step */
    double Ppend[3], Lpend[3];    /* cover/uncover impulse carried into the next step */
    double ledger[2];             /* mass removed from component l by the particle this step */
    double delta[2];              /* per-node mass correction applied in the next collision */
    int64_t nfluid;
    int64_t step;
    double mp, Ip, Fp;
} oracle;

static inline int64_t nidx(const oracle* o, int64_t x, int64_t y, int64_t z)
{
    return x + o->p.lx * (y + o->p.ly * z);
}

/* Neighbour of (x,y,z) along c_i. Returns 1 if it lies beyond a wall (a
 * ghost node), 0 otherwise; periodic axes wrap. Ghost coordinates are left
 * unwrapped in g[]. */
static int neighbour(const oracle* o, int64_t x, int64_t y, int64_t z, int i, int64_t g[3])
{
    const int64_t L[3] = {o->p.lx, o->p.ly, o->p.lz};
    int64_t q[3] = {x + CV[i][0], y + CV[i][1], z + CV[i][2]};
    int ghost = 0;
    for (int a = 0; a < 3; ++a) {
        if (q[a] < 0 || q[a] >= L[a]) {
            if (o->p.wall[a]) ghost = 1;
            else q[a] = (q[a] + L[a]) % L[a];
        }
    }
    g[0] = q[0]; g[1] = q[1]; g[2] = q[2];
    return ghost;
}

/* Same as neighbour() but starting from an arbitrary (possibly ghost) point. */
static int neighbour_of_point(const oracle* o, const int64_t s[3], int i, int64_t g[3])
{
    const int64_t L[3] = {o->p.lx, o->p.ly, o->p.lz};
    int64_t q[3] = {s[0] + CV[i][0], s[1] + CV[i][1], s[2] + CV[i][2]};
    int ghost = 0;
    for (int a = 0; a < 3; ++a) {
        if (q[a] < 0 || q[a] >= L[a]) {
            if (o->p.wall[a]) ghost = 1;
            else q[a] = ((q[a] % L[a]) + L[a]) % L[a];
        }
    }
    g[0] = q[0]; g[1] = q[1]; g[2] = q[2];
    return ghost;
}

/* Vector from the particle centre to point r, minimum image on periodic axes. */
static void rel_to_centre(const oracle* o, const double X[3], const double r[3], double d[3])
{
    const double L[3] = {(double)o->p.lx, (double)o->p.ly, (double)o->p.lz};
    for (int a = 0; a < 3; ++a) {
        d[a] = r[a] - X[a];
        if (!o->p.wall[a]) d[a] -= L[a] * floor(d[a] / L[a] + 0.5);
    }
}

/* Particle nodes: lattice nodes whose centre lies strictly inside the sphere
 * (Section 2: "declaring the fluid nodes belonging to the particle"). [R] */
static int inside_sphere(const oracle* o, const double X[3], int64_t x, int64_t y, int64_t z)
{
    if (o->p.radius <= 0.0) return 0;
    double r[3] = {(double)x, (double)y, (double)z}, d[3];
    rel_to_centre(o, X, r, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < o->p.radius * o->p.radius;
}

static void mark_solid(const oracle* o, const double X[3], unsigned char* mask)
{
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) mask[nidx(o, x, y, z)] = (unsigned char)inside_sphere(o, X, x, y, z);
}

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Second-order equilibrium w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2). */
static double feq(int i, double rho, const double u[3])
{
    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return WT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

#define F_AT(arr, l, i, n) (arr)[((int64_t)(l) * 19 + (i)) * o->N + (n)]

static void count_fluid(oracle* o)
{
    int64_t c = 0;
    for (int64_t n = 0; n < o->N; ++n) c += !o->solid[n];
    o->nfluid = c;
}

oracle* oracle_create(const oracle_params* p)
{
    lattice_init();
    oracle* o = (oracle*)calloc(1, sizeof(oracle));
    if (!o) return NULL;
    o->p = *p;
    o->N = p->lx * p->ly * p->lz;
    size_t nf = (size_t)2 * 19 * o->N;
    o->f = (double*)calloc(nf, sizeof(double));
    o->fn = (double*)calloc(nf, sizeof(double));
    o->fs = (double*)calloc(nf, sizeof(double));
    o->rho = (double*)calloc(2 * o->N, sizeof(double));
    o->psi = (double*)calloc(2 * o->N, sizeof(double));
    o->force = (double*)calloc(6 * o->N, sizeof(double));
    o->solid = (unsigned char*)calloc(o->N, 1);
    o->solid2 = (unsigned char*)calloc(o->N, 1);
    o->unc = (unsigned char*)calloc(o->N, 1);
    if (!o->f || !o->fn || !o->fs || !o->rho || !o->psi || !o->force || !o->solid || !o->solid2 || !o->unc) {
        free(o->f); free(o->fn); free(o->fs); free(o->rho); free(o->psi); free(o->force);
        free(o->solid); free(o->solid2); free(o->unc); free(o);
        return NULL;
    }
    /* Initial state: f = w_i rho_l0 (1 + a (2u - 1)), one uniform per (node, component),
     * Philox counter (0, node, 0, 1). [R] */
    uint32_t key[2];
    philox_key(p, key);
    for (int64_t n = 0; n < o->N; ++n) {
        uint32_t ctr[4] = {0u, (uint32_t)n, 0u, 1u}, r[4];
        philox4x32_10(ctr, key, r);
        for (int l = 0; l < 2; ++l) {
            double rl = p->rho0[l] * (1.0 + p->init_pert * (2.0 * uniform_open(r[l]) - 1.0));
            for (int i = 0; i < 19; ++i) F_AT(o->f, l, i, n) = WT[i] * rl;
        }
    }
    /* Particle: starts at rest at pos0. Mass and driving force, Eq. (fp):
     * F_p = (4/3) pi R^3 (rho_p - rho_tot) g, m_p = (4/3) pi R^3 rho_p. [R: nominal volume] */
    for (int a = 0; a < 3; ++a) o->X[a] = p->pos0[a];
    if (p->radius > 0.0) {
        double vol = 4.0 / 3.0 * M_PI * p->radius * p->radius * p->radius;
        double rho_tot = p->rho0[0] + p->rho0[1];
        double rho_p = p->rho_p_ratio * rho_tot;
        o->mp = vol * rho_p;
        o->Ip = 0.4 * o->mp * p->radius * p->radius;
        o->Fp = vol * (rho_p - rho_tot) * p->g;
    }
    mark_solid(o, o->X, o->solid);
    count_fluid(o);
    return o;
}

void oracle_destroy(oracle* o)
{
    if (!o) return;
    free(o->f); free(o->fn); free(o->fs); free(o->rho); free(o->psi); free(o->force);
    free(o->solid); free(o->solid2); free(o->unc);
    free(o);
}

/* Mean of rho_l over the fluid neighbours of point s (a particle node or a
 * wall ghost). Returns the number of fluid neighbours. */
static int fluid_neighbour_mean(const oracle* o, const int64_t s[3], const unsigned char* solid,
                                const double* rho, double mean[2])
{
    int cnt = 0;
    mean[0] = mean[1] = 0.0;
    for (int j = 1; j < 19; ++j) {
        int64_t q[3];
        if (neighbour_of_point(o, s, j, q)) continue;
        int64_t m = nidx(o, q[0], q[1], q[2]);
        if (solid[m]) continue;
        mean[0] += rho[m];
        mean[1] += rho[o->N + m];
        ++cnt;
    }
    if (cnt) { mean[0] /= cnt; mean[1] /= cnt; }
    return cnt;
}

/* Pseudo-potential seen by a fluid node along direction i. psi = rho on
 * fluid nodes; on particle nodes the virtual layer (Section 2: neighbour
 * average plus a wetting shift, +delta_rho for A and -delta_rho for B [R]);
 * on wall ghosts the same average with no shift (neutral walls, Section 3). */
static double psi_neighbour(const oracle* o, int l, int64_t x, int64_t y, int64_t z, int i)
{
    int64_t q[3];
    if (neighbour(o, x, y, z, i, q)) {
        double mean[2];
        fluid_neighbour_mean(o, q, o->solid, o->rho, mean);
        return mean[l];
    }
    return o->psi[l * o->N + nidx(o, q[0], q[1], q[2])];
}

/* Densities (Eq. density), virtual layer, and the force density on each
 * component: Shan-Chen, Eq. (sc-force), with omega_i the D3Q19 weights [R],
 * plus the constant fluid body force split in proportion to rho_l. Also
 * returns the Shan-Chen reaction on the particle (force and torque). */
static void densities_and_forces(oracle* o, double Fsc[3], double Tsc[3])
{
    const int64_t N = o->N;
    for (int64_t n = 0; n < N; ++n) {
        for (int l = 0; l < 2; ++l) {
            double s = 0.0;
            if (!o->solid[n])
                for (int i = 0; i < 19; ++i) s += F_AT(o->f, l, i, n);
            o->rho[l * N + n] = s;
        }
    }
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                if (!o->solid[n]) {
                    o->psi[n] = o->rho[n];
                    o->psi[N + n] = o->rho[N + n];
                } else {
                    int64_t s[3] = {x, y, z};
                    double mean[2];
                    if (fluid_neighbour_mean(o, s, o->solid, o->rho, mean)) {
                        double a = mean[0] + o->p.delta_rho, b = mean[1] - o->p.delta_rho;
                        o->psi[n] = a > 0.0 ? a : 0.0;
                        o->psi[N + n] = b > 0.0 ? b : 0.0;
                    } else {
                        o->psi[n] = o->psi[N + n] = 0.0;
                    }
                }
            }
    double fc = 0.0;
    if (o->p.fluid_counterforce && o->p.radius > 0.0 && o->nfluid > 0) fc = -o->Fp / (double)o->nfluid;
    for (int a = 0; a < 3; ++a) { Fsc[a] = 0.0; Tsc[a] = 0.0; }
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                for (int l = 0; l < 2; ++l)
                    for (int a = 0; a < 3; ++a) o->force[(l * 3 + a) * N + n] = 0.0;
                if (o->solid[n]) continue;
                double rt = o->rho[n] + o->rho[N + n];
                for (int l = 0; l < 2; ++l) {
                    int lo = 1 - l;
                    double acc[3] = {0.0, 0.0, 0.0};
                    for (int i = 1; i < 19; ++i) {
                        double ps = psi_neighbour(o, lo, x, y, z, i);
                        for (int a = 0; a < 3; ++a) acc[a] += WT[i] * ps * CV[i][a];
                    }
                    double frac = rt > 0.0 ? o->rho[l * N + n] / rt : 0.0;
                    double ext[3] = {o->p.fluid_force[0], o->p.fluid_force[1], o->p.fluid_force[2] + fc};
                    for (int a = 0; a < 3; ++a)
                        o->force[(l * 3 + a) * N + n] = -o->p.G * o->psi[l * N + n] * acc[a] + frac * ext[a];
                }
                /* Reaction on the particle of the pair forces between this
                 * fluid node and neighbouring particle nodes. */
                for (int i = 1; i < 19; ++i) {
                    int64_t q[3];
                    if (neighbour(o, x, y, z, i, q)) continue;
                    int64_t m = nidx(o, q[0], q[1], q[2]);
                    if (!o->solid[m]) continue;
                    double mag = o->p.G * WT[i] *
                                 (o->psi[n] * o->psi[N + m] + o->psi[N + n] * o->psi[m]);
                    double fr[3] = {mag * CV[i][0], mag * CV[i][1], mag * CV[i][2]};
                    double r[3] = {x + 0.5 * CV[i][0], y + 0.5 * CV[i][1], z + 0.5 * CV[i][2]}, d[3], t[3];
                    rel_to_centre(o, o->X, r, d);
                    cross(d, fr, t);
                    for (int a = 0; a < 3; ++a) { Fsc[a] += fr[a]; Tsc[a] += t[a]; }
                }
            }
}

/* MRT collision of Eq. (lbe) at one fluid node, both components, with the
 * Shan-Chen/body force as source term and thermal noise on the
 * non-conserved modes (Section 2). Writes post-collision populations. */
static void collide_node(oracle* o, int64_t n)
{
    const int64_t N = o->N;
    const double gs = 1.0 - 1.0 / o->p.tau_s;
    const double gd = 1.0 - 1.0 / o->p.tau_d;
    const double gg = 1.0 - 1.0 / o->p.tau_g;
    double m[2][19], rho[2], F[2][3];
    for (int l = 0; l < 2; ++l) {
        for (int k = 0; k < 19; ++k) {
            double s = 0.0;
            for (int i = 0; i < 19; ++i) s += EM[k][i] * F_AT(o->f, l, i, n);
            m[l][k] = s;
        }
        rho[l] = m[l][0];
        for (int a = 0; a < 3; ++a) F[l][a] = o->force[(l * 3 + a) * N + n];
    }
    /* Common velocity: the hydrodynamical velocity v^(H) = v + (F_A+F_B)/(2 rho_tot). */
    double rt = rho[0] + rho[1], u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[0][1 + a] + m[1][1 + a] + 0.5 * (F[0][a] + F[1][a])) / rt;

    double r[36] = {0};
    if (o->p.kT > 0.0) node_normals(&o->p, (uint32_t)o->step, (uint32_t)n, r);

    double ms[2][19];
    for (int l = 0; l < 2; ++l) {
        const double* Fl = F[l];
        double rl = rho[l];
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double uF = u[0] * Fl[0] + u[1] * Fl[1] + u[2] * Fl[2];
        double meq[19] = {0}, S[19] = {0};
        meq[4] = rl * uu;
        meq[5] = rl * (3.0 * u[0] * u[0] - uu);
        meq[6] = rl * (u[1] * u[1] - u[2] * u[2]);
        meq[7] = rl * u[0] * u[1];
        meq[8] = rl * u[1] * u[2];
        meq[9] = rl * u[0] * u[2];
        /* Second moment of the source u F + F u. */
        S[4] = 2.0 * uF;
        S[5] = 2.0 * (3.0 * u[0] * Fl[0] - uF);
        S[6] = 2.0 * (u[1] * Fl[1] - u[2] * Fl[2]);
        S[7] = u[0] * Fl[1] + u[1] * Fl[0];
        S[8] = u[1] * Fl[2] + u[2] * Fl[1];
        S[9] = u[0] * Fl[2] + u[2] * Fl[0];
        ms[l][0] = rl;
        for (int a = 0; a < 3; ++a)
            ms[l][1 + a] = rl * u[a] + gd * (m[l][1 + a] + 0.5 * Fl[a] - rl * u[a]) + 0.5 * Fl[a];
        for (int k = 4; k <= 9; ++k) ms[l][k] = meq[k] + gs * (m[l][k] - meq[k]) + 0.5 * (1.0 + gs) * S[k];
        for (int k = 10; k < 19; ++k) ms[l][k] = gg * m[l][k];
        if (o->p.kT > 0.0) {
            /* Fluctuation-dissipation: variance 3 kT rho_l b_k (1 - gamma_k^2). */
            double rp = rl > 0.0 ? rl : 0.0;
            for (int k = 4; k < 19; ++k) {
                double gk = (k <= 9) ? gs : gg;
                ms[l][k] += sqrt(3.0 * o->p.kT * rp * BN[k] * (1.0 - gk * gk)) * r[15 * l + (k - 4)];
            }
        }
    }
    if (o->p.kT > 0.0) {
        /* Interdiffusion noise: equal and opposite on the two components, so
         * that total momentum receives none. [R] */
        double ra = rho[0] > 0.0 ? rho[0] : 0.0, rb = rho[1] > 0.0 ? rho[1] : 0.0;
        double var = rt > 0.0 ? 3.0 * o->p.kT * (1.0 / 3.0) * (1.0 - gd * gd) * ra * rb / rt : 0.0;
        double amp = sqrt(var > 0.0 ? var : 0.0);
        for (int a = 0; a < 3; ++a) {
            ms[0][1 + a] += amp * r[30 + a];
            ms[1][1 + a] -= amp * r[30 + a];
        }
    }
    for (int l = 0; l < 2; ++l)
        for (int i = 0; i < 19; ++i) {
            double s = 0.0;
            for (int k = 0; k < 19; ++k) s += EM[k][i] * ms[l][k] / BN[k];
            F_AT(o->fs, l, i, n) = WT[i] * s + WT[i] * o->delta[l];
        }
}

/* Streaming of Eq. (lbe) with bounce-back: halfway at walls, and the moving
 * link rule at the particle (Ladd 1994, cited in Section 2) with momentum
 * exchange. Returns the exchanged force and torque; adds the mass removed by
 * the moving-wall term to the ledger. */
static void stream(oracle* o, double Fbb[3], double Tbb[3])
{
    const int64_t N = o->N;
    memcpy(o->fn, o->f, sizeof(double) * 2 * 19 * N);
    for (int a = 0; a < 3; ++a) { Fbb[a] = 0.0; Tbb[a] = 0.0; }
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                if (o->solid[n]) continue;
                for (int i = 0; i < 19; ++i) {
                    int64_t q[3];
                    int ghost = neighbour(o, x, y, z, i, q);
                    if (ghost) {
                        for (int l = 0; l < 2; ++l) F_AT(o->fn, l, OPP[i], n) = F_AT(o->fs, l, i, n);
                        continue;
                    }
                    int64_t m = nidx(o, q[0], q[1], q[2]);
                    if (!o->solid[m]) {
                        for (int l = 0; l < 2; ++l) F_AT(o->fn, l, i, m) = F_AT(o->fs, l, i, n);
                        continue;
                    }
                    /* Link to a particle node: boundary point halfway along the link. */
                    double r[3] = {x + 0.5 * CV[i][0], y + 0.5 * CV[i][1], z + 0.5 * CV[i][2]}, d[3], w[3];
                    rel_to_centre(o, o->X, r, d);
                    cross(o->Om, d, w);
                    double ub[3] = {o->V[0] + w[0], o->V[1] + w[1], o->V[2] + w[2]};
                    double ubc = ub[0] * CV[i][0] + ub[1] * CV[i][1] + ub[2] * CV[i][2];
                    double dp = 0.0;
                    for (int l = 0; l < 2; ++l) {
                        double corr = 6.0 * WT[i] * o->rho[l * N + n] * ubc;
                        double out = F_AT(o->fs, l, i, n);
                        double back = out - corr;
                        F_AT(o->fn, l, OPP[i], n) = back;
                        dp += out + back;
                        o->ledger[l] += corr;
                    }
                    double fr[3] = {dp * CV[i][0], dp * CV[i][1], dp * CV[i][2]}, t[3];
                    cross(d, fr, t);
                    for (int a = 0; a < 3; ++a) { Fbb[a] += fr[a]; Tbb[a] += t[a]; }
                }
            }
}

/* Cover/uncover after the particle moved from Xold to o->X (Section 2,
 * following Aidun et al. 1998 and Jansen & Harting 2011), and the mass
 * ledger of the mass-correction algorithm. */
static void cover_uncover(oracle* o, const double Xold[3])
{
    const int64_t N = o->N;
    mark_solid(o, o->X, o->solid2);
    for (int64_t n = 0; n < N; ++n) o->unc[n] = (unsigned char)(o->solid[n] && !o->solid2[n]);
    /* Covered nodes: their momentum goes to the particle, their mass to the ledger. */
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                if (o->solid[n] || !o->solid2[n]) continue;
                double j[3] = {0, 0, 0};
                for (int l = 0; l < 2; ++l) {
                    double rl = 0.0;
                    for (int i = 0; i < 19; ++i) {
                        double fv = F_AT(o->fn, l, i, n);
                        rl += fv;
                        for (int a = 0; a < 3; ++a) j[a] += fv * CV[i][a];
                    }
                    o->ledger[l] += rl;
                }
                double r[3] = {(double)x, (double)y, (double)z}, d[3], t[3];
                rel_to_centre(o, o->X, r, d);
                cross(d, j, t);
                for (int a = 0; a < 3; ++a) { o->Ppend[a] += j[a]; o->Lpend[a] += t[a]; }
            }
    /* Uncovered nodes: equilibrium at the neighbour-mean densities and the
     * local surface velocity; the particle pays the momentum. [R]
     * Section 2 defers this rule to Jansen and Harting (2011). Pinned by a
     * sphere moving with a uniform flow through uncover events (the refill
     * must reproduce the flow exactly, with arbitrary values inside the
     * sphere), by exact mass and momentum closure and by the square
     * channel's symmetries. The rotational part of the surface velocity is
     * pinned only through the moving link rule, which uses the same formula. */
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                if (!o->unc[n]) continue;
                double mean[2] = {0, 0};
                int cnt = 0;
                for (int j = 1; j < 19; ++j) {
                    int64_t q[3];
                    if (neighbour(o, x, y, z, j, q)) continue;
                    int64_t m = nidx(o, q[0], q[1], q[2]);
                    if (o->solid2[m] || o->unc[m]) continue;
                    for (int l = 0; l < 2; ++l) {
                        double rl = 0.0;
                        for (int i = 0; i < 19; ++i) rl += F_AT(o->fn, l, i, m);
                        mean[l] += rl;
                    }
                    ++cnt;
                }
                for (int l = 0; l < 2; ++l) mean[l] = cnt ? mean[l] / cnt : o->p.rho0[l];
                double r[3] = {(double)x, (double)y, (double)z}, d[3], w[3], t[3];
                rel_to_centre(o, o->X, r, d);
                cross(o->Om, d, w);
                double ub[3] = {o->V[0] + w[0], o->V[1] + w[1], o->V[2] + w[2]};
                double pm[3] = {0, 0, 0};
                for (int l = 0; l < 2; ++l) {
                    for (int i = 0; i < 19; ++i) F_AT(o->fn, l, i, n) = feq(i, mean[l], ub);
                    for (int a = 0; a < 3; ++a) pm[a] += mean[l] * ub[a];
                    o->ledger[l] -= mean[l];
                }
                cross(d, pm, t);
                for (int a = 0; a < 3; ++a) { o->Ppend[a] -= pm[a]; o->Lpend[a] -= t[a]; }
            }
    (void)Xold;
    unsigned char* tmp = o->solid;
    o->solid = o->solid2;
    o->solid2 = tmp;
    count_fluid(o);
}

static void step_once(oracle* o)
{
    const int64_t N = o->N;
    double Fsc[3], Tsc[3], Fbb[3], Tbb[3];
    densities_and_forces(o, Fsc, Tsc);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n)
        if (!o->solid[n]) collide_node(o, n);
    o->ledger[0] = o->ledger[1] = 0.0;
    stream(o, Fbb, Tbb);
    if (o->p.radius > 0.0) {
        /* Newton-Euler with leap-frog (Section 2); the boundary velocity used
         * in this step was V_{n-1/2}. */
        double Xold[3] = {o->X[0], o->X[1], o->X[2]};
        const double L[3] = {(double)o->p.lx, (double)o->p.ly, (double)o->p.lz};
        for (int a = 0; a < 3; ++a) {
            o->Fh[a] = Fbb[a] + Fsc[a] + o->Ppend[a];
            o->Th[a] = Tbb[a] + Tsc[a] + o->Lpend[a];
            o->Ppend[a] = o->Lpend[a] = 0.0;
        }
        for (int a = 0; a < 3; ++a) {
            double ext = (a == 2) ? o->Fp : 0.0;
            double vn = o->V[a] + (o->Fh[a] + ext) / o->mp;
            o->Vavg[a] = 0.5 * (o->V[a] + vn);
            o->V[a] = vn;
            o->Om[a] += o->Th[a] / o->Ip;
            o->X[a] += vn;
            if (!o->p.wall[a]) o->X[a] -= L[a] * floor(o->X[a] / L[a]);
        }
        cover_uncover(o, Xold);
        o->delta[0] = o->ledger[0] / (double)o->nfluid;
        o->delta[1] = o->ledger[1] / (double)o->nfluid;
    } else {
        o->delta[0] = o->delta[1] = 0.0;
    }
    double* t = o->f;
    o->f = o->fn;
    o->fn = t;
    o->step += 1;
}

/* ------------------------------------------------------------------ */
/* Exported interface (ctypes)                                          */
/* ------------------------------------------------------------------ */
void oracle_step(oracle* o, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) step_once(o);
}

int64_t oracle_num_nodes(const oracle* o) { return o->N; }

/* Populations in [component][direction][z][y][x] order. */
void oracle_get_f(const oracle* o, double* out) { memcpy(out, o->f, sizeof(double) * 2 * 19 * o->N); }
void oracle_set_f(oracle* o, const double* in) { memcpy(o->f, in, sizeof(double) * 2 * 19 * o->N); }

/* Particle record: X[3] V[3] Vavg[3] Omega[3] F[3] T[3] Ppend[3] Lpend[3]
 * delta[2] nfluid step mp Fp (32 doubles). V is V_{n+1/2} after a step. */
void oracle_get_particle(const oracle* o, double* out)
{
    int k = 0;
    for (int a = 0; a < 3; ++a) out[k++] = o->X[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->V[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Vavg[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Om[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Fh[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Th[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Ppend[a];
    for (int a = 0; a < 3; ++a) out[k++] = o->Lpend[a];
    out[k++] = o->delta[0];
    out[k++] = o->delta[1];
    out[k++] = (double)o->nfluid;
    out[k++] = (double)o->step;
    out[k++] = o->mp;
    out[k++] = o->Fp;
}

/* Set position, velocity (V_{n-1/2}) and angular velocity; re-marks the particle nodes. */
void oracle_set_particle(oracle* o, const double* X, const double* V, const double* Om)
{
    for (int a = 0; a < 3; ++a) { o->X[a] = X[a]; o->V[a] = V[a]; o->Om[a] = Om[a]; }
    mark_solid(o, o->X, o->solid);
    count_fluid(o);
}

/* Densities, pseudo-potential and force density of the current state,
 * without stepping: rho[2][N], psi[2][N], force[2][3][N], solid[N] (as doubles),
 * and the Shan-Chen reaction on the particle fsc[6] = (force, torque). */
void oracle_fields(oracle* o, double* rho, double* psi, double* force, double* solid, double* fsc)
{
    double F[3], T[3];
    densities_and_forces(o, F, T);
    if (rho) memcpy(rho, o->rho, sizeof(double) * 2 * o->N);
    if (psi) memcpy(psi, o->psi, sizeof(double) * 2 * o->N);
    if (force) memcpy(force, o->force, sizeof(double) * 6 * o->N);
    if (solid)
        for (int64_t n = 0; n < o->N; ++n) solid[n] = o->solid[n];
    if (fsc) {
        for (int a = 0; a < 3; ++a) { fsc[a] = F[a]; fsc[3 + a] = T[a]; }
    }
}

/* Observables of the current state: mass[2], fluid momentum[3], kinetic
 * energy sum |j|^2/(2 rho), particle momentum m_p V[3], pending mass
 * correction delta_l * N_fluid [2], nfluid (11 doubles). */
void oracle_observables(const oracle* o, double* out)
{
    double mass[2] = {0, 0}, mom[3] = {0, 0, 0}, ke = 0.0;
    for (int64_t n = 0; n < o->N; ++n) {
        if (o->solid[n]) continue;
        double rt = 0.0, j[3] = {0, 0, 0};
        for (int l = 0; l < 2; ++l)
            for (int i = 0; i < 19; ++i) {
                double fv = o->f[((int64_t)l * 19 + i) * o->N + n];
                mass[l] += fv;
                rt += fv;
                for (int a = 0; a < 3; ++a) j[a] += fv * CV[i][a];
            }
        for (int a = 0; a < 3; ++a) mom[a] += j[a];
        if (rt > 0.0) ke += (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / (2.0 * rt);
    }
    out[0] = mass[0]; out[1] = mass[1];
    out[2] = mom[0]; out[3] = mom[1]; out[4] = mom[2];
    out[5] = ke;
    for (int a = 0; a < 3; ++a) out[6 + a] = o->mp * o->V[a];
    out[9] = o->delta[0] * (double)o->nfluid;
    out[10] = o->delta[1] * (double)o->nfluid;
}

/* Temperatures of the fluctuating modes (Section 2: thermal noise on the
 * non-conserved modes, in compliance with the fluctuation-dissipation
 * relation; none on mass and total momentum). Sums over the bulk fluid nodes,
 * the fluid nodes with no particle node among their 18 neighbours. With the
 * modes m_lk = sum_i e_k(c_i) f_li of each component, u = (j_A + j_B)/rho_tot
 * and m_lk^eq = sum_i e_k(c_i) f_eq,i(rho_l, u):
 *   out[19 l + k] = sum (m_lk - m_lk^eq)^2 / (3 b_k sum rho_l), k = 4..18 (0 for k < 4)
 *   out[38 + a]   = sum d_a^2 / sum (rho_A rho_B / rho_tot), d = (rho_B j_A - rho_A j_B)/rho_tot
 *   out[41 + a]   = sum j_a^2 / sum rho_tot, j = j_A + j_B
 *   out[44]       = number of bulk fluid nodes.
 * In a thermalised ideal mixture each temperature equals kT. */
void oracle_mode_temps(const oracle* o, double* out)
{
    double s2[2][19], sr[2] = {0, 0}, sd[3] = {0, 0, 0}, sdr = 0.0, sj[3] = {0, 0, 0};
    int64_t cnt = 0;
    memset(s2, 0, sizeof(s2));
    for (int64_t z = 0; z < o->p.lz; ++z)
        for (int64_t y = 0; y < o->p.ly; ++y)
            for (int64_t x = 0; x < o->p.lx; ++x) {
                int64_t n = nidx(o, x, y, z);
                if (o->solid[n]) continue;
                int next_to_particle = 0;
                for (int i = 1; i < 19; ++i) {
                    int64_t q[3];
                    if (!neighbour(o, x, y, z, i, q) && o->solid[nidx(o, q[0], q[1], q[2])]) next_to_particle = 1;
                }
                if (next_to_particle) continue;
                double m[2][19];
                for (int l = 0; l < 2; ++l)
                    for (int k = 0; k < 19; ++k) {
                        m[l][k] = 0.0;
                        for (int i = 0; i < 19; ++i) m[l][k] += EM[k][i] * F_AT(o->f, l, i, n);
                    }
                double rt = m[0][0] + m[1][0];
                double j[3] = {m[0][1] + m[1][1], m[0][2] + m[1][2], m[0][3] + m[1][3]};
                double u[3] = {j[0] / rt, j[1] / rt, j[2] / rt};
                for (int l = 0; l < 2; ++l) {
                    for (int k = 4; k < 19; ++k) {
                        double meq = 0.0;
                        for (int i = 0; i < 19; ++i) meq += EM[k][i] * feq(i, m[l][0], u);
                        s2[l][k] += (m[l][k] - meq) * (m[l][k] - meq);
                    }
                    sr[l] += m[l][0];
                }
                for (int a = 0; a < 3; ++a) {
                    double d = (m[1][0] * m[0][1 + a] - m[0][0] * m[1][1 + a]) / rt;
                    sd[a] += d * d;
                    sj[a] += j[a] * j[a];
                }
                sdr += m[0][0] * m[1][0] / rt;
                ++cnt;
            }
    for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 19; ++k) out[19 * l + k] = (k >= 4 && sr[l] > 0.0) ? s2[l][k] / (3.0 * BN[k] * sr[l]) : 0.0;
    for (int a = 0; a < 3; ++a) {
        out[38 + a] = sdr > 0.0 ? sd[a] / sdr : 0.0;
        out[41 + a] = (sr[0] + sr[1]) > 0.0 ? sj[a] / (sr[0] + sr[1]) : 0.0;
    }
    out[44] = (double)cnt;
}

/* Lattice tables for the tests: c[19][3], w[19], opp[19], e[19][19] (mode
 * k, direction i), b[19]. */
void oracle_lattice(double* c, double* w, int64_t* opp, double* e, double* b)
{
    lattice_init();
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = WT[i];
        opp[i] = OPP[i];
        b[i] = BN[i];
        for (int k = 0; k < 19; ++k) e[19 * k + i] = EM[k][i];
    }
}

void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

void oracle_normals(uint64_t seed, int64_t replica, uint32_t step, uint32_t node, double* out)
{
    oracle_params p;
    memset(&p, 0, sizeof(p));
    p.seed = seed;
    p.replica = replica;
    node_normals(&p, step, node, out);
}

double oracle_uniform(uint32_t x) { return uniform_open(x); }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the OpenMP loops of later calls (n >= 1; ignored without OpenMP). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * flbm.h - C ABI of the GB300 (sm_103a) library for one time step of the
 * fluctuating lattice Boltzmann method (FLBM) for a two-component Shan-Chen
 * mixture coupled to a wetted finite-size spherical particle.
 *
 * Method: X. Xue, L. Biferale, M. Sbragaglia, F. Toschi, "A lattice Boltzmann
 * study of particle settling in a fluctuating multicomponent fluid under
 * confinement", arXiv:1909.01092.
 *   - Section 2, Eq. (density): component densities and mixture momentum.
 *   - Section 2, Eq. (lbe): collision (MRT), source term, thermal noise, streaming.
 *   - Section 2, Eq. (sc-force): Shan-Chen inter-component force.
 *   - Section 2, particle paragraph: particle nodes, moving bounce-back with
 *     momentum exchange, leap-frog Newton-Euler update, cover/uncover, mass
 *     correction, virtual fluid layer for wettability.
 *   - Section 3, Eq. (fp): driving force on the particle; square channel walls.
 *
 * Conventions for every function:
 *   - Return 0 (FLBM_OK) on success, a negative FLBM_E_* code on failure;
 *     flbm_error_string() names the code and flbm_last_error() gives the
 *     message of the handle's last failure.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 *   - All device work is issued on the handle's stream (the one passed to
 *     flbm_create; NULL means the legacy default stream). Functions that
 *     return data to host memory synchronise that stream before returning.
 *   - Host pointers are plain host memory (pageable or pinned); pinned memory
 *     makes flbm_run_host's copies faster. Device pointers are CUDA global
 *     memory on the current device.
 *
 * Population layout (host and device): float32 f[l][i][z][y][x], l = 0 (A),
 * 1 (B); D3Q19 direction i in the order
 *   0:(0,0,0)  1:(+1,0,0)  2:(-1,0,0)  3:(0,+1,0)  4:(0,-1,0)  5:(0,0,+1)  6:(0,0,-1)
 *   7:(+1,+1,0) 8:(-1,-1,0) 9:(+1,-1,0) 10:(-1,+1,0)
 *   11:(+1,0,+1) 12:(-1,0,-1) 13:(+1,0,-1) 14:(-1,0,+1)
 *   15:(0,+1,+1) 16:(0,-1,-1) 17:(0,+1,-1) 18:(0,-1,+1)
 * The stored state is the post-streaming (pre-collision) population of the
 * current time. Values at particle nodes are not part of the state.
 */
#ifndef FLBM_H
#define FLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FLBM_OK = 0,
    FLBM_E_INVAL = -1,       /* invalid argument or parameter set */
    FLBM_E_NOMEM = -2,       /* device or host allocation failed */
    FLBM_E_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    FLBM_E_NONFINITE = -4,   /* a NaN/Inf was found in the state */
    FLBM_E_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    FLBM_E_UNSUPPORTED = -6  /* valid request this build does not implement */
};

/* Parameters of one simulation; host memory, copied by flbm_create. */
typedef struct flbm_params {
    int32_t lx, ly, lz;             /* lattice nodes per axis, each >= 1 */
    int32_t wall_x, wall_y, wall_z; /* 1: halfway bounce-back walls at -1/2 and L-1/2; 0: periodic */
    double tau_s;                   /* relaxation time of the stress modes (viscosity nu = (tau_s-1/2)/3) */
    double tau_d;                   /* relaxation time of the component momenta (diffusivity D = (tau_d-1/2)/3) */
    double tau_g;                   /* relaxation time of the ghost modes */
    double G;                       /* Shan-Chen coupling of Eq. (sc-force), psi = rho */
    double rho_a0, rho_b0;          /* initial densities of components A and B */
    double init_pert;               /* relative amplitude of the uniform random initial density perturbation */
    double kT;                      /* thermal energy; 0 switches the noise off */
    double radius;                  /* sphere radius in lattice units; <= 0: no particle */
    double rho_p_ratio;             /* particle density / (rho_a0 + rho_b0) */
    double g;                       /* body-force density along z of Eq. (fp): F_p = 4/3 pi R^3 (rho_p - rho_tot) g */
    double delta_rho;               /* wetting shift of the virtual layer: +delta_rho on A, -delta_rho on B */
    double fluid_force[3];          /* constant body-force density on the fluid, split over A/B by rho_l/rho_tot */
    int32_t fluid_counterforce;     /* 1: also apply -F_p/N_fluid along z on the fluid (zero net external force) */
    uint32_t replica;               /* replica index, folded into the Philox key */
    uint64_t seed;                  /* Philox key */
    double pos0[3];                 /* initial particle centre (lattice coordinates, node centres at integers) */
} flbm_params;

/* Particle record (host memory, filled by the library). */
typedef struct flbm_particle {
    double X[3];          /* centre after the last step */
    double V[3];          /* velocity V_{n+1/2} of the last leap-frog update */
    double Vavg[3];       /* (V_{n-1/2} + V_{n+1/2}) / 2: the velocity reported for step n */
    double Omega[3];      /* angular velocity Omega_{n+1/2} */
    double F[3];          /* hydrodynamic force of the last step (exchange + Shan-Chen reaction + cover/uncover) */
    double T[3];          /* hydrodynamic torque of the last step */
    double P_pending[3];  /* cover/uncover impulse carried into the next step */
    double L_pending[3];  /* cover/uncover angular impulse carried into the next step */
    double delta[2];      /* per-node mass correction of A and B applied in the next collision */
    double mp;            /* particle mass 4/3 pi R^3 rho_p */
    double Fp;            /* driving force of Eq. (fp) */
    int64_t nfluid;       /* number of fluid nodes */
    int64_t step;         /* completed steps */
} flbm_particle;

/* Observables of the current state (host memory, filled by the library).
 *
 * The "temperatures" below check the fluctuation-dissipation requirement of
 * Section 2 (thermal noise on the non-conserved modes, none on mass and total
 * momentum). They are reduced over the bulk fluid nodes: fluid nodes with no
 * particle node among their 18 neighbours. With m_lk = sum_i e_k(c_i) f_li the
 * modes of component l (the basis of Section 2's MRT collision, in the order
 * 1, c, c^2-1, 3c_x^2-c^2, c_y^2-c_z^2, c_xc_y, c_yc_z, c_xc_z, (3c^2-5)c,
 * (c_y^2-c_z^2)c_x and cyclic, 3c^4-6c^2+1, (2c^2-3)(3c_x^2-c^2),
 * (2c^2-3)(c_y^2-c_z^2)), b_k their norms sum_i w_i e_k(c_i)^2, and
 * n_lk = m_lk - m_lk^eq(rho_l, u) with u = (j_A + j_B)/rho_tot:
 *   mode_temp[l][k] = sum n_lk^2 / (3 b_k sum rho_l), k = 4..18;
 *   diff_temp[a]    = sum d_a^2 / sum (rho_A rho_B / rho_tot),
 *                     d = (rho_B j_A - rho_A j_B)/rho_tot (interdiffusion current);
 *   mom_temp[a]     = sum j_a^2 / sum rho_tot, j = j_A + j_B.
 * In a thermalised ideal mixture (G = 0) every one of them equals kT. */
typedef struct flbm_obs {
    double mass[2];              /* sum over fluid nodes of rho_A, rho_B */
    double momentum[3];          /* sum over fluid nodes of sum_l sum_i f_li c_i */
    double kinetic;              /* sum over fluid nodes of |j|^2 / (2 rho_tot) */
    double particle_momentum[3]; /* m_p V */
    double pending_mass[2];      /* delta_l * N_fluid, still to be added by the next collision */
    int64_t nfluid;
    int64_t step;
    int64_t nonfinite;           /* number of non-finite populations on fluid nodes */
    double mode_temp[2][19];     /* per component and mode, as above; entries k = 0..3 are 0 */
    double diff_temp[3];         /* interdiffusion current per axis, as above */
    double mom_temp[3];          /* total momentum per axis, as above */
    int64_t n_bulk;              /* bulk fluid nodes the temperatures are reduced over */
} flbm_obs;

typedef struct flbm_sim flbm_t;

/* Device bytes of the population storage (two float32 copies of
 * 2 x 19 x lx*ly*lz values) for these parameters; 0 if they are invalid. */
size_t flbm_state_bytes(const flbm_params* p);

/* Create a simulation on the current CUDA device.
 *   p        : parameters (validated; FLBM_E_INVAL if out of range).
 *   f_dev    : NULL, or device memory of at least flbm_state_bytes(p) bytes,
 *              256-byte aligned, that the library borrows for the populations
 *              (the caller keeps it alive until flbm_destroy). NULL: the
 *              library allocates it.
 *   f_dev_bytes : size of f_dev in bytes (ignored when f_dev is NULL).
 *   stream   : cudaStream_t to issue all work on (NULL: default stream).
 *   out      : receives the handle.
 * Initial state (Section 2 set-up): f_li = w_i rho_l0 (1 + a (2u-1)) with one
 * Philox uniform u per (node, component); the particle at pos0, at rest.
 * Errors: FLBM_E_INVAL, FLBM_E_NOMEM, FLBM_E_CUDA. */
int flbm_create(const flbm_params* p, void* f_dev, size_t f_dev_bytes, void* stream, flbm_t** out);

/* Advance nsteps >= 0 time steps (Eq. (lbe) with all of Section 2's particle
 * coupling). Asynchronous on the handle's stream. Within a step the
 * near-particle collide runs on a second, higher-priority stream that the
 * handle owns, forked from and joined back to the handle's stream by events,
 * so every step is complete in the handle's stream order. Errors:
 * FLBM_E_INVAL, FLBM_E_CUDA (launch failure). */
int flbm_step(flbm_t* h, int64_t nsteps);

/* Copy the particle record (the sphere of Section 2, advanced by Newton's
 * equation with leap-frog; F_p of Eq. (fp)) to host memory `out`;
 * synchronises the stream. Errors: FLBM_E_INVAL (NULL argument), FLBM_E_CUDA,
 * FLBM_E_TIMEOUT if a bounded device-side wait of an earlier step gave up. */
int flbm_particle_state(flbm_t* h, flbm_particle* out);

/* Reduce the observables of the current state (FP64) into `out`: the
 * component masses and the total momentum of Eq. (density) over the fluid
 * nodes, the kinetic energy, the particle's momentum, the pending mass
 * correction and the mode, interdiffusion and momentum temperatures of the
 * fluctuating modes (Section 2; definitions at flbm_obs); synchronises the
 * stream. Errors: FLBM_E_INVAL (NULL argument),
 * FLBM_E_CUDA, FLBM_E_NONFINITE if any fluid population is not finite (out
 * is still filled), FLBM_E_TIMEOUT as flbm_particle_state. */
int flbm_observables(flbm_t* h, flbm_obs* out);

/* Copy the current populations to host_f (2*19*N float32, layout above) and,
 * if host_rho is not NULL, the densities used by the Shan-Chen force of the
 * next step (2*N float32: rho on fluid nodes, virtual-layer values on surface
 * particle nodes, 0 elsewhere). Either pointer may be NULL. Synchronises.
 * Errors: FLBM_E_INVAL (NULL handle), FLBM_E_CUDA. */
int flbm_read_fields(flbm_t* h, float* host_f, float* host_rho);

/* Overwrite the current populations from host_f (2*19*N float32, host
 * memory, layout above). Errors: FLBM_E_INVAL (NULL argument), FLBM_E_CUDA. */
int flbm_write_fields(flbm_t* h, const float* host_f);

/* Set the particle centre, velocity (V_{n-1/2}) and angular velocity, and
 * re-mark the particle nodes. Pending impulses and mass corrections are
 * cleared. Errors: FLBM_E_INVAL (NULL argument, a non-finite value, or a
 * centre that puts the sphere outside the walls), FLBM_E_UNSUPPORTED if the simulation has no
 * particle, FLBM_E_CUDA. */
int flbm_set_particle(flbm_t* h, const double X[3], const double V[3], const double Omega[3]);

/* End-to-end call from host memory: copy host_f_in (2*19*N float32) to the
 * device, advance nsteps, write the particle record of every step to
 * traj[0..nsteps-1] (may be NULL), copy the final populations to host_f_out
 * (may be NULL). With flbm_use_graphs on, the steps replay captured graphs as
 * flbm_step does, each step followed by a small kernel that stores its record
 * on the device. Synchronises before returning. Errors: FLBM_E_INVAL (NULL
 * handle or input, nsteps < 0, or more than 2^31 - 1 steps with a
 * trajectory), FLBM_E_NOMEM (host or device staging of the trajectory),
 * FLBM_E_CUDA. */
int flbm_run_host(flbm_t* h, const float* host_f_in, int64_t nsteps, float* host_f_out, flbm_particle* traj);

/* Kernel classes of one step. Two-pass steps launch them in this order;
 * fused steps (flbm_set_density_mode) launch the collide first, then the
 * particle kernels, the completion of the densities and the shell. */
enum {
    FLBM_K_DENSITY = 0,  /* densities of fluid nodes (Eq. (density)): the density pass (two-pass), or
                            the completion of the densities the collide summed (fused) */
    FLBM_K_SHELL = 1,    /* periodic copies and neutral wall ghosts of the density field, and the
                            virtual wetting layer on particle surface nodes (one launch) */
    FLBM_K_COLLIDE = 2,  /* force, MRT collision, noise, streaming, bounce-back, exchange; with a
                            particle also its leap-frog update (last block of the near-particle launch) */
    FLBM_K_PARTICLE = 3, /* next-position particle nodes, cover/uncover, mass correction, step count */
    FLBM_NKERNELS = 4
};

/* Same as flbm_step, and measures the device time of each kernel class with
 * CUDA events recorded between the kernels on the handle's stream (no extra
 * synchronisation between steps). On return ms[FLBM_NKERNELS] (host memory,
 * caller-owned) holds the summed milliseconds of each class over the nsteps
 * steps. Synchronises the stream. Errors: FLBM_E_INVAL, FLBM_E_CUDA. */
int flbm_step_timed(flbm_t* h, int64_t nsteps, double* ms);

/* Static name of kernel class k ("" if out of range). */
const char* flbm_kernel_name(int k);

/* Number of kernel launches the last flbm_step / flbm_step_timed / flbm_run_host issued. */
int64_t flbm_last_launch_count(const flbm_t* h);

/* Write the whole simulation state to the file `path` (host path string):
 * the parameters, the FP64 particle record (position, velocities, pending
 * impulses, mass-correction ledger, step counter), the particle-node masks
 * and the current populations. Synchronises the stream. The paper has no
 * counterpart; this serves runs longer than one process (the paper's
 * production runs take 10^6 steps, Section 3).
 * Errors: FLBM_E_INVAL (NULL argument, file cannot be written), FLBM_E_CUDA. */
int flbm_checkpoint(flbm_t* h, const char* path);

/* Read a file written by flbm_checkpoint into h. The file's lattice sizes,
 * walls and particle radius must equal h's (they fix the state layout); the
 * other parameters (kT, G, forces, seed, ...) stay those h was created with,
 * so a state may be equilibrated under one set and continued under another.
 * With equal parameters, stepping after a restore gives the same populations
 * and particle record, bit for bit, as stepping on without the checkpoint.
 * Synchronises the stream. Errors: FLBM_E_INVAL (NULL, unreadable or
 * truncated file, wrong format, layout mismatch), FLBM_E_CUDA. */
int flbm_restore(flbm_t* h, const char* path);

/* CUDA-graph replay for flbm_step: with enable = 1, flbm_step replays a
 * captured graph of eight steps (captured on first use; a remainder of fewer
 * than eight steps runs as plain launches) instead of issuing each kernel,
 * which removes the per-launch host cost that dominates small lattices. Results are identical to plain launches. The handle's stream
 * must not be the legacy default stream (capture is not allowed there):
 * FLBM_E_UNSUPPORTED then. enable = 0 returns to plain launches.
 * Errors: FLBM_E_INVAL, FLBM_E_UNSUPPORTED, FLBM_E_CUDA (capture failed). */
int flbm_use_graphs(flbm_t* h, int enable);

/* Bulk collide-stream with its inputs staged by the Tensor Memory Accelerator
 * (same node update, Section 2, Eq. (lbe)): a persistent grid copies each
 * tile's 38 x 256 populations and its padded density stencil into shared
 * memory with tensor copies, double-buffered, while the previous tile is
 * computed. Available when the lattice allows it (lx % 4 == 0 and
 * lx >= 32); off by default, since the kernel that reads global memory
 * directly keeps twice as many warps resident and runs this issue-bound
 * update faster. Both give identical results. Captured step graphs are dropped on
 * a change (the stream is synchronised). A bounded wait in this kernel that
 * gives up makes flbm_particle_state and flbm_observables return
 * FLBM_E_TIMEOUT. Errors: FLBM_E_INVAL, FLBM_E_UNSUPPORTED (enable = 1 on a
 * lattice that does not allow it), FLBM_E_CUDA. */
int flbm_use_tma(flbm_t* h, int enable);

/* How each step forms the densities of Eq. (density) that the Shan-Chen force
 * of Eq. (sc-force) reads at the next step.
 *   mode 0 (two-pass): a density pass re-reads every population at the start
 *     of each step (152 B per node of extra HBM traffic);
 *   mode 1 (fused): the collide-stream
 *     sums the populations it pushes into each node as it writes them, and a
 *     small completion kernel adds the partial sums across tile and chunk
 *     boundaries and recomputes the densities next to the particle after
 *     cover/uncover. The densities are then carried from step to step (and
 *     saved by flbm_checkpoint).
 * The two modes compute the same sums in different orders: they agree to
 * float32 rounding, and each is bit-reproducible. Mode 0 is the default: on
 * GB300 the fused collide's exchange of pushed values between the threads of
 * a block (two barriers per plane, about 600 more instructions per node)
 * costs more than the density pass it removes. planes_per_block (fused
 * only) is how many consecutive z-planes one block of the fused collide walks;
 * 0 chooses about two waves of blocks for this GPU. The TMA-staged collide
 * (flbm_use_tma) always runs two-pass. Captured step graphs are dropped.
 * Errors: FLBM_E_INVAL (mode not 0 or 1, planes_per_block < 0 or > lz),
 * FLBM_E_UNSUPPORTED (mode 1 on a lattice whose tiles are narrower than 8
 * nodes, or with fewer than 3 tiles along a periodic x or y), FLBM_E_NOMEM,
 * FLBM_E_CUDA. */
int flbm_set_density_mode(flbm_t* h, int32_t mode, int32_t planes_per_block);

/* The density mode the next step takes (host memory, caller-owned outputs):
 * mode 1 with its planes per block, or mode 0 with 0. Errors: FLBM_E_INVAL. */
int flbm_get_density_mode(const flbm_t* h, int32_t* mode, int32_t* planes_per_block);

/* Limit, in SM clock cycles, of each wait of the TMA-staged collide for a
 * tile's tensor copies (cycles = 0 restores the default of 2^31, about a
 * second). A block whose wait runs out sets the handle's error flag, waits
 * with the default limit for its copies still in flight, and returns, so the
 * kernel ends without touching the rest of its tiles. The next
 * flbm_particle_state or flbm_observables then returns FLBM_E_TIMEOUT, and
 * the handle's state is no longer a step of the method: destroy it. This
 * exists to exercise the error path of the bounded waits: a limit near 0
 * makes them give up (the paper has no counterpart). Captured step graphs are
 * dropped on a change (the stream is synchronised).
 * Errors: FLBM_E_INVAL (cycles < 0), FLBM_E_CUDA. */
int flbm_set_tma_wait(flbm_t* h, int64_t cycles);

/* Observables of a population field, allocating nothing.
 *
 * For callers that cannot allocate device memory: code whose device memory is
 * owned by a pool or arena, host plugins that must not call cudaMalloc or
 * cudaFree (cudaFree synchronises the device), or code that must not grow the
 * process's device footprint after start-up. The paper has no counterpart:
 * this is an alternative entry to the observables reduction of
 * flbm_observables.
 *   p       : parameters of the field (sizes and walls are used); the
 *             simulation must have no particle (radius <= 0), else
 *             FLBM_E_UNSUPPORTED.
 *   f_dev   : device memory, 2*19*N float32 populations in the layout above.
 *   out_dev : device memory for 8 doubles, written in stream order:
 *             mass A, mass B, momentum x, y, z, kinetic energy, number of
 *             non-finite populations, 0.
 *   stream  : cudaStream_t (NULL: default stream). Asynchronous.
 * Scratch: a file-scope device array of FLBM_NOALLOC_MAX_TILES x 8 doubles
 * (2 MiB), held by every GPU that loads the library until the process exits.
 * A lattice that needs more tiles (more than 128x128x512 nodes or equivalent)
 * is rejected with FLBM_E_INVAL and a message on stderr. The first call on a
 * device looks up the array's device address with that device current, and
 * so does the first call from any other CUDA context (the address belongs to
 * the context: a primary context re-created after cudaDeviceReset, or a
 * context made current through the driver API, gets its own lookup); make
 * those first calls before any stream capture. All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. Every scratch slot a call reads is
 * written earlier in the same call, so no clearing is needed. */
#define FLBM_NOALLOC_MAX_TILES 32768
int flbm_observables_noalloc(const flbm_params* p, const float* f_dev, double* out_dev, void* stream);

/* Release the handle and the device memory the library allocated. */
void flbm_destroy(flbm_t* h);

/* Static name of an FLBM_E_* code. */
const char* flbm_error_string(int code);

/* Message of the handle's last failure ("" if none); valid until the next call. */
const char* flbm_last_error(const flbm_t* h);

/* ------------------------------------------------------------------------
 * Adjoint of the noise-free step.
 * ------------------------------------------------------------------------ */

/* Result of flbm_adjoint_run (host memory, filled by the library). */
typedef struct flbm_adjoint_result {
    double J;                /* (1/T) sum_{n<T} Vavg_z(n): time-averaged settling velocity */
    double dJ_dg;            /* dJ / d g (body-force density of Section 3, Eq. (fp)) */
    double dJ_ddelta_rho;    /* dJ / d delta_rho (wetting shift of the virtual layer, Section 2) */
    double dJ_dG;            /* dJ / d G (Shan-Chen coupling, Eq. (sc-force)) */
    int64_t steps;           /* T */
    int32_t checkpoint_every;/* K actually used (min(K, T)): segment length of the reverse sweep */
    int32_t whole_tape;      /* 1: the forward run kept the whole tape (no recompute); 0: checkpoints */
    double device_bytes;     /* device memory the call allocated (checkpoints or tape store, tape, adjoint fields) */
    double ms_forward;       /* device time of the forward run (with checkpoints or the tape) */
    double ms_reverse;       /* device time of the reverse sweep (with the segment recomputes, if any) */
} flbm_adjoint_result;

/* Run T = nsteps steps from h's current state and return J and its gradient
 * with respect to (g, delta_rho, G) by the discrete adjoint of the step. The
 * reverse sweep reads a tape of the moments rho_l, j_l of every step (8
 * floats per node), the particle records and the masks, segment by segment
 * of K = checkpoint_every steps. Where the tape of all T steps fits within
 * the limit that flbm_adjoint_tape_limit sets (by default half of the free
 * device memory), the forward run writes it and nothing is recomputed:
 * memory (T + 1) x (8 floats per node + masks). Otherwise the state is
 * checkpointed every K steps and each segment recomputed, with its tape,
 * before it is swept backwards: memory (T/K) x populations + K x 8 floats
 * per node. Both give the same J and gradient, bit for bit. The
 * adjoint holds the step's discrete sets fixed (particle nodes, links,
 * covered and uncovered nodes): J is differentiated along the forward
 * trajectory. On return h has advanced T steps, exactly as flbm_step(h, T)
 * would leave it. The paper computes no gradients; this differentiates its
 * noise-free method.
 * The repeated step sequences of the forward run and of the recomputes
 * are replayed as CUDA graphs (two-pass density mode); on a handle whose
 * stream is the legacy default stream, which graphs cannot capture, the
 * call runs on a private stream ordered after and before the handle's.
 * Requires a particle (radius > 0), kT = 0, every relaxation time 1 and
 * fluid_counterforce = 0: FLBM_E_UNSUPPORTED otherwise. Synchronises.
 * Errors: FLBM_E_INVAL, FLBM_E_UNSUPPORTED, FLBM_E_NOMEM, FLBM_E_CUDA. */
int flbm_adjoint_run(flbm_t* h, int64_t nsteps, int32_t checkpoint_every, flbm_adjoint_result* out);

/* Device bytes up to which flbm_adjoint_run keeps the tape of every step
 * instead of recomputing segments from checkpoints: bytes < 0 (the default)
 * half of the device memory free at the call, 0 never, > 0 that many bytes
 * (a store that then cannot be allocated falls back to checkpoints).
 * Errors: FLBM_E_INVAL (NULL handle). */
int flbm_adjoint_tape_limit(flbm_t* h, int64_t bytes);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent simulations (replicas) advanced
 * together. The paper's velocity statistics (Section 3) are averages over
 * noise realisations and channel geometries; an ensemble runs them as one
 * set of batched launches per step instead of one set per replica. Each
 * replica is exactly the simulation flbm_create would make from its
 * parameters (same initial state, same Philox stream, same step), so an
 * ensemble member and a single simulation agree bit for bit under tile
 * policy 0; other tile policies change only the FP64 summation order of the
 * particle force.
 * ------------------------------------------------------------------------ */
typedef struct flbm_ens flbm_ens_t;

/* Launch configuration of an ensemble (host memory). */
typedef struct flbm_ens_config {
    int32_t packing;     /* order of work items in each launch: 0 replica after replica,
                            1 interleaved (item k of every replica, then item k+1),
                            2 replica after replica, largest lattice first */
    int32_t ctas_per_sm; /* persistent blocks per SM of every batched launch (1..8);
                            0: one block per work item, and the bulk collide in
                            launches of up to 48 replicas of similar tile counts
                            whose descriptors are a kernel parameter */
    int32_t tile_policy; /* 0: tile width min(32, next power of two >= lx), as flbm_create;
                            1: the largest of 32, 16, 8 that divides lx (else as 0) */
} flbm_ens_config;

/* Create n >= 1 replicas on the current device from the parameter array
 * p[0..n-1] (host memory; each validated as by flbm_create). cfg NULL
 * selects {packing 0, ctas_per_sm 4, tile_policy 0}. The library owns all
 * device memory. With a stream other than the legacy default stream,
 * flbm_ensemble_step replays captured CUDA graphs of two steps.
 * Errors: FLBM_E_INVAL (a parameter set is invalid: the message names it),
 * FLBM_E_NOMEM, FLBM_E_CUDA. */
int flbm_ensemble_create(const flbm_params* p, int32_t n, const flbm_ens_config* cfg, void* stream,
                         flbm_ens_t** out);

/* Advance every replica by nsteps >= 0 steps (asynchronous on the stream).
 * Errors: FLBM_E_INVAL, FLBM_E_CUDA. */
int flbm_ensemble_step(flbm_ens_t* e, int64_t nsteps);

/* Autotuner: time `steps` >= 2 steps of every candidate configuration (the
 * three packings x ctas_per_sm in {0, 2, 4} x the two tile policies) with
 * CUDA events on the stream, keep the fastest, then put every replica back
 * to its initial state. best (may be NULL) receives the chosen
 * configuration and ms_best (may be NULL) its milliseconds per step.
 * Synchronises. Errors: FLBM_E_INVAL, FLBM_E_NOMEM, FLBM_E_CUDA. */
int flbm_ensemble_tune(flbm_ens_t* e, int32_t steps, flbm_ens_config* best, double* ms_best);

/* Current configuration (host memory, caller-owned out). */
int flbm_ensemble_config(const flbm_ens_t* e, flbm_ens_config* out);

/* Particle records of all replicas into out[0..n-1] (host memory; replicas
 * without a particle report their step and fluid count only). Synchronises. */
int flbm_ensemble_particles(flbm_ens_t* e, flbm_particle* out);

/* Populations of replica r (layout as flbm_read_fields) into host_f.
 * Synchronises. Errors: FLBM_E_INVAL (r out of range), FLBM_E_CUDA. */
int flbm_ensemble_read_fields(flbm_ens_t* e, int32_t r, float* host_f);

/* Observables of replica r, as flbm_observables. Synchronises. */
int flbm_ensemble_observables(flbm_ens_t* e, int32_t r, flbm_obs* out);

/* Total lattice nodes over all replicas (the unit of ensemble MLUPS). */
int64_t flbm_ensemble_nodes(const flbm_ens_t* e);

/* Kernel launches issued by the last flbm_ensemble_step (graph replays
 * count the kernels inside the graph). */
int64_t flbm_ensemble_last_launch_count(const flbm_ens_t* e);

/* Message of the ensemble's last failure ("" if none). */
const char* flbm_ensemble_last_error(const flbm_ens_t* e);

/* Free everything the ensemble owns; synchronises its stream. */
void flbm_ensemble_destroy(flbm_ens_t* e);

#ifdef __cplusplus
}
#endif

#endif /* FLBM_H */

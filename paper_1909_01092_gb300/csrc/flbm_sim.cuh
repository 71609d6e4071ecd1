// The simulation handle behind flbm_t and the step launcher, shared by the
// translation units of the library (single simulation and adjoint).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "flbm_fused.cuh"
#include "flbm_host.cuh"

using flbm::DevState;
using flbm::KParams;

struct flbm_sim {
    flbm_params p;
    KParams kp;
    cudaStream_t stream = nullptr;
    float* fbuf[2] = {nullptr, nullptr};
    void* f_owned = nullptr;
    int cur = 0;  // fbuf[cur] holds the current state
    // Padded density fields: psibuf[c] holds the densities of the state in
    // fbuf[c] (Shan-Chen pseudo-potential with its shell and virtual layer).
    // psi_valid: psibuf[cur] is up to date with fbuf[cur]; the fused step keeps
    // it so (it writes psibuf[1 - cur] as it streams), the two-pass step
    // recomputes it at the start of every step.
    float* psibuf[2] = {nullptr, nullptr};
    bool psi_valid = false;
    // Density mode: 0 two-pass (density pass every step), 1 fused (densities
    // as a by-product of the collide); fused only where fused_ok allows it.
    int density_mode = 0;
    bool fused_allowed = false;
    flbm::FusedGeom fg{};
    float2* ring = nullptr;        // ring partials: tiles x lz x fg.ring
    float2* seam = nullptr;        // seam partials: tiles x nchunk x 2 x fg.fp
    size_t seam_cap = 0;           // float2 slots allocated for seam
    DevState* st = nullptr;
    uint8_t* masks = nullptr;
    double* partials = nullptr;    // per candidate near tile: force, torque, ledger
    int* box_counts = nullptr;      // per block of the particle box: particle nodes
    double* box_parts = nullptr;    // per block of the particle box: cover/uncover sums
    int box_blocks = 0;
    long long ncand = 0;
    double* obs_tiles = nullptr;
    double* obs_out = nullptr;
    double* obs_mode_tiles = nullptr;  // per tile: kObsModes sums of k_obs_modes
    double* obs_mode_out = nullptr;
    float* scratch_rho = nullptr;
    DevState* traj_dev = nullptr;  // per-step particle records of flbm_run_host
    size_t traj_cap = 0;
    int* traj_count = nullptr;     // records written so far in this call (k_record)
    DevState* traj_host = nullptr;
    size_t traj_host_cap = 0;
    std::vector<cudaEvent_t> events;  // pool for flbm_step_timed
    bool use_graphs = false;
    // Captured steps starting from cur = 0 / 1; graph_rec also records each
    // step's particle state into traj_dev (flbm_run_host with a trajectory).
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_rec[2] = {nullptr, nullptr};
    int64_t graph_launches[2] = {0, 0};      // kernels in each graph
    int64_t graph_rec_launches[2] = {0, 0};
    dim3 grid, block;
    // Bulk collide with TMA-staged inputs (k_collide_bulk_tma): tensor maps of
    // the two population copies and of the padded densities; tma_ok when the
    // lattice allows it, tma when it is in use; persistent grid size.
    CUtensorMap tm_f[2];
    CUtensorMap tm_psi[2];
    bool tma_ok = false;
    bool tma = false;
    int tma_grid = 0;
    long long tma_wait = 0;  // limit of its waits for a tile's inputs, SM cycles (set at creation)
    // The near-particle collide runs on a second, higher-priority stream,
    // concurrently with the bulk collide (they write disjoint populations);
    // fork and join by events.
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    long long ntiles = 0;
    int64_t launches = 0;
    int64_t adj_tape_limit = -1;  // flbm_adjoint_tape_limit: < 0 automatic, 0 never, > 0 bytes
    float* tape_out = nullptr;    // set by sim_step_tape: the step's density pass also writes this tape
    std::string err;
};

namespace flbm {

// Densities of the current state.
inline float* psi_cur(flbm_sim* h) { return h->psibuf[h->cur]; }

// Launch one time step on h's stream (h->cur flips). With ev, events
// ev[0..5] are recorded between its kernel classes.
int sim_step(flbm_sim* h, cudaEvent_t* ev = nullptr);

// One two-pass step whose density pass also writes the adjoint's moment
// tape of the current state (8 fields of N floats) to tape.
int sim_step_tape(flbm_sim* h, float* tape);

// Record an error message on h and return code.
int sim_fail(flbm_sim* h, int code, const std::string& msg);

// Make psibuf[cur] hold the current state's densities (a density pass if
// they are stale).
int sim_ensure_psi(flbm_sim* h);

// Does the next step take the fused path (densities carried from step to step)?
bool sim_fused(const flbm_sim* h);

}  // namespace flbm

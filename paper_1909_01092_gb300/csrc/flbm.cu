// C-ABI of the FLBM step library (declared in include/flbm.h): handle
// management, validation, launch sequence of one time step (on the handle's
// stream and its second stream), and the host copies. All compute runs in the
// kernels of flbm_kernels.cuh, flbm_step.cuh and flbm_tma.cuh.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "flbm.h"
#include "flbm_sim.cuh"
#include "flbm_tma.cuh"

using namespace flbm;

namespace {

int fail(flbm_sim* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(flbm_sim* h, cudaError_t e, const char* what)
{
    return fail(h, FLBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                             \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

void fill_kparams(flbm_sim* h)
{
    KParams& k = h->kp;
    make_kparams(h->p, 0, k);
    h->block = dim3(k.tx, k.ty, 1);
    h->grid = dim3(k.gx, k.gy, k.lz);
    h->ntiles = tile_count(k);
    h->ncand = cand_count(k);
    h->box_blocks = box_block_count(k);
}

int launch_check(flbm_sim* h, const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    h->launches += 1;
    return FLBM_OK;
}

void record(flbm_sim* h, cudaEvent_t* ev, int k)
{
    if (ev) cudaEventRecord(ev[k], h->stream);
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor maps and launch shape of k_collide_bulk_tma. The populations of one
// copy are a 4-D float tensor (lx, ly, lz, 38) and the padded densities one of
// (px, py, pz, 2); both need rows of a multiple of 16 bytes (lx % 4 == 0,
// px is rounded up) and the 32 x 8 tile. Otherwise, or if the driver refuses
// a map, the kernel is unavailable. It is off by default: holding two stages
// of 256 nodes in shared memory leaves room for two blocks (16 warps) per
// SM, and the direct kernel with 32 resident warps runs the issue-bound
// update faster.
void setup_tma(flbm_sim* h)
{
    const KParams& k = h->kp;
    h->tma_ok = h->tma = false;
    h->tma_wait = kTmaWaitCycles;
    if (k.lx % 4 != 0 || k.tx != kTmaTX || k.ty != kTmaTY || k.px % 4 != 0) return;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return;
    const cuuint32_t one[4] = {1, 1, 1, 1};
    for (int c = 0; c < 2; ++c) {
        const cuuint64_t dims[4] = {(cuuint64_t)k.lx, (cuuint64_t)k.ly, (cuuint64_t)k.lz, 38};
        const cuuint64_t strides[3] = {(cuuint64_t)k.lx * 4, (cuuint64_t)k.lx * k.ly * 4, (cuuint64_t)k.N * 4};
        const cuuint32_t box[4] = {kTmaTX, kTmaTY, 1, 38};
        if (enc(&h->tm_f[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->fbuf[c], dims, strides, box, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    }
    for (int c = 0; c < 2; ++c) {
        const cuuint64_t dims[4] = {(cuuint64_t)k.px, (cuuint64_t)k.py, (cuuint64_t)k.pz, 2};
        const cuuint64_t strides[3] = {(cuuint64_t)k.px * 4, (cuuint64_t)k.px * k.py * 4, (cuuint64_t)k.padn * 4};
        const cuuint32_t box[4] = {kTmaPX, kTmaPY, 3, 2};
        if (enc(&h->tm_psi[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->psibuf[c], dims, strides, box, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return;
    void (*kern[4])(const CUtensorMap, const CUtensorMap, float*, DevState*, KParams, long long) = {
        k_collide_bulk_tma<false, false>, k_collide_bulk_tma<false, true>, k_collide_bulk_tma<true, false>,
        k_collide_bulk_tma<true, true>};
    for (auto* f : kern)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemBytes) != cudaSuccess)
            return;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[3], kThreadsStep, kTmaSmemBytes) !=
            cudaSuccess ||
        per_sm < 1)
        return;
    h->tma_grid = (int)std::min<long long>(h->ntiles, (long long)sms * per_sm);
    h->tma_ok = true;  // available; flbm_use_tma switches it on
}

// Densities, then the psi shell and the virtual layer (one launch), of the
// current state into psibuf[cur]. With ev, events ev[0..2] bracket the two
// kernels.
int launch_psi(flbm_sim* h, cudaEvent_t* ev = nullptr)
{
    const KParams& k = h->kp;
    float* psi = psi_cur(h);
    record(h, ev, 0);
    if (h->tape_out) {
        k_density_tape<<<h->grid, h->block, 0, h->stream>>>(h->fbuf[h->cur], psi, h->st, h->masks, k, h->tape_out);
        if (int rc = launch_check(h, "k_density_tape")) return rc;
    } else {
        k_density<<<h->grid, h->block, 0, h->stream>>>(h->fbuf[h->cur], psi, h->st, h->masks, k);
        if (int rc = launch_check(h, "k_density")) return rc;
    }
    record(h, ev, 1);
    const int nbs = (int)((shell_count(k) + kThreads - 1) / kThreads);
    const int nbv = virtual_blocks(k);
    k_shell_virtual<<<nbs + nbv, kThreads, 0, h->stream>>>(psi, h->st, h->masks, k, nbs);
    if (int rc = launch_check(h, "k_shell_virtual")) return rc;
    record(h, ev, 2);
    h->psi_valid = true;
    return FLBM_OK;
}

// Does the next step take the fused path (densities as a by-product)?
bool use_fused(const flbm_sim* h) { return h->density_mode == 1 && h->fused_allowed && !h->tma; }

// The current state's densities, if the next step needs them and they are stale.
int ensure_psi(flbm_sim* h)
{
    return h->psi_valid ? FLBM_OK : launch_psi(h);
}

// Kernel classes in the order each step launches them; step_timed assigns
// the time between consecutive events to these classes.
constexpr int kTwoPassOrder[FLBM_NKERNELS] = {FLBM_K_DENSITY, FLBM_K_SHELL, FLBM_K_COLLIDE, FLBM_K_PARTICLE};
constexpr int kFusedOrder[FLBM_NKERNELS] = {FLBM_K_COLLIDE, FLBM_K_PARTICLE, FLBM_K_DENSITY, FLBM_K_SHELL};

// Collide-stream of the current state: the near-particle tiles on the side
// stream (higher priority, so its few blocks start first), the bulk tiles on
// the handle's stream, joined before the particle kernels (the near launch
// and its particle update overlap the bulk launch). Fused: the bulk launch
// also writes the next state's densities (psibuf[1 - cur], ring, seams).
int launch_collide(flbm_sim* h, bool fused)
{
    const KParams& k = h->kp;
    const float* fin = h->fbuf[h->cur];
    float* fout = h->fbuf[1 - h->cur];
    const float* psi = psi_cur(h);
    const bool noise = k.kT > 0.0f;
    const bool part = k.has_particle != 0;
    const dim3 gnear(k.ncx, k.ncy, k.ncz);
    const dim3 gfused(k.gx, k.gy, h->fg.nchunk);
#define FLBM_COLLIDE(NZ, T1)                                                                                  \
    do {                                                                                                      \
        if (part) {                                                                                           \
            CK(h, cudaEventRecord(h->fork_ev, h->stream));                                                    \
            CK(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));                                               \
            k_collide_near<NZ, T1><<<gnear, h->block, 0, h->side>>>(fin, fout, psi, h->st, h->masks,          \
                                                                    h->partials, k);                          \
            if (int rc = launch_check(h, "k_collide_near")) return rc;                                        \
            CK(h, cudaEventRecord(h->join_ev, h->side));                                                      \
        }                                                                                                     \
        if (fused) {                                                                                          \
            k_collide_bulk_fused<NZ, T1><<<gfused, h->block, fused_smem_bytes(k), h->stream>>>(                \
                fin, fout, psi, h->psibuf[1 - h->cur], h->ring, h->seam, h->st, k, h->fg);                    \
            if (int rc = launch_check(h, "k_collide_bulk_fused")) return rc;                                  \
        } else if (h->tma) {                                                                                  \
            k_collide_bulk_tma<NZ, T1><<<h->tma_grid, h->block, kTmaSmemBytes, h->stream>>>(                   \
                h->tm_f[h->cur], h->tm_psi[h->cur], fout, h->st, k, h->tma_wait);                             \
            if (int rc = launch_check(h, "k_collide_bulk_tma")) return rc;                                    \
        } else {                                                                                              \
            k_collide_bulk<NZ, T1><<<h->grid, h->block, 0, h->stream>>>(fin, fout, psi, h->st, k);            \
            if (int rc = launch_check(h, "k_collide_bulk")) return rc;                                        \
        }                                                                                                     \
        if (part) CK(h, cudaStreamWaitEvent(h->stream, h->join_ev, 0));                                      \
    } while (0)
    if (noise && k.tau1) FLBM_COLLIDE(true, true);
    else if (noise) FLBM_COLLIDE(true, false);
    else if (k.tau1) FLBM_COLLIDE(false, true);
    else FLBM_COLLIDE(false, false);
#undef FLBM_COLLIDE
    return FLBM_OK;
}

// Particle kernels after the collide (the particle update ran in the near
// kernel's last block): next-position masks, cover/uncover and the step's
// bookkeeping; without a particle only the bookkeeping.
int launch_particle(flbm_sim* h)
{
    const KParams& k = h->kp;
    if (k.has_particle) {
        k_mark_next<<<h->box_blocks, 256, 0, h->stream>>>(h->st, h->masks, h->box_counts, k);
        if (int rc = launch_check(h, "k_mark_next")) return rc;
        k_cover<<<h->box_blocks, 256, 0, h->stream>>>(h->fbuf[1 - h->cur], h->st, h->masks, h->box_parts,
                                                       h->box_counts, k);
        if (int rc = launch_check(h, "k_cover")) return rc;
    } else {
        k_finish<<<1, 256, 0, h->stream>>>(h->st, h->box_counts, h->box_parts, h->box_blocks, k);
        if (int rc = launch_check(h, "k_finish")) return rc;
    }
    return FLBM_OK;
}

// One time step. With ev, events ev[0..4] bracket its four kernel classes
// (in the order kTwoPassOrder or kFusedOrder).
int launch_step(flbm_sim* h, cudaEvent_t* ev = nullptr)
{
    const KParams& k = h->kp;
    if (!use_fused(h)) {
        if (int rc = launch_psi(h, ev)) return rc;
        if (int rc = launch_collide(h, false)) return rc;
        record(h, ev, 3);
        if (int rc = launch_particle(h)) return rc;
        record(h, ev, 4);
        h->cur = 1 - h->cur;
        h->psi_valid = false;  // psibuf[cur] belongs to an older state
        return FLBM_OK;
    }
    if (int rc = ensure_psi(h)) return rc;
    record(h, ev, 0);
    if (int rc = launch_collide(h, true)) return rc;
    record(h, ev, 1);
    if (int rc = launch_particle(h)) return rc;
    record(h, ev, 2);
    float* psi_next = h->psibuf[1 - h->cur];
    const int nB = k.gx * k.gy * h->fg.nchunk;
    const int nA = (int)((near_box_nodes(k) + kThreadsStep - 1) / kThreadsStep);
    k_psi_finish<<<nB + nA, kThreadsStep, 0, h->stream>>>(h->fbuf[1 - h->cur], psi_next, h->ring, h->seam, h->st,
                                                          h->masks, k, h->fg, nB);
    if (int rc = launch_check(h, "k_psi_finish")) return rc;
    record(h, ev, 3);
    const int nbs = (int)((shell_count(k) + kThreads - 1) / kThreads);
    const int nbv = virtual_blocks(k);
    k_shell_virtual<<<nbs + nbv, kThreads, 0, h->stream>>>(psi_next, h->st, h->masks, k, nbs);
    if (int rc = launch_check(h, "k_shell_virtual")) return rc;
    record(h, ev, 4);
    h->cur = 1 - h->cur;
    h->psi_valid = true;
    return FLBM_OK;
}

// Planes per block of the fused collide by default: enough chunks for about
// two waves of resident blocks (4 per SM) over the lattice's tiles.
int auto_chunk(const KParams& k)
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    const long long tiles = (long long)k.gx * k.gy;
    const long long target = 2LL * sms * FLBM_BULK_MINBLOCKS;
    const long long nch = std::max(1LL, std::min<long long>(k.lz, target / tiles));
    return (int)((k.lz + nch - 1) / nch);
}

// Fused geometry for K planes per block; the seam buffer grows if needed.
int set_fused_geometry(flbm_sim* h, int K)
{
    const KParams& k = h->kp;
    K = std::max(K, (k.lz + 65534) / 65535);  // grid z limit
    FusedGeom g;
    g.K = K;
    g.nchunk = (k.lz + K - 1) / K;
    g.ring = 2 * (k.tx + 2) + 2 * k.ty;
    g.fp = (k.tx + 2) * (k.ty + 2);
    const size_t need = (size_t)k.gx * k.gy * g.nchunk * 2 * g.fp;
    if (need > h->seam_cap) {
        if (h->seam) cudaFree(h->seam);
        h->seam = nullptr;
        h->seam_cap = 0;
        if (cudaMalloc(&h->seam, sizeof(float2) * need) != cudaSuccess) return fail(h, FLBM_E_NOMEM, "seam buffer");
        h->seam_cap = need;
    }
    h->fg = g;
    return FLBM_OK;
}

// Captured graphs replay the kernels and parameters of their capture; drop
// them (with rec_only, only those that record the trajectory).
int drop_graphs(flbm_sim* h, bool rec_only = false)
{
    bool any = false;
    for (int c = 0; c < 2; ++c) any = any || h->graph_rec[c] || (!rec_only && h->graph[c]);
    if (!any) return FLBM_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    for (int c = 0; c < 2; ++c) {
        if (h->graph_rec[c]) cudaGraphExecDestroy(h->graph_rec[c]);
        h->graph_rec[c] = nullptr;
        if (!rec_only && h->graph[c]) {
            cudaGraphExecDestroy(h->graph[c]);
            h->graph[c] = nullptr;
        }
    }
    return FLBM_OK;
}

// The particle record of the step just finished into the next free slot of
// traj (count of them kept on the device, so that captured steps can record).
static __global__ void __launch_bounds__(64) k_record(const DevState* __restrict__ st, DevState* __restrict__ traj,
                                                      int* __restrict__ count, int cap)
{
    const int slot = *count;
    if (slot >= cap) return;  // the same for the whole block
    const uint32_t* src = reinterpret_cast<const uint32_t*>(st);
    uint32_t* dst = reinterpret_cast<uint32_t*>(traj + slot);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();  // every thread has read the count
    if (threadIdx.x == 0) *count = slot + 1;
}
static_assert(sizeof(DevState) % 4 == 0, "DevState is copied as 32-bit words");

// One step and, with rec, its particle record (flbm_run_host).
int launch_step_rec(flbm_sim* h, bool rec)
{
    if (int rc = launch_step(h)) return rc;
    if (!rec) return FLBM_OK;
    k_record<<<1, 64, 0, h->stream>>>(h->st, h->traj_dev, h->traj_count, (int)h->traj_cap);
    return launch_check(h, "k_record");
}

// Steps per captured graph (even, so that a replay brings cur back). More
// steps per graph spread the replay's own launch cost over more steps.
constexpr int kGraphSteps = 8;

// Capture kGraphSteps steps starting from cur = c (with rec, each followed by
// its particle record) into h->graph[c] or h->graph_rec[c] (once).
int ensure_graph(flbm_sim* h, int c, bool rec = false)
{
    cudaGraphExec_t& ge = rec ? h->graph_rec[c] : h->graph[c];
    if (ge) return FLBM_OK;
    const int64_t before = h->launches;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = FLBM_OK;
    for (int k = 0; k < kGraphSteps && !rc; ++k) rc = launch_step_rec(h, rec);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ge = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    // Capturing only recorded the kernels: nothing ran, cur is back at c.
    (rec ? h->graph_rec_launches[c] : h->graph_launches[c]) = h->launches - before;
    h->launches = before;
    return FLBM_OK;
}

// nsteps steps: replayed graphs of kGraphSteps steps while they fit (with
// use_graphs), plain launches for the rest; with rec each step's particle
// record follows it.
int run_steps(flbm_sim* h, int64_t nsteps, bool rec)
{
    int64_t s = 0;
    if (h->use_graphs) {
        // A graph captures steps that start from valid densities.
        if (use_fused(h) && nsteps >= kGraphSteps)
            if (int rc = ensure_psi(h)) return rc;
        for (; s + kGraphSteps <= nsteps; s += kGraphSteps) {
            if (int rc = ensure_graph(h, h->cur, rec)) return rc;
            CK(h, cudaGraphLaunch(rec ? h->graph_rec[h->cur] : h->graph[h->cur], h->stream));
            // an even number of steps brings cur back
            h->launches += rec ? h->graph_rec_launches[h->cur] : h->graph_launches[h->cur];
        }
    }
    for (; s < nsteps; ++s)
        if (int rc = launch_step_rec(h, rec)) return rc;
    return FLBM_OK;
}

// Fixed-size head of a checkpoint file, followed by flbm_params, DevState,
// the two particle masks, the current populations and (version 2) the padded
// density field of the current state, which the fused step carries from one
// step to the next.
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t lx, ly, lz, wall[3], B;
    double radius;
    uint64_t params_bytes, state_bytes, mask_bytes, f_bytes;
};

void fill_header(const flbm_sim* h, CkptHeader* hd)
{
    std::memset(hd, 0, sizeof(*hd));
    std::memcpy(hd->magic, "FLBMCKP", 8);
    hd->version = 2;
    hd->lx = h->p.lx; hd->ly = h->p.ly; hd->lz = h->p.lz;
    hd->wall[0] = h->p.wall_x; hd->wall[1] = h->p.wall_y; hd->wall[2] = h->p.wall_z;
    hd->B = h->kp.B;
    hd->radius = h->kp.has_particle ? h->p.radius : 0.0;
    hd->params_bytes = sizeof(flbm_params);
    hd->state_bytes = sizeof(DevState);
    hd->mask_bytes = (uint64_t)2 * h->kp.B * h->kp.B * h->kp.B;
    hd->f_bytes = (uint64_t)sizeof(float) * 2 * 19 * h->kp.N;
}

}  // namespace

namespace flbm {
int sim_step(flbm_sim* h, cudaEvent_t* ev) { return launch_step(h, ev); }
int sim_step_tape(flbm_sim* h, float* tape)
{
    if (use_fused(h)) return fail(h, FLBM_E_UNSUPPORTED, "a taped step needs the two-pass density mode");
    h->tape_out = tape;
    const int rc = launch_step(h);
    h->tape_out = nullptr;
    return rc;
}
int sim_fail(flbm_sim* h, int code, const std::string& msg) { return fail(h, code, msg); }
int sim_ensure_psi(flbm_sim* h) { return ensure_psi(h); }
bool sim_fused(const flbm_sim* h) { return use_fused(h); }
}  // namespace flbm

extern "C" {

size_t flbm_state_bytes(const flbm_params* p)
{
    if (!validate(p).empty()) return 0;
    return (size_t)2 * 2 * 19 * (size_t)p->lx * p->ly * p->lz * sizeof(float);
}

int flbm_create(const flbm_params* p, void* f_dev, size_t f_dev_bytes, void* stream, flbm_t** out)
{
    if (!out) return FLBM_E_INVAL;
    *out = nullptr;
    std::string v = validate(p);
    if (!v.empty()) {
        std::fprintf(stderr, "flbm_create: %s\n", v.c_str());
        return FLBM_E_INVAL;
    }
    flbm_sim* h = new (std::nothrow) flbm_sim();
    if (!h) return FLBM_E_NOMEM;
    h->p = *p;
    h->stream = (cudaStream_t)stream;
    fill_kparams(h);
    const KParams& k = h->kp;
    const size_t need = flbm_state_bytes(p);
    auto bail = [&](int code) {
        flbm_destroy(h);
        return code;
    };
    if (f_dev) {
        if (f_dev_bytes < need || ((uintptr_t)f_dev % 256) != 0) {
            std::fprintf(stderr, "flbm_create: borrowed buffer too small or not 256-byte aligned\n");
            return bail(FLBM_E_INVAL);
        }
        h->fbuf[0] = (float*)f_dev;
    } else {
        if (cudaMalloc(&h->f_owned, need) != cudaSuccess) return bail(FLBM_E_NOMEM);
        h->fbuf[0] = (float*)h->f_owned;
    }
    h->fbuf[1] = h->fbuf[0] + (size_t)2 * 19 * k.N;
    const size_t B3 = (size_t)k.B * k.B * k.B;
    if (cudaMalloc(&h->psibuf[0], sizeof(float) * 2 * k.padn) != cudaSuccess ||
        cudaMalloc(&h->psibuf[1], sizeof(float) * 2 * k.padn) != cudaSuccess ||
        cudaMalloc(&h->st, sizeof(DevState)) != cudaSuccess ||
        cudaMalloc(&h->masks, 2 * B3) != cudaSuccess ||
        cudaMalloc(&h->partials, sizeof(double) * 8 * h->ncand) != cudaSuccess ||
        cudaMalloc(&h->box_counts, sizeof(int) * h->box_blocks) != cudaSuccess ||
        cudaMalloc(&h->box_parts, sizeof(double) * 8 * h->box_blocks) != cudaSuccess ||
        cudaMalloc(&h->obs_tiles, sizeof(double) * 8 * h->ntiles) != cudaSuccess ||
        cudaMalloc(&h->obs_out, sizeof(double) * 8) != cudaSuccess ||
        cudaMalloc(&h->obs_mode_tiles, sizeof(double) * kObsModes * h->ntiles) != cudaSuccess ||
        cudaMalloc(&h->obs_mode_out, sizeof(double) * kObsModes) != cudaSuccess)
        return bail(FLBM_E_NOMEM);

    {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(FLBM_E_CUDA);
    }

    // Particle state (FP64): Eq. (fp) and the nominal sphere mass and inertia.
    const DevState s = initial_state(*p, k);
    if (cudaMemcpyAsync(h->st, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return bail(FLBM_E_CUDA);
    if (cudaMemsetAsync(h->masks, 0, 2 * B3, h->stream) != cudaSuccess) return bail(FLBM_E_CUDA);
    for (int c = 0; c < 2; ++c)
        if (cudaMemsetAsync(h->psibuf[c], 0, sizeof(float) * 2 * k.padn, h->stream) != cudaSuccess)
            return bail(FLBM_E_CUDA);
    if (cudaMemsetAsync(h->partials, 0, sizeof(double) * 8 * h->ncand, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->box_counts, 0, sizeof(int) * h->box_blocks, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->box_parts, 0, sizeof(double) * 8 * h->box_blocks, h->stream) != cudaSuccess)
        return bail(FLBM_E_CUDA);
    k_init<<<h->grid, h->block, 0, h->stream>>>(h->fbuf[0], k, (float)p->rho_a0, (float)p->rho_b0,
                                                 (float)p->init_pert);
    if (launch_check(h, "k_init")) return bail(FLBM_E_CUDA);
    // Both copies start equal, so particle nodes (never written by the step) hold defined values.
    if (cudaMemcpyAsync(h->fbuf[1], h->fbuf[0], need / 2, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return bail(FLBM_E_CUDA);
    if (k.has_particle) {
        k_mark<<<1, 1024, 0, h->stream>>>(h->st, h->masks, k);
        if (launch_check(h, "k_mark")) return bail(FLBM_E_CUDA);
    }
    // The densities of the initial state; later steps keep them (fused) or
    // recompute them (two-pass).
    if (launch_psi(h)) return bail(FLBM_E_CUDA);
    // The fused collide is available where the lattice allows it (ring buffer
    // for every plane, seams for the default chunking); steps are two-pass
    // until flbm_set_density_mode selects it.
    h->fused_allowed = fused_ok(k);
    if (h->fused_allowed) {
        // Exchange arrays and rolling sums in dynamic shared memory (above the
        // 48 KB default for 32 x 8 tiles).
        void (*fused_kern[4])(const float*, float*, const float*, float*, float2*, float2*, const DevState*, KParams,
                              FusedGeom) = {k_collide_bulk_fused<false, false>, k_collide_bulk_fused<false, true>,
                                            k_collide_bulk_fused<true, false>, k_collide_bulk_fused<true, true>};
        for (auto* fk : fused_kern)
            if (cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem_bytes(k)) !=
                cudaSuccess)
                return bail(FLBM_E_CUDA);
        const FusedGeom g{1, 1, 2 * (k.tx + 2) + 2 * k.ty, (k.tx + 2) * (k.ty + 2)};
        if (cudaMalloc(&h->ring, sizeof(float2) * (size_t)k.gx * k.gy * k.lz * g.ring) != cudaSuccess)
            return bail(FLBM_E_NOMEM);
        if (set_fused_geometry(h, auto_chunk(k))) return bail(FLBM_E_NOMEM);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(FLBM_E_CUDA);
    setup_tma(h);
    h->launches = 0;
    *out = h;
    return FLBM_OK;
}

int flbm_step(flbm_t* h, int64_t nsteps)
{
    if (!h || nsteps < 0) return fail(h, FLBM_E_INVAL, "invalid handle or step count");
    h->launches = 0;
    return run_steps(h, nsteps, false);
}

int flbm_use_tma(flbm_t* h, int enable)
{
    if (!h || (enable != 0 && enable != 1)) return fail(h, FLBM_E_INVAL, "invalid argument");
    if (enable && !h->tma_ok)
        return fail(h, FLBM_E_UNSUPPORTED, "TMA-staged collide needs lx % 4 == 0 and lx >= 32");
    if (h->tma != (enable != 0))
        if (int rc = drop_graphs(h)) return rc;  // captured graphs hold the other bulk kernel
    h->tma = enable != 0;
    return FLBM_OK;
}

int flbm_set_density_mode(flbm_t* h, int32_t mode, int32_t planes_per_block)
{
    if (!h || (mode != 0 && mode != 1) || planes_per_block < 0 || planes_per_block > h->kp.lz)
        return fail(h, FLBM_E_INVAL, "invalid argument");
    if (mode == 1 && !h->fused_allowed)
        return fail(h, FLBM_E_UNSUPPORTED,
                    "fused densities need tiles at least 8 wide and 3 tiles along a periodic x or y");
    if (int rc = drop_graphs(h)) return rc;
    if (mode == 1) {
        if (int rc = set_fused_geometry(h, planes_per_block ? planes_per_block : auto_chunk(h->kp))) return rc;
    }
    h->density_mode = mode;
    return FLBM_OK;
}

int flbm_get_density_mode(const flbm_t* h, int32_t* mode, int32_t* planes_per_block)
{
    if (!h || !mode || !planes_per_block) return FLBM_E_INVAL;
    *mode = use_fused(h) ? 1 : 0;
    *planes_per_block = *mode ? h->fg.K : 0;
    return FLBM_OK;
}

int flbm_set_tma_wait(flbm_t* h, int64_t cycles)
{
    if (!h || cycles < 0) return fail(h, FLBM_E_INVAL, "invalid argument");
    if (cycles == 0) cycles = kTmaWaitCycles;
    if (h->tma_wait != cycles)
        if (int rc = drop_graphs(h)) return rc;  // captured graphs hold the old limit
    h->tma_wait = cycles;
    return FLBM_OK;
}

int flbm_use_graphs(flbm_t* h, int enable)
{
    if (!h || (enable != 0 && enable != 1)) return fail(h, FLBM_E_INVAL, "invalid argument");
    if (enable && h->stream == nullptr)
        return fail(h, FLBM_E_UNSUPPORTED, "graph capture needs a stream other than the legacy default stream");
    h->use_graphs = enable != 0;
    return FLBM_OK;
}

int flbm_checkpoint(flbm_t* h, const char* path)
{
    if (!h || !path) return fail(h, FLBM_E_INVAL, "NULL argument");
    const KParams& k = h->kp;
    CkptHeader hd;
    fill_header(h, &hd);
    std::vector<unsigned char> masks(hd.mask_bytes);
    std::vector<float> f((size_t)2 * 19 * k.N);
    std::vector<float> psi((size_t)2 * k.padn);
    DevState st;
    if (int rc = ensure_psi(h)) return rc;
    CK(h, cudaMemcpyAsync(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(masks.data(), h->masks, hd.mask_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(f.data(), h->fbuf[h->cur], hd.f_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(psi.data(), psi_cur(h), sizeof(float) * psi.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(h, FLBM_E_INVAL, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(&h->p, sizeof(h->p), 1, fp) == 1 &&
              std::fwrite(&st, sizeof(st), 1, fp) == 1 &&
              std::fwrite(masks.data(), 1, hd.mask_bytes, fp) == hd.mask_bytes &&
              std::fwrite(f.data(), 1, hd.f_bytes, fp) == hd.f_bytes &&
              std::fwrite(psi.data(), sizeof(float), psi.size(), fp) == psi.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? FLBM_OK : fail(h, FLBM_E_INVAL, std::string("write to ") + path + " failed");
}

int flbm_restore(flbm_t* h, const char* path)
{
    if (!h || !path) return fail(h, FLBM_E_INVAL, "NULL argument");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(h, FLBM_E_INVAL, std::string("cannot open ") + path);
    CkptHeader want, got;
    fill_header(h, &want);
    flbm_params fp_params;
    DevState st;
    std::vector<unsigned char> masks(want.mask_bytes);
    std::vector<float> f((size_t)2 * 19 * h->kp.N);
    bool ok = std::fread(&got, sizeof(got), 1, fp) == 1;
    if (ok && (std::memcmp(got.magic, want.magic, sizeof(got.magic)) != 0 || got.version < 1 ||
               got.version > want.version ||
               got.params_bytes != want.params_bytes || got.state_bytes != want.state_bytes)) {
        std::fclose(fp);
        return fail(h, FLBM_E_INVAL, std::string(path) + ": not a checkpoint of this library version");
    }
    if (ok && (got.lx != want.lx || got.ly != want.ly || got.lz != want.lz || got.wall[0] != want.wall[0] ||
               got.wall[1] != want.wall[1] || got.wall[2] != want.wall[2] || got.B != want.B ||
               got.radius != want.radius || got.mask_bytes != want.mask_bytes || got.f_bytes != want.f_bytes)) {
        std::fclose(fp);
        return fail(h, FLBM_E_INVAL, std::string(path) + ": lattice, walls or radius differ from this simulation");
    }
    ok = ok && std::fread(&fp_params, sizeof(fp_params), 1, fp) == 1 && std::fread(&st, sizeof(st), 1, fp) == 1 &&
         std::fread(masks.data(), 1, want.mask_bytes, fp) == want.mask_bytes &&
         std::fread(f.data(), 1, want.f_bytes, fp) == want.f_bytes;
    // Version 2 carries the state's densities; version 1 files get them recomputed.
    std::vector<float> psi(got.version >= 2 ? (size_t)2 * h->kp.padn : 0);
    ok = ok && (psi.empty() || std::fread(psi.data(), sizeof(float), psi.size(), fp) == psi.size());
    std::fclose(fp);
    if (!ok) return fail(h, FLBM_E_INVAL, std::string(path) + ": truncated checkpoint");
    const std::string bad = check_restored_state(st, h->kp);
    if (!bad.empty()) return fail(h, FLBM_E_INVAL, std::string(path) + ": " + bad);
    // Values derived from the parameters follow this handle's parameters.
    if (h->kp.has_particle) {
        const DevState s0 = initial_state(h->p, h->kp);
        st.mp = s0.mp;
        st.Ip = s0.Ip;
        st.Fp = s0.Fp;
        st.fc = (h->p.fluid_counterforce && st.nfluid > 0) ? -st.Fp / (double)st.nfluid : 0.0;
        st.fc_f = (float)st.fc;
    }
    // Counters of the step's launches start from zero on this handle.
    st.err = 0;
    st.near_done = 0;
    st.cover_done = 0;
    CK(h, cudaMemcpyAsync(h->st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->masks, masks.data(), want.mask_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->fbuf[h->cur], f.data(), want.f_bytes, cudaMemcpyHostToDevice, h->stream));
    if (!psi.empty()) {
        CK(h, cudaMemcpyAsync(psi_cur(h), psi.data(), sizeof(float) * psi.size(), cudaMemcpyHostToDevice, h->stream));
        h->psi_valid = true;
    } else if (int rc = launch_psi(h)) {
        return rc;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return FLBM_OK;
}

int flbm_particle_state(flbm_t* h, flbm_particle* out)
{
    if (!h || !out) return fail(h, FLBM_E_INVAL, "NULL argument");
    DevState s;
    CK(h, cudaMemcpyAsync(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (s.err) return fail(h, FLBM_E_TIMEOUT, "a bounded device-side wait gave up");
    return copy_particle(s, out);
}

int flbm_observables(flbm_t* h, flbm_obs* out)
{
    if (!h || !out) return fail(h, FLBM_E_INVAL, "NULL argument");
    const KParams& k = h->kp;
    k_obs_tiles<<<h->grid, h->block, 0, h->stream>>>(h->fbuf[h->cur], h->st, h->masks, h->obs_tiles, k);
    if (int rc = launch_check(h, "k_obs_tiles")) return rc;
    k_obs_final<<<1, 1024, 0, h->stream>>>(h->obs_tiles, h->ntiles, h->obs_out);
    if (int rc = launch_check(h, "k_obs_final")) return rc;
    k_obs_modes<<<h->grid, h->block, 0, h->stream>>>(h->fbuf[h->cur], h->st, h->masks, h->obs_mode_tiles, k);
    if (int rc = launch_check(h, "k_obs_modes")) return rc;
    k_obs_final_n<kObsModes><<<1, 1024, 0, h->stream>>>(h->obs_mode_tiles, h->ntiles, h->obs_mode_out);
    if (int rc = launch_check(h, "k_obs_final_n")) return rc;
    double v[8], vm[kObsModes];
    DevState s;
    CK(h, cudaMemcpyAsync(v, h->obs_out, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(vm, h->obs_mode_out, sizeof(vm), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    fill_obs(v, s, out);
    fill_mode_obs(vm, out);
    if (s.err) return fail(h, FLBM_E_TIMEOUT, "a bounded device-side wait gave up");
    return out->nonfinite ? fail(h, FLBM_E_NONFINITE, "non-finite populations") : FLBM_OK;
}

int flbm_read_fields(flbm_t* h, float* host_f, float* host_rho)
{
    if (!h) return FLBM_E_INVAL;
    const KParams& k = h->kp;
    if (host_f)
        CK(h, cudaMemcpyAsync(host_f, h->fbuf[h->cur], sizeof(float) * 2 * 19 * k.N, cudaMemcpyDeviceToHost,
                              h->stream));
    if (host_rho) {
        if (!h->scratch_rho) CK(h, cudaMalloc(&h->scratch_rho, sizeof(float) * 2 * k.N));
        if (int rc = ensure_psi(h)) return rc;
        k_unpad<<<h->grid, h->block, 0, h->stream>>>(psi_cur(h), h->scratch_rho, k);
        if (int rc = launch_check(h, "k_unpad")) return rc;
        CK(h, cudaMemcpyAsync(host_rho, h->scratch_rho, sizeof(float) * 2 * k.N, cudaMemcpyDeviceToHost,
                              h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return FLBM_OK;
}

int flbm_write_fields(flbm_t* h, const float* host_f)
{
    if (!h || !host_f) return fail(h, FLBM_E_INVAL, "NULL argument");
    CK(h, cudaMemcpyAsync(h->fbuf[h->cur], host_f, sizeof(float) * 2 * 19 * h->kp.N, cudaMemcpyHostToDevice,
                          h->stream));
    if (int rc = launch_psi(h)) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return FLBM_OK;
}

int flbm_set_particle(flbm_t* h, const double X[3], const double V[3], const double Omega[3])
{
    if (!h || !X || !V || !Omega) return fail(h, FLBM_E_INVAL, "NULL argument");
    if (!h->kp.has_particle) return fail(h, FLBM_E_UNSUPPORTED, "simulation has no particle");
    for (int a = 0; a < 3; ++a) {
        const int L[3] = {h->p.lx, h->p.ly, h->p.lz};
        const int w[3] = {h->p.wall_x, h->p.wall_y, h->p.wall_z};
        if (!std::isfinite(X[a]) || !std::isfinite(V[a]) || !std::isfinite(Omega[a]))
            return fail(h, FLBM_E_INVAL, "non-finite particle state");
        if (w[a] && (X[a] - h->p.radius < -0.5 || X[a] + h->p.radius > L[a] - 0.5))
            return fail(h, FLBM_E_INVAL, "the sphere must lie inside the walls");
    }
    DevState s;
    CK(h, cudaMemcpyAsync(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int a = 0; a < 3; ++a) {
        s.X[a] = X[a];
        if (!h->p.wall_x && a == 0) s.X[a] -= h->p.lx * std::floor(s.X[a] / h->p.lx);
        if (!h->p.wall_y && a == 1) s.X[a] -= h->p.ly * std::floor(s.X[a] / h->p.ly);
        if (!h->p.wall_z && a == 2) s.X[a] -= h->p.lz * std::floor(s.X[a] / h->p.lz);
        s.V[a] = V[a];
        s.Om[a] = Omega[a];
        s.Ppend[a] = s.Lpend[a] = 0.0;
    }
    s.delta[0] = s.delta[1] = 0.0;
    CK(h, cudaMemcpyAsync(h->st, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    k_mark<<<1, 1024, 0, h->stream>>>(h->st, h->masks, h->kp);
    if (int rc = launch_check(h, "k_mark")) return rc;
    if (int rc = launch_psi(h)) return rc;  // particle nodes and virtual layer moved
    CK(h, cudaStreamSynchronize(h->stream));
    return FLBM_OK;
}

int flbm_run_host(flbm_t* h, const float* host_f_in, int64_t nsteps, float* host_f_out, flbm_particle* traj)
{
    if (!h || !host_f_in || nsteps < 0) return fail(h, FLBM_E_INVAL, "invalid argument");
    const KParams& k = h->kp;
    const size_t fbytes = sizeof(float) * 2 * 19 * k.N;
    if (traj && nsteps > 0x7fffffff) return fail(h, FLBM_E_INVAL, "too many steps for a trajectory");
    if (traj && (size_t)nsteps > h->traj_cap) {
        if (int rc = drop_graphs(h, true)) return rc;  // they hold the old record buffer
        if (h->traj_dev) cudaFree(h->traj_dev);
        h->traj_dev = nullptr;
        h->traj_cap = 0;
        CK(h, cudaMalloc(&h->traj_dev, sizeof(DevState) * (size_t)nsteps));
        h->traj_cap = (size_t)nsteps;
    }
    if (traj && !h->traj_count) CK(h, cudaMalloc(&h->traj_count, sizeof(int)));
    CK(h, cudaMemcpyAsync(h->fbuf[h->cur], host_f_in, fbytes, cudaMemcpyHostToDevice, h->stream));
    if (traj) CK(h, cudaMemsetAsync(h->traj_count, 0, sizeof(int), h->stream));
    h->launches = 0;
    // New populations: the densities are stale (a two-pass step computes its
    // own; the fused one needs them first).
    h->psi_valid = false;
    if (use_fused(h))
        if (int rc = ensure_psi(h)) return rc;
    if (int rc = run_steps(h, nsteps, traj != nullptr)) return rc;
    if (host_f_out)
        CK(h, cudaMemcpyAsync(host_f_out, h->fbuf[h->cur], fbytes, cudaMemcpyDeviceToHost, h->stream));
    if (traj && nsteps > 0) {
        if ((size_t)nsteps > h->traj_host_cap) {
            delete[] h->traj_host;
            h->traj_host = new (std::nothrow) DevState[(size_t)nsteps];
            if (!h->traj_host) {
                h->traj_host_cap = 0;
                return fail(h, FLBM_E_NOMEM, "trajectory staging");
            }
            h->traj_host_cap = (size_t)nsteps;
        }
        CK(h, cudaMemcpyAsync(h->traj_host, h->traj_dev, sizeof(DevState) * (size_t)nsteps, cudaMemcpyDeviceToHost,
                              h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (traj)
        for (int64_t s = 0; s < nsteps; ++s) copy_particle(h->traj_host[s], traj + s);
    return FLBM_OK;
}

int flbm_step_timed(flbm_t* h, int64_t nsteps, double* ms)
{
    if (!h || nsteps < 0 || !ms) return fail(h, FLBM_E_INVAL, "invalid argument");
    const size_t need = (size_t)(FLBM_NKERNELS + 1) * (size_t)nsteps;
    while (h->events.size() < need) {
        cudaEvent_t e;
        CK(h, cudaEventCreate(&e));
        h->events.push_back(e);
    }
    h->launches = 0;
    const int* order = use_fused(h) ? kFusedOrder : kTwoPassOrder;
    for (int64_t s = 0; s < nsteps; ++s)
        if (int rc = launch_step(h, h->events.data() + (FLBM_NKERNELS + 1) * s)) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < FLBM_NKERNELS; ++k) ms[k] = 0.0;
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaEvent_t* ev = h->events.data() + (FLBM_NKERNELS + 1) * s;
        for (int k = 0; k < FLBM_NKERNELS; ++k) {
            float t = 0.0f;
            CK(h, cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            ms[order[k]] += t;
        }
    }
    return FLBM_OK;
}

const char* flbm_kernel_name(int k)
{
    static const char* names[FLBM_NKERNELS] = {"k_density", "k_shell_virtual", "k_collide", "k_particle"};
    return (k >= 0 && k < FLBM_NKERNELS) ? names[k] : "";
}

int64_t flbm_last_launch_count(const flbm_t* h) { return h ? h->launches : 0; }

void flbm_destroy(flbm_t* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->f_owned);
    cudaFree(h->psibuf[0]);
    cudaFree(h->psibuf[1]);
    cudaFree(h->ring);
    cudaFree(h->seam);
    cudaFree(h->st);
    cudaFree(h->masks);
    cudaFree(h->partials);
    cudaFree(h->box_counts);
    cudaFree(h->box_parts);
    cudaFree(h->obs_tiles);
    cudaFree(h->obs_out);
    cudaFree(h->obs_mode_tiles);
    cudaFree(h->obs_mode_out);
    cudaFree(h->scratch_rho);
    cudaFree(h->traj_dev);
    cudaFree(h->traj_count);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    for (cudaGraphExec_t g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    for (cudaGraphExec_t g : h->graph_rec)
        if (g) cudaGraphExecDestroy(g);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    delete[] h->traj_host;
    delete h;
}

const char* flbm_error_string(int code)
{
    switch (code) {
    case FLBM_OK: return "FLBM_OK";
    case FLBM_E_INVAL: return "FLBM_E_INVAL: invalid argument";
    case FLBM_E_NOMEM: return "FLBM_E_NOMEM: allocation failed";
    case FLBM_E_CUDA: return "FLBM_E_CUDA: CUDA error";
    case FLBM_E_NONFINITE: return "FLBM_E_NONFINITE: non-finite state";
    case FLBM_E_TIMEOUT: return "FLBM_E_TIMEOUT: device wait timed out";
    case FLBM_E_UNSUPPORTED: return "FLBM_E_UNSUPPORTED: not supported";
    }
    return "unknown FLBM error code";
}

const char* flbm_last_error(const flbm_t* h) { return h ? h->err.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Observables without any allocation.
//
// For callers that cannot allocate device memory themselves: code running
// inside a memory pool or arena that owns every byte of the device, plugins
// of host applications that forbid cudaMalloc/cudaFree on their streams, or
// callers that must not synchronise the device (cudaFree does). They pass the
// population field and a place for the result; the per-tile partial sums go
// to the file-scope array below, which every GPU that loads this library
// holds until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_tiles[FLBM_NOALLOC_MAX_TILES * 8];

namespace {

// Device address of g_noalloc_tiles, looked up on the first call made with a
// device current (host code may not use the symbol itself: in host code its
// name is only a stand-in, not a device address). The address belongs to the
// CUDA context the lookup ran in, so each slot remembers that context's
// unique ID and the lookup runs again when a call comes from another context
// (a primary context re-created after cudaDeviceReset, or a context the
// caller made current through the driver API).
struct NoallocSlot {
    double* ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool ready = false;
};
NoallocSlot g_noalloc_slots[64];
std::mutex g_noalloc_mutex;

// Unique ID of the calling thread's current CUDA context (0 if there is none
// or the driver cannot tell), from the driver's cuCtxGetCurrent and
// cuCtxGetId reached through the runtime (no link to libcuda).
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

}  // namespace

extern "C" int flbm_observables_noalloc(const flbm_params* p, const float* f_dev, double* out_dev, void* stream)
{
    if (!p || !f_dev || !out_dev) return FLBM_E_INVAL;
    if (p->lx < 1 || p->ly < 1 || p->lz < 1 || p->lz > 65535 ||
        (double)p->lx * p->ly * p->lz > 4294967295.0) {
        std::fprintf(stderr, "flbm_observables_noalloc: invalid lattice size\n");
        return FLBM_E_INVAL;
    }
    if (p->radius > 0.0) {
        std::fprintf(stderr, "flbm_observables_noalloc: only for simulations without a particle\n");
        return FLBM_E_UNSUPPORTED;
    }
    flbm_sim tmp;  // launch geometry only; nothing is allocated
    tmp.p = *p;
    fill_kparams(&tmp);
    if (tmp.ntiles > FLBM_NOALLOC_MAX_TILES) {
        std::fprintf(stderr, "flbm_observables_noalloc: lattice needs %lld tiles, more than the %d of the static "
                             "scratch (at most 128x128x512 nodes or equivalent)\n",
                     tmp.ntiles, FLBM_NOALLOC_MAX_TILES);
        return FLBM_E_INVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FLBM_E_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocSlot& s = g_noalloc_slots[dev];
        const unsigned long long id = current_context_id();
        if (!s.ready || id == 0 || id != s.ctx_id) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_tiles) != cudaSuccess) return FLBM_E_CUDA;
            s.ptr = (double*)ptr;
            // The lookup made the runtime's context current if none was.
            s.ctx_id = current_context_id();
            s.ready = s.ctx_id != 0;
        }
        scratch = s.ptr;
    }
    // Every tile slot the final sum reads is written by k_obs_tiles in this
    // same call, so nothing has to be cleared first.
    cudaStream_t st = (cudaStream_t)stream;
    k_obs_tiles<<<tmp.grid, tmp.block, 0, st>>>(f_dev, nullptr, nullptr, scratch, tmp.kp);
    if (cudaGetLastError() != cudaSuccess) return FLBM_E_CUDA;
    k_obs_final<<<1, 1024, 0, st>>>(scratch, tmp.ntiles, out_dev);
    if (cudaGetLastError() != cudaSuccess) return FLBM_E_CUDA;
    return FLBM_OK;
}

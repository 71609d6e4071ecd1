// Batched ensemble of independent FLBM simulations (declared in include/flbm.h).
//
// The paper's statistics of the settling velocity (Section 3) are averages
// over noise realisations and channel geometries. An ensemble advances all
// its replicas with one set of batched launches per step: every launch walks
// a flat list of work items (replica and block of that replica, with the
// block's tile coordinates decoded on the host), one block per item or a
// fixed number of persistent blocks per SM striding over the list. A block
// stages the descriptor of its current replica (kernel parameters and device
// pointers) in shared memory and runs the same device bodies as the
// single-simulation kernels, so each replica computes exactly what
// flbm_create/flbm_step would. With one block per item, the bulk collide
// instead takes the descriptors of up to kChunkReps replicas as a kernel
// parameter (kb_bulk_rep). The step sequence (densities; density shell;
// collide-stream of the bulk tiles; on a side stream meanwhile the virtual
// layer, the near tiles, whose launch ends with each replica's particle
// update, and the next-position masks; cover/uncover ending with each
// replica's bookkeeping) is captured into a CUDA graph of two steps when the
// stream allows capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "flbm_host.cuh"

using namespace flbm;

namespace flbm_ensemble {

// Everything a block needs to run one replica's work item.
struct RepDesc {
    KParams P;
    float* f[2];          // population copies; step s reads f[s % 2]
    float* psi;           // padded density field
    DevState* st;         // particle record and step counter
    uint8_t* masks;       // two particle-node masks of the box
    double* partials;     // per candidate near tile: force, torque, ledger
    int* box_counts;      // per block of the particle box
    double* box_parts;    // per block of the particle box
    int box_blocks;
    int pad_;
};
static_assert(sizeof(RepDesc) % 4 == 0, "RepDesc is copied as 32-bit words");

// Copy the descriptor of replica r into shared memory unless the block holds
// it already (r is the same for every thread of the block).
__device__ __forceinline__ void stage_rep(const RepDesc* __restrict__ reps, int r, RepDesc& s, int& have)
{
    if (r == have) return;
    __syncthreads();  // every thread is done with the previous replica
    const uint32_t* src = reinterpret_cast<const uint32_t*>(reps + r);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s);
    for (int w = threadIdx.x; w < (int)(sizeof(RepDesc) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    have = r;
}

// Work item of a batched launch: x the replica; for tile lists (density,
// bulk collide) y, z, w the tile (bx, by, bz), for near lists the candidate
// (cx, cy, cz); for the others y the block of the replica.
using Item = int4;

// This thread's place (tx, ty) in a tile: the tile width is a power of two.
struct TileCoord {
    int bx, by, bz, tx, ty;
};
__device__ __forceinline__ TileCoord tile_of(const Item& it, const KParams& P)
{
    TileCoord c;
    c.bx = it.y;
    c.by = it.z;
    c.bz = it.w;
    c.tx = threadIdx.x & (P.tx - 1);
    c.ty = threadIdx.x >> (__ffs(P.tx) - 1);
    return c;
}

// Every batched kernel: 256 threads, items[i] as above.
#define FLBM_FOR_ITEMS                                                     \
    __shared__ RepDesc sR;                                                 \
    int have = -1;                                                         \
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {                 \
        const Item it = items[i];                                          \
        stage_rep(reps, it.x, sR, have);                                   \
        const KParams& P = sR.P;
#define FLBM_END_ITEMS }

static __global__ void __launch_bounds__(256) kb_density(const RepDesc* __restrict__ reps,
                                                         const Item* __restrict__ items, int nitems, int par)
{
    FLBM_FOR_ITEMS
    const TileCoord c = tile_of(it, P);
    density_node(c.bx * P.tx + c.tx, c.by * P.ty + c.ty, c.bz, sR.f[par], sR.psi, sR.st, sR.masks, P);
    FLBM_END_ITEMS
}

// Shell blocks of the replica first, then the blocks of its particle box.
static __global__ void __launch_bounds__(256) kb_shell(const RepDesc* __restrict__ reps,
                                                       const Item* __restrict__ items, int nitems)
{
    FLBM_FOR_ITEMS
    const int nbs = (int)((shell_count(P) + 255) / 256);
    if (it.y < nbs)
        shell_node(it.y * 256LL + threadIdx.x, sR.psi, sR.st, sR.masks, P);
    else
        virtual_node((it.y - nbs) * 256 + threadIdx.x, sR.psi, sR.st, sR.masks, P);
    FLBM_END_ITEMS
}

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(256, 3)
    kb_bulk(const RepDesc* __restrict__ reps, const Item* __restrict__ items, int nitems, int par)
{
    FLBM_FOR_ITEMS
    const TileCoord c = tile_of(it, P);
    bulk_tile<NOISE, TAU1>(c.bx, c.by, c.bz, c.tx, c.ty, sR.f[par], sR.f[1 - par], sR.psi, sR.st, P);
    FLBM_END_ITEMS
}

// Bulk collide with the replicas' descriptors as a kernel parameter (up to
// kChunkReps of them per launch): blockIdx.y picks the replica and blockIdx.x
// the tile. The descriptor's fields are then read from the constant bank at
// an index the same for the whole block, as a single simulation reads its
// kernel parameters, instead of from shared memory into registers: the
// kernel fits four blocks per SM. Blocks past the replica's tile count return.
constexpr int kChunkReps = 48;
struct RepChunk {
    RepDesc r[kChunkReps];
};
static_assert(sizeof(RepChunk) + 64 <= 32764, "kernel parameters are at most 32764 bytes");

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(256, 4) kb_bulk_rep(const __grid_constant__ RepChunk c, int par)
{
    const RepDesc& R = c.r[blockIdx.y];
    const KParams& P = R.P;
    const int plane = P.gx * P.gy;
    const int t = blockIdx.x;
    if (t >= plane * P.lz) return;
    const int bz = t / plane, w = t - bz * plane;
    const int by = w / P.gx, bx = w - by * P.gx;
    const int tx = threadIdx.x & (P.tx - 1), ty = threadIdx.x >> (__ffs(P.tx) - 1);
    bulk_tile<NOISE, TAU1>(bx, by, bz, tx, ty, R.f[par], R.f[1 - par], R.psi, R.st, P);
}

// Three blocks per SM: the register cap costs some spills, and the extra
// resident warps hide more of the near tiles' latency (measured faster).
template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(256, 3)
    kb_near(const RepDesc* __restrict__ reps, const Item* __restrict__ items, int nitems, int par)
{
    FLBM_FOR_ITEMS
    const TileCoord c = tile_of(it, P);
    near_tile<NOISE, TAU1>(c.bx, c.by, c.bz, c.tx, c.ty, threadIdx.x, sR.f[par],
                           sR.f[1 - par], sR.psi, sR.st, sR.masks, sR.partials, P);
    FLBM_END_ITEMS
}

static __global__ void __launch_bounds__(256) kb_mark_next(const RepDesc* __restrict__ reps,
                                                           const Item* __restrict__ items, int nitems)
{
    FLBM_FOR_ITEMS
    mark_next_block(it.y, sR.st, sR.masks, sR.box_counts, P);
    FLBM_END_ITEMS
}

static __global__ void __launch_bounds__(256) kb_cover(const RepDesc* __restrict__ reps,
                                                       const Item* __restrict__ items, int nitems, int par)
{
    FLBM_FOR_ITEMS
    cover_then_finish(it.y, sR.f[1 - par], sR.st, sR.masks, sR.box_parts, sR.box_counts, P);
    FLBM_END_ITEMS
}

static __global__ void __launch_bounds__(256) kb_finish(const RepDesc* __restrict__ reps,
                                                        const Item* __restrict__ items, int nitems)
{
    FLBM_FOR_ITEMS
    finish_step(sR.st, sR.box_counts, sR.box_parts, sR.box_blocks, P);
    __syncthreads();
    FLBM_END_ITEMS
}

#undef FLBM_FOR_ITEMS
#undef FLBM_END_ITEMS

// Work lists of one step, in launch order. The collide lists are split by
// kernel variant (noise on/off x all relaxation times 1 or not).
enum WorkKind {
    W_DENSITY = 0,
    W_SHELL,           // shell
    W_VIRT,            // virtual layer (blocks of kb_shell after the shell's)
    W_BULK,            // + variant (4 lists)
    W_NEAR = W_BULK + 4,  // + variant (4 lists)
    W_MARK = W_NEAR + 4,
    W_COVER,
    W_FINISH,
    W_COUNT
};

}  // namespace flbm_ensemble

using namespace flbm_ensemble;

struct flbm_ens {
    int n = 0;
    std::vector<flbm_params> p;
    std::vector<KParams> kp;       // for the current tile policy
    std::vector<RepDesc> rd;
    flbm_ens_config cfg{0, 4, 0};
    cudaStream_t stream = nullptr;
    // Virtual layers, near-particle collide and next-position masks on a
    // higher-priority side stream, concurrent with the shells and the bulk
    // collide (disjoint writes), forked (psi_ev, fork_ev) and joined by events.
    cudaStream_t side = nullptr;
    cudaEvent_t psi_ev = nullptr, fork_ev = nullptr, join_ev = nullptr;
    int nsm = 0;
    void* arena = nullptr;
    RepDesc* d_reps = nullptr;
    DevState* d_states = nullptr;  // n records, contiguous
    Item* d_items = nullptr;
    size_t items_cap = 0;
    long long off[W_COUNT + 1] = {};  // work list k = d_items[off[k] .. off[k+1])
    // Bulk collide launches of one block per tile (ctas_per_sm 0), per
    // variant: replicas of similar tile counts grouped, kChunkReps at most
    // per launch.
    struct RepLaunch {
        RepChunk c;
        int n = 0;
        int max_blocks = 0;
    };
    std::vector<RepLaunch> rep_launches[4];
    double* obs_tiles = nullptr;
    double* obs_out = nullptr;
    double* obs_mode_tiles = nullptr;
    double* obs_mode_out = nullptr;
    long long max_tiles = 0;
    int cur = 0;                   // all replicas read f[cur] in the next step
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_launches[2] = {0, 0};
    int64_t launches = 0;
    long long nodes = 0;
    std::string err;
};

namespace {

int efail(flbm_ens* e, int code, const std::string& msg)
{
    if (e) e->err = msg;
    return code;
}

#define ECK(e, call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return efail((e), FLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int elaunch(flbm_ens* e, const char* what)
{
    cudaError_t c = cudaGetLastError();
    if (c != cudaSuccess) return efail(e, FLBM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(c));
    e->launches += 1;
    return FLBM_OK;
}

int variant(const KParams& k) { return (k.kT > 0.0f ? 2 : 0) + (k.tau1 ? 1 : 0); }

// Blocks of replica r in work list w.
long long blocks_of(const KParams& k, int w)
{
    const bool part = k.has_particle != 0;
    if (w == W_DENSITY) return tile_count(k);
    if (w == W_SHELL) return (shell_count(k) + 255) / 256;
    if (w == W_VIRT) return part ? box_block_count(k) : 0;
    if (w >= W_BULK && w < W_BULK + 4) return variant(k) == w - W_BULK ? tile_count(k) : 0;
    if (w >= W_NEAR && w < W_NEAR + 4) return (part && variant(k) == w - W_NEAR) ? cand_count(k) : 0;
    if (w == W_MARK || w == W_COVER) return part ? box_block_count(k) : 0;
    return part ? 0 : 1;  // W_FINISH: with a particle the cover launch finishes the step
}

void destroy_graphs(flbm_ens* e)
{
    for (int c = 0; c < 2; ++c) {
        if (e->graph[c]) cudaGraphExecDestroy(e->graph[c]);
        e->graph[c] = nullptr;
        e->graph_launches[c] = 0;
    }
}

// Kernel parameters, descriptors and work lists for configuration e->cfg.
int apply_config(flbm_ens* e)
{
    destroy_graphs(e);
    for (int r = 0; r < e->n; ++r) {
        make_kparams(e->p[r], e->cfg.tile_policy, e->kp[r]);
        e->rd[r].P = e->kp[r];
    }
    std::vector<int> order(e->n);
    std::iota(order.begin(), order.end(), 0);
    if (e->cfg.packing == 2)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e->kp[a].N > e->kp[b].N; });
    std::vector<Item> items;
    // Block b of replica r in list w, with its tile or candidate decoded.
    auto item = [&](int r, long long b, int w) {
        const KParams& k = e->kp[r];
        if (w == W_DENSITY || (w >= W_BULK && w < W_BULK + 4))
            return make_int4(r, (int)(b % k.gx), (int)(b / k.gx % k.gy), (int)(b / ((long long)k.gx * k.gy)));
        if (w >= W_NEAR && w < W_NEAR + 4)
            return make_int4(r, (int)(b % k.ncx), (int)(b / k.ncx % k.ncy), (int)(b / ((long long)k.ncx * k.ncy)));
        if (w == W_VIRT) return make_int4(r, (int)(blocks_of(k, W_SHELL) + b), 0, 0);
        return make_int4(r, (int)b, 0, 0);
    };
    for (int w = 0; w < W_COUNT; ++w) {
        e->off[w] = (long long)items.size();
        if (e->cfg.packing == 1) {
            long long most = 0;
            for (int r = 0; r < e->n; ++r) most = std::max(most, blocks_of(e->kp[r], w));
            for (long long b = 0; b < most; ++b)
                for (int r = 0; r < e->n; ++r)
                    if (b < blocks_of(e->kp[r], w)) items.push_back(item(r, b, w));
        } else {
            for (int r : order)
                for (long long b = 0, nb = blocks_of(e->kp[r], w); b < nb; ++b) items.push_back(item(r, b, w));
        }
    }
    e->off[W_COUNT] = (long long)items.size();
    // Bulk launches with descriptor chunks, per variant (group_by_blocks;
    // the blocks past a replica's own tiles return at once).
    for (int k = 0; k < 4; ++k) {
        std::vector<long long> tiles(e->n);
        for (int r = 0; r < e->n; ++r) {
            tiles[r] = blocks_of(e->kp[r], W_BULK + k);
            if (tiles[r] > 0x7fffffffLL) return efail(e, FLBM_E_INVAL, "too many tiles in one replica");
        }
        auto& ch = e->rep_launches[k];
        ch.clear();
        for (const auto& g : group_by_blocks(tiles, kChunkReps)) {
            ch.emplace_back();
            ch.back().max_blocks = (int)tiles[g[0]];
            for (int r : g) ch.back().c.r[ch.back().n++] = e->rd[r];
        }
    }
    if (items.size() > (size_t)0x7fffffff) return efail(e, FLBM_E_INVAL, "too many work items");
    if (items.size() > e->items_cap) {
        cudaFree(e->d_items);
        e->d_items = nullptr;
        e->items_cap = 0;
        if (cudaMalloc(&e->d_items, sizeof(Item) * items.size()) != cudaSuccess)
            return efail(e, FLBM_E_NOMEM, "work lists");
        e->items_cap = items.size();
    }
    ECK(e, cudaMemcpyAsync(e->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, e->stream));
    ECK(e, cudaMemcpyAsync(e->d_reps, e->rd.data(), sizeof(RepDesc) * e->n, cudaMemcpyHostToDevice, e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));  // host vectors go out of scope
    return FLBM_OK;
}

// Every replica back to its initial state (as flbm_create makes it).
int init_replicas(flbm_ens* e)
{
    destroy_graphs(e);
    std::vector<DevState> st(e->n);
    for (int r = 0; r < e->n; ++r) st[r] = initial_state(e->p[r], e->kp[r]);
    ECK(e, cudaMemcpyAsync(e->d_states, st.data(), sizeof(DevState) * e->n, cudaMemcpyHostToDevice, e->stream));
    for (int r = 0; r < e->n; ++r) {
        const KParams& k = e->kp[r];
        const RepDesc& d = e->rd[r];
        const size_t B3 = (size_t)k.B * k.B * k.B;
        ECK(e, cudaMemsetAsync(d.masks, 0, 2 * B3, e->stream));
        ECK(e, cudaMemsetAsync(d.psi, 0, sizeof(float) * 2 * k.padn, e->stream));
        k_init<<<dim3(k.gx, k.gy, k.lz), dim3(k.tx, k.ty, 1), 0, e->stream>>>(
            d.f[0], k, (float)e->p[r].rho_a0, (float)e->p[r].rho_b0, (float)e->p[r].init_pert);
        if (int rc = elaunch(e, "k_init")) return rc;
        ECK(e, cudaMemcpyAsync(d.f[1], d.f[0], sizeof(float) * 2 * 19 * k.N, cudaMemcpyDeviceToDevice, e->stream));
        if (k.has_particle) {
            k_mark<<<1, 1024, 0, e->stream>>>(d.st, d.masks, k);
            if (int rc = elaunch(e, "k_mark")) return rc;
        }
    }
    e->cur = 0;
    ECK(e, cudaStreamSynchronize(e->stream));
    return FLBM_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device memory of all replicas in one allocation; partials sized for the
// larger candidate grid of the two tile policies.
int allocate(flbm_ens* e)
{
    std::vector<size_t> at(e->n);
    size_t off = align256(sizeof(DevState) * e->n);
    struct Sizes {
        size_t f, psi, masks, partials, counts, parts;
    };
    std::vector<Sizes> sz(e->n);
    std::vector<int> nbox(e->n);
    for (int r = 0; r < e->n; ++r) {
        KParams k0, k1;
        make_kparams(e->p[r], 0, k0);
        make_kparams(e->p[r], 1, k1);
        const size_t B3 = (size_t)k0.B * k0.B * k0.B;
        const long long nb = box_block_count(k0);
        nbox[r] = (int)nb;
        sz[r] = {align256(sizeof(float) * 2 * 19 * k0.N), align256(sizeof(float) * 2 * k0.padn), align256(2 * B3),
                 align256(sizeof(double) * 8 * std::max(cand_count(k0), cand_count(k1))),
                 align256(sizeof(int) * nb), align256(sizeof(double) * 8 * nb)};
        at[r] = off;
        off += 2 * sz[r].f + sz[r].psi + sz[r].masks + sz[r].partials + sz[r].counts + sz[r].parts;
        e->nodes += k0.N;
        e->max_tiles = std::max({e->max_tiles, tile_count(k0), tile_count(k1)});
    }
    if (cudaMalloc(&e->arena, off) != cudaSuccess) return efail(e, FLBM_E_NOMEM, "ensemble state");
    ECK(e, cudaMemsetAsync(e->arena, 0, off, e->stream));
    if (cudaMalloc(&e->d_reps, sizeof(RepDesc) * e->n) != cudaSuccess ||
        cudaMalloc(&e->obs_tiles, sizeof(double) * 8 * e->max_tiles) != cudaSuccess ||
        cudaMalloc(&e->obs_out, sizeof(double) * 8) != cudaSuccess ||
        cudaMalloc(&e->obs_mode_tiles, sizeof(double) * kObsModes * e->max_tiles) != cudaSuccess ||
        cudaMalloc(&e->obs_mode_out, sizeof(double) * kObsModes) != cudaSuccess)
        return efail(e, FLBM_E_NOMEM, "ensemble descriptors");
    char* base = static_cast<char*>(e->arena);
    e->d_states = reinterpret_cast<DevState*>(base);
    for (int r = 0; r < e->n; ++r) {
        RepDesc& d = e->rd[r];
        std::memset(&d, 0, sizeof(d));
        char* q = base + at[r];
        d.f[0] = reinterpret_cast<float*>(q); q += sz[r].f;
        d.f[1] = reinterpret_cast<float*>(q); q += sz[r].f;
        d.psi = reinterpret_cast<float*>(q); q += sz[r].psi;
        d.masks = reinterpret_cast<uint8_t*>(q); q += sz[r].masks;
        d.partials = reinterpret_cast<double*>(q); q += sz[r].partials;
        d.box_counts = reinterpret_cast<int*>(q); q += sz[r].counts;
        d.box_parts = reinterpret_cast<double*>(q);
        d.st = e->d_states + r;
        d.box_blocks = nbox[r];
    }
    return FLBM_OK;
}

}  // namespace

namespace {

// Launch work list w of kernel K with its trailing arguments on stream s.
template <typename... Args>
int launch_on(flbm_ens* e, cudaStream_t s, int w, void (*kern)(const RepDesc*, const Item*, int, Args...),
              const char* what, Args... args)
{
    const long long nitems = e->off[w + 1] - e->off[w];
    if (nitems == 0) return FLBM_OK;
    long long grid = nitems;
    if (e->cfg.ctas_per_sm > 0) grid = std::min(grid, (long long)e->cfg.ctas_per_sm * e->nsm);
    kern<<<(unsigned)grid, 256, 0, s>>>(e->d_reps, e->d_items + e->off[w], (int)nitems, args...);
    return elaunch(e, what);
}

template <typename... Args>
int launch_list(flbm_ens* e, int w, void (*kern)(const RepDesc*, const Item*, int, Args...), const char* what,
                Args... args)
{
    return launch_on(e, e->stream, w, kern, what, args...);
}

// The bulk collide launches with descriptor chunks.
int launch_bulk_reps(flbm_ens* e, int par)
{
    void (*kern[4])(const RepChunk, int) = {kb_bulk_rep<false, false>, kb_bulk_rep<false, true>,
                                            kb_bulk_rep<true, false>, kb_bulk_rep<true, true>};
    for (int k = 0; k < 4; ++k)
        for (const auto& ch : e->rep_launches[k]) {
            kern[k]<<<dim3((unsigned)ch.max_blocks, (unsigned)ch.n), 256, 0, e->stream>>>(ch.c, par);
            if (int rc = elaunch(e, "kb_bulk_rep")) return rc;
        }
    return FLBM_OK;
}

// One step of every replica: reads f[cur], writes f[1 - cur].
int ens_step(flbm_ens* e)
{
    const int par = e->cur;
    if (int rc = launch_list(e, W_DENSITY, kb_density, "kb_density", par)) return rc;
    // The particles' share of the step runs on the side stream: the virtual
    // layers once the densities are in, the near tiles once the shells are
    // in too, then the next-position masks. The shells and the bulk tiles,
    // which read neither, run on the main stream meanwhile.
    const bool near = e->off[W_NEAR + 4] > e->off[W_NEAR];
    if (near) {
        ECK(e, cudaEventRecord(e->psi_ev, e->stream));
        ECK(e, cudaStreamWaitEvent(e->side, e->psi_ev, 0));
        if (int rc = launch_on(e, e->side, W_VIRT, kb_shell, "kb_shell")) return rc;
    } else if (int rc = launch_list(e, W_VIRT, kb_shell, "kb_shell")) {
        return rc;
    }
    if (int rc = launch_list(e, W_SHELL, kb_shell, "kb_shell")) return rc;
    if (near) {
        ECK(e, cudaEventRecord(e->fork_ev, e->stream));
        ECK(e, cudaStreamWaitEvent(e->side, e->fork_ev, 0));
        if (int rc = launch_on(e, e->side, W_NEAR + 0, kb_near<false, false>, "kb_near", par)) return rc;
        if (int rc = launch_on(e, e->side, W_NEAR + 1, kb_near<false, true>, "kb_near", par)) return rc;
        if (int rc = launch_on(e, e->side, W_NEAR + 2, kb_near<true, false>, "kb_near", par)) return rc;
        if (int rc = launch_on(e, e->side, W_NEAR + 3, kb_near<true, true>, "kb_near", par)) return rc;
        if (int rc = launch_on(e, e->side, W_MARK, kb_mark_next, "kb_mark_next")) return rc;
        ECK(e, cudaEventRecord(e->join_ev, e->side));
    }
    if (e->cfg.ctas_per_sm == 0) {
        if (int rc = launch_bulk_reps(e, par)) return rc;
    } else {
        if (int rc = launch_list(e, W_BULK + 0, kb_bulk<false, false>, "kb_bulk", par)) return rc;
        if (int rc = launch_list(e, W_BULK + 1, kb_bulk<false, true>, "kb_bulk", par)) return rc;
        if (int rc = launch_list(e, W_BULK + 2, kb_bulk<true, false>, "kb_bulk", par)) return rc;
        if (int rc = launch_list(e, W_BULK + 3, kb_bulk<true, true>, "kb_bulk", par)) return rc;
    }
    if (near) ECK(e, cudaStreamWaitEvent(e->stream, e->join_ev, 0));
    else if (int rc = launch_list(e, W_MARK, kb_mark_next, "kb_mark_next")) return rc;
    if (int rc = launch_list(e, W_COVER, kb_cover, "kb_cover", par)) return rc;
    if (int rc = launch_list(e, W_FINISH, kb_finish, "kb_finish")) return rc;
    e->cur = 1 - e->cur;
    return FLBM_OK;
}

// Two steps from cur = c captured into e->graph[c] (once per configuration).
int ens_graph(flbm_ens* e, int c)
{
    if (e->graph[c]) return FLBM_OK;
    const int64_t before = e->launches;
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    int rc = ens_step(e);
    if (!rc) rc = ens_step(e);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return efail(e, FLBM_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&e->graph[c], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        e->graph[c] = nullptr;
        return efail(e, FLBM_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    }
    e->graph_launches[c] = e->launches - before;
    e->launches = before;
    return FLBM_OK;
}

int ens_advance(flbm_ens* e, int64_t nsteps)
{
    int64_t s = 0;
    if (e->stream != nullptr) {
        for (; s + 2 <= nsteps; s += 2) {
            if (int rc = ens_graph(e, e->cur)) return rc;
            ECK(e, cudaGraphLaunch(e->graph[e->cur], e->stream));
            e->launches += e->graph_launches[e->cur];
        }
    }
    for (; s < nsteps; ++s)
        if (int rc = ens_step(e)) return rc;
    return FLBM_OK;
}

bool config_ok(const flbm_ens_config& c)
{
    return c.packing >= 0 && c.packing <= 2 && c.ctas_per_sm >= 0 && c.ctas_per_sm <= 8 && c.tile_policy >= 0 &&
           c.tile_policy <= 1;
}

}  // namespace

extern "C" {

int flbm_ensemble_create(const flbm_params* p, int32_t n, const flbm_ens_config* cfg, void* stream,
                         flbm_ens_t** out)
{
    if (!out) return FLBM_E_INVAL;
    *out = nullptr;
    if (!p || n < 1) return FLBM_E_INVAL;
    if (cfg && !config_ok(*cfg)) {
        std::fprintf(stderr, "flbm_ensemble_create: invalid configuration\n");
        return FLBM_E_INVAL;
    }
    for (int r = 0; r < n; ++r) {
        const std::string v = validate(p + r);
        if (!v.empty()) {
            std::fprintf(stderr, "flbm_ensemble_create: replica %d: %s\n", r, v.c_str());
            return FLBM_E_INVAL;
        }
    }
    flbm_ens* e = new (std::nothrow) flbm_ens();
    if (!e) return FLBM_E_NOMEM;
    e->n = n;
    e->p.assign(p, p + n);
    e->kp.resize(n);
    e->rd.resize(n);
    if (cfg) e->cfg = *cfg;
    e->stream = (cudaStream_t)stream;
    int dev = 0, lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&e->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->psi_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        flbm_ensemble_destroy(e);
        return FLBM_E_CUDA;
    }
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        flbm_ensemble_destroy(e);
        return FLBM_E_CUDA;
    }
    int rc = allocate(e);
    if (!rc) rc = apply_config(e);
    if (!rc) rc = init_replicas(e);
    if (rc) {
        std::fprintf(stderr, "flbm_ensemble_create: %s\n", e->err.c_str());
        flbm_ensemble_destroy(e);
        return rc;
    }
    *out = e;
    return FLBM_OK;
}

int flbm_ensemble_step(flbm_ens_t* e, int64_t nsteps)
{
    if (!e || nsteps < 0) return efail(e, FLBM_E_INVAL, "invalid handle or step count");
    e->launches = 0;
    return ens_advance(e, nsteps);
}

int flbm_ensemble_tune(flbm_ens_t* e, int32_t steps, flbm_ens_config* best, double* ms_best)
{
    if (!e || steps < 2) return efail(e, FLBM_E_INVAL, "tuning needs at least 2 steps per candidate");
    cudaEvent_t t0, t1;
    ECK(e, cudaEventCreate(&t0));
    if (cudaEventCreate(&t1) != cudaSuccess) {
        cudaEventDestroy(t0);
        return efail(e, FLBM_E_CUDA, "cudaEventCreate");
    }
    const flbm_ens_config start = e->cfg;
    flbm_ens_config pick = start;
    double pick_ms = 1e300;
    int rc = FLBM_OK;
    for (int pol = 0; pol <= 1 && !rc; ++pol)
        for (int pk = 0; pk <= 2 && !rc; ++pk)
            for (int ct : {0, 2, 4}) {
                e->cfg = flbm_ens_config{pk, ct, pol};
                if ((rc = apply_config(e))) break;
                if ((rc = ens_advance(e, 2))) break;  // warm-up and graph capture
                cudaEventRecord(t0, e->stream);
                if ((rc = ens_advance(e, steps))) break;
                cudaEventRecord(t1, e->stream);
                if (cudaEventSynchronize(t1) != cudaSuccess) {
                    rc = efail(e, FLBM_E_CUDA, "tuning run failed");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ms / steps < pick_ms) {
                    pick_ms = ms / steps;
                    pick = e->cfg;
                }
            }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) return rc;
    e->cfg = pick;
    if ((rc = apply_config(e)) || (rc = init_replicas(e))) return rc;
    if (best) *best = pick;
    if (ms_best) *ms_best = pick_ms;
    return FLBM_OK;
}

int flbm_ensemble_config(const flbm_ens_t* e, flbm_ens_config* out)
{
    if (!e || !out) return FLBM_E_INVAL;
    *out = e->cfg;
    return FLBM_OK;
}

int flbm_ensemble_particles(flbm_ens_t* e, flbm_particle* out)
{
    if (!e || !out) return efail(e, FLBM_E_INVAL, "NULL argument");
    std::vector<DevState> st(e->n);
    ECK(e, cudaMemcpyAsync(st.data(), e->d_states, sizeof(DevState) * e->n, cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    for (int r = 0; r < e->n; ++r) copy_particle(st[r], out + r);
    return FLBM_OK;
}

int flbm_ensemble_read_fields(flbm_ens_t* e, int32_t r, float* host_f)
{
    if (!e || !host_f || r < 0 || r >= e->n) return efail(e, FLBM_E_INVAL, "invalid argument");
    ECK(e, cudaMemcpyAsync(host_f, e->rd[r].f[e->cur], sizeof(float) * 2 * 19 * e->kp[r].N, cudaMemcpyDeviceToHost,
                           e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    return FLBM_OK;
}

int flbm_ensemble_observables(flbm_ens_t* e, int32_t r, flbm_obs* out)
{
    if (!e || !out || r < 0 || r >= e->n) return efail(e, FLBM_E_INVAL, "invalid argument");
    const KParams& k = e->kp[r];
    const RepDesc& d = e->rd[r];
    k_obs_tiles<<<dim3(k.gx, k.gy, k.lz), dim3(k.tx, k.ty, 1), 0, e->stream>>>(d.f[e->cur], d.st, d.masks,
                                                                               e->obs_tiles, k);
    if (int rc = elaunch(e, "k_obs_tiles")) return rc;
    k_obs_final<<<1, 1024, 0, e->stream>>>(e->obs_tiles, tile_count(k), e->obs_out);
    if (int rc = elaunch(e, "k_obs_final")) return rc;
    k_obs_modes<<<dim3(k.gx, k.gy, k.lz), dim3(k.tx, k.ty, 1), 0, e->stream>>>(d.f[e->cur], d.st, d.masks,
                                                                               e->obs_mode_tiles, k);
    if (int rc = elaunch(e, "k_obs_modes")) return rc;
    k_obs_final_n<kObsModes><<<1, 1024, 0, e->stream>>>(e->obs_mode_tiles, tile_count(k), e->obs_mode_out);
    if (int rc = elaunch(e, "k_obs_final_n")) return rc;
    double v[8], vm[kObsModes];
    DevState s;
    ECK(e, cudaMemcpyAsync(v, e->obs_out, sizeof(v), cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaMemcpyAsync(vm, e->obs_mode_out, sizeof(vm), cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaMemcpyAsync(&s, d.st, sizeof(s), cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    fill_obs(v, s, out);
    fill_mode_obs(vm, out);
    return out->nonfinite ? efail(e, FLBM_E_NONFINITE, "non-finite populations") : FLBM_OK;
}

int64_t flbm_ensemble_nodes(const flbm_ens_t* e) { return e ? e->nodes : 0; }

int64_t flbm_ensemble_last_launch_count(const flbm_ens_t* e) { return e ? e->launches : 0; }

const char* flbm_ensemble_last_error(const flbm_ens_t* e) { return e ? e->err.c_str() : ""; }

void flbm_ensemble_destroy(flbm_ens_t* e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    else cudaDeviceSynchronize();
    destroy_graphs(e);
    if (e->side) {
        cudaStreamSynchronize(e->side);
        cudaStreamDestroy(e->side);
    }
    if (e->psi_ev) cudaEventDestroy(e->psi_ev);
    if (e->fork_ev) cudaEventDestroy(e->fork_ev);
    if (e->join_ev) cudaEventDestroy(e->join_ev);
    cudaFree(e->arena);
    cudaFree(e->d_reps);
    cudaFree(e->d_items);
    cudaFree(e->obs_tiles);
    cudaFree(e->obs_out);
    cudaFree(e->obs_mode_tiles);
    cudaFree(e->obs_mode_out);
    delete e;
}

}  // extern "C"

// Bulk collide-stream with its inputs staged by the Tensor Memory Accelerator
// (arXiv:1909.01092, Section 2: Eq. (lbe), Eq. (sc-force)).
//
// The same node update as k_collide_bulk (collide_core), for lattices whose
// rows are a multiple of 16 bytes (lx % 4 == 0) and whose tiles are 32 x 8
// nodes of one z-plane. A persistent grid (two blocks per SM) walks the
// tiles that are not next to the particle. For each tile one thread issues
// two tensor copies into a shared-memory stage: the 38 populations of the
// tile's 256 nodes (38 x 8 x 32 floats) and the padded densities the
// Shan-Chen stencil reads (2 components x 3 planes x 10 rows x 36 columns).
// Two stages alternate: while the block works on one tile, the copies of its
// next tile are in flight, so the HBM reads no longer wait on the warps. The
// stores of the streamed populations go straight to global memory as before.
//
// Every wait on a stage's mbarrier is bounded: the waits for a tile's inputs
// by the launch's wait_cycles (default about a second of SM clock, set with
// flbm_set_tma_wait), the final waits for a leaving block's own copies by
// that default. A block that gives up sets DevState::err, waits for its
// copies still in flight and returns; the host reports FLBM_E_TIMEOUT.
#pragma once

#include <cuda.h>

#include "flbm_step.cuh"

namespace flbm {

constexpr int kTmaTX = 32, kTmaTY = 8;                 // tile: 256 nodes of one plane
constexpr int kTmaPX = kTmaTX + 4;                     // psi box row: x0 - 1 .. x0 + 32, padded to 16 bytes
constexpr int kTmaPY = kTmaTY + 2;                     // psi box rows: y0 - 1 .. y0 + 8
constexpr int kTmaFBytes = 38 * kTmaTX * kTmaTY * 4;   // 38912
constexpr int kTmaPsiBytes = 2 * 3 * kTmaPY * kTmaPX * 4;  // 8640
constexpr int kTmaStageBytes = (kTmaFBytes + kTmaPsiBytes + 127) / 128 * 128;
constexpr int kTmaSmemBytes = 2 * kTmaStageBytes + 16;  // two stages and two mbarriers
constexpr long long kTmaWaitCycles = 1LL << 31;         // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity` of the mbarrier.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the mbarrier for at most `limit` SM cycles.
// With the default limit the thread waits in try_wait, which the hardware may
// suspend until the phase completes. A shorter limit polls with test_wait,
// which returns at once, so that the limit itself decides.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit = kTmaWaitCycles)
{
    const long long t0 = clock64();
    if (limit >= kTmaWaitCycles) {
        while (!mbar_try_wait(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    while (!mbar_test_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// 4-D tiled tensor copy global -> shared, completing on the mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Inputs of node (tx, ty) of the tile held in one shared-memory stage.
struct StagedInputs {
    const float* f_;  // population q at f_[256 q]
    const float* p_;  // psi_A at the node; neighbour i at p_[off(i)], psi_B one component further
    __device__ __forceinline__ StagedInputs(const float* stage, int tx, int ty)
        : f_(stage + ty * kTmaTX + tx),
          p_(stage + kTmaFBytes / 4 + (kTmaPY + ty + 1) * kTmaPX + tx + 1)
    {
    }
    __device__ __forceinline__ float f(int q, const KParams&) const { return f_[q * kTmaTX * kTmaTY]; }
    static __device__ __forceinline__ int off(int i) { return cxv(i) + kTmaPX * (cyv(i) + kTmaPY * czv(i)); }
    __device__ __forceinline__ float psa(int i) const { return p_[off(i)]; }
    __device__ __forceinline__ float psb(int i) const { return p_[3 * kTmaPY * kTmaPX + off(i)]; }
};

// Tile t of the plane-tile grid (x fastest, as the grid of k_collide_bulk).
__device__ __forceinline__ void tile_coords(long long t, const KParams& P, int& bx, int& by, int& bz)
{
    bx = (int)(t % P.gx);
    const long long r = t / P.gx;
    by = (int)(r % P.gy);
    bz = (int)(r / P.gy);
}

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(kThreadsStep, 2)
    k_collide_bulk_tma(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_psi,
                       float* __restrict__ fout, DevState* __restrict__ st, KParams P, long long wait_cycles)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool leader = tx == 0 && ty == 0;
    const uint32_t s0 = smem_addr(smem);
    const uint32_t bar = s0 + 2 * kTmaStageBytes;  // bar + 8 s: mbarrier of stage s
    const long long ntiles = (long long)P.gx * P.gy * P.lz;
    const long long G = gridDim.x;

    int o[3] = {0, 0, 0};
    if (P.has_particle) {
        o[0] = st->box0[0];
        o[1] = st->box0[1];
        o[2] = st->box0[2];
    }
    // The tiles of this block: blockIdx.x + k G, skipping the near tiles.
    auto skip = [&](long long t) {
        int bx, by, bz;
        tile_coords(t, P, bx, by, bz);
        return P.has_particle && tile_near(bx, by, bz, o, P);
    };
    auto next = [&](long long t) {
        if (t >= ntiles) return ntiles;
        t += G;
        while (t < ntiles && skip(t)) t += G;
        return t < ntiles ? t : ntiles;
    };
    auto issue = [&](long long t, int s) {
        int bx, by, bz;
        tile_coords(t, P, bx, by, bz);
        const uint32_t b = bar + 8 * s;
        mbar_expect_tx(b, (uint32_t)(kTmaFBytes + kTmaPsiBytes));
        // Populations: box (32, 8, 1, 38) at (x0, y0, z, 0). Densities: box
        // (36, 10, 3, 2) at padded (x0, y0, z, 0), i.e. nodes x0 - 1, y0 - 1, z - 1.
        tma_load_4d(s0 + s * kTmaStageBytes, &tm_f, bx * kTmaTX, by * kTmaTY, bz, 0, b);
        tma_load_4d(s0 + s * kTmaStageBytes + kTmaFBytes, &tm_psi, bx * kTmaTX, by * kTmaTY, bz, 0, b);
    };

    if (s0 & 127u) {  // tensor copies need 128-byte aligned stages
        if (leader) atomicExch(&st->err, 2);
        return;
    }
    long long t = blockIdx.x < ntiles ? blockIdx.x : ntiles;
    if (t < ntiles && skip(t)) t = next(t);
    long long tn = next(t);
    if (leader) {
        mbar_init(bar, 1);
        mbar_init(bar + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (t < ntiles) issue(t, 0);
        if (tn < ntiles) issue(tn, 1);
    }
    __syncthreads();

    for (int k = 0; t < ntiles; ++k) {
        const int s = k & 1;
        const bool ready = mbar_wait_bounded(bar + 8 * s, (uint32_t)(k >> 1) & 1u, wait_cycles);
        if (__syncthreads_or(!ready)) {  // the whole block leaves together
            if (leader) atomicExch(&st->err, 1);
            // Let the copies this block issued land before its shared memory is released.
            mbar_wait_bounded(bar + 8 * s, (uint32_t)(k >> 1) & 1u);
            if (tn < ntiles) mbar_wait_bounded(bar + 8 * (1 - s), (uint32_t)((k + 1) >> 1) & 1u);
            return;
        }
        int bx, by, bz;
        tile_coords(t, P, bx, by, bz);
        const int x = bx * kTmaTX + tx, y = by * kTmaTY + ty;
        if (x < P.lx && y < P.ly) {
            const uint32_t n = (uint32_t)x + (uint32_t)P.lx * ((uint32_t)y + (uint32_t)P.ly * (uint32_t)bz);
            const StagedInputs in(reinterpret_cast<const float*>(smem + s * kTmaStageBytes), tx, ty);
            collide_core<NOISE, false, TAU1>(x, y, bz, n, in, fout, st, P, 0u, nullptr);
        }
        __syncthreads();  // every thread is done with stage s
        const long long t2 = next(tn);
        if (leader && t2 < ntiles) issue(t2, s);
        t = tn;
        tn = t2;
    }
}

}  // namespace flbm

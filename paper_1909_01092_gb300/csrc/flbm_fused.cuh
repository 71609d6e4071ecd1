// Fused collide-stream that also produces the next step's densities
// (arXiv:1909.01092, Section 2: Eq. (density), Eq. (lbe), Eq. (sc-force)).
//
// The Shan-Chen force of step t + 1 needs rho_l(x, t + 1) = sum_i f_li(x, t + 1)
// at every node. In the push scheme those 19 values are exactly what the
// collide of step t writes into the node's slots, so the collide can sum them
// on the fly instead of a separate pass re-reading all 38 populations per
// node (152 B/node, a quarter of the two-pass step's time).
//
// Work split. A block owns one tile column (TX x TY nodes, TX >= 8) over a
// chunk of K consecutive planes and walks the chunk in z. For each plane it
// collides and pushes its nodes as k_collide_bulk does, and every pushed
// value goes to a receiver (DensitySink):
//   - the node's own column (rest population, +z, -z, and everything a wall
//     bounced back into the node) is summed in registers;
//   - the 16 values that leave the column go to shared memory, one array per
//     direction; after a barrier each thread gathers, for its own column, the
//     values its neighbours in the tile pushed into it.
// Each thread keeps two rolling partial sums per component in shared memory:
// the densities of its column at planes z and z + 1. The density of plane
// z - 1 is complete once plane z has been pushed. Values bound for columns
// outside the tile are gathered the same way by "ring" threads, one per
// node of the one-node ring around the tile, and stored per (tile, plane,
// ring slot). Values bound for the planes just below and above the chunk are
// stored per (tile, chunk, side, footprint position): the "seams".
//
// k_psi_finish then completes the field:
//   - part B: nodes on a tile edge or on a chunk's first or last plane add
//     the ring and seam partials of the neighbouring blocks, in a fixed order;
//   - part A: nodes within one node of a tile the near-particle collide ran
//     (their sources bounced off the moving sphere, were covered or refilled)
//     are summed directly from the populations after cover/uncover, and
//     particle nodes get 0, as k_density does.
// Every sum is taken in a fixed order, so runs are bit-reproducible. Summation
// order differs from k_density's, so the two paths agree to float32 rounding.
//
// Requirements (checked by fused_ok): TX >= 8 (at most 84 ring slots, one per
// thread), and at least 3 tiles along a periodic x or y (the neighbouring
// tiles on either side are then distinct).
#pragma once

#include "flbm_kernels.cuh"

namespace flbm {

// Chunks of planes per block and the sizes of the ring and seam buffers.
struct FusedGeom {
    int K;       // planes per block: chunk c holds planes [c K, min((c + 1) K, lz))
    int nchunk;  // chunks along z
    int ring;    // ring slots per tile and plane: 2 (TX + 2) + 2 TY
    int fp;      // footprint positions per tile: (TX + 2) (TY + 2)
};

constexpr int kRingMax = 84;  // 2 (TX + 2) + 2 TY for TX >= 8, TX TY = 256
constexpr int kXchDirs = 16;  // directions that leave the node's column

// The 16 directions that change x or y, in slot order, and back.
__host__ __device__ constexpr int xch_slot(int i) { return i <= 4 ? i - 1 : i - 3; }
__host__ __device__ constexpr int xch_dir(int s) { return s < 4 ? s + 1 : s + 3; }

__host__ __device__ __forceinline__ bool fused_ok(const KParams& P)
{
    return P.tx >= 8 && (P.wall[0] || P.gx >= 3) && (P.wall[1] || P.gy >= 3);
}

__host__ __device__ __forceinline__ int tile_w(int bx, const KParams& P) { return min(P.tx, P.lx - bx * P.tx); }
__host__ __device__ __forceinline__ int tile_h(int by, const KParams& P) { return min(P.ty, P.ly - by * P.ty); }

// Ring slot of position (fx, fy), relative to the corner of a tile of extent
// w x h: south row (fy = -1), north row (fy = h), west column (fx = -1) and
// east column (fx = w), corners in the rows. -1 inside the tile or outside
// the one-node ring.
__host__ __device__ __forceinline__ int ring_slot(int fx, int fy, int w, int h, const KParams& P)
{
    if (fx < -1 || fx > w || fy < -1 || fy > h) return -1;
    const int R = P.tx + 2;
    if (fy == -1) return fx + 1;
    if (fy == h) return R + fx + 1;
    if (fx == -1) return 2 * R + fy;
    if (fx == w) return 2 * R + P.ty + fy;
    return -1;
}

// Position of ring slot r of a tile of extent w x h; false if the tile does
// not use that slot.
__host__ __device__ __forceinline__ bool ring_pos(int r, int w, int h, const KParams& P, int& fx, int& fy)
{
    const int R = P.tx + 2;
    if (r < R) { fx = r - 1; fy = -1; return fx <= w; }
    if (r < 2 * R) { fx = r - R - 1; fy = h; return fx <= w; }
    if (r < 2 * R + P.ty) { fx = -1; fy = r - 2 * R; return fy < h; }
    if (r < 2 * R + 2 * P.ty) { fx = w; fy = r - 2 * R - P.ty; return fy < h; }
    return false;
}

__host__ __device__ __forceinline__ int fp_index(int fx, int fy, const KParams& P) { return (fx + 1) + (P.tx + 2) * (fy + 1); }

// Is position (fx, fy) of tile (bx, by) a node of the lattice (not across a wall)?
__host__ __device__ __forceinline__ bool fp_node(int bx, int by, int fx, int fy, const KParams& P)
{
    const int x = bx * P.tx + fx, y = by * P.ty + fy;
    return !(P.wall[0] && (x < 0 || x >= P.lx)) && !(P.wall[1] && (y < 0 || y >= P.ly));
}

__host__ __device__ __forceinline__ long long ring_index(int tile, int z, int slot, const KParams& P, const FusedGeom& G)
{
    return ((long long)tile * P.lz + z) * G.ring + slot;
}

// side 0: plane z0 - 1 below the chunk; side 1: plane z1 above it.
__host__ __device__ __forceinline__ long long seam_index(int tile, int c, int side, int pos, const FusedGeom& G)
{
    return (((long long)tile * G.nchunk + c) * 2 + side) * G.fp + pos;
}

// Near-particle region of the step, dilated by one node: the nodes with a
// node of a near tile (tile_near with the box origin o the step's collide
// used) among their 26 neighbours or themselves. tile_near is a product of
// one test per axis, so the dilated set is too.
__host__ __device__ __forceinline__ bool near_dilated(int x, int y, int z, const int o[3], const KParams& P)
{
    const int B2 = P.B + 2;
    bool nx = false, ny = false, nz = false;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int q = x + d;
        if (q < 0 || q >= P.lx) {
            if (P.wall[0]) continue;
            q += q < 0 ? P.lx : -P.lx;
        }
        const int b = q / P.tx;
        nx = nx || ranges_meet(b * P.tx, min(P.tx, P.lx - b * P.tx), o[0] - 1, B2, P.lx, P.wall[0]);
    }
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int q = y + d;
        if (q < 0 || q >= P.ly) {
            if (P.wall[1]) continue;
            q += q < 0 ? P.ly : -P.ly;
        }
        const int b = q / P.ty;
        ny = ny || ranges_meet(b * P.ty, min(P.ty, P.ly - b * P.ty), o[1] - 1, B2, P.ly, P.wall[1]);
    }
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int q = z + d;
        if (q < 0 || q >= P.lz) {
            if (P.wall[2]) continue;
            q += q < 0 ? P.lz : -P.lz;
        }
        nz = nz || ranges_meet(q, 1, o[2] - 1, B2, P.lz, P.wall[2]);
    }
    return nx && ny && nz;
}

// One axis of the box part A walks: start (one node before the first
// candidate tile) and length (candidate tiles plus one node on either side,
// at most the axis on a periodic axis, so that no node is visited twice).
__host__ __device__ __forceinline__ void near_box_axis(int o, int T, int nc, int g, int L, int wall, int& start, int& len)
{
    start = candidate_tile(0, o, T, g, L, wall) * T - 1;
    len = nc * T + 2;
    if (!wall && len > L) len = L;
}

// Shared-memory exchange of the values that leave a node's column: per
// direction one float2 (A, B) array over the tile padded by two columns on
// either side and one row above and below, (TX + 4) x (TY + 2). The padding
// and the cells of a ragged tile's missing nodes are zero and stay zero, so
// a column (or a ring position) gathers its incoming values at fixed offsets
// without tests: values from outside the tile read as 0.
__host__ __device__ __forceinline__ int xch_pitch(const KParams& P) { return P.tx + 4; }
__host__ __device__ __forceinline__ int xch_size(const KParams& P) { return (P.tx + 4) * (P.ty + 2); }
__host__ __device__ __forceinline__ int xch_pos(int fx, int fy, const KParams& P) { return (fx + 2) + (P.tx + 4) * (fy + 1); }
__host__ __device__ __forceinline__ size_t fused_smem_bytes(const KParams& P)
{
    return sizeof(float2) * (size_t)(kXchDirs * xch_size(P) + 2 * kThreadsStep + 2 * kRingMax);
}

// Receiver of one node's pushed populations (see collide_core): the own
// column's contributions per component to the planes z - 1, z, z + 1
// (everything a wall bounced back counts for plane z), and the 16 values
// leaving the column into the exchange arrays (component l in .x or .y).
struct DensitySink {
    static constexpr bool active = true;
    float* xch;  // float2 [16][xch_size], viewed as floats
    int pos;     // xch_pos of the node
    int size;    // xch_size
    float own[2][3];
    __host__ __device__ __forceinline__ DensitySink(float* x, int p, int sz) : xch(x), pos(p), size(sz)
    {
#pragma unroll
        for (int l = 0; l < 2; ++l) own[l][0] = own[l][1] = own[l][2] = 0.0f;
    }
    __host__ __device__ __forceinline__ void put(int l, int i, float v, bool bounced)
    {
        if (i == 0) {
            own[l][1] += v;
            return;
        }
        if (bounced) own[l][1] += v;
        if (i == 5) {
            if (!bounced) own[l][2] += v;
        } else if (i == 6) {
            if (!bounced) own[l][0] += v;
        } else {
            // A bounced value is stored too: its target lies across the wall,
            // where no node and no ring position gathers it.
            xch[2 * (xch_slot(i) * size + pos) + l] = v;
        }
    }
};

// Values pushed into the column at exchange position p from the tile's
// nodes at the plane just pushed, per destination plane (index cz + 1). For
// a node of the tile all 16 directions; the missing ones read as 0.
__host__ __device__ __forceinline__ void gather_column(int p, const float2* xch, const KParams& P, float2 inc[3])
{
    const int pitch = xch_pitch(P), size = xch_size(P);
#pragma unroll
    for (int s = 0; s < kXchDirs; ++s) {
        const int d = xch_dir(s);
        const float2 v = xch[s * size + p - cxv(d) - pitch * cyv(d)];
        inc[czv(d) + 1].x += v.x;
        inc[czv(d) + 1].y += v.y;
    }
}

// The same for a ring position on side `side` (0 south row, 1 north row, 2
// west column, 3 east column): only the five directions that cross that side
// can bring values from the tile (corners lie in the rows and read zeros
// for the directions that miss the tile).
__host__ __device__ __forceinline__ void gather_ring(int side, int p, const float2* xch, const KParams& P,
                                                     float2 inc[3])
{
    const int pitch = xch_pitch(P), size = xch_size(P);
#pragma unroll
    for (int s = 0; s < kXchDirs; ++s) {
        const int d = xch_dir(s);
        const bool take = side == 0 ? cyv(d) < 0 : side == 1 ? cyv(d) > 0 : side == 2 ? cxv(d) < 0 : cxv(d) > 0;
        if (!take) continue;
        const float2 v = xch[s * size + p - cxv(d) - pitch * cyv(d)];
        inc[czv(d) + 1].x += v.x;
        inc[czv(d) + 1].y += v.y;
    }
}

// Side of ring slot r (see ring_pos).
__host__ __device__ __forceinline__ int ring_side(int r, const KParams& P)
{
    const int R = P.tx + 2;
    return r < R ? 0 : r < 2 * R ? 1 : r < 2 * R + P.ty ? 2 : 3;
}

// Stores a density (both components) of destination plane zd for footprint
// position (fx, fy) of the block's tile: the tile's own nodes into psi_next
// (zd inside the chunk), ring positions into the ring buffer, and the planes
// just outside the chunk into the seams. Planes across a z wall are skipped.
__host__ __device__ __forceinline__ void put_density(int zd, int fx, int fy, bool in_tile, int slot, float2 v,
                                                     int tile, int bx, int by, int c, int z0, int z1,
                                                     float* __restrict__ psi_next, float2* __restrict__ ring,
                                                     float2* __restrict__ seam, const KParams& P,
                                                     const FusedGeom& G)
{
    if (zd >= z0 && zd < z1) {
        if (in_tile) {
            const long long q = pad_index(bx * P.tx + fx, by * P.ty + fy, zd, P);
            psi_next[q] = v.x;
            psi_next[P.padn + q] = v.y;
        } else {
            ring[ring_index(tile, zd, slot, P, G)] = v;
        }
        return;
    }
    if ((zd < 0 || zd >= P.lz) && P.wall[2]) return;
    const int side = zd < z0 ? 0 : 1;
    seam[seam_index(tile, c, side, fp_index(fx, fy, P), G)] = v;
}

// One plane's update of a column's rolling sums, for the plane z just
// pushed. Before, roll[0] and roll[1] hold the partial densities (A, B) of
// planes z - 1 and z; after, those of planes z and z + 1, and the result is
// the complete density of plane z - 1. own: the column's own contributions
// to planes z - 1, z, z + 1 (none for ring positions); inc: what the tile's
// other nodes pushed into the column, per destination plane.
__host__ __device__ __forceinline__ float2 roll_update(float2 roll[2], const float own[2][3], const float2 inc[3])
{
    const float2 r = make_float2(roll[0].x + own[0][0] + inc[0].x, roll[0].y + own[1][0] + inc[0].y);
    roll[0] = make_float2(roll[1].x + own[0][1] + inc[1].x, roll[1].y + own[1][1] + inc[1].y);
    roll[1] = make_float2(own[0][2] + inc[2].x, own[1][2] + inc[2].y);
    return r;
}

// Does tile (bx, by) meet the particle box grown by one node in x and y
// (tile_near without its z test)?
__host__ __device__ __forceinline__ bool tile_near_xy(int bx, int by, const int o[3], const KParams& P)
{
    const int B2 = P.B + 2;
    return ranges_meet(bx * P.tx, min(P.tx, P.lx - bx * P.tx), o[0] - 1, B2, P.lx, P.wall[0]) &&
           ranges_meet(by * P.ty, min(P.ty, P.ly - by * P.ty), o[1] - 1, B2, P.ly, P.wall[1]);
}

// The ring position a thread gathers for (threads below the tile's ring
// length, when the position is a node of the lattice).
struct RingDuty {
    bool on;
    int fx, fy, side, pos;
    __device__ __forceinline__ RingDuty(int tid, int bx, int by, int w, int h, const KParams& P, const FusedGeom& G)
    {
        fx = fy = 0;
        on = tid < G.ring && ring_pos(tid, w, h, P, fx, fy) && fp_node(bx, by, fx, fy, P);
        side = ring_side(tid, P);
        pos = xch_pos(fx, fy, P);
    }
};

template <bool NOISE, bool TAU1>
static __global__ void __launch_bounds__(kThreadsStep, FLBM_BULK_MINBLOCKS)
    k_collide_bulk_fused(const float* __restrict__ fin, float* __restrict__ fout, const float* __restrict__ psi,
                         float* __restrict__ psi_next, float2* __restrict__ ring, float2* __restrict__ seam,
                         const DevState* __restrict__ st, KParams P, FusedGeom G)
{
    extern __shared__ float2 s_fused[];
    const int xsize = xch_size(P);
    float2* s_xch = s_fused;                           // [16][xsize]
    float2* s_roll = s_fused + kXchDirs * xsize;       // [2][256]: rolling sums of the tile's columns
    float2* s_rollr = s_roll + 2 * kThreadsStep;       // [2][kRingMax]: the same for ring positions
    const int tid = threadIdx.x + P.tx * threadIdx.y;
    const float2 zero = make_float2(0.f, 0.f);
    const int z0 = blockIdx.z * G.K, z1 = min(z0 + G.K, P.lz);
    // Planes of this tile that belong to the near launch: [zn0, zn0 + nzn)
    // (periodic along z), none without a particle or when the tile is not
    // next to it in x and y.
    int zn0 = 0, nzn = 0;
    if (P.has_particle) {
        const int o[3] = {st->box0[0], st->box0[1], st->box0[2]};
        if (tile_near_xy(blockIdx.x, blockIdx.y, o, P)) {
            zn0 = o[2] - 1;
            nzn = P.B + 2;
        }
    }
    for (int k = tid; k < kXchDirs * xsize; k += kThreadsStep) s_xch[k] = zero;
    auto reset = [&] {
        s_roll[tid] = s_roll[kThreadsStep + tid] = zero;
        if (tid < kRingMax) s_rollr[tid] = s_rollr[kRingMax + tid] = zero;
    };
    reset();
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
        // Tiles next to the particle belong to the near launch: the densities
        // around them are recomputed after cover/uncover (part A of
        // k_psi_finish), so the partial sums just restart.
        if (nzn && ranges_meet(z, 1, zn0, nzn, P.lz, P.wall[2])) {
            reset();
            continue;
        }
        const int w = tile_w(blockIdx.x, P), h = tile_h(blockIdx.y, P);
        const bool node = (int)threadIdx.x < w && (int)threadIdx.y < h;
        DensitySink sink(reinterpret_cast<float*>(s_xch), xch_pos(threadIdx.x, threadIdx.y, P), xsize);
        if (node) {
            const int x = blockIdx.x * P.tx + threadIdx.x, y = blockIdx.y * P.ty + threadIdx.y;
            const uint32_t n = (uint32_t)x + (uint32_t)P.lx * ((uint32_t)y + (uint32_t)P.ly * (uint32_t)z);
            const GlobalInputs in(fin, psi, x, y, z, n, P);
            collide_core<NOISE, false, TAU1>(x, y, z, n, in, fout, st, P, 0u, nullptr, &sink);
        }
        __syncthreads();
        const int tile = blockIdx.x + P.gx * blockIdx.y;
        if (node) {
            float2 inc[3] = {zero, zero, zero};
            gather_column(sink.pos, s_xch, P, inc);
            float2 roll[2] = {s_roll[tid], s_roll[kThreadsStep + tid]};
            const float2 r = roll_update(roll, sink.own, inc);
            s_roll[tid] = roll[0];
            s_roll[kThreadsStep + tid] = roll[1];
            put_density(z - 1, threadIdx.x, threadIdx.y, true, -1, r, tile, blockIdx.x, blockIdx.y, blockIdx.z, z0,
                        z1, psi_next, ring, seam, P, G);
        }
        if (tid < G.ring) {
            const RingDuty rd(tid, blockIdx.x, blockIdx.y, w, h, P, G);
            if (rd.on) {
                float2 inc[3] = {zero, zero, zero};
                gather_ring(rd.side, rd.pos, s_xch, P, inc);
                const float none[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                float2 roll[2] = {s_rollr[tid], s_rollr[kRingMax + tid]};
                const float2 r = roll_update(roll, none, inc);
                s_rollr[tid] = roll[0];
                s_rollr[kRingMax + tid] = roll[1];
                put_density(z - 1, rd.fx, rd.fy, false, tid, r, tile, blockIdx.x, blockIdx.y, blockIdx.z, z0, z1,
                            psi_next, ring, seam, P, G);
            }
        }
        __syncthreads();  // the next plane overwrites the exchange arrays
    }
    // The chunk's last plane still lacks what the plane above pushes down,
    // and the plane above the chunk has only this chunk's share.
    const int tile = blockIdx.x + P.gx * blockIdx.y;
    const int w = tile_w(blockIdx.x, P), h = tile_h(blockIdx.y, P);
    if ((int)threadIdx.x < w && (int)threadIdx.y < h) {
        put_density(z1 - 1, threadIdx.x, threadIdx.y, true, -1, s_roll[tid], tile, blockIdx.x, blockIdx.y, blockIdx.z,
                    z0, z1, psi_next, ring, seam, P, G);
        put_density(z1, threadIdx.x, threadIdx.y, true, -1, s_roll[kThreadsStep + tid], tile, blockIdx.x, blockIdx.y,
                    blockIdx.z, z0, z1, psi_next, ring, seam, P, G);
    }
    if (tid < G.ring) {
        const RingDuty rd(tid, blockIdx.x, blockIdx.y, w, h, P, G);
        if (rd.on) {
            put_density(z1 - 1, rd.fx, rd.fy, false, tid, s_rollr[tid], tile, blockIdx.x, blockIdx.y, blockIdx.z, z0,
                        z1, psi_next, ring, seam, P, G);
            put_density(z1, rd.fx, rd.fy, false, tid, s_rollr[kRingMax + tid], tile, blockIdx.x, blockIdx.y,
                        blockIdx.z, z0, z1, psi_next, ring, seam, P, G);
        }
    }
}

// Number of nodes part B visits on one plane of a tile of extent w x h: the
// whole tile on a seam plane, else its edge.
__host__ __device__ __forceinline__ int edge_count(int w, int h)
{
    return h == 1 ? w : (w == 1 ? h : 2 * w + 2 * (h - 2));
}

__host__ __device__ __forceinline__ void edge_node(int i, int w, int h, int& fx, int& fy)
{
    if (h == 1) { fx = i; fy = 0; return; }
    if (w == 1) { fx = 0; fy = i; return; }
    if (i < w) { fx = i; fy = 0; return; }
    if (i < 2 * w) { fx = i - w; fy = h - 1; return; }
    i -= 2 * w;
    if (i < h - 2) { fx = 0; fy = 1 + i; return; }
    fx = w - 1;
    fy = 1 + i - (h - 2);
}

// Items part B visits for one (tile, chunk): planes z0 .. z1 - 1 of a tile of
// extent w x h. A plane that receives a seam (the chunk's first plane from
// the chunk below, its last plane from the chunk above, unless a z wall is
// there) needs every node; the other planes only the tile's edge nodes.
struct FinishItems {
    int z0, z1, w, h, ne, n_first, n_last;
    __host__ __device__ __forceinline__ FinishItems(int z0_, int z1_, int w_, int h_, const KParams& P)
        : z0(z0_), z1(z1_), w(w_), h(h_)
    {
        const bool lo = z0 > 0 || !P.wall[2];
        const bool hi = z1 < P.lz || !P.wall[2];
        ne = edge_count(w, h);
        n_first = (lo || (z1 - z0 == 1 && hi)) ? w * h : ne;
        n_last = z1 - z0 > 1 ? (hi ? w * h : ne) : 0;
    }
    __host__ __device__ __forceinline__ long long count() const
    {
        return (long long)n_first + n_last + (long long)max(z1 - z0 - 2, 0) * ne;
    }
    __host__ __device__ __forceinline__ void item(long long it, int& z, int& fx, int& fy) const
    {
        if (it < n_first) {
            z = z0;
            const int i = (int)it;
            if (n_first == w * h) { fx = i % w; fy = i / w; } else edge_node(i, w, h, fx, fy);
        } else if (it < n_first + n_last) {
            z = z1 - 1;
            const int i = (int)(it - n_first);
            if (n_last == w * h) { fx = i % w; fy = i / w; } else edge_node(i, w, h, fx, fy);
        } else {
            const long long j = it - n_first - n_last;
            z = z0 + 1 + (int)(j / ne);
            edge_node((int)(j % ne), w, h, fx, fy);
        }
    }
};

// The tiles around tile (bx, by) that part B reads: index, extent, and
// whether it exists (not across a wall). Slot k = (dbx + 1) + 3 (dby + 1).
struct TileRing {
    int t[9], w[9], h[9];
    bool ok[9];
    __host__ __device__ __forceinline__ TileRing(int bx, int by, const KParams& P)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            int tbx = bx + k % 3 - 1, tby = by + k / 3 - 1;
            ok[k] = true;
            if (tbx < 0 || tbx >= P.gx) {
                if (P.wall[0]) ok[k] = false;
                tbx += tbx < 0 ? P.gx : -P.gx;
            }
            if (tby < 0 || tby >= P.gy) {
                if (P.wall[1]) ok[k] = false;
                tby += tby < 0 ? P.gy : -P.gy;
            }
            t[k] = ok[k] ? tbx + P.gx * tby : 0;
            w[k] = ok[k] ? tile_w(tbx, P) : 0;
            h[k] = ok[k] ? tile_h(tby, P) : 0;
        }
    }
};

// Density of node (fx, fy) of tile (bx, by) (ring R of its tiles), plane z,
// chunk c, from its home partial (psi_next) and the partials of the blocks
// whose footprint holds it: for each tile k of the 3 x 3 block around it (in
// slot order) whose ring or footprint contains the node, the ring partial of
// plane z (other tiles only) and the seams of the chunks below and above
// when z is the chunk's first or last plane. A node on a tile edge sits on
// the ring of one side tile, a corner node on the rings of three tiles.
__host__ __device__ __forceinline__ void finish_node(int fx, int fy, int z, int bx, int by, int c, const TileRing& R,
                                                    float* __restrict__ psi_next, const float2* __restrict__ ring,
                                                    const float2* __restrict__ seam, const KParams& P,
                                                    const FusedGeom& G)
{
    const int w = R.w[4], h = R.h[4];
    const int z0 = c * G.K, z1 = min(z0 + G.K, P.lz);
    const bool lo = z == z0 && (z0 > 0 || !P.wall[2]);
    const bool hi = z == z1 - 1 && (z1 < P.lz || !P.wall[2]);
    const int cb = c == 0 ? G.nchunk - 1 : c - 1;
    const int ca = c == G.nchunk - 1 ? 0 : c + 1;
    const long long q = pad_index(bx * P.tx + fx, by * P.ty + fy, z, P);
    float a = psi_next[q], b = psi_next[P.padn + q];
    const int dxs[3] = {fx == 0 ? -1 : 0, 0, fx == w - 1 ? 1 : 0};  // candidate side columns
    const int dys[3] = {fy == 0 ? -1 : 0, 0, fy == h - 1 ? 1 : 0};
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int dbx = kx - 1, dby = ky - 1;
            if ((dbx != 0 && dxs[kx] != dbx) || (dby != 0 && dys[ky] != dby)) continue;
            const int k = kx + 3 * ky;
            if (!R.ok[k]) continue;
            // Position of the node relative to tile k.
            const int fxk = dbx < 0 ? R.w[k] : (dbx > 0 ? -1 : fx);
            const int fyk = dby < 0 ? R.h[k] : (dby > 0 ? -1 : fy);
            if (k != 4) {
                const float2 v = ring[ring_index(R.t[k], z, ring_slot(fxk, fyk, R.w[k], R.h[k], P), P, G)];
                a += v.x;
                b += v.y;
            }
            const int p = fp_index(fxk, fyk, P);
            if (lo) {
                const float2 v = seam[seam_index(R.t[k], cb, 1, p, G)];
                a += v.x;
                b += v.y;
            }
            if (hi) {
                const float2 v = seam[seam_index(R.t[k], ca, 0, p, G)];
                a += v.x;
                b += v.y;
            }
        }
    }
    psi_next[q] = a;
    psi_next[P.padn + q] = b;
}

// Can the dilated near-particle region meet tile (bx, by) over planes
// [z0, z1)? Only then do part B's nodes of that block need the per-node test.
__host__ __device__ __forceinline__ bool block_meets_near(int bx, int by, int z0, int z1, const int o[3],
                                                          const KParams& P)
{
    bool nx = false, ny = false;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int b = bx + d;
        if (b < 0 || b >= P.gx) {
            if (P.wall[0]) continue;
            b += b < 0 ? P.gx : -P.gx;
        }
        nx = nx || ranges_meet(b * P.tx, min(P.tx, P.lx - b * P.tx), o[0] - 1, P.B + 2, P.lx, P.wall[0]);
    }
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int b = by + d;
        if (b < 0 || b >= P.gy) {
            if (P.wall[1]) continue;
            b += b < 0 ? P.gy : -P.gy;
        }
        ny = ny || ranges_meet(b * P.ty, min(P.ty, P.ly - b * P.ty), o[1] - 1, P.B + 2, P.ly, P.wall[1]);
    }
    const int zl = min(z1 - z0 + 2, P.lz);
    const int zs = (z0 == 0 && !P.wall[2]) ? P.lz - 1 : max(z0 - 1, 0);
    return nx && ny && ranges_meet(zs, zl, o[2] - 1, P.B + 2, P.lz, P.wall[2]);
}

// Completes psi_next after the fused collide and the particle kernels.
// Blocks [0, nB): part B, one block per (tile, chunk), over the tile's edge
// nodes on every plane of the chunk and all its nodes on seam planes.
// Blocks [nB, ...): part A, the near-particle region dilated by one node, in
// the box around the candidate tiles of the step's collide (box origin
// st->box_prev); densities straight from the populations f (after
// cover/uncover), 0 on particle nodes at the new position.
static __global__ void __launch_bounds__(kThreadsStep) k_psi_finish(const float* __restrict__ f,
                                                                    float* __restrict__ psi_next,
                                                                    const float2* __restrict__ ring,
                                                                    const float2* __restrict__ seam,
                                                                    const DevState* __restrict__ st,
                                                                    const uint8_t* __restrict__ masks, KParams P,
                                                                    FusedGeom G, int nB)
{
    int o[3] = {0, 0, 0};
    if (P.has_particle) {
        o[0] = st->box_prev[0];
        o[1] = st->box_prev[1];
        o[2] = st->box_prev[2];
    }
    if ((int)blockIdx.x < nB) {
        const int ntile = P.gx * P.gy;
        const int tile = blockIdx.x % ntile, c = blockIdx.x / ntile;
        const int bx = tile % P.gx, by = tile / P.gx;
        const TileRing R(bx, by, P);
        const int z0 = c * G.K, z1 = min(z0 + G.K, P.lz);
        const bool check = P.has_particle && block_meets_near(bx, by, z0, z1, o, P);
        const FinishItems items(z0, z1, R.w[4], R.h[4], P);
        const long long total = items.count();
        for (long long it = threadIdx.x; it < total; it += blockDim.x) {
            int z, fx, fy;
            items.item(it, z, fx, fy);
            if (check && near_dilated(bx * P.tx + fx, by * P.ty + fy, z, o, P)) continue;
            finish_node(fx, fy, z, bx, by, c, R, psi_next, ring, seam, P, G);
        }
        return;
    }
    if (!P.has_particle) return;
    int xs, nxb, ys, nyb, zs, nzb;
    near_box_axis(o[0], P.tx, P.ncx, P.gx, P.lx, P.wall[0], xs, nxb);
    near_box_axis(o[1], P.ty, P.ncy, P.gy, P.ly, P.wall[1], ys, nyb);
    near_box_axis(o[2], 1, P.ncz, P.lz, P.lz, P.wall[2], zs, nzb);
    const long long t = (long long)(blockIdx.x - nB) * blockDim.x + threadIdx.x;
    if (t >= (long long)nxb * nyb * nzb) return;
    int x = xs + (int)(t % nxb), y = ys + (int)((t / nxb) % nyb), z = zs + (int)(t / ((long long)nxb * nyb));
    const int L[3] = {P.lx, P.ly, P.lz};
    int q[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (q[a] < 0 || q[a] >= L[a]) {
            if (P.wall[a]) return;
            q[a] += q[a] < 0 ? L[a] : -L[a];
        }
    }
    x = q[0];
    y = q[1];
    z = q[2];
    if (!near_dilated(x, y, z, o, P)) return;
    density_node(x, y, z, f, psi_next, st, masks, P);
}

// Part A's launch size: its box (candidate tiles plus one node per side).
__host__ __device__ __forceinline__ long long near_box_nodes(const KParams& P)
{
    if (!P.has_particle) return 0;
    auto len = [](int T, int nc, int L, int wall) {
        const int l = nc * T + 2;
        return (!wall && l > L) ? L : l;
    };
    return (long long)len(P.tx, P.ncx, P.lx, P.wall[0]) * len(P.ty, P.ncy, P.ly, P.wall[1]) *
           len(1, P.ncz, P.lz, P.wall[2]);
}

}  // namespace flbm

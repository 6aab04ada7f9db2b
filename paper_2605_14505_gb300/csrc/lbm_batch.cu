// Batched update of many independent lattices (a parameter sweep over size,
// Froude number, forcing scheme and stencil pair).
//
// Two drivers live here:
//   k_batch_variant  per time step one launch per (pair, forcing) variant
//                    over that variant's tiles of bx x by nodes of one z-plane
//                    (graph-captured by the host);
//   k_batch_flow     one persistent launch that advances `steps` time steps
//                    of every instance with no grid-wide barrier (below).
//
// k_batch_flow. Each step's work is one list of tiles, every instance cut
// into runs of flow_nodes consecutive nodes (node index x + nx (y + ny z)).
// Queue position q = s * flow_tiles + r stands for tile r of step s; blocks
// claim positions from one global counter in increasing order, so every tile
// of step s is claimed before any tile of step s + 1. Instances depend only
// on themselves: a tile of instance i at step s > 0 starts once all nflow_i
// tiles of instance i at step s - 1 are done (a per-instance completion
// counter), because the AA step of a node reads and writes its neighbours'
// slots. The next position is claimed while the current tile runs. A block
// claims positions only while it is running, so whatever a block waits for
// is held by running blocks that will finish it: the launch needs no
// co-residency guarantee (a plain launch, capturable in a CUDA graph, of any
// grid size). Every wait polls at most spin_limit times; a wait that runs out
// raises the error flag, and any block that sees the flag stops, so the
// kernel always ends.
#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"

namespace lbm {

// One node of one instance: identical arithmetic to k_step.
template <class P, int FORCING, bool ODD>
__device__ __forceinline__ void batch_node(const BatchInstance& I, int x, int y, int z)
{
    update_node<P, FORCING, float, ODD>(I.f, I.g, I.geo, I.ph, x, y, z);
}

// Tile t of the global list: its instance and this thread's node; false if
// the node lies outside the instance (ragged tiles).
__device__ __forceinline__ bool tile_node(const BatchArgs& A, uint32_t t, const BatchInstance*& inst, int& x, int& y,
                                          int& z)
{
    const BatchInstance& I = A.inst[A.tile_inst[t]];
    inst = &I;
    const uint32_t lt = t - I.tile0;
    const uint32_t plane = I.tx * I.ty;
    z = (int)(lt / plane);
    const uint32_t r = lt - (uint32_t)z * plane;
    x = (int)((r % I.tx) * blockDim.x + threadIdx.x);
    y = (int)((r / I.tx) * blockDim.y + threadIdx.y);
    return x < I.geo.nx && y < I.geo.ny;
}

template <bool ODD>
__device__ __forceinline__ void batch_tile(const BatchArgs& A, uint32_t t)
{
    const BatchInstance* I;
    int x, y, z;
    if (!tile_node(A, t, I, x, y, z)) return;
    switch (I->variant) {
    case 0: batch_node<Pair<27, 19>, kGuo, ODD>(*I, x, y, z); break;
    case 1: batch_node<Pair<27, 19>, kShanChen, ODD>(*I, x, y, z); break;
    case 2: batch_node<Pair<27, 19>, kEDM, ODD>(*I, x, y, z); break;
    case 3: batch_node<Pair<27, 19>, kHCZ, ODD>(*I, x, y, z); break;
    case 4: batch_node<Pair<19, 7>, kGuo, ODD>(*I, x, y, z); break;
    case 5: batch_node<Pair<19, 7>, kShanChen, ODD>(*I, x, y, z); break;
    case 6: batch_node<Pair<19, 7>, kEDM, ODD>(*I, x, y, z); break;
    default: batch_node<Pair<19, 7>, kHCZ, ODD>(*I, x, y, z); break;
    }
}

// Per-step driver: one launch per (pair, forcing) variant over that variant's
// tiles, which the host lists contiguously. Without the other variants'
// code the kernel fits three 256-thread blocks per SM, as k_step does.
template <class P, int FORCING, bool ODD>
__global__ void __launch_bounds__(256, 3) k_batch_variant(BatchArgs A)
{
    for (uint32_t t = A.tile_begin + blockIdx.x; t < A.tile_end; t += gridDim.x) {
        const BatchInstance* I;
        int x, y, z;
        if (tile_node(A, t, I, x, y, z)) batch_node<P, FORCING, ODD>(*I, x, y, z);
    }
}

// Nodes [n0, n1) of one instance, consecutive nodes on consecutive threads.
// A thread's coordinates are divided out of its first node index once and
// then advanced by the block size (dx, dy) with carries, instead of two
// divisions and two remainders by the run-time sizes per node (dx < nx, so x
// carries into y at most once; y carries into z once per plane advanced).
template <class P, int FORCING, bool ODD>
__device__ __forceinline__ void flow_nodes(const BatchInstance& I, uint32_t n0, uint32_t n1)
{
    uint32_t n = n0 + threadIdx.x;
    if (n >= n1) return;
    int x, y, z;
    node_xyz(I.geo, n, x, y, z);
    const int nx = I.geo.nx, ny = I.geo.ny;
    const int dy = (int)(blockDim.x / (unsigned)nx), dx = (int)blockDim.x - dy * nx;
    for (; n < n1; n += blockDim.x) {
        batch_node<P, FORCING, ODD>(I, x, y, z);
        x += dx;
        y += dy;
        if (x >= nx) {
            x -= nx;
            ++y;
        }
        while (y >= ny) {
            y -= ny;
            ++z;
        }
    }
}

// Variants compiled into a persistent kernel: bit v of MASK for variant v.
constexpr int kFlowAll = 0xff;
constexpr int kFlowGuoSC = 0x33;   // Guo and Shan-Chen on both pairs

template <int MASK, bool ODD>
__device__ __forceinline__ void flow_tile(const BatchInstance& I, uint32_t n0, uint32_t n1)
{
    switch (I.variant) {
    case 0: if constexpr ((MASK & 1) != 0) flow_nodes<Pair<27, 19>, kGuo, ODD>(I, n0, n1); break;
    case 1: if constexpr ((MASK & 2) != 0) flow_nodes<Pair<27, 19>, kShanChen, ODD>(I, n0, n1); break;
    case 2: if constexpr ((MASK & 4) != 0) flow_nodes<Pair<27, 19>, kEDM, ODD>(I, n0, n1); break;
    case 3: if constexpr ((MASK & 8) != 0) flow_nodes<Pair<27, 19>, kHCZ, ODD>(I, n0, n1); break;
    case 4: if constexpr ((MASK & 16) != 0) flow_nodes<Pair<19, 7>, kGuo, ODD>(I, n0, n1); break;
    case 5: if constexpr ((MASK & 32) != 0) flow_nodes<Pair<19, 7>, kShanChen, ODD>(I, n0, n1); break;
    case 6: if constexpr ((MASK & 64) != 0) flow_nodes<Pair<19, 7>, kEDM, ODD>(I, n0, n1); break;
    default: if constexpr ((MASK & 128) != 0) flow_nodes<Pair<19, 7>, kHCZ, ODD>(I, n0, n1); break;
    }
}

// Thread 0: wait until `need` tiles of an instance are complete. False (with
// the error flag raised) after spin_limit polls or once another block has
// raised the flag.
__device__ __forceinline__ bool flow_wait(const BatchArgs& A, uint32_t inst, uint32_t need)
{
    volatile unsigned* done = A.flow + 1 + inst;
    volatile unsigned* flag = A.sync + 2;
    unsigned polls = 0;
    while (*done < need) {
        if (++polls > A.spin_limit || *flag != 0u) {
            atomicExch(A.sync + 2, 1u);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();   // acquire: the producers' stores are visible to this block after the barrier
    return true;
}

static_assert(sizeof(FlowArgs) <= 32000, "persistent arguments within the kernel parameter limit");

template <int MASK, int MINB>
__global__ void __launch_bounds__(256, MINB) k_batch_flow(const __grid_constant__ FlowArgs F)
{
    const BatchArgs& A = F.a;
    __shared__ uint32_t s_q;
    __shared__ int s_go;
    const uint32_t total = (uint32_t)A.steps * A.flow_tiles;
    uint32_t next = 0;   // thread 0: the position claimed for the next tile
    if (threadIdx.x == 0) {
        s_q = atomicAdd(A.flow, 1u);
        next = atomicAdd(A.flow, 1u);
    }
    __syncthreads();
    uint32_t q = s_q;
    while (q < total) {
        const uint32_t s = q / A.flow_tiles;
        const uint32_t r = q - s * A.flow_tiles;
        const uint32_t ii = A.flow_inst[r];
        const BatchInstance& I = F.inst[ii];
        if (threadIdx.x == 0) s_go = (s == 0) ? 1 : (int)flow_wait(A, ii, s * I.nflow + A.extra_dep);
        __syncthreads();
        if (!s_go) return;
        const uint32_t n0 = (r - I.flow0) * A.flow_nodes;
        const uint32_t n1 = min(n0 + A.flow_nodes, I.geo.n3);
        if (((uint32_t)A.odd0 + s) & 1u)
            flow_tile<MASK, true>(I, n0, n1);
        else
            flow_tile<MASK, false>(I, n0, n1);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();   // release: this block's stores before the completion count
            atomicAdd(A.flow + 1 + ii, 1u);
            s_q = next;
            if (next < total) next = atomicAdd(A.flow, 1u);
        }
        __syncthreads();
        q = s_q;
    }
}

template <class P, int F>
const void* variant_kernel(int odd)
{
    return odd ? (const void*)k_batch_variant<P, F, true> : (const void*)k_batch_variant<P, F, false>;
}

const void* batch_variant_kernel(int variant, int odd)
{
    switch (variant) {
    case 0: return variant_kernel<Pair<27, 19>, kGuo>(odd);
    case 1: return variant_kernel<Pair<27, 19>, kShanChen>(odd);
    case 2: return variant_kernel<Pair<27, 19>, kEDM>(odd);
    case 3: return variant_kernel<Pair<27, 19>, kHCZ>(odd);
    case 4: return variant_kernel<Pair<19, 7>, kGuo>(odd);
    case 5: return variant_kernel<Pair<19, 7>, kShanChen>(odd);
    case 6: return variant_kernel<Pair<19, 7>, kEDM>(odd);
    default: return variant_kernel<Pair<19, 7>, kHCZ>(odd);
    }
}

// Guo / Shan-Chen only (80 registers, three blocks per SM as k_step), or every variant.
const void* batch_flow_kernel(bool guo_sc_only)
{
    return guo_sc_only ? (const void*)k_batch_flow<kFlowGuoSC, 3> : (const void*)k_batch_flow<kFlowAll, 1>;
}

}  // namespace lbm

// Batched update of many independent lattices (a parameter sweep over size,
// Froude number, forcing scheme and stencil pair) in one launch.
//
// The lattices are cut into tiles of blockDim.x x blockDim.y nodes of one
// z-plane; one global tile list covers every instance. A block updates whole
// tiles; the (pair, forcing) variant is uniform over a tile, so the switch
// below never diverges inside a block. Two drivers:
//   k_batch_variant     per time step one launch per (pair, forcing) variant over
//                       that variant's tiles (graph-captured by the host);
//   k_batch_persistent  a cooperative launch that advances `steps` time steps,
//                       with a grid-wide barrier between steps. Every wait of
//                       the barrier is bounded: after `spin_limit` polls the
//                       block raises the error flag and returns, so a barrier
//                       that cannot complete ends the kernel instead of hanging.
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

// Grid-wide barrier for a cooperative launch. sync[0] counts arrivals,
// sync[1] is the generation, sync[2] the error flag. Thread 0 of each block
// reads the generation before arriving; the last block to arrive resets the
// count and advances the generation. Returns false (after raising the flag)
// if the generation did not move within spin_limit polls.
__device__ __forceinline__ bool grid_barrier(const BatchArgs& A)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* vsync = A.sync;
        const unsigned gen = vsync[1];
        int ok = 1;
        __threadfence();
        const unsigned arrived = atomicAdd(A.sync, 1u);
        if (arrived == A.nblocks - 1) {
            A.sync[0] = 0u;
            __threadfence();
            atomicAdd(A.sync + 1, 1u);
        } else {
            unsigned polls = 0;
            while (vsync[1] == gen) {
                if (++polls > A.spin_limit || vsync[2] != 0u) {
                    atomicExch(A.sync + 2, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(256) k_batch_persistent(BatchArgs A)
{
    int odd = A.odd0;
    for (int s = 0; s < A.steps; ++s) {
        for (uint32_t t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
            if (odd)
                batch_tile<true>(A, t);
            else
                batch_tile<false>(A, t);
        }
        if (s + 1 < A.steps && !grid_barrier(A)) return;
        odd ^= 1;
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

const void* batch_persistent_kernel() { return (const void*)k_batch_persistent; }

}  // namespace lbm

// 16-bit storage, two nodes per thread, with the populations of each tile
// brought into shared memory by bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier) one tile ahead of the compute.
//
// The store is in half-row order (row_pos): word k of a row holds nodes k and
// k + nx / 2. A tile is W = 2 * blockDim.x consecutive elements of one x-row
// (y, z), the words of blockDim.x pairs; thread p takes word xs / 2 + p. For
// every slot the AA step reads one row segment: slot i of row (y, z) on the
// even step, slot opp(i) of row (y - e_y, z - e_z) on the odd step. Each such
// segment is one bulk copy of W elements (even) or W + 16 elements from 8
// before the tile to 8 after it (odd: the words k - 1 and k + 1 are read);
// at either end of the row the 8-element pad wraps to the other end and is a
// separate 16-byte copy. A tile that is a whole row (W = nx) needs no pads:
// the words across its ends are the row's own, read modulo W from the staged
// row, so every slot row is one copy on both AA steps. Warp 0 issues the copies of tile k + 1 into the
// other half of a two-stage ring while the block computes tile k from shared
// memory, so the DRAM latency is covered by the ring rather than by
// registers held in flight. Results are stored straight to global memory as
// in k_step2 (aligned 32-bit words). Blocks are persistent: block b takes
// tiles b, b + grid, ...
//
// Every mbarrier wait is bounded (spin_limit polls). A wait that runs out
// raises *err; the block then drains: it waits for the barriers of the copies
// it has issued, with its own fixed limit (kStageDrainPolls, independent of
// spin_limit), and returns, so a barrier that cannot complete ends the kernel
// and no bulk copy is still writing shared memory when the block exits. The
// test hook's phantom bytes are counted on a barrier of their own that no
// copy signals, so the real copies' barriers always complete and the drain
// observes every copy landing.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct StageArgs {
    void* f;                // QF * n3 elements, then g: QG * n3 (one store)
    void* g;
    Geometry geo;
    Phys ph;
    int W;                  // tile width in nodes: 2 * blockDim.x, divides nx, multiple of 8
    int ntx;                // nx / W
    uint32_t ntiles;        // ntx * ny * nz
    int* err;               // set to 1 when a wait gives up
    uint32_t spin_limit;    // polls per wait
    uint32_t extra_tx;      // test hook: bytes a separate barrier expects and no copy delivers (0 in use)
};

// Polls of the drain after a wait ran out: long enough for any copy in
// flight to land (~0.3-1 s), and bounded so that the block always returns.
constexpr uint32_t kStageDrainPolls = 1u << 22;

constexpr int kStagePad = 8;   // staged row element j holds row element xs - 8 + j

// Shared-memory bytes of one block: two stages of Q rows of W + 16 elements,
// three mbarriers (one per stage, one for the test hook), Q row codes.
__host__ __device__ constexpr size_t stage_smem_bytes(int q, int W)
{
    return (size_t)2 * q * (W + 2 * kStagePad) * 2 + 24 + (size_t)q * 4;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// True once the phase of the given parity has completed; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Row r of a stage (f slots 0..QF-1, then g slots): the store slot it is
// copied from (g slots follow the QF f slots) and its row shift,
// packed as slot | (dy + 1) << 8 | (dz + 1) << 10.
template <class P, bool ODD>
__device__ __forceinline__ uint32_t stage_row_code(int r)
{
    const bool isg = r >= P::QF;
    const int i = isg ? r - P::QF : r;
    const int ey = isg ? P::LG::ey(i) : P::LF::ey(i);
    const int ez = isg ? P::LG::ez(i) : P::LF::ez(i);
    const int op = isg ? P::LG::opp(i) : P::LF::opp(i);
    const int slot = (isg ? P::QF : 0) + (ODD ? op : i);
    const int dy = ODD ? -ey : 0, dz = ODD ? -ez : 0;
    return (uint32_t)slot | (uint32_t)(dy + 1) << 8 | (uint32_t)(dz + 1) << 10;
}

// Warp 0: the copies of tile t into one stage, counted on `bar`.
template <class P, bool ODD>
__device__ __forceinline__ void stage_issue(const StageArgs& A, uint16_t* st, uint64_t* bar, const uint32_t* code,
                                            uint32_t t)
{
    constexpr int Q = P::QF + P::QG;
    const int lane = threadIdx.x & 31;
    const int W = A.W, RS = W + 2 * kStagePad;
    const int nx = A.geo.nx, ny = A.geo.ny, nz = A.geo.nz;
    const uint32_t xt = t % (uint32_t)A.ntx;
    const uint32_t row = t / (uint32_t)A.ntx;
    const int y = (int)(row % (uint32_t)ny), z = (int)(row / (uint32_t)ny);
    const int xs = (int)xt * W;
    const bool whole = (W == nx);   // a whole row: no pads (read modulo W)
    const uint32_t row_bytes = (uint32_t)((ODD && !whole) ? W + 2 * kStagePad : W) * 2u;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)Q * row_bytes);
    __syncwarp();
    const uint16_t* base = static_cast<const uint16_t*>(A.f);
    for (int r = lane; r < Q; r += 32) {
        const uint32_t c = code[r];
        const int slot = (int)(c & 0xffu);
        int yy = y + (int)((c >> 8) & 3u) - 1;
        int zz = z + (int)((c >> 10) & 3u) - 1;
        yy = yy < 0 ? ny - 1 : (yy == ny ? 0 : yy);
        zz = zz < 0 ? nz - 1 : (zz == nz ? 0 : zz);
        const uint16_t* src = base + (size_t)slot * A.geo.n3 + ((size_t)zz * ny + yy) * nx;
        uint16_t* dst = st + (size_t)r * RS;
        if (!ODD || whole) {
            bulk_copy_g2s(dst + kStagePad, src + xs, (uint32_t)W * 2u, bar);
        } else if (xs > 0 && xs + W < nx) {
            bulk_copy_g2s(dst, src + (xs - kStagePad), row_bytes, bar);
        } else {
            // head and tail pads wrap at the ends of the row
            bulk_copy_g2s(dst, src + (xs > 0 ? xs - kStagePad : nx - kStagePad), kStagePad * 2u, bar);
            bulk_copy_g2s(dst + kStagePad, src + xs, (uint32_t)W * 2u, bar);
            bulk_copy_g2s(dst + kStagePad + W, src + (xs + W < nx ? xs + W : 0), kStagePad * 2u, bar);
        }
    }
}

__device__ __forceinline__ uint32_t lds_word(const uint16_t* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

// The pair's words of lattice L from its stage rows (rows = first row of L):
// word p of the tile on the even step, word p - e_x on the odd step (modulo
// the tile for a whole-row tile, W = nx), with the halves exchanged where the
// row wraps (as load_pair).
template <class L, bool ODD>
__device__ __forceinline__ void stage_load(const uint16_t* rows, int RS, int W, bool whole, int p, const Seam& sm,
                                           uint32_t* w)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ex = ODD ? L::ex(i) : 0;
        int e = 2 * p - 2 * ex;
        if constexpr (ex != 0) {
            if (whole) e = (e < 0) ? e + W : (e >= W ? e - W : e);
        }
        w[i] = lds_word(rows + i * RS + kStagePad + e);
    });
    if constexpr (ODD) {
        if (sm.warp_first) {
            sfor<0, L::kQ>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr (L::ex(i) == 1) w[i] = seam_word(w[i], sm.sel_first);
            });
        }
        if (sm.warp_last) {
            sfor<0, L::kQ>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr (L::ex(i) == -1) w[i] = seam_word(w[i], sm.sel_last);
            });
        }
    }
}

template <class P>
constexpr int kStageMinBlocks = (P::QF + P::QG <= 34) ? 6 : 4;

template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(128, kStageMinBlocks<P>) k_step_staged(const __grid_constant__ StageArgs A)
{
    constexpr int Q = P::QF + P::QG;
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = A.W, RS = W + 2 * kStagePad;
    uint16_t* stages = reinterpret_cast<uint16_t*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)2 * Q * RS * 2);
    uint32_t* code = reinterpret_cast<uint32_t*>(bar + 3);
    for (int r = (int)threadIdx.x; r < Q; r += (int)blockDim.x) code[r] = stage_row_code<P, ODD>(r);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        // test hook: phase 0 of bar[2] expects bytes that no copy delivers
        if (A.extra_tx) mbar_arrive_expect_tx(&bar[2], A.extra_tx);
        fence_mbarrier_init();
    }
    __syncthreads();
    if (blockIdx.x >= A.ntiles) return;
    const bool producer = threadIdx.x < 32;
    if (producer) stage_issue<P, ODD>(A, stages, &bar[0], code, blockIdx.x);

    unsigned short* fb = static_cast<unsigned short*>(A.f);
    unsigned short* gb = static_cast<unsigned short*>(A.g);
    const int p = (int)threadIdx.x;
    uint32_t k = 0;
    for (uint32_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++k) {
        const uint32_t s = k & 1u;
        const uint32_t tn = t + gridDim.x;
        if (producer && tn < A.ntiles) {
            // stage s ^ 1 was last read for tile k - 1, before the barrier that ended it
            fence_proxy_async_smem();
            stage_issue<P, ODD>(A, stages + (size_t)(s ^ 1u) * Q * RS, &bar[s ^ 1u], code, tn);
        }
        bool ok = mbar_wait(&bar[s], (k >> 1) & 1u, A.spin_limit);
        if (A.extra_tx && ok) ok = mbar_wait(&bar[2], 0u, A.spin_limit);
        if (ok) {
            const uint16_t* st = stages + (size_t)s * Q * RS;
            const uint32_t row = t / (uint32_t)A.ntx;
            const int x0 = (int)(t - row * (uint32_t)A.ntx) * W + 2 * p;
            const Seam sm(A.geo, x0);
            uint32_t wf[P::QF], wg[P::QG];
            const bool whole = (W == A.geo.nx);
            stage_load<typename P::LF, ODD>(st, RS, W, whole, p, sm, wf);
            stage_load<typename P::LG, ODD>(st + (size_t)P::QF * RS, RS, W, whole, p, sm, wg);
            collide_pair_words<P, FORCING, T>(wf, wg, A.ph);
            const int y = (int)(row % (uint32_t)A.geo.ny), z = (int)(row / (uint32_t)A.geo.ny);
            const PairAddr b(A.geo, (int)launder(x0), (int)launder(y), (int)launder(z));
            store_pair<typename P::LF, ODD>(fb, A.geo.n3, b, sm, wf);
            store_pair<typename P::LG, ODD>(gb, A.geo.n3, b, sm, wg);
        }
        if (__syncthreads_or(!ok)) {
            // a wait ran out: report, wait for this block's copies in flight
            // (the two stage barriers; the hook's barrier has none), stop
            if (threadIdx.x == 0) atomicExch(A.err, 1);
            mbar_wait(&bar[s], (k >> 1) & 1u, kStageDrainPolls);
            if (tn < A.ntiles) mbar_wait(&bar[s ^ 1u], ((k + 1) >> 1) & 1u, kStageDrainPolls);
            return;
        }
    }
}

}  // namespace lbm

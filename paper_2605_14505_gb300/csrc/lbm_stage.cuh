// 16-bit storage, two nodes per thread, with the populations of each tile
// brought into shared memory by bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier) ahead of the compute, by a warp of its
// own.
//
// The store is in half-row order (row_pos): word k of a row holds nodes k and
// k + nx / 2. A tile is W consecutive elements of one x-row (y, z), the words
// of W / 2 pairs; consumer thread p takes word xs / 2 + p. For every slot the
// AA step reads one row segment: slot i of row (y, z) on the even step, slot
// opp(i) of row (y - e_y, z - e_z) on the odd step. Each such segment is one
// bulk copy of W elements. The odd step also reads the words k - 1 and k + 1:
// a tile that is a whole row (W = nx) finds the words across its ends in the
// row itself, read modulo W from the staged row; a narrower tile gets 8
// elements on either side (wrapping at the row's ends) as two plain 16-byte
// loads per slot row, which the producer lanes store beside the copy.
//
// Warp specialisation: a block is W / 64 consumer warps and one producer
// warp around a ring of kStageRing stages. Stage s has a "full" barrier (the
// producer's expected bytes, completed by the copies) and an "empty" barrier
// (one arrival per consumer warp). A consumer warp waits for full[s], loads
// its pair's words into registers, arrives on empty[s] and only then
// collides and stores, so the producer refills the stage while the
// consumers compute; no block-wide barrier is taken per tile and each
// consumer warp runs at its own pace. Results are stored straight to global
// memory as in k_step2 (aligned 32-bit words). Blocks are persistent: block b
// takes tiles b, b + grid, ...
//
// Every mbarrier wait is bounded (spin_limit polls). A consumer warp whose
// wait runs out raises *err and returns; the producer, whose empty-barrier
// wait then runs out too, raises *err and stops issuing. Whatever happens,
// the producer waits for the full barriers of the last stages it filled
// (with a fixed limit of its own, kStageDrainPolls) before it returns: the
// block's shared memory lives until its last thread exits, so no bulk copy
// is still writing it then. The test hook's phantom bytes are counted on a
// barrier of their own that no copy signals, so the real copies' barriers
// always complete and the drain observes every copy landing.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct StageArgs {
    void* f;                // QF * n3 elements, then g: QG * n3 (one store)
    void* g;
    Geometry geo;
    Phys ph;
    int W;                  // tile width in nodes: a multiple of 64 that divides nx
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
#ifndef LBM_STAGE_RING
#define LBM_STAGE_RING 2
#endif
constexpr int kStageRing = LBM_STAGE_RING;  // stages of the ring

// Threads of a block for tile width W: one consumer thread per word, one producer warp.
__host__ __device__ constexpr int stage_threads(int W) { return W / 2 + 32; }

// Shared-memory bytes of one block: kStageRing stages of Q rows of W + 16
// elements, the mbarriers (full and empty per stage, one for the test hook),
// Q row codes.
__host__ __device__ constexpr size_t stage_smem_bytes(int q, int W)
{
    return (size_t)kStageRing * q * (W + 2 * kStagePad) * 2 + 8 * (2 * kStageRing + 1) + (size_t)q * 4;
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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

// The producer warp: the copies of tile t into one stage, counted on `bar`.
// Each slot row's tile body is one bulk copy. Where the odd step needs the
// words across the ends of a tile narrower than the row, the 8-element pads
// on either side (wrapping at the row's ends) are two plain 16-byte loads per
// slot row, stored to the stage by the producer lanes; those stages' barrier
// expects one arrival from each producer lane besides the copies' bytes, so
// a lane's arrival releases its pad stores to the consumers.
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
    const bool pads = ODD && W != nx;   // a whole row reads across its ends modulo W
    const uint16_t* base = static_cast<const uint16_t*>(A.f);
    auto src_row = [&](int r) {
        const uint32_t c = code[r];
        const int slot = (int)(c & 0xffu);
        int yy = y + (int)((c >> 8) & 3u) - 1;
        int zz = z + (int)((c >> 10) & 3u) - 1;
        yy = yy < 0 ? ny - 1 : (yy == ny ? 0 : yy);
        zz = zz < 0 ? nz - 1 : (zz == nz ? 0 : zz);
        return base + (size_t)slot * A.geo.n3 + ((size_t)zz * ny + yy) * nx;
    };
    // pads first, all of a lane's loads in flight together (two rows per lane)
    static_assert(Q <= 64, "two stage rows per producer lane");
    uint4 head[2], tail[2];
    if (pads) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = lane + 32 * k;
            if (r < Q) {
                const uint16_t* src = src_row(r);
                head[k] = *reinterpret_cast<const uint4*>(src + (xs > 0 ? xs - kStagePad : nx - kStagePad));
                tail[k] = *reinterpret_cast<const uint4*>(src + (xs + W < nx ? xs + W : 0));
            }
        }
    }
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)Q * (uint32_t)W * 2u);
    __syncwarp();
    for (int r = lane; r < Q; r += 32)
        bulk_copy_g2s(st + (size_t)r * RS + kStagePad, src_row(r) + xs, (uint32_t)W * 2u, bar);
    if (pads) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = lane + 32 * k;
            if (r < Q) {
                uint16_t* dst = st + (size_t)r * RS;
                *reinterpret_cast<uint4*>(dst) = head[k];
                *reinterpret_cast<uint4*>(dst + kStagePad + W) = tail[k];
            }
        }
        mbar_arrive(bar);
    }
}

__device__ __forceinline__ uint32_t lds_word(const uint16_t* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

// Element offsets, within a staged row, of the words a consumer thread reads:
// o[0] = word p - 1, o[1] = word p + 1, o[2] = word p (of the tile). For a
// whole-row tile (W = nx, a power of two here) the words across the ends are
// the row's own, modulo W; otherwise the pads hold them.
struct StageOff {
    int o[3];
    __device__ __forceinline__ StageOff(int W, bool whole, int p)
    {
        const int m = whole ? W - 1 : -1;   // all ones: no wrap
        o[0] = kStagePad + ((2 * p - 2) & m);
        o[1] = kStagePad + ((2 * p + 2) & m);
        o[2] = kStagePad + 2 * p;
    }
};

// The pair's words of lattice L from its stage rows (rows = first row of L):
// word p of the tile on the even step, word p - e_x on the odd step, with the
// halves exchanged where the row wraps (as load_pair).
template <class L, bool ODD>
__device__ __forceinline__ void stage_load(const uint16_t* rows, int RS, const StageOff& so, const Seam& sm,
                                           uint32_t* w)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ex = ODD ? L::ex(i) : 0;
        constexpr int k = ex == 1 ? 0 : ex == -1 ? 1 : 2;
        w[i] = lds_word(rows + i * RS + so.o[k]);
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

// Collision form and occupancy per pair, from sweeps at 256^3 (FP16, ms per
// step even / odd): D3Q27xD3Q19 holds each node's FP32 values in an array
// (collide_pair_words, 128 registers, three blocks of four consumer warps
// per SM: 0.490 / 0.498) rather than streaming them from the packed words
// (96 registers, four blocks: 0.545 / 0.561; 80 registers with a one-stage
// ring, five blocks: 0.505 / 0.550); the smaller pairs stream (D3Q19xD3Q7
// 0.302 / 0.305 against 0.320 / 0.334 with the array form).
template <class P>
constexpr bool kStageStream = (P::QF + P::QG <= 34);
template <class P>
constexpr int kStageMinBlocks = kStageStream<P> ? 6 : 3;

template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(160, kStageMinBlocks<P>) k_step_staged(const __grid_constant__ StageArgs A)
{
    constexpr int Q = P::QF + P::QG;
    constexpr uint32_t S = kStageRing;
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = A.W, RS = W + 2 * kStagePad;
    const int nc = W / 2;   // consumer threads
    uint16_t* stages = reinterpret_cast<uint16_t*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * Q * RS * 2);
    uint64_t* empty = full + S;
    uint64_t* hook = empty + S;
    uint32_t* code = reinterpret_cast<uint32_t*>(hook + 1);
    for (int r = (int)threadIdx.x; r < Q; r += (int)blockDim.x) code[r] = stage_row_code<P, ODD>(r);
    if (threadIdx.x == 0) {
        // full: the expected bytes' arrival, and one per producer lane where it stores pads
        const uint32_t full_count = (ODD && W != A.geo.nx) ? 33u : 1u;
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&full[s], full_count);
            mbar_init(&empty[s], (uint32_t)nc / 32u);
        }
        mbar_init(hook, 1);
        // test hook: phase 0 of its barrier expects bytes that no copy delivers
        if (A.extra_tx) mbar_arrive_expect_tx(hook, A.extra_tx);
        fence_mbarrier_init();
    }
    __syncthreads();
    if (blockIdx.x >= A.ntiles) return;
    const int lane = (int)(threadIdx.x & 31);

    if ((int)threadIdx.x >= nc) {
        // producer: tile j of this block goes to stage j % S, use j / S
        uint32_t j = 0;
        bool ok = true;
        for (uint32_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++j) {
            const uint32_t s = j % S, u = j / S;
            if (j >= S) {
                // the consumers have loaded the stage's previous use
                ok = __all_sync(0xffffffffu, mbar_wait(&empty[s], (u - 1u) & 1u, A.spin_limit));
                if (!ok) break;
            }
            fence_proxy_async_smem();
            stage_issue<P, ODD>(A, stages + (size_t)s * Q * RS, &full[s], code, t);
        }
        if (!ok && lane == 0) atomicExch(A.err, 1);
        // the copies of the last stages filled land before the block can exit
        for (uint32_t i = j > S ? j - S : 0u; i < j; ++i) mbar_wait(&full[i % S], (i / S) & 1u, kStageDrainPolls);
        return;
    }

    unsigned short* fb = static_cast<unsigned short*>(A.f);
    unsigned short* gb = static_cast<unsigned short*>(A.g);
    const int p = (int)threadIdx.x;
    const StageOff so(W, W == A.geo.nx, p);
    uint32_t j = 0;
    for (uint32_t t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++j) {
        const uint32_t s = j % S, u = j / S;
        bool ok = mbar_wait(&full[s], u & 1u, A.spin_limit);
        if (A.extra_tx && j == 0 && ok) ok = mbar_wait(hook, 0u, A.spin_limit);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(A.err, 1);
            return;
        }
        const uint32_t row = t / (uint32_t)A.ntx;
        const int x0 = (int)(t - row * (uint32_t)A.ntx) * W + 2 * p;
        const Seam sm(A.geo, x0);
        uint32_t wf[P::QF], wg[P::QG];
        {
            const uint16_t* st = stages + (size_t)s * Q * RS;
            stage_load<typename P::LF, ODD>(st, RS, so, sm, wf);
            stage_load<typename P::LG, ODD>(st + (size_t)P::QF * RS, RS, so, sm, wg);
        }
        // the warp's words are in registers: hand the stage back
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if constexpr (kStageStream<P>) {
            collide_half_stream<P, FORCING, T, 0>(wf, wg, A.ph);
            collide_half_stream<P, FORCING, T, 1>(wf, wg, A.ph);
        } else {
            collide_pair_words<P, FORCING, T>(wf, wg, A.ph);
        }
        const int y = (int)(row % (uint32_t)A.geo.ny), z = (int)(row / (uint32_t)A.geo.ny);
        const PairAddr b(A.geo, (int)launder(x0), (int)launder(y), (int)launder(z));
        store_pair<typename P::LF, ODD>(fb, A.geo.n3, b, sm, wf);
        store_pair<typename P::LG, ODD>(gb, A.geo.n3, b, sm, wg);
    }
}

}  // namespace lbm

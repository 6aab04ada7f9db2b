// Kernel templates of the library: the fused AA stream-and-collide step,
// initialisation, population/field transfer and the diagnostics reduction.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Diagnostics (Eqs. 22-26), three deterministic passes.
// ---------------------------------------------------------------------------
enum DiagSlot : int {
    kDEk = 0, kDEp, kDEpsK, kDDrho, kDA, kDJx, kDJy, kDJz, kDUmax,   // pass 1
    kDEpsP, kDEpsKCurl,                                            // pass 2
    kDNumSlots
};
constexpr int kDiagPass1 = 9;
constexpr int kDiagPass2 = 2;
constexpr int kDiagBlock = 256;

struct DiagArgs {
    const void* f;
    const void* g;
    Geometry geo;
    Phys ph;
    int odd;
    float ep_scale;      // (G/N)^2 / (2 rho0^2)
    float epsk_scale;    // 2 nu
    float s_scale;       // -1 / (2 cs^2 tau_f)
    float epsp_scale;    // D (G/N)^2 / rho0^2
    float nu;
    float* fields;       // 4 * n3: rho', ux, uy, uz (written by pass 1, read by pass 2)
    double* partials;    // gridDim.x * kDNumSlots
    uint32_t idx0, idx1; // pass 1 reduces nodes [idx0, idx1) (a z-slab: its own planes only)
};

// Compensated (Kahan) FP32 running sum for a thread's share of a diagnostics
// reduction: within a few FP32 ulps of the exact sum of its terms, on the FP32
// pipes (this GPU's FP64 rate is a small fraction of its FP32 rate). The
// thread partials are then combined in FP64.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Block sum (the last slot a maximum if MAXLAST) of v into out[0..NV), for
// blocks of up to 256 threads, a whole number of warps, in any shape.
template <int NV, bool MAXLAST>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* out)
{
    __shared__ double sh[kDiagBlock / 32][NV];
    const int tid = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z));
    const int nwarps = (int)(blockDim.x * blockDim.y * blockDim.z) / 32;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double t = __shfl_down_sync(0xffffffffu, v[q], o);
            v[q] = (MAXLAST && q == NV - 1) ? fmax(v[q], t) : v[q] + t;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[wid][q] = v[q];
    }
    __syncthreads();
    if (tid < NV) {
        const int q = tid;
        double acc = sh[0][q];
        for (int w = 1; w < nwarps; ++w) acc = (MAXLAST && q == NV - 1) ? fmax(acc, sh[w][q]) : acc + sh[w][q];
        out[q] = acc;
    }
}

// What a kernel needs to add one node's diagnostics (pass 1): the scales of
// Eqs. 22-24 and of the non-equilibrium eps_k, the fields for pass 2 and the
// per-block partials.
struct DiagSink {
    float ep_scale;      // (G/N)^2 / (2 rho0^2)
    float epsk_scale;    // 2 nu
    float s_scale;       // -1 / (2 cs^2 tau_f)
    float* fields;       // 4 * n3: rho', ux, uy, uz
    double* partials;    // one row of kDNumSlots per block
};

// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

struct DiagAcc {
    KahanF acc[kDiagPass1 - 1];
    float umax = 0.f;
    // The pass-1 slots of this thread into one block row. The block sum is
    // carried as an unevaluated FP32 pair (hi + lo, two-sum at every add), so
    // the step kernels, which write one row per block, keep FP64-like
    // accuracy on the FP32 pipes; one thread per slot converts the pair.
    __device__ __forceinline__ void store_block(double* row)
    {
        __shared__ float sh[kDiagBlock / 32][kDiagPass1][2];
        const int tid = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z));
        const int nwarps = (int)(blockDim.x * blockDim.y * blockDim.z) / 32;
        const int lane = tid & 31, wid = tid >> 5;
        float hi[kDiagPass1], lo[kDiagPass1];
#pragma unroll
        for (int q = 0; q < kDiagPass1 - 1; ++q) {
            hi[q] = acc[q].s;
            lo[q] = -acc[q].c;
        }
        hi[kDUmax] = umax;
        lo[kDUmax] = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < kDiagPass1; ++q) {
                const float oh = __shfl_down_sync(0xffffffffu, hi[q], o);
                const float ol = __shfl_down_sync(0xffffffffu, lo[q], o);
                if (q == kDUmax) {
                    hi[q] = fmaxf(hi[q], oh);
                } else {
                    float t, e;
                    two_sum(hi[q], oh, t, e);
                    hi[q] = t;
                    lo[q] = lo[q] + ol + e;
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kDiagPass1; ++q) {
                sh[wid][q][0] = hi[q];
                sh[wid][q][1] = lo[q];
            }
        }
        __syncthreads();
        if (tid < kDiagPass1) {
            const int q = tid;
            float h = sh[0][q][0], l = sh[0][q][1];
            for (int w = 1; w < nwarps; ++w) {
                if (q == kDUmax) {
                    h = fmaxf(h, sh[w][q][0]);
                } else {
                    float t, e;
                    two_sum(h, sh[w][q][0], t, e);
                    h = t;
                    l = l + sh[w][q][1] + e;
                }
            }
            // the pair itself, in the slot's 8 bytes (k_diag_final with pass1_pairs)
            reinterpret_cast<float2*>(row)[q] = make_float2(h, l);
        }
    }
};

// One node's pass-1 diagnostics from its post-stream, pre-collision
// populations and moments, and its FP32 fields for pass 2. PAIRSUM: h holds
// each opposite pair as (sum, difference), the exact node_macro form;
// otherwise the raw deviations. Second moment of the deviations:
// M2 = sum e e h, Pi_neq = M2 - rho u u - drho cs^2 I; e e is the same for e
// and -e, so a pair contributes e e (h_i + h_j). D3Q7 lacks the fourth-order
// isotropy behind sum e e f_eq = rho u u + rho cs^2 I, so there the pair sums
// of f_eq(rho, u) are subtracted explicitly and the closed-form terms are not.
template <class P, bool PAIRSUM>
__device__ __forceinline__ void diag_node(const float* h, const Macro& m, const DiagSink& s, uint32_t n3,
                                          uint32_t idx, DiagAcc& d)
{
    using LF = typename P::LF;
    constexpr bool kExplicit = (LF::kQ == 7);
    const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
    sfor<0, kPairs<LF>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        float sp = PAIRSUM ? h[i] : h[i] + h[i + 1];
        if constexpr (kExplicit) {
            const float eu = e_dot<LF, i>(m.ux, m.uy, m.uz);
            sp -= 2.f * LF::w(i) * (m.drho + m.rho * (LF::half_inv_cs4 * eu * eu - LF::half_inv_cs2 * usq));
        }
        if constexpr (LF::ex(i) != 0) mxx += sp;
        if constexpr (LF::ey(i) != 0) myy += sp;
        if constexpr (LF::ez(i) != 0) mzz += sp;
        if constexpr (LF::ex(i) * LF::ey(i) == 1) mxy += sp;
        if constexpr (LF::ex(i) * LF::ey(i) == -1) mxy -= sp;
        if constexpr (LF::ex(i) * LF::ez(i) == 1) mxz += sp;
        if constexpr (LF::ex(i) * LF::ez(i) == -1) mxz -= sp;
        if constexpr (LF::ey(i) * LF::ez(i) == 1) myz += sp;
        if constexpr (LF::ey(i) * LF::ez(i) == -1) myz -= sp;
    });
    const float dc = kExplicit ? 0.f : m.drho * LF::cs2;
    const float rr = kExplicit ? 0.f : m.rho;
    // S = s_scale / rho * (Pi_neq + (u F + F u) / 2), F = (0, 0, Fz)
    const float pxx = mxx - rr * m.ux * m.ux - dc;
    const float pyy = myy - rr * m.uy * m.uy - dc;
    const float pzz = mzz - rr * m.uz * m.uz - dc + m.uz * m.Fz;
    const float pxy = mxy - rr * m.ux * m.uy;
    const float pxz = mxz - rr * m.ux * m.uz + 0.5f * m.ux * m.Fz;
    const float pyz = myz - rr * m.uy * m.uz + 0.5f * m.uy * m.Fz;
    const float ss = pxx * pxx + pyy * pyy + pzz * pzz + 2.f * (pxy * pxy + pxz * pxz + pyz * pyz);
    const float sfac = s.s_scale * m.irho;
    d.acc[kDEk].add(0.5f * usq);
    d.acc[kDEp].add(s.ep_scale * m.rho_p * m.rho_p);
    d.acc[kDEpsK].add(s.epsk_scale * sfac * sfac * ss);
    d.acc[kDDrho].add(m.drho);
    d.acc[kDA].add(m.a);
    d.acc[kDJx].add(m.jx);
    d.acc[kDJy].add(m.jy);
    d.acc[kDJz].add(m.jz);
    d.umax = fmaxf(d.umax, sqrtf(usq));
    if (s.fields) {
        s.fields[idx] = m.rho_p;
        s.fields[(size_t)n3 + idx] = m.ux;
        s.fields[2 * (size_t)n3 + idx] = m.uy;
        s.fields[3 * (size_t)n3 + idx] = m.uz;
    }
}

struct StepArgs {
    void* f;          // QF * n3 elements, slot-major (f[i][z][y][x])
    void* g;          // QG * n3 elements
    Geometry geo;
    Phys ph;
    DiagSink dg;      // used by the diagnosing variants only
    int z0;           // first z-plane of the launch (1 for a z-slab with ghost planes, else 0)
};

// The fused AA update of one node: load the QF + QG populations (coalesced
// along x), moments, coupled rho'/u solve, f and g collisions, store.
// hook(h, m) runs between the moments and the collisions (the diagnosing
// step kernels read the pre-collision state there).
template <class P, int FORCING, class T, bool ODD, class Hook>
__device__ __forceinline__ void update_node(void* fv, void* gv, const Geometry& geo, const Phys& ph, int x,
                                            int y, int z, Hook&& hook)
{
    const NodeAddr a = node_addr<T>(geo, x, y, z);
    T* __restrict__ f = static_cast<T*>(fv);
    T* __restrict__ g = static_cast<T*>(gv);
    const uint32_t n3 = geo.n3;
    constexpr bool kExact = std::is_same<T, float>::value;
    float h[P::QF], k[P::QG];
    load_node<typename P::LF, ODD, T>(f, n3, a, h);
    load_node<typename P::LG, ODD, T>(g, n3, a, k);
    collide_node<P, FORCING, kExact>(h, k, ph, hook);
    const NodeAddr b = node_addr<T>(geo, (int)launder(x), (int)launder(y), (int)launder(z));
    store_node<typename P::LF, ODD, T>(f, n3, b, h);
    store_node<typename P::LG, ODD, T>(g, n3, b, k);
}

template <class P, int FORCING, class T, bool ODD>
__device__ __forceinline__ void update_node(void* fv, void* gv, const Geometry& geo, const Phys& ph, int x,
                                            int y, int z)
{
    update_node<P, FORCING, T, ODD>(fv, gv, geo, ph, x, y, z, [](const float*, const Macro&) {});
}

// Three 256-thread blocks per SM (<= 85 registers): measured on the 256^3
// D3Q27xD3Q19 lattice, 2% faster for FP32 Shan-Chen and 16% for FP16 with one
// node per thread than the unconstrained allocation (up to 124 registers).
// D3Q27xD3Q27, whose 54 values per node spill up to 180 bytes at that cap,
// takes two (<= 128 registers). Pairs of at most 26 values (D3Q19xD3Q7,
// D3Q15xD3Q7) fit four blocks (64 registers) without spilling: D3Q19xD3Q7
// FP32 at 256^3 0.516 against 0.543 ms per step with three.
#ifndef LBM_STEP_MINBLOCKS
#define LBM_STEP_MINBLOCKS 3
#endif
template <class P>
constexpr int kStepMinBlocks = (P::QF + P::QG > 46) ? 2 : (P::QF + P::QG <= 26) ? 4 : LBM_STEP_MINBLOCKS;
// One AA step for every node of one lattice.
template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(256, kStepMinBlocks<P>) k_step(StepArgs args)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + args.z0;
    if (x >= args.geo.nx || y >= args.geo.ny) return;
    update_node<P, FORCING, T, ODD>(args.f, args.g, args.geo, args.ph, x, y, z);
}

// The same step, also reducing the diagnostics (pass 1) of its input state,
// the post-stream pre-collision populations of every node: one row of
// partials per block (blocks numbered x fastest), FP32 fields for pass 2.
// Three 256-thread blocks per SM, as k_step (80 registers, up to 8 bytes of
// spill): 1.22 ms at 256^3 against 1.41 ms with two blocks and no spill.
template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(256, 3) k_step_diag(StepArgs args)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    constexpr bool kExact = std::is_same<T, float>::value;
    DiagAcc d;
    if (x < args.geo.nx && y < args.geo.ny) {
        const uint32_t idx = (uint32_t)x + (uint32_t)args.geo.nx * ((uint32_t)y + (uint32_t)args.geo.ny * (uint32_t)z);
        update_node<P, FORCING, T, ODD>(args.f, args.g, args.geo, args.ph, x, y, z,
                                        [&](const float* h, const Macro& m) {
                                            diag_node<P, kExact>(h, m, args.dg, args.geo.n3, idx, d);
                                        });
    }
    const uint32_t blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    d.store_block(args.dg.partials + (size_t)blk * kDNumSlots);
}

// ---------------------------------------------------------------------------
// 16-bit storage, two nodes per thread, nx even, in the half-row order of the
// store (row_pos): thread k < half takes the 32-bit word k of its row, nodes
// k (low half) and k + half (high half), on both AA steps. The odd step reads
// slot opp(i) at x - e_i and writes slot i at x + e_i; both nodes move by the
// same e_x, so every access is the aligned word k - e_x or k + e_x of a
// neighbouring row. Where the row wraps the word arrives with its halves
// exchanged: word half - 1 read from k = 0 (e_x = 1) and written from k = 0
// (e_x = -1), word 0 read from k = half - 1 (e_x = -1) and written from
// k = half - 1 (e_x = 1). Those lanes exchange the halves in registers, in
// code that only the warps holding word 0 or word half - 1 run. Loads, stores
// and address arithmetic are shared by the two nodes.
// ---------------------------------------------------------------------------
template <class T>
struct Pack16;
template <>
struct Pack16<__half> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __low2float(*reinterpret_cast<const __half2*>(&w)); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __high2float(*reinterpret_cast<const __half2*>(&w)); }
    static __device__ __forceinline__ uint32_t pack(float a, float b)
    {
        const __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&v);
    }    static __device__ __forceinline__ uint32_t bits(float a) { return __half_as_ushort(__float2half_rn(a)); }
};
template <>
struct Pack16<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ uint32_t pack(float a, float b)
    {
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&v);
    }    static __device__ __forceinline__ uint32_t bits(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
};

// Element offsets of the words around the pair's word k within one slot
// array: X[0] = word k - 1, X[1] = word k + 1 (both wrapped), X[2] = word k
// (element 2 k = x0); Y and Z for y -1, 0, +1 and z -1, 0, +1.
struct PairAddr {
    uint32_t X[3], Y[3], Z[3];
    __device__ __forceinline__ PairAddr(const Geometry& g, int x0, int y, int z)
    {
        const int wm = (x0 == 0) ? g.nx - 2 : x0 - 2;
        const int wp = (x0 == g.nx - 2) ? 0 : x0 + 2;
        const int ym = (y == 0) ? g.ny - 1 : y - 1, yp = (y == g.ny - 1) ? 0 : y + 1;
        const int zm = (z == 0) ? g.nz - 1 : z - 1, zp = (z == g.nz - 1) ? 0 : z + 1;
        const uint32_t nxy = (uint32_t)g.nx * (uint32_t)g.ny;
        X[0] = wm; X[1] = wp; X[2] = x0;
        Y[0] = ym * g.nx; Y[1] = y * g.nx; Y[2] = yp * g.nx;
        Z[0] = zm * nxy; Z[1] = z * nxy; Z[2] = zp * nxy;
    }
    __device__ __forceinline__ uint32_t off(int p, int sy, int sz) const { return Z[sz + 1] + Y[sy + 1] + X[p]; }
};

// The seam lanes of a pair: k = 0 (first) and k = half - 1 (last), and
// whether any lane of the warp is one (a warp-uniform branch condition).
struct Seam {
    bool first, last, warp_first, warp_last;
    uint32_t sel_first, sel_last;   // byte-permute selectors: exchange halves on the seam lanes
    __device__ __forceinline__ Seam(const Geometry& g, int x0)
    {
        first = x0 == 0;
        last = x0 == g.nx - 2;
        sel_first = first ? 0x1032u : 0x3210u;
        sel_last = last ? 0x1032u : 0x3210u;
        const unsigned m = __activemask();
        warp_first = __any_sync(m, first);
        warp_last = __any_sync(m, last);
    }
};

// A seam slot's word in a warp that holds a seam lane: one byte permute with
// the lane's own selector, which exchanges the halves on the seam lane and
// keeps the word elsewhere (a select between the word and its permutation
// gives the same words, measured slower: D3Q19xD3Q7 FP16 odd step 0.287
// against 0.269 ms at 256^3).
__device__ __forceinline__ uint32_t seam_word(uint32_t w, uint32_t sel) { return __byte_perm(w, 0u, sel); }

// Streaming (evict-first) word loads that ask L2 for the whole 256-byte
// block, as the FP32 loads do: D3Q19xD3Q7 FP16 at 256^3 0.2638 against
// 0.2694 ms per step with plain loads, D3Q27xD3Q19 unchanged (0.4536 ms).
__device__ __forceinline__ uint32_t ld_word(const unsigned short* p)
{
    uint32_t v;
    asm volatile("ld.global.cs.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_word(unsigned short* p, uint32_t w)
{
    __stcs(reinterpret_cast<unsigned int*>(p), w);
}

template <class L, bool ODD>
__device__ __forceinline__ void load_pair(const unsigned short* __restrict__ b16, uint32_t n3, const PairAddr& a,
                                          const Seam& sm, uint32_t* w)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        if constexpr (!ODD) {
            w[i] = ld_word(b16 + (size_t)i * n3 + a.off(2, 0, 0));
        } else {
            // slot opp(i) at x - e_i: word k - e_x
            constexpr int p = ex == 1 ? 0 : ex == -1 ? 1 : 2;
            w[i] = ld_word(b16 + ((uint32_t)L::opp(i) * n3 + a.off(p, -ey, -ez)));
        }
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

template <class L, bool ODD>
__device__ __forceinline__ void store_pair(unsigned short* __restrict__ b16, uint32_t n3, const PairAddr& a,
                                           const Seam& sm, uint32_t* w)
{
    if constexpr (ODD) {
        if (sm.warp_first) {
            sfor<0, L::kQ>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr (L::ex(i) == -1) w[i] = seam_word(w[i], sm.sel_first);
            });
        }
        if (sm.warp_last) {
            sfor<0, L::kQ>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr (L::ex(i) == 1) w[i] = seam_word(w[i], sm.sel_last);
            });
        }
    }
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        if constexpr (!ODD) {
            st_word(b16 + (size_t)L::opp(i) * n3 + a.off(2, 0, 0), w[i]);
        } else {
            // slot i at x + e_i: word k + e_x
            constexpr int p = ex == 1 ? 1 : ex == -1 ? 0 : 2;
            st_word(b16 + ((uint32_t)i * n3 + a.off(p, ey, ez)), w[i]);
        }
    });
}

// Both nodes of a pair on the packed words, each node's values held as an
// FP32 array (for the diagnosing step, whose hook reads them, and the staged
// kernel; the plain step streams them, collide_half_stream): the low-half
// node, then the high-half node. Each node's results are packed two slots to a word by one
// conversion (slots 2m, 2m + 1; the last slot of an odd count alone); once
// the high-half node is unpacked the loaded words are dead, so at most one
// node's FP32 values and the other's packed results are live. One byte
// permute per slot then forms the stored words (low node, high node).
// hook(which, h, m) sees node `which` (0 low, 1 high) between its moments
// and its collisions.
template <int Q, class T>
__device__ __forceinline__ void pack_slots(const float* h, uint32_t* t)
{
#pragma unroll
    for (int i = 0; i < Q / 2; ++i) t[i] = Pack16<T>::pack(h[2 * i], h[2 * i + 1]);
    if constexpr (Q % 2) t[Q / 2] = Pack16<T>::pack(h[Q - 1], 0.f);
}
template <int Q>
__device__ __forceinline__ void merge_slots(const uint32_t* tlo, const uint32_t* thi, uint32_t* w)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) w[i] = __byte_perm(tlo[i / 2], thi[i / 2], (i & 1) ? 0x7632 : 0x5410);
}

template <class P, int FORCING, class T, class Hook>
__device__ __forceinline__ void collide_pair_words(uint32_t* wf, uint32_t* wg, const Phys& ph, Hook&& hook)
{
    uint32_t tf[(P::QF + 1) / 2], tg[(P::QG + 1) / 2];
    {
        float h[P::QF], k[P::QG];
#pragma unroll
        for (int i = 0; i < P::QF; ++i) h[i] = Pack16<T>::lo(wf[i]);
#pragma unroll
        for (int i = 0; i < P::QG; ++i) k[i] = Pack16<T>::lo(wg[i]);
        collide_node<P, FORCING, false>(h, k, ph, [&](const float* hh, const Macro& m) { hook(0, hh, m); });
        pack_slots<P::QF, T>(h, tf);
        pack_slots<P::QG, T>(k, tg);
    }
    {
        float h[P::QF], k[P::QG];
#pragma unroll
        for (int i = 0; i < P::QF; ++i) h[i] = Pack16<T>::hi(wf[i]);
#pragma unroll
        for (int i = 0; i < P::QG; ++i) k[i] = Pack16<T>::hi(wg[i]);
        collide_node<P, FORCING, false>(h, k, ph, [&](const float* hh, const Macro& m) { hook(1, hh, m); });
        uint32_t uf[(P::QF + 1) / 2], ug[(P::QG + 1) / 2];
        pack_slots<P::QF, T>(h, uf);
        pack_slots<P::QG, T>(k, ug);
        merge_slots<P::QF>(tf, uf, wf);
        merge_slots<P::QG>(tg, ug, wg);
    }
}

template <class P, int FORCING, class T>
__device__ __forceinline__ void collide_pair_words(uint32_t* wf, uint32_t* wg, const Phys& ph)
{
    collide_pair_words<P, FORCING, T>(wf, wg, ph, [](int, const float*, const Macro&) {});
}

// One node of a pair (HALF 0: low halves, 1: high halves) straight from the
// packed words: the moments in a first pass, then each opposite pair of
// slots unpacked again, updated and merged back into its half. The words are
// laundered between the passes so that the first pass's values die there:
// through the collision only the packed words, the node's coefficients and
// running values are live (80 registers, 24 warps per SM, against 128
// registers and 16 warps with the node's FP32 values held in an array).
// Unpacking every value twice costs less than the occupancy gains: at 256^3
// FP16 0.457 against 0.469 ms per step, D3Q19xD3Q7 0.264 against 0.282 ms.
// Per node the arithmetic is collide_node's short form.
template <class P, int FORCING, class T, int HALF>
__device__ __forceinline__ void collide_half_stream(uint32_t* wf, uint32_t* wg, const Phys& ph)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    using K = Pack16<T>;
    constexpr uint32_t sel = HALF ? 0x5410 : 0x3254;
    auto un = [](uint32_t w) { return HALF ? K::hi(w) : K::lo(w); };
    FastMoments<P> s(un(wf[0]), un(wg[0]));
    sfor<0, kPairs<LF>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        s.template f_pair<i>(un(wf[i]), un(wf[i + 1]));
    });
    sfor<0, kPairs<LG>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        s.template g_pair<i>(un(wg[i]), un(wg[i + 1]));
    });
    const Macro m = s.solve(ph);
#pragma unroll
    for (int i = 0; i < P::QF; ++i) wf[i] = launder(wf[i]);
#pragma unroll
    for (int i = 0; i < P::QG; ++i) wg[i] = launder(wg[i]);
    {
        const FastF<P, FORCING> c(m, ph);
        wf[0] = __byte_perm(wf[0], K::bits(c.rest(un(wf[0]))), sel);
        sfor<0, kPairs<LF>>([&](auto mc) {
            constexpr int i = 2 * decltype(mc)::value + 1;
            float a = un(wf[i]), b = un(wf[i + 1]);
            c.template pair<i>(a, b);
            wf[i] = __byte_perm(wf[i], K::bits(a), sel);
            wf[i + 1] = __byte_perm(wf[i + 1], K::bits(b), sel);
        });
    }
    {
        const FastG<P> c(m, ph);
        wg[0] = __byte_perm(wg[0], K::bits(c.rest(un(wg[0]))), sel);
        sfor<0, kPairs<LG>>([&](auto mc) {
            constexpr int i = 2 * decltype(mc)::value + 1;
            float a = un(wg[i]), b = un(wg[i + 1]);
            c.template pair<i>(a, b);
            wg[i] = __byte_perm(wg[i], K::bits(a), sel);
            wg[i + 1] = __byte_perm(wg[i + 1], K::bits(b), sel);
        });
    }
}

struct NoHook {
    __device__ void operator()(int, const float*, const Macro&) const {}
};

// One pair's AA update: loads, both collisions (streamed from the words for
// the plain step; collide_pair_words where a hook reads the nodes' values),
// stores.
template <class P, int FORCING, class T, bool ODD, class Hook>
__device__ __forceinline__ void update_pair(const StepArgs& args, int x0, int y, int z, Hook&& hook)
{
    const uint32_t n3 = args.geo.n3;
    unsigned short* fb = static_cast<unsigned short*>(args.f);
    unsigned short* gb = static_cast<unsigned short*>(args.g);
    uint32_t wf[P::QF], wg[P::QG];
    const Seam sm(args.geo, x0);
    {
        const PairAddr a(args.geo, x0, y, z);
        load_pair<typename P::LF, ODD>(fb, n3, a, sm, wf);
        load_pair<typename P::LG, ODD>(gb, n3, a, sm, wg);
    }
    if constexpr (std::is_same_v<std::decay_t<Hook>, NoHook>) {
        collide_half_stream<P, FORCING, T, 0>(wf, wg, args.ph);
        collide_half_stream<P, FORCING, T, 1>(wf, wg, args.ph);
    } else {
        collide_pair_words<P, FORCING, T>(wf, wg, args.ph, hook);
    }
    const PairAddr b(args.geo, (int)launder(x0), (int)launder(y), (int)launder(z));
    store_pair<typename P::LF, ODD>(fb, n3, b, sm, wf);
    store_pair<typename P::LG, ODD>(gb, n3, b, sm, wg);
}

// Three 256-thread blocks per SM (<= 85 registers) for D3Q27xD3Q19, whose
// 46 packed words stay live through the streaming collision; four (<= 64)
// for the smaller pairs.
template <class P>
constexpr int kStep2MinBlocks = (P::QF + P::QG <= 34) ? 4 : 3;

template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(256, kStep2MinBlocks<P>) k_step2(StepArgs args)
{
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + args.z0;
    if (x0 >= args.geo.nx || y >= args.geo.ny) return;
    update_pair<P, FORCING, T, ODD>(args, x0, y, z, NoHook{});
}

// k_step2 that also reduces the diagnostics (pass 1) of its input state, as
// k_step_diag does.
template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(256, 2) k_step2_diag(StepArgs args)
{
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    DiagAcc d;
    if (x0 < args.geo.nx && y < args.geo.ny) {
        const uint32_t row = (uint32_t)args.geo.nx * ((uint32_t)y + (uint32_t)args.geo.ny * (uint32_t)z);
        // nodes of the pair's word k = x0 / 2: k and k + half
        const uint32_t lo = row + (uint32_t)(x0 / 2);
        const uint32_t hi = lo + (uint32_t)(args.geo.nx / 2);
        update_pair<P, FORCING, T, ODD>(args, x0, y, z, [&](int which, const float* h, const Macro& m) {
            diag_node<P, false>(h, m, args.dg, args.geo.n3, which ? hi : lo, d);
        });
    }
    const uint32_t blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    d.store_block(args.dg.partials + (size_t)blk * kDNumSlots);
}

// Batched update: per-instance descriptor and launch arguments.
struct BatchInstance {
    void* f;
    void* g;
    Geometry geo;
    Phys ph;
    int variant;      // 4 * (0: D3Q27xD3Q19, 1: D3Q19xD3Q7) + forcing
    uint32_t tile0;   // first tile of this instance in the global tile list
    uint32_t tx, ty;  // tiles along x and y of one z-plane
    uint32_t flow0;   // persistent driver: first of its tiles in one step's list
    uint32_t nflow;   // and their number (ceil(n3 / flow_nodes))
};

struct BatchArgs {
    const BatchInstance* inst;
    const uint16_t* tile_inst;  // instance index of every tile
    uint32_t ntiles;
    uint32_t tile_begin;        // per-variant launches: the variant's tiles [tile_begin, tile_end)
    uint32_t tile_end;
    int steps;                  // time steps of one persistent launch
    int odd0;                   // AA layout parity at the start
    unsigned* sync;             // [2]: error flag raised by a wait that ran out
    unsigned spin_limit;        // polls before a wait gives up
    // persistent driver
    const uint16_t* flow_inst;  // instance of every tile of one step's list
    uint32_t flow_tiles;        // tiles in one step's list
    uint32_t flow_nodes;        // nodes per tile (a multiple of the block size)
    unsigned* flow;             // [0]: queue position counter; [1 + i]: tiles of instance i completed
    unsigned extra_dep;         // test hook: completions every dependency wait expects beyond the real ones
};

// Persistent driver: the descriptors travel by value in the kernel's
// parameter block (constant bank), like the single-lattice kernel's
// arguments, so the per-node code reads them as constant loads that the
// compiler can repeat instead of keeping ~18 values in registers.
constexpr int kFlowMaxInst = 320;   // 320 * 96 bytes + the arguments stay under the 32 KB parameter limit
struct FlowArgs {
    BatchArgs a;
    BatchInstance inst[kFlowMaxInst];
};

__device__ __forceinline__ void node_xyz(const Geometry& geo, uint32_t idx, int& x, int& y, int& z)
{
    x = (int)(idx % (uint32_t)geo.nx);
    uint32_t r = idx / (uint32_t)geo.nx;
    y = (int)(r % (uint32_t)geo.ny);
    z = (int)(r / (uint32_t)geo.ny);
}

// Populations from macroscopic fields, natural layout: f = f_eq(rho, u) + amp w xi_f,
// g = (rho' + rho0) Theta(u) + amp w xi_g, evaluated in FP64 then rounded to T.
// xi arrays are (27, n3) FP64 indexed by the canonical velocity code
// (ex+1)*9 + (ey+1)*3 + (ez+1), or null.
struct InitArgs {
    void* f;
    void* g;
    Geometry geo;
    const double* rho;
    const double* u;       // 3 * n3
    const double* rho_p;
    const double* xi_f;
    const double* xi_g;
    float amp_f;      // perturbation amplitude (the perturbation is arithmetic in FP32)
    double rho0;
};

// Equilibrium deviations w_i (rho_m1 + rho P_i) (Eq. 9). Evaluated in FP32 on
// these small numbers (relative error ~1e-7, below the FP32 store's own
// rounding); GB300's FP64 rate would make FP64 here the slowest part of an
// initialisation.
template <class L>
__device__ __forceinline__ void eq_dev(float rho_m1, float rho, float ux, float uy, float uz, float* out)
{
    const float usq = ux * ux + uy * uy + uz * uz;
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float eu = e_dot<L, i>(ux, uy, uz);
        const float Pi = eu * (L::inv_cs2 + L::half_inv_cs4 * eu) - L::half_inv_cs2 * usq;
        out[i] = L::w(i) * fmaf(rho, Pi, rho_m1);
    });
}

// IEEE 754 binary64 -> binary32 conversion, round to nearest, ties to even,
// on the integer pipes: this GPU's FP64 pipe runs at a small fraction of its
// FP32 rate, and with the hardware conversion (seven per node) the field
// initialisation was bound by it. The float keeps the double's sign, its
// exponent rebiased (1023 -> 127) and the top 23 of its 52 fraction bits; the
// 29 bits below decide the rounding, and a carry out of the fraction moves
// into the exponent (up to infinity) as IEEE rounding does. Zero is copied;
// doubles whose float is subnormal or out of range, infinities and NaNs take
// the hardware conversion.
__device__ __forceinline__ float d2f_rn(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    if ((b << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e < 1 || e > 254) return __double2float_rn(v);
    uint32_t r = (hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ++r;
    return __uint_as_float(r);
}

template <class L>
__device__ __forceinline__ int canon_code(int i)
{
    return (L::ex(i) + 1) * 9 + (L::ey(i) + 1) * 3 + (L::ez(i) + 1);
}

template <class P, class T>
__global__ void k_init_fields(InitArgs a)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    const uint32_t n3 = a.geo.n3;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        const double rho = a.rho[idx];
        const double ux = a.u[idx], uy = a.u[n3 + idx], uz = a.u[2 * (size_t)n3 + idx];
        const double rp = a.rho_p[idx];
        float hf[P::QF], hg[P::QG];
        const float uxf = d2f_rn(ux), uyf = d2f_rn(uy), uzf = d2f_rn(uz);
        eq_dev<LF>(d2f_rn(rho - 1.0), d2f_rn(rho), uxf, uyf, uzf, hf);
        // g_eq - w rho0 = w (rho' + (rho' + rho0) P)
        eq_dev<LG>(d2f_rn(rp), d2f_rn(rp + a.rho0), uxf, uyf, uzf, hg);
        T* f = static_cast<T*>(a.f);
        T* g = static_cast<T*>(a.g);
        const uint32_t sidx = store_index_t<T>(a.geo, idx);
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            float v = hf[i];
            if (a.xi_f) v += a.amp_f * LF::w(i) * d2f_rn(a.xi_f[(size_t)canon_code<LF>(i) * n3 + idx]);
            st_pop<T>(f + (size_t)i * n3 + sidx, v);
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            float v = hg[i];
            if (a.xi_g) v += a.amp_f * LG::w(i) * d2f_rn(a.xi_g[(size_t)canon_code<LG>(i) * n3 + idx]);
            st_pop<T>(g + (size_t)i * n3 + sidx, v);
        });
    }
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator: draw c of
// stream `seed` is the finaliser of seed + (c + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

struct TgvArgs {
    void* f;
    void* g;
    Geometry geo;
    const double* trig;   // sin(2 pi i / n), cos(2 pi i / n), i < n (n = nx = ny = nz)
    double U0;
    double noise;     // noise amplitude relative to U0 (0: pure Eq. 20)
    uint64_t seed;
    double rho0;
};

// Eq. 20 on the vertex grid x_i = 2 pi i / n, rho = 1, rho' = 0.
template <class P, class T>
__global__ void k_init_tgv(TgvArgs a)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    const uint32_t n3 = a.geo.n3;
    // the factors of Eq. 20 depend on one coordinate each: tabulated once
    // (FP64, by the host) instead of five FP64 trigonometric calls per node
    const double* sn = a.trig;
    const double* cs = a.trig + a.geo.nx;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        double ux = a.U0 * sn[x] * cs[y] * cs[z];
        double uy = -a.U0 * cs[x] * sn[y] * cs[z];
        double uz = 0.0;
        if (a.noise != 0.0) {
            ux += a.noise * a.U0 * uniform_pm1(a.seed, idx);
            uy += a.noise * a.U0 * uniform_pm1(a.seed, (uint64_t)n3 + idx);
            uz += a.noise * a.U0 * uniform_pm1(a.seed, 2ull * n3 + idx);
        }
        float hf[P::QF], hg[P::QG];
        eq_dev<LF>(0.f, 1.f, (float)ux, (float)uy, (float)uz, hf);
        eq_dev<LG>(0.f, (float)a.rho0, (float)ux, (float)uy, (float)uz, hg);
        T* f = static_cast<T*>(a.f);
        T* g = static_cast<T*>(a.g);
        const uint32_t sidx = store_index_t<T>(a.geo, idx);
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(f + (size_t)i * n3 + sidx, hf[i]);
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(g + (size_t)i * n3 + sidx, hg[i]);
        });
    }
}

// Full populations (FP64, natural order f[i][node] with this library's slot
// order) from/to the store, reading with the AA parity of the current layout.
struct PopArgs {
    void* f;
    void* g;
    Geometry geo;
    double* fout;     // QF * n3  (or input for k_set_pops)
    double* gout;     // QG * n3
    double rho0;
    int odd;          // layout parity
};

template <class P, class T>
__global__ void k_get_pops(PopArgs a)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    const uint32_t n3 = a.geo.n3;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na = node_addr<T>(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<LF, true, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<LG, true, T>(static_cast<const T*>(a.g), n3, na, k);
        } else {
            load_node<LF, false, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<LG, false, T>(static_cast<const T*>(a.g), n3, na, k);
        }
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.fout[(size_t)i * n3 + idx] = LF::wd(i) + (double)h[i];
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.gout[(size_t)i * n3 + idx] = LG::wd(i) * a.rho0 + (double)k[i];
        });
    }
}

// Populations of a list of nodes (FP64, node-major: out[k * Q + i]).
struct SampleArgs {
    const void* f;
    const void* g;
    Geometry geo;
    const int64_t* nodes;
    int64_t count;
    double* fout;
    double* gout;
    double rho0;
    int odd;
};

template <class P, class T>
__global__ void k_sample_pops(SampleArgs a)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.count; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t idx = (uint32_t)a.nodes[s];
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na = node_addr<T>(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<LF, true, T>(static_cast<const T*>(a.f), a.geo.n3, na, h);
            load_node<LG, true, T>(static_cast<const T*>(a.g), a.geo.n3, na, k);
        } else {
            load_node<LF, false, T>(static_cast<const T*>(a.f), a.geo.n3, na, h);
            load_node<LG, false, T>(static_cast<const T*>(a.g), a.geo.n3, na, k);
        }
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.fout[s * P::QF + i] = LF::wd(i) + (double)h[i];
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.gout[s * P::QG + i] = LG::wd(i) * a.rho0 + (double)k[i];
        });
    }
}

// Writes the natural layout.
template <class P, class T>
__global__ void k_set_pops(PopArgs a)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    const uint32_t n3 = a.geo.n3;
    T* f = static_cast<T*>(a.f);
    T* g = static_cast<T*>(a.g);
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        const uint32_t sidx = store_index_t<T>(a.geo, idx);
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(f + (size_t)i * n3 + sidx, (float)(a.fout[(size_t)i * n3 + idx] - LF::wd(i)));
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(g + (size_t)i * n3 + sidx,
                      (float)(a.gout[(size_t)i * n3 + idx] - LG::wd(i) * a.rho0));
        });
    }
}

template <class P, class T>
__global__ void __launch_bounds__(kDiagBlock) k_diag_moments(DiagArgs a)
{
    using LF = typename P::LF;
    const uint32_t n3 = a.geo.n3;
    const DiagSink sink{a.ep_scale, a.epsk_scale, a.s_scale, a.fields, a.partials};
    DiagAcc d;
    for (uint32_t idx = a.idx0 + blockIdx.x * blockDim.x + threadIdx.x; idx < a.idx1;
         idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na = node_addr<T>(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<LF, true, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, true, T>(static_cast<const T*>(a.g), n3, na, k);
        } else {
            load_node<LF, false, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, false, T>(static_cast<const T*>(a.g), n3, na, k);
        }
        const Macro m = node_macro<P>(h, k, a.ph);
        diag_node<P, true>(h, m, sink, n3, idx, d);
    }
    d.store_block(a.partials + (size_t)blockIdx.x * kDNumSlots);
}

#ifdef LBM_REDUCTION_KERNELS  // defined in exactly one translation unit
// Eqs. 25, 26 with second-order central differences of the pass-1 fields.
__global__ void __launch_bounds__(kDiagBlock) k_diag_gradients(DiagArgs a)
{
    const uint32_t n3 = a.geo.n3;
    const float* rp = a.fields;
    const float* ux = a.fields + n3;
    const float* uy = a.fields + 2 * (size_t)n3;
    const float* uz = a.fields + 3 * (size_t)n3;
    KahanF acc[kDiagPass2];
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na(a.geo, x, y, z);   // the FP32 fields are in node order
        const uint32_t xp = na.off(1, 0, 0), xm = na.off(-1, 0, 0);
        const uint32_t yp = na.off(0, 1, 0), ym = na.off(0, -1, 0);
        const uint32_t zp = na.off(0, 0, 1), zm = na.off(0, 0, -1);
        const float gx = 0.5f * (rp[xp] - rp[xm]);
        const float gy = 0.5f * (rp[yp] - rp[ym]);
        const float gz = 0.5f * (rp[zp] - rp[zm]);
        const float wx = 0.5f * (uz[yp] - uz[ym]) - 0.5f * (uy[zp] - uy[zm]);
        const float wy = 0.5f * (ux[zp] - ux[zm]) - 0.5f * (uz[xp] - uz[xm]);
        const float wz = 0.5f * (uy[xp] - uy[xm]) - 0.5f * (ux[yp] - ux[ym]);
        acc[0].add(a.epsp_scale * (gx * gx + gy * gy + gz * gz));
        acc[1].add(a.nu * (wx * wx + wy * wy + wz * wz));
    }
    double v[kDiagPass2] = {acc[0].value(), acc[1].value()};
    block_reduce_store<kDiagPass2, false>(v, a.partials + (size_t)blockIdx.x * kDNumSlots + kDiagPass1);
}

// Final pass: one block adds the per-block partials in a fixed order.
// Block b of the grid sums its share of the rows: pass-1 slots from the first
// nb1 rows, pass-2 slots from the first nb2, split into gridDim.x contiguous
// ranges in order. The pass-1 slots hold FP32 (hi, lo) pairs (DiagAcc; the
// diagnosing step kernels write one row per step block, 65536 rows at
// 256^3), summed with two-sum on the FP32 pipes; the pass-2 slots FP64
// values. With one block the totals go to out[0..kDNumSlots) as FP64; with
// more (a first level that spreads the row reads over the SMs) each block
// writes its row of out in the input's format.
__global__ void __launch_bounds__(kDiagBlock) k_diag_final(const double* partials, int nb1, int nb2, double* out)
{
    constexpr bool pass1_pairs = true;
    const int per1 = (nb1 + (int)gridDim.x - 1) / (int)gridDim.x;
    const int per2 = (nb2 + (int)gridDim.x - 1) / (int)gridDim.x;
    const int b1 = (int)blockIdx.x * per1, e1 = min(nb1, b1 + per1);
    const int b2 = (int)blockIdx.x * per2, e2 = min(nb2, b2 + per2);
    const bool pairs_out = pass1_pairs && gridDim.x > 1;
    double acc[kDNumSlots];
#pragma unroll
    for (int q = 0; q < kDNumSlots; ++q) acc[q] = 0.0;
    float hi[kDiagPass1], lo[kDiagPass1];
#pragma unroll
    for (int q = 0; q < kDiagPass1; ++q) hi[q] = lo[q] = 0.f;
    {
        for (int b = b1 + (int)threadIdx.x; b < e1; b += blockDim.x) {
            const float2* row = reinterpret_cast<const float2*>(partials + (size_t)b * kDNumSlots);
#pragma unroll
            for (int q = 0; q < kDiagPass1; ++q) {
                const float2 v = row[q];
                if (q == kDUmax) {
                    hi[q] = fmaxf(hi[q], v.x);
                } else {
                    float t, e;
                    two_sum(hi[q], v.x, t, e);
                    hi[q] = t;
                    lo[q] = lo[q] + v.y + e;
                }
            }
        }
        if (!pairs_out) {
#pragma unroll
            for (int q = 0; q < kDiagPass1; ++q) acc[q] = (double)hi[q] + (double)lo[q];
        }
    }
    for (int b = b2 + (int)threadIdx.x; b < e2; b += blockDim.x) {
#pragma unroll
        for (int q = kDiagPass1; q < kDNumSlots; ++q) acc[q] += partials[(size_t)b * kDNumSlots + q];
    }
    double* dst = out + (size_t)blockIdx.x * kDNumSlots;
    if (pairs_out) {
        // pass-1 pairs through the block in FP32 two-sum, pass-2 in FP64 below
        __shared__ float shp[kDiagBlock / 32][kDiagPass1][2];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < kDiagPass1; ++q) {
                const float oh = __shfl_down_sync(0xffffffffu, hi[q], o);
                const float ol = __shfl_down_sync(0xffffffffu, lo[q], o);
                if (q == kDUmax) {
                    hi[q] = fmaxf(hi[q], oh);
                } else {
                    float t, e;
                    two_sum(hi[q], oh, t, e);
                    hi[q] = t;
                    lo[q] = lo[q] + ol + e;
                }
            }
        }
        if (lane == 0)
            for (int q = 0; q < kDiagPass1; ++q) {
                shp[wid][q][0] = hi[q];
                shp[wid][q][1] = lo[q];
            }
        __syncthreads();
        if (threadIdx.x < kDiagPass1) {
            const int q = threadIdx.x;
            float h = shp[0][q][0], l = shp[0][q][1];
            for (int w = 1; w < kDiagBlock / 32; ++w) {
                if (q == kDUmax) {
                    h = fmaxf(h, shp[w][q][0]);
                } else {
                    float t, e;
                    two_sum(h, shp[w][q][0], t, e);
                    h = t;
                    l = l + shp[w][q][1] + e;
                }
            }
            reinterpret_cast<float2*>(dst)[q] = make_float2(h, l);
        }
    }
    __shared__ double sh[kDiagBlock / 32][kDNumSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q0 = pairs_out ? kDiagPass1 : 0;   // slots reduced in FP64 here
#pragma unroll
    for (int q = 0; q < kDNumSlots; ++q) {
        if (q < q0) continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, acc[q], o);
            acc[q] = (q == kDUmax) ? fmax(acc[q], t) : acc[q] + t;
        }
    }
    if (lane == 0)
        for (int q = q0; q < kDNumSlots; ++q) sh[wid][q] = acc[q];
    __syncthreads();
    if ((int)threadIdx.x >= q0 && threadIdx.x < kDNumSlots) {
        const int q = threadIdx.x;
        double v = sh[0][q];
        for (int w = 1; w < kDiagBlock / 32; ++w) v = (q == kDUmax) ? fmax(v, sh[w][q]) : v + sh[w][q];
        dst[q] = v;
    }
}

#endif  // LBM_REDUCTION_KERNELS

// Macroscopic fields (FP64) for the host: rho, u (3 blocks), rho'.
struct FieldArgs {
    const void* f;
    const void* g;
    Geometry geo;
    Phys ph;
    int odd;
    double* rho;
    double* u;
    double* rho_p;
};

template <class P, class T>
__global__ void k_get_fields(FieldArgs a)
{
    const uint32_t n3 = a.geo.n3;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na = node_addr<T>(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<typename P::LF, true, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, true, T>(static_cast<const T*>(a.g), n3, na, k);
        } else {
            load_node<typename P::LF, false, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, false, T>(static_cast<const T*>(a.g), n3, na, k);
        }
        const Macro m = node_macro<P>(h, k, a.ph);
        if (a.rho) a.rho[idx] = (double)m.rho;
        if (a.u) {
            a.u[idx] = (double)m.ux;
            a.u[(size_t)n3 + idx] = (double)m.uy;
            a.u[2 * (size_t)n3 + idx] = (double)m.uz;
        }
        if (a.rho_p) a.rho_p[idx] = (double)m.rho_p;
    }
}

}  // namespace lbm

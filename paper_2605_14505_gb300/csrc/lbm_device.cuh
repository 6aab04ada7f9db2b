// Device building blocks of the DDF lattice Boltzmann update (paper Section 2):
// velocity sets of Table A.1 in this library's slot order, the storage codec,
// the per-node moments and coupled rho'/u solve (Eqs. 6, 7, 12, 16-18), the
// BGK collisions with the four forcing schemes (Eqs. 5, 8-10, 11, 14, 15) and
// the AA-pattern address arithmetic.
//
// Populations are kept as deviations from the rest state: the store holds
// h_i = f_i - w_i (momentum, reference density 1) and k_i = g_i - w_i rho0
// (scalar). All arithmetic is FP32 on these small numbers; FP16/BF16 storage
// only changes the element type of the store.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

// Per-node arithmetic is host-callable as well, so that it can be checked
// against the oracle without a GPU.
#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

// ---------------------------------------------------------------------------
// Velocity sets. Slot order: rest, the 6 axis directions, the 12 edge
// directions, the 8 corners; for i >= 1 slots (2m-1, 2m) are opposite. D3Q19
// and D3Q7 are prefixes of D3Q27; D3Q15 is rest + axes + corners.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int q27_ex(int i)
{
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1,
                           0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int q27_ey(int i)
{
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0,
                           1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int q27_ez(int i)
{
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1,
                           1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
    return t[i];
}

template <int Q>
struct Lattice {
    static_assert(Q == 7 || Q == 15 || Q == 19 || Q == 27, "velocity set");
    static constexpr int kQ = Q;
    __host__ __device__ static constexpr int slot27(int i) { return (Q == 15 && i >= 7) ? i + 12 : i; }
    __host__ __device__ static constexpr int ex(int i) { return q27_ex(slot27(i)); }
    __host__ __device__ static constexpr int ey(int i) { return q27_ey(slot27(i)); }
    __host__ __device__ static constexpr int ez(int i) { return q27_ez(slot27(i)); }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr int norm2(int i) { return ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i); }
    // Table A.1 weights
    __host__ __device__ static constexpr double wd(int i)
    {
        return Q == 7    ? (norm2(i) == 0 ? 1.0 / 4.0 : 1.0 / 8.0)
               : Q == 15 ? (norm2(i) == 0 ? 2.0 / 9.0 : norm2(i) == 1 ? 1.0 / 9.0 : 1.0 / 72.0)
               : Q == 19 ? (norm2(i) == 0 ? 1.0 / 3.0 : norm2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                         : (norm2(i) == 0   ? 8.0 / 27.0
                            : norm2(i) == 1 ? 2.0 / 27.0
                            : norm2(i) == 2 ? 1.0 / 54.0
                                            : 1.0 / 216.0);
    }
    __host__ __device__ static constexpr float w(int i) { return (float)wd(i); }
    // lattice speed of sound squared (Table A.1) and the Hermite coefficients of Eq. 9
    static constexpr double cs2d = (Q == 7) ? 0.25 : 1.0 / 3.0;
    static constexpr float cs2 = (float)cs2d;
    static constexpr float inv_cs2 = (Q == 7) ? 4.0f : 3.0f;         // 1 / cs^2
    static constexpr float half_inv_cs4 = (Q == 7) ? 8.0f : 4.5f;    // 1 / (2 cs^4)
    static constexpr float half_inv_cs2 = (Q == 7) ? 2.0f : 1.5f;    // 1 / (2 cs^2)

    // The FP32 weights do not sum to exactly 1 (e.g. D3Q19: 1 + 1.5e-8), nor
    // does sum w e_x^2 equal cs^2 exactly. Summed over i, the FP32 equilibrium
    // w_i (X + Y P_i) then carries X (sum w - 1) + 1.5 Y |u|^2 (sum w e_x^2 /
    // cs^2 - sum w): a bias with a fixed sign every step. For the scalar
    // (X = rho', up to ~5 with the G = N/1024 split) it grows rho' by ~3e-5
    // over 1000 steps. The rest slot absorbs the exact residual:
    //   w_0 (...) += kMassCorr * X + kUsqCorr * Y |u|^2.
    __host__ __device__ static constexpr double sum_w_fp32()
    {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += (double)w(i);
        return s;
    }
    __host__ __device__ static constexpr double sum_wxx_fp32()
    {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += (double)w(i) * (double)(ex(i) * ex(i));
        return s;
    }
    static constexpr float kMassCorr = (float)(1.0 - sum_w_fp32());
    static constexpr float kUsqCorr = (float)(-1.5 * (sum_wxx_fp32() / cs2d - sum_w_fp32()));
};

template <int QF_, int QG_>
struct Pair {
    using LF = Lattice<QF_>;
    using LG = Lattice<QG_>;
    static constexpr int QF = QF_;
    static constexpr int QG = QG_;
};

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
LBM_HD void sfor(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------------------
// Storage codec (round to nearest even on store).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ float ld_pop(const T* p);
// Population loads are streaming (evict-first) and ask L2 to fetch the whole
// 256-byte block around the address. A warp's row segment is 128 bytes in
// FP32 (64 in 16-bit storage) and the next warps read the next ones, so the
// rest of the block arrives early: FP32 D3Q27xD3Q19 at 256^3 0.9087 against
// 0.9121-0.9128 ms per step (two boxes), D3Q19xD3Q7 0.5433 against 0.5509;
// the one-node 16-bit kernel 0.3-0.8 % faster. The block lies in the same
// mapped page as the address, so the hint never reaches past the
// allocation's pages.
__device__ __forceinline__ uint16_t ld_u16_stream(const void* p)
{
    uint16_t v;
    asm volatile("ld.global.cs.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ float ld_pop<float>(const float* p)
{
    float v;
    asm volatile("ld.global.cs.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ float ld_pop<__half>(const __half* p)
{
    return __half2float(__ushort_as_half(ld_u16_stream(p)));
}
template <>
__device__ __forceinline__ float ld_pop<__nv_bfloat16>(const __nv_bfloat16* p)
{
    return __bfloat162float(__ushort_as_bfloat16(ld_u16_stream(p)));
}
template <class T>
__device__ __forceinline__ void st_pop(T* p, float v);
template <>
__device__ __forceinline__ void st_pop<float>(float* p, float v) { __stcs(p, v); }
template <>
__device__ __forceinline__ void st_pop<__half>(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
template <>
__device__ __forceinline__ void st_pop<__nv_bfloat16>(__nv_bfloat16* p, float v)
{
    __stcs(p, __float2bfloat16_rn(v));
}

// ---------------------------------------------------------------------------
// Parameters (lattice units, FP32 for the update).
// ---------------------------------------------------------------------------
enum Forcing : int { kGuo = 0, kShanChen = 1, kEDM = 2, kHCZ = 3 };

// BGK with omega = 1/tau close to 2 (tau - 1/2 ~ 0.006 in the workloads):
// omega rounded to FP32 would move nu = cs^2 (tau - 1/2) by ~5e-6 relative, so
// the relaxation is written with delta = 2 - omega = (2 tau - 1) / tau, which
// FP32 holds to full relative precision:
//   f* = f + omega (f_eq - f) = 2 f_eq - f + delta (f - f_eq).
struct Phys {
    float delta_f;    // 2 - 1 / tau_f
    float delta_g;    // 2 - 1 / tau_g
    float G;          // gravity (Eq. 18)
    float beta;       // (d rho_b / dz)_LU (Eqs. 12, 13)
    float rho0;       // reference density (Eq. 15)
    float kappa;      // c_mom * (-beta): rho' = a + kappa * u_z (Eqs. 16, 17)
    float c_lbe;      // factor of S_i in the g update (Eq. 11)
    float guo_pref;   // 1 - 1 / (2 tau_f)
    float sc_tau;     // shift * tau_f of the Shan-Chen equilibrium velocity (Eq. 10)
    float guo_tau;    // tau_f - 1/2 = (1 - 1 / (2 tau_f)) tau_f: the Guo source over 1 / tau_f
};

struct Geometry {
    int nx, ny, nz;
    uint32_t n3;      // nx * ny * nz
};

// Order of the nodes of one row within each slot array. FP32 stores, and
// 16-bit stores with odd nx: node x at position x. 16-bit stores with even nx
// (half-row order, half = nx / 2): position 2 (x mod half) + (x >= half), so
// the 32-bit word w of a row holds nodes w (low half) and w + half (high
// half). A shift of the row by one node then moves both nodes of every word
// to the next word, so the two-nodes-per-thread kernel reads and writes whole
// aligned words on both AA steps; only where the row wraps (words 0 and
// half - 1) the two halves arrive exchanged.
__host__ __device__ __forceinline__ int row_pos(int x, int half)
{
    return half == 0 ? x : (x < half ? 2 * x : 2 * (x - half) + 1);
}

// half of a 16-bit store: nx / 2 for even nx, 0 (node order) for odd nx.
__host__ __device__ __forceinline__ int row_half(const Geometry& g)
{
    return (g.nx & 1) ? 0 : g.nx / 2;
}

// Element index, within a slot array of a 16-bit store, of the node with
// linear index idx.
__host__ __device__ __forceinline__ uint32_t store_index(const Geometry& g, uint32_t idx)
{
    const int half = row_half(g);
    if (half == 0) return idx;
    const int x = (int)(idx % (uint32_t)g.nx);
    return idx - (uint32_t)x + (uint32_t)row_pos(x, half);
}

// Neighbour offsets of one node with periodic wrap. off(s) with s = (sx, sy, sz)
// in {-1, 0, 1}^3 is the element index, within a slot array, of node
// (x + sx, y + sy, z + sz): its linear index, or with a row order (half > 0)
// the row's start plus the node's position in the row.
struct RowOrder {
    int half;
};
struct NodeAddr {
    uint32_t X[3], Y[3], Z[3];
    __device__ __forceinline__ NodeAddr(const Geometry& g, int x, int y, int z)
    {
        int xm = (x == 0) ? g.nx - 1 : x - 1, xp = (x == g.nx - 1) ? 0 : x + 1;
        int ym = (y == 0) ? g.ny - 1 : y - 1, yp = (y == g.ny - 1) ? 0 : y + 1;
        int zm = (z == 0) ? g.nz - 1 : z - 1, zp = (z == g.nz - 1) ? 0 : z + 1;
        uint32_t nxy = (uint32_t)g.nx * (uint32_t)g.ny;
        X[0] = xm; X[1] = x; X[2] = xp;
        Y[0] = ym * g.nx; Y[1] = y * g.nx; Y[2] = yp * g.nx;
        Z[0] = zm * nxy; Z[1] = z * nxy; Z[2] = zp * nxy;
    }
    __device__ __forceinline__ NodeAddr(const Geometry& g, int x, int y, int z, RowOrder r) : NodeAddr(g, x, y, z)
    {
        X[0] = row_pos((int)X[0], r.half);
        X[1] = row_pos(x, r.half);
        X[2] = row_pos((int)X[2], r.half);
    }
    __device__ __forceinline__ uint32_t off(int sx, int sy, int sz) const
    {
        return Z[sz + 1] + Y[sy + 1] + X[sx + 1];
    }
};

// NodeAddr in the order of a store of element type T: FP32 stores are never
// reordered, so their addressing has no run-time row order at all.
template <class T>
__device__ __forceinline__ NodeAddr node_addr(const Geometry& g, int x, int y, int z)
{
    if constexpr (std::is_same_v<T, float>) {
        return NodeAddr(g, x, y, z);
    } else {
        return NodeAddr(g, x, y, z, RowOrder{row_half(g)});
    }
}
template <class T>
__host__ __device__ __forceinline__ uint32_t store_index_t(const Geometry& g, uint32_t idx)
{
    if constexpr (std::is_same_v<T, float>) {
        return idx;
    } else {
        return store_index(g, idx);
    }
}

// AA pattern, in place. Natural layout (after an even number of steps): slot i at
// node x holds f_i(x). The even step reads slot i at x and writes the
// post-collision f_i* to slot opp(i) at x. The odd step reads f_i(x) =
// f_i*(x - e_i) from slot opp(i) at x - e_i and writes f_i* to slot i at
// x + e_i, which restores the natural layout. Each location is read and then
// written by the same thread only, so the update is race-free in place.
template <class L, bool ODD>
struct AA {
    template <int I>
    __device__ __forceinline__ static uint32_t read_slot() { return ODD ? L::opp(I) : I; }
    template <int I>
    __device__ __forceinline__ static uint32_t read_off(const NodeAddr& a)
    {
        return ODD ? a.off(-L::ex(I), -L::ey(I), -L::ez(I)) : a.off(0, 0, 0);
    }
    template <int I>
    __device__ __forceinline__ static uint32_t write_slot() { return ODD ? I : L::opp(I); }
    template <int I>
    __device__ __forceinline__ static uint32_t write_off(const NodeAddr& a)
    {
        return ODD ? a.off(L::ex(I), L::ey(I), L::ez(I)) : a.off(0, 0, 0);
    }
};

// Element offsets are 32-bit (slot * n3 + node < 2^32 for every supported
// size); the 64-bit address is formed at each access.
#ifndef LBM_ADDR64
#define LBM_ADDR64 0
#endif
template <class L, bool ODD, class T>
__device__ __forceinline__ void load_node(const T* __restrict__ base, uint32_t n3, const NodeAddr& a,
                                          float* v)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
#if LBM_ADDR64
        const T* p = base + AA<L, ODD>::template read_off<i>(a);
        v[i] = ld_pop<T>(p + (size_t)AA<L, ODD>::template read_slot<i>() * n3);
#else
        v[i] = ld_pop<T>(base + (AA<L, ODD>::template read_slot<i>() * n3 +
                                 AA<L, ODD>::template read_off<i>(a)));
#endif
    });
}

template <class L, bool ODD, class T>
__device__ __forceinline__ void store_node(T* __restrict__ base, uint32_t n3, const NodeAddr& a,
                                           const float* v)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
#if LBM_ADDR64
        T* p = base + AA<L, ODD>::template write_off<i>(a);
        st_pop<T>(p + (size_t)AA<L, ODD>::template write_slot<i>() * n3, v[i]);
#else
        st_pop<T>(base + (AA<L, ODD>::template write_slot<i>() * n3 +
                          AA<L, ODD>::template write_off<i>(a)),
                  v[i]);
#endif
    });
}

// Returns v through an empty inline-asm move, so that the compiler cannot
// prove the result equal to v. The step kernel rebuilds its store addresses
// from laundered coordinates: otherwise common-subexpression elimination keeps
// all load addresses live through the collision (two registers each).
__device__ __forceinline__ uint32_t launder(uint32_t v)
{
    uint32_t r;
    asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
    return r;
}

// ---------------------------------------------------------------------------
// Moments and the coupled local solve.
// ---------------------------------------------------------------------------
// Near 1, FP32 resolves rho and 1/rho only to ~6e-8 absolute, and the
// rounding of rho * fl(1/rho) stays fixed at a node for many steps (drho moves
// slowly), rescaling the momentum coherently (E_k off by ~4e-5 after 1000
// steps). The update therefore uses the deviations drho = rho - 1 and
// dirho = 1/rho - 1, with rho X = X + drho X and X / rho = X + dirho X.
struct Macro {
    float drho;      // rho - 1
    float dirho;     // 1/rho - 1
    float rho, irho; // for the diagnostics only
    float jx, jy, jz;
    float a;         // sum g - rho0
    float rho_p;     // Eq. 16
    float Fz;        // Eq. 18
    float ux, uy, uz;  // Eq. 7
};

// Opposite slots (2m-1, 2m) carry e and -e, so their contributions to the
// moments are the pair sum and difference, and their equilibria share the
// even part of P and flip the odd part.
template <class L>
constexpr int kPairs = (L::kQ - 1) / 2;

template <class L, int I>
LBM_HD float e_dot(float ux, float uy, float uz)
{
    float eu = 0.f;
    if constexpr (L::ex(I) == 1) eu += ux;
    if constexpr (L::ex(I) == -1) eu -= ux;
    if constexpr (L::ey(I) == 1) eu += uy;
    if constexpr (L::ey(I) == -1) eu -= uy;
    if constexpr (L::ez(I) == 1) eu += uz;
    if constexpr (L::ez(I) == -1) eu -= uz;
    return eu;
}

// Moments of one node. EXACT (FP32 storage): on return each opposite pair
// (2m-1, 2m) of h and k holds its sum and difference, the form the exact
// collisions take, and rho, 1/rho enter only through their deviations from 1.
// !EXACT (16-bit storage, whose rounding of ~5e-4 per step dwarfs the 1e-8
// effects the exact forms remove): h and k are left as they are and the
// plain reciprocal is used.
// Quotient within 2 ulp (__fdividef on the device; the host build, used only
// to study the arithmetic, divides exactly).
LBM_HD float fast_div(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// Moment sums of one node for the short forms (16-bit storage), accumulated
// opposite pair by opposite pair, and the coupled solve. node_macro's short
// path and the two-node word kernels share it, so both give the same bits.
template <class P>
struct FastMoments {
    using LF = typename P::LF;
    float drho, jx, jy, jz, a;
    LBM_HD FastMoments(float h0, float k0) : drho(h0), jx(0.f), jy(0.f), jz(0.f), a(k0) {}
    template <int I>
    LBM_HD void f_pair(float hi, float hj)
    {
        const float sum = hi + hj;
        const float dif = hi - hj;
        drho += sum;
        if constexpr (LF::ex(I) == 1) jx += dif;
        if constexpr (LF::ex(I) == -1) jx -= dif;
        if constexpr (LF::ey(I) == 1) jy += dif;
        if constexpr (LF::ey(I) == -1) jy -= dif;
        if constexpr (LF::ez(I) == 1) jz += dif;
        if constexpr (LF::ez(I) == -1) jz -= dif;
    }
    template <int I>
    LBM_HD void g_pair(float ki, float kj) { a += ki + kj; }
    LBM_HD Macro solve(const Phys& ph) const
    {
        Macro m;
        m.drho = drho;
        m.jx = jx; m.jy = jy; m.jz = jz;
        m.a = a;
        m.rho = 1.f + drho;
        m.irho = 1.f / m.rho;
        m.dirho = m.irho - 1.f;
        // rho' = a + d, d = kappa j_z / rho - num x / (1 + x), as node_macro
        // forms it: a coherent rounding of the tiny x would compound over the
        // steps where the storage's own rounding averages out
        const float kj = ph.kappa * jz * m.irho;
        const float x = 0.5f * ph.kappa * ph.G * m.irho;
        m.rho_p = a + fmaf(-(a + kj), fast_div(x, 1.f + x), kj);
        m.Fz = -ph.G * m.rho_p;
        m.ux = jx * m.irho;
        m.uy = jy * m.irho;
        m.uz = (jz + 0.5f * m.Fz) * m.irho;
        return m;
    }
};

template <class P, bool EXACT = true>
LBM_HD Macro node_macro(float* h, float* k, const Phys& ph)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    if constexpr (!EXACT) {
        FastMoments<P> s(h[0], k[0]);
        sfor<0, kPairs<LF>>([&](auto mc) {
            constexpr int i = 2 * decltype(mc)::value + 1;
            s.template f_pair<i>(h[i], h[i + 1]);
        });
        sfor<0, kPairs<LG>>([&](auto mc) {
            constexpr int i = 2 * decltype(mc)::value + 1;
            s.template g_pair<i>(k[i], k[i + 1]);
        });
        return s.solve(ph);
    }
    Macro m;
    float drho = h[0], jx = 0.f, jy = 0.f, jz = 0.f, a = k[0];
    sfor<0, kPairs<LF>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        const float sum = h[i] + h[i + 1];
        const float dif = h[i] - h[i + 1];
        h[i] = sum;       // pair form, see collide_f
        h[i + 1] = dif;
        drho += sum;
        if constexpr (LF::ex(i) == 1) jx += dif;
        if constexpr (LF::ex(i) == -1) jx -= dif;
        if constexpr (LF::ey(i) == 1) jy += dif;
        if constexpr (LF::ey(i) == -1) jy -= dif;
        if constexpr (LF::ez(i) == 1) jz += dif;
        if constexpr (LF::ez(i) == -1) jz -= dif;
    });
    sfor<0, kPairs<LG>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        const float sum = k[i] + k[i + 1];
        k[i + 1] = k[i] - k[i + 1];
        k[i] = sum;
        a += sum;
    });
    m.drho = drho;
    m.jx = jx; m.jy = jy; m.jz = jz;
    m.a = a;
    m.dirho = -drho / (1.f + drho);
    m.rho = 1.f + drho;
    m.irho = 1.f + m.dirho;
    // rho' = a + kappa * u_z with u_z = (j_z - G rho' / 2) / rho  (Eqs. 7, 12, 16-18),
    // solved in closed form: rho' = num / (1 + x), num = a + kappa j_z / rho,
    // x = kappa G / (2 rho). In the workloads x ~ 1e-8 to 1e-6, so 1 + x
    // rounded in FP32 would be one fixed value for every node and step, and
    // num x / (1 + x) is itself below an ulp of num: subtracted from num it
    // rounds to a whole ulp (or none), on every node and step the same way, a
    // coherent shrinkage of rho' (E_p -2.5e-5 after 1000 steps at 128^3,
    // D3Q19xD3Q7, Fr 0.5). So the small part d = rho' - a = kappa j_z / rho -
    // num x / (1 + x) is formed first, where FP32 holds it to full relative
    // precision, and rho' = a + d is rounded once.
    const float kg = 0.5f * ph.kappa * ph.G;
    const float kj = ph.kappa * fmaf(jz, m.dirho, jz);
    const float num = a + kj;
    const float x = fmaf(kg, m.dirho, kg);
    m.rho_p = a + fmaf(-num, x / (1.f + x), kj);
    m.Fz = -ph.G * m.rho_p;
    const float jzf = jz + 0.5f * m.Fz;
    m.ux = fmaf(jx, m.dirho, jx);
    m.uy = fmaf(jy, m.dirho, jy);
    m.uz = fmaf(jzf, m.dirho, jzf);
    return m;
}

// BGK step of one population: f + omega (f_eq - f) = 2 f_eq - f + delta (f - f_eq).
LBM_HD float bgk(float f, float feq, float dl)
{
    return fmaf(dl, f - feq, 2.f * feq - f);
}

// Eq. 9 for deviations: f_eq_i - w_i = w_i (drho + rho P_i), with
// P_i = e.u / cs^2 + (e.u)^2 / (2 cs^4) - u^2 / (2 cs^2). For the pair (i, opp):
// f_eq = w (base + rho (e.u)^2 / (2 cs^4)) +- w rho e.u / cs^2, base = drho - rho u^2 / (2 cs^2).
//
// f collision (Eqs. 5, 8, 9) with the forcing scheme, in place on h.
template <class P, int FORCING>
LBM_HD void collide_f(float* h, const Macro& m, const Phys& ph)
{
    using LF = typename P::LF;
    constexpr float c1 = LF::inv_cs2, c2 = LF::half_inv_cs4, c0 = LF::half_inv_cs2;
    const float dl = ph.delta_f;
    // velocity of the equilibrium: u of Eq. 7 (Guo, HCZ), the Shan-Chen shifted
    // velocity of Eq. 10, or j / rho (EDM). Its momentum rho v is formed
    // without dividing by rho, so that the odd (momentum) part of f_eq,
    // w e.(rho v) / cs^2, carries no rounding of 1/rho: with rho = 1 + drho
    // rounded near 1, rho * (j / rho) differs from j by a rounding error that
    // follows the smooth fields and rescales the momentum coherently.
    float mx = m.jx, my = m.jy, mz;
    if constexpr (FORCING == kGuo || FORCING == kHCZ) {
        mz = m.jz + 0.5f * m.Fz;
    } else if constexpr (FORCING == kShanChen) {
        mz = m.jz + ph.sc_tau * m.Fz;
    } else {
        mz = m.jz;
    }
    const float vx = fmaf(mx, m.dirho, mx), vy = fmaf(my, m.dirho, my), vz = fmaf(mz, m.dirho, mz);
    const float vsq = vx * vx + vy * vy + vz * vz;
    float base = m.drho - c0 * (mx * vx + my * vy + mz * vz);
    // Guo: the source is linear in F, so it folds into the equilibrium that
    // the relaxation weights by 1/tau: S_i tau = (tau - 1/2) w [(e - v)/cs^2 +
    // (e.v) e / cs^4] . F adds (tau - 1/2) F_z to the momentum of the odd part
    // (mzo), 2 (tau - 1/2) F_z to the e.(rho v) factor of the even part (mze)
    // and -(tau - 1/2) F_z v_z / cs^2 to its base. Other schemes: mzo = mze = mz.
    float mze = mz, mzo = mz;
    if constexpr (FORCING == kGuo) {
        const float gFo = ph.guo_tau * m.Fz;
        base = fmaf(-gFo * c1, vz, base);
        mze = fmaf(2.f, gFo, mz);
        mzo = mz + gFo;
    }
    // forcing coefficients
    const float gF = ph.guo_pref * m.Fz;     // HCZ: (1 - 1/(2 tau)) F_z
    const float du = fmaf(m.Fz, m.dirho, m.Fz);  // EDM: velocity increment F/rho (z only)
    const float dusq = du * (2.f * vz + du); // |v + du|^2 - |v|^2

    // rest slot (e = 0), with the exact FP32 weight-sum residual
    {
        float heq = LF::w(0) * base + LF::kMassCorr * m.drho + LF::kUsqCorr * (mx * vx + my * vy + mz * vz);
        float F0 = 0.f;   // (Guo: folded into base)
        if constexpr (FORCING == kHCZ) F0 = -gF * c1 * vz * LF::w(0) * (1.f - c0 * vsq);
        if constexpr (FORCING == kEDM) {
            const float rdusq = fmaf(m.drho, dusq, dusq);   // rho (|v + du|^2 - |v|^2)
            F0 = (-c0 * LF::w(0) + LF::kUsqCorr) * rdusq;
        }
        h[0] = bgk(h[0], heq, dl) + F0;
    }
    // Odd (momentum) parts: sum over pairs of e (f_eq_i - f_eq_j) must be the
    // momentum rho v exactly. With FP32 weights, sum w e_x^2 / cs^2 = 1 + eps
    // (eps ~ 1e-8), so the plain form w e.(rho v) / cs^2 would rescale the
    // momentum by ~(1 + 2 eps) every step (E_k off by ~5e-5 after 1000 steps).
    // The edge and corner pairs use the plain form; each axis pair takes the
    // residual. That residual is formed without rounding: on the smooth,
    // nearly two-dimensional Taylor-Green momenta the rounding errors of a
    // plain FP32 running sum of the edge/corner parts (and even a single
    // rounding of the exact residual, whose low bits sit near ties) follow
    // the momentum, a relative momentum bias of ~6e-9 (D3Q19) / ~2e-9
    // (D3Q27) per step that drifts E_k by ~5e-6 in 600 steps. So the sum is
    // compensated (Knuth's TwoSum), the residual stays an unevaluated pair
    // hi + lo, and the axis pair's new populations are formed so that each is
    // rounded once (relax_axis).
    float ox = 0.f, oy = 0.f, oz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    auto two_sum = [](float& s, float& c, float x) {
        const float t = s + x;
        const float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    };
    auto relax_pair = [&](auto mc, float ha) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        constexpr int j = i + 1;
        constexpr float w = LF::w(i);
        constexpr int ez = LF::ez(i);
        const float eu = e_dot<LF, i>(vx, vy, vz);
        const float em = e_dot<LF, i>(mx, my, mze);
        const float hs = w * fmaf(c2 * em, eu, base);
        float Fs = 0.f, Fa = 0.f;
        if constexpr (FORCING == kHCZ) {
            // (1 - 1/(2 tau)) (e - u).F / (rho cs^2) f_eq, f_eq = w rho (1 + P)
            const float ps = 1.f + c2 * eu * eu - c0 * vsq;
            const float pa = c1 * eu;
            const float c = gF * c1 * w;
            Fs = c * ((float)ez * pa - vz * ps);
            Fa = c * ((float)ez * ps - vz * pa);
        } else if constexpr (FORCING == kEDM) {
            // f_eq(v + du) - f_eq(v) in closed form
            float ps = -c0 * dusq;
            if constexpr (ez != 0) ps += c2 * du * (2.f * (float)ez * eu + du);
            Fs = w * fmaf(m.drho, ps, ps);
            Fa = (ez != 0) ? w * c1 * (float)ez * m.Fz : 0.f;     // w rho e_z du / cs^2
        }
        // Even and odd parts relax separately: forming hs +- ha first would round
        // the even part (density, stress) to the ulp of the much larger odd part.
        const float sp = bgk(h[i], 2.f * hs, dl) + 2.f * Fs;   // h_i + h_j
        const float dp = bgk(h[j], 2.f * ha, dl) + 2.f * Fa;   // h_i - h_j
        h[i] = 0.5f * (sp + dp);
        h[j] = 0.5f * (sp - dp);
    };
    sfor<3, kPairs<LF>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        const float ha = LF::w(i) * c1 * e_dot<LF, i>(mx, my, mzo);
        if constexpr (LF::ex(i) != 0) two_sum(ox, cx, (float)LF::ex(i) * ha);
        if constexpr (LF::ey(i) != 0) two_sum(oy, cy, (float)LF::ey(i) * ha);
        if constexpr (LF::ez(i) != 0) two_sum(oz, cz, (float)LF::ez(i) * ha);
        relax_pair(mc, ha);
    });
    // Axis pair with the odd part ha = hi + lo: the exact update
    // h_i' = (sp + dp) / 2, dp = bgk(d, 2 ha) + 2 Fa, is
    // hi + [sp / 2 + (delta - 1) n / 2 + (2 - delta) lo + Fa] with n = d - 2 hi
    // (exact near equilibrium); the bracket is far below hi in magnitude, so
    // its own roundings vanish in the final one. r0 = m / 2 - (sum) is exact
    // whenever the sum lies between m / 4 and m (Sterbenz; it is ~m / 3 for
    // D3Q19, ~5 m / 18 for D3Q27), and hi + lo = r0 - comp exactly (|r0| >>
    // |comp|).
    auto relax_axis = [&](auto mc, float r0, float comp) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        constexpr int j = i + 1;
        constexpr float w = LF::w(i);
        constexpr int ez = LF::ez(i);
        const float hi = r0 - comp;
        const float lo = (r0 - hi) - comp;
        const float eu = e_dot<LF, i>(vx, vy, vz);
        const float em = e_dot<LF, i>(mx, my, mze);
        const float hs = w * fmaf(c2 * em, eu, base);
        float Fs = 0.f, Fa = 0.f;
        if constexpr (FORCING == kHCZ) {
            const float ps = 1.f + c2 * eu * eu - c0 * vsq;
            const float pa = c1 * eu;
            const float c = gF * c1 * w;
            Fs = c * ((float)ez * pa - vz * ps);
            Fa = c * ((float)ez * ps - vz * pa);
        } else if constexpr (FORCING == kEDM) {
            float ps = -c0 * dusq;
            if constexpr (ez != 0) ps += c2 * du * (2.f * (float)ez * eu + du);
            Fs = w * fmaf(m.drho, ps, ps);
            Fa = (ez != 0) ? w * c1 * (float)ez * m.Fz : 0.f;
        }
        const float sp = bgk(h[i], 2.f * hs, dl) + 2.f * Fs;
        const float n = h[j] - 2.f * hi;
        const float t = fmaf(0.5f * dl, n, fmaf(-0.5f, n, fmaf(2.f - dl, lo, Fa)));   // delta kept exact
        h[i] = hi + fmaf(0.5f, sp, t);
        h[j] = -hi + fmaf(0.5f, sp, -t);
    };
    relax_axis(std::integral_constant<int, 0>{}, fmaf(0.5f, mx, -ox), cx);    // slots 1, 2: +-x
    relax_axis(std::integral_constant<int, 1>{}, fmaf(0.5f, my, -oy), cy);    // slots 3, 4: +-y
    relax_axis(std::integral_constant<int, 2>{}, fmaf(0.5f, mzo, -oz), cz);   // slots 5, 6: +-z
}

// g collision (Eqs. 11, 12, 14, 15): g_eq = (rho' + rho0) Theta(u), S_i = w_i (-u_z beta).
// For deviations: g_eq_i - w_i rho0 = w_i (rho' + (rho' + rho0) P_i).
template <class P>
LBM_HD void collide_g(float* k, const Macro& m, const Phys& ph)
{
    using LG = typename P::LG;
    constexpr float c1 = LG::inv_cs2, c2 = LG::half_inv_cs4, c0 = LG::half_inv_cs2;
    const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const float rr = m.rho_p + ph.rho0;
    const float src = ph.c_lbe * (-m.uz * ph.beta);
    const float base = m.rho_p - c0 * rr * usq;
    const float dl = ph.delta_g;
    {
        const float keq = LG::w(0) * base + LG::kMassCorr * m.rho_p + LG::kUsqCorr * rr * usq;
        k[0] = bgk(k[0], keq, dl) + (LG::w(0) + LG::kMassCorr) * src;
    }
    sfor<0, kPairs<LG>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        constexpr float w = LG::w(i);
        const float eu = e_dot<LG, i>(m.ux, m.uy, m.uz);
        const float ks = w * fmaf(rr * c2, eu * eu, base);
        const float ka = w * rr * c1 * eu;
        const float sp = bgk(k[i], 2.f * ks, dl) + 2.f * w * src;
        const float dp = bgk(k[i + 1], 2.f * ka, dl);
        k[i] = 0.5f * (sp + dp);
        k[i + 1] = 0.5f * (sp - dp);
    });
}

// ---------------------------------------------------------------------------
// Collisions for 16-bit storage. The same update as collide_f / collide_g
// written for fewer instructions: BGK as f* = (1 - omega) f + omega f_eq, with
// omega, the weight and the 1/rho of the equilibrium folded into one
// coefficient per weight class, and rho (e.u)^2 = (e.j)^2 / rho, so that each
// opposite pair costs e.j, two multiplies, three FMAs and an add/subtract.
// FP32 arithmetic still; its rounding is ~1e-7 of values stored to 2^-11
// (FP16) or 2^-8 (BF16). FastF and FastG hold one node's coefficients and
// update one opposite pair at a time: collide_f_fast / collide_g_fast apply
// them to one node's array, the two-node kernels to both halves of each
// packed 32-bit word.
// ---------------------------------------------------------------------------
template <class P, int FORCING>
struct FastF {
    using LF = typename P::LF;
    static constexpr float c1 = LF::inv_cs2, c2 = LF::half_inv_cs4, c0 = LF::half_inv_cs2;
    float om, cm;               // 1 / tau_f, 1 - 1 / tau_f
    float mx, my, mz;           // momentum of the equilibrium velocity (as in collide_f)
    float mv, base, vz, gFo, ob, o2, o1, gF, du, dusq, irho, rho, Fz, drho;
    LBM_HD FastF(const Macro& m, const Phys& ph)
    {
        om = 2.f - ph.delta_f;
        cm = ph.delta_f - 1.f;
        mx = m.jx;
        my = m.jy;
        if constexpr (FORCING == kGuo || FORCING == kHCZ) {
            mz = m.jz + 0.5f * m.Fz;
        } else if constexpr (FORCING == kShanChen) {
            mz = m.jz + ph.sc_tau * m.Fz;
        } else {
            mz = m.jz;
        }
        mv = (mx * mx + my * my + mz * mz) * m.irho;       // rho |v|^2
        base = m.drho - c0 * mv;
        // forcing (Eqs. 8-10 and the cited schemes); v = j_eq / rho
        vz = mz * m.irho;
        // Guo folded into the equilibrium as in collide_f: base - (tau - 1/2) F_z v_z / cs^2,
        // e.j + 2 (tau - 1/2) F_z e_z in the even part, e.j + (tau - 1/2) F_z e_z in the odd part
        gFo = (FORCING == kGuo) ? ph.guo_tau * m.Fz : 0.f;
        if constexpr (FORCING == kGuo) base = fmaf(-gFo * c1, vz, base);
        ob = om * base;               // omega (f_eq_i - w_i) / w_i without the e terms
        o2 = om * c2 * m.irho;        // omega rho (e.v)^2 / (2 cs^4) per (e.j)^2
        o1 = om * c1;                 // omega rho e.v / cs^2 per e.j
        gF = ph.guo_pref * m.Fz;
        du = m.Fz * m.irho;
        dusq = du * (2.f * vz + du);
        irho = m.irho;
        rho = m.rho;
        Fz = m.Fz;
        drho = m.drho;
    }
    // the rest population
    LBM_HD float rest(float h0) const
    {
        const float heq = LF::w(0) * base + LF::kMassCorr * drho + LF::kUsqCorr * mv;
        float F0 = 0.f;   // (Guo: folded into base)
        if constexpr (FORCING == kHCZ) {
            const float vsq = mv * irho;
            F0 = -gF * c1 * vz * LF::w(0) * (1.f - c0 * vsq);
        }
        if constexpr (FORCING == kEDM) F0 = (-c0 * LF::w(0) + LF::kUsqCorr) * (rho * dusq);
        return fmaf(cm, h0, fmaf(om, heq, F0));
    }
    // the opposite pair (I, I + 1), in place
    template <int I>
    LBM_HD void pair(float& hi, float& hj) const
    {
        constexpr float w = LF::w(I);
        constexpr int ez = LF::ez(I);
        const float em = e_dot<LF, I>(mx, my, mz);
        float emo = em;          // e.j of the odd part
        float hs;
        if constexpr (FORCING == kGuo && ez != 0) {
            hs = fmaf((w * o2) * em, fmaf(2.f * (float)ez, gFo, em), w * ob);
            emo = fmaf((float)ez, gFo, em);
        } else {
            hs = fmaf((w * o2) * em, em, w * ob);
        }
        float ha = 0.f;          // forcing part of the odd term; the equilibrium part is (w o1) e.j
        if constexpr (FORCING == kHCZ) {
            const float eu = em * irho;
            const float ps = 1.f + c2 * eu * eu - c0 * mv * irho;
            const float pa = c1 * eu;
            const float c = gF * c1 * w;
            hs += c * ((float)ez * pa - vz * ps);
            ha += c * ((float)ez * ps - vz * pa);
        } else if constexpr (FORCING == kEDM) {
            float ps = -c0 * dusq;
            if constexpr (ez != 0) ps += c2 * du * (2.f * (float)ez * (em * irho) + du);
            hs += w * rho * ps;
            if constexpr (ez != 0) ha += w * c1 * (float)ez * Fz;
        }
        float hp = hs, hm = hs;
        if constexpr (FORCING == kHCZ || FORCING == kEDM) {
            hp = hs + ha;
            hm = hs - ha;
        }
        hi = fmaf(cm, hi, fmaf(w * o1, emo, hp));
        hj = fmaf(cm, hj, fmaf(-(w * o1), emo, hm));
    }
};

template <class P, int FORCING>
LBM_HD void collide_f_fast(float* h, const Macro& m, const Phys& ph)
{
    const FastF<P, FORCING> c(m, ph);
    h[0] = c.rest(h[0]);
    sfor<0, kPairs<typename P::LF>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        c.template pair<i>(h[i], h[i + 1]);
    });
}

template <class P>
struct FastG {
    using LG = typename P::LG;
    static constexpr float c1 = LG::inv_cs2, c2 = LG::half_inv_cs4, c0 = LG::half_inv_cs2;
    float om, cm;               // 1 / tau_g, 1 - 1 / tau_g
    float ux, uy, uz, usq, rr, src, base, rho_p, obs, a2, a1;
    LBM_HD FastG(const Macro& m, const Phys& ph)
    {
        om = 2.f - ph.delta_g;
        cm = ph.delta_g - 1.f;
        ux = m.ux; uy = m.uy; uz = m.uz;
        usq = ux * ux + uy * uy + uz * uz;
        rr = m.rho_p + ph.rho0;
        src = ph.c_lbe * (-uz * ph.beta);                  // S_i / w_i (Eq. 12)
        base = m.rho_p - c0 * rr * usq;
        rho_p = m.rho_p;
        obs = fmaf(om, base, src);
        a2 = om * rr * c2;
        a1 = om * rr * c1;
    }
    LBM_HD float rest(float k0) const
    {
        const float keq = LG::w(0) * base + LG::kMassCorr * rho_p + LG::kUsqCorr * rr * usq;
        return fmaf(cm, k0, fmaf(om, keq, (LG::w(0) + LG::kMassCorr) * src));
    }
    template <int I>
    LBM_HD void pair(float& ki, float& kj) const
    {
        constexpr float w = LG::w(I);
        const float eu = e_dot<LG, I>(ux, uy, uz);
        const float ks = fmaf((w * a2) * eu, eu, w * obs);
        ki = fmaf(cm, ki, fmaf(w * a1, eu, ks));
        kj = fmaf(cm, kj, fmaf(-(w * a1), eu, ks));
    }
};

template <class P>
LBM_HD void collide_g_fast(float* k, const Macro& m, const Phys& ph)
{
    const FastG<P> c(m, ph);
    k[0] = c.rest(k[0]);
    sfor<0, kPairs<typename P::LG>>([&](auto mc) {
        constexpr int i = 2 * decltype(mc)::value + 1;
        c.template pair<i>(k[i], k[i + 1]);
    });
}

// Moments, coupled solve and both collisions of one node, in place on h, k:
// the exact FP32 forms for FP32 storage, the short forms for 16-bit storage.
template <class P, int FORCING, bool EXACT, class Hook>
LBM_HD Macro collide_node(float* h, float* k, const Phys& ph, Hook&& hook)
{
    const Macro m = node_macro<P, EXACT>(h, k, ph);
    hook(static_cast<const float*>(h), m);
    if constexpr (EXACT) {
        collide_f<P, FORCING>(h, m, ph);
        collide_g<P>(k, m, ph);
    } else {
        collide_f_fast<P, FORCING>(h, m, ph);
        collide_g_fast<P>(k, m, ph);
    }
    return m;
}

template <class P, int FORCING, bool EXACT>
LBM_HD Macro collide_node(float* h, float* k, const Phys& ph)
{
    return collide_node<P, FORCING, EXACT>(h, k, ph, [](const float*, const Macro&) {});
}

}  // namespace lbm

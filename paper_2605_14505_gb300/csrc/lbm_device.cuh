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
__device__ __forceinline__ void sfor(F&& f)
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
template <>
__device__ __forceinline__ float ld_pop<float>(const float* p) { return __ldcs(p); }
template <>
__device__ __forceinline__ float ld_pop<__half>(const __half* p) { return __half2float(__ldcs(p)); }
template <>
__device__ __forceinline__ float ld_pop<__nv_bfloat16>(const __nv_bfloat16* p)
{
    return __bfloat162float(__ldcs(p));
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

struct Phys {
    float omega_f;    // 1 / tau_f
    float omega_g;    // 1 / tau_g
    float G;          // gravity (Eq. 18)
    float beta;       // (d rho_b / dz)_LU (Eqs. 12, 13)
    float rho0;       // reference density (Eq. 15)
    float kappa;      // c_mom * (-beta): rho' = a + kappa * u_z (Eqs. 16, 17)
    float c_lbe;      // factor of S_i in the g update (Eq. 11)
    float guo_pref;   // 1 - 1 / (2 tau_f)
    float sc_tau;     // shift * tau_f of the Shan-Chen equilibrium velocity (Eq. 10)
};

struct Geometry {
    int nx, ny, nz;
    uint32_t n3;      // nx * ny * nz
};

// Neighbour offsets of one node with periodic wrap. off(s) with s = (sx, sy, sz)
// in {-1, 0, 1}^3 is the linear index of node (x + sx, y + sy, z + sz).
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
    __device__ __forceinline__ uint32_t off(int sx, int sy, int sz) const
    {
        return Z[sz + 1] + Y[sy + 1] + X[sx + 1];
    }
};

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
template <class L, bool ODD, class T>
__device__ __forceinline__ void load_node(const T* __restrict__ base, uint32_t n3, const NodeAddr& a,
                                          float* v)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        v[i] = ld_pop<T>(base + (AA<L, ODD>::template read_slot<i>() * n3 +
                                 AA<L, ODD>::template read_off<i>(a)));
    });
}

template <class L, bool ODD, class T>
__device__ __forceinline__ void store_node(T* __restrict__ base, uint32_t n3, const NodeAddr& a,
                                           const float* v)
{
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        st_pop<T>(base + (AA<L, ODD>::template write_slot<i>() * n3 +
                          AA<L, ODD>::template write_off<i>(a)),
                  v[i]);
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
struct Macro {
    float drho;      // rho - 1
    float rho, irho;
    float jx, jy, jz;
    float a;         // sum g - rho0
    float rho_p;     // Eq. 16
    float Fz;        // Eq. 18
    float ux, uy, uz;  // Eq. 7
};

template <class P>
__device__ __forceinline__ Macro node_macro(const float* h, const float* k, const Phys& ph)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    Macro m;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, a = 0.f;
    sfor<0, LF::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        drho += h[i];
        if constexpr (LF::ex(i) == 1) jx += h[i];
        if constexpr (LF::ex(i) == -1) jx -= h[i];
        if constexpr (LF::ey(i) == 1) jy += h[i];
        if constexpr (LF::ey(i) == -1) jy -= h[i];
        if constexpr (LF::ez(i) == 1) jz += h[i];
        if constexpr (LF::ez(i) == -1) jz -= h[i];
    });
    sfor<0, LG::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        a += k[i];
    });
    m.drho = drho;
    m.rho = 1.f + drho;
    m.irho = 1.f / m.rho;
    m.jx = jx; m.jy = jy; m.jz = jz;
    m.a = a;
    // rho' = a + kappa * u_z with u_z = (j_z - G rho' / 2) / rho  (Eqs. 7, 12, 16-18),
    // solved in closed form.
    m.rho_p = (a + ph.kappa * jz * m.irho) / (1.f + 0.5f * ph.kappa * ph.G * m.irho);
    m.Fz = -ph.G * m.rho_p;
    m.ux = jx * m.irho;
    m.uy = jy * m.irho;
    m.uz = (jz + 0.5f * m.Fz) * m.irho;
    return m;
}

// Eq. 9 written for deviations: f_eq_i - w_i = w_i (drho + rho * P_i(u)),
// P_i = e.u / cs^2 + (e.u)^2 / (2 cs^4) - u^2 / (2 cs^2).
template <class L, int I>
__device__ __forceinline__ float hermite_P(float ux, float uy, float uz, float usq)
{
    float eu = 0.f;
    if constexpr (L::ex(I) == 1) eu += ux;
    if constexpr (L::ex(I) == -1) eu -= ux;
    if constexpr (L::ey(I) == 1) eu += uy;
    if constexpr (L::ey(I) == -1) eu -= uy;
    if constexpr (L::ez(I) == 1) eu += uz;
    if constexpr (L::ez(I) == -1) eu -= uz;
    return eu * (L::inv_cs2 + L::half_inv_cs4 * eu) - L::half_inv_cs2 * usq;
}

template <class L, int I>
__device__ __forceinline__ float e_dot(float ux, float uy, float uz)
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

// f collision (Eqs. 5, 8, 9 with the forcing scheme), in place on h.
template <class P, int FORCING>
__device__ __forceinline__ void collide_f(float* h, const Macro& m, const Phys& ph)
{
    using LF = typename P::LF;
    const float om = ph.omega_f;
    if constexpr (FORCING == kGuo || FORCING == kHCZ) {
        const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
        const float pref = ph.guo_pref * m.Fz;
        sfor<0, LF::kQ>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float Pi = hermite_P<LF, i>(m.ux, m.uy, m.uz, usq);
            const float heq = LF::w(i) * (m.drho + m.rho * Pi);
            float Fi;
            if constexpr (FORCING == kGuo) {
                // Guo, Zheng & Shi: (1 - 1/(2 tau)) w [ (e - u)/cs^2 + (e.u) e / cs^4 ] . F
                const float eu = e_dot<LF, i>(m.ux, m.uy, m.uz);
                Fi = pref * LF::w(i) *
                     (LF::inv_cs2 * ((float)LF::ez(i) - m.uz) + 2.f * LF::half_inv_cs4 * eu * (float)LF::ez(i));
            } else {
                // He-Chen-Zhang: (1 - 1/(2 tau)) (e - u).F / (rho cs^2) f_eq
                Fi = pref * LF::inv_cs2 * ((float)LF::ez(i) - m.uz) * LF::w(i) * (1.f + Pi);
            }
            h[i] = h[i] + om * (heq - h[i]) + Fi;
        });
    } else if constexpr (FORCING == kShanChen) {
        // Eq. 10: equilibrium at u_eq = j / rho + shift * tau_f F / rho
        const float vx = m.jx * m.irho, vy = m.jy * m.irho;
        const float vz = (m.jz + ph.sc_tau * m.Fz) * m.irho;
        const float vsq = vx * vx + vy * vy + vz * vz;
        sfor<0, LF::kQ>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float heq = LF::w(i) * (m.drho + m.rho * hermite_P<LF, i>(vx, vy, vz, vsq));
            h[i] = h[i] + om * (heq - h[i]);
        });
    } else {
        // Exact difference method: BGK toward f_eq(rho, j/rho) plus
        // f_eq(rho, j/rho + F/rho) - f_eq(rho, j/rho)
        const float vx = m.jx * m.irho, vy = m.jy * m.irho, vz = m.jz * m.irho;
        const float vsq = vx * vx + vy * vy + vz * vz;
        const float wz = vz + m.Fz * m.irho;
        const float wsq = vx * vx + vy * vy + wz * wz;
        sfor<0, LF::kQ>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float P1 = hermite_P<LF, i>(vx, vy, vz, vsq);
            const float P2 = hermite_P<LF, i>(vx, vy, wz, wsq);
            const float heq = LF::w(i) * (m.drho + m.rho * P1);
            h[i] = h[i] + om * (heq - h[i]) + LF::w(i) * m.rho * (P2 - P1);
        });
    }
}

// g collision (Eqs. 11, 12, 14, 15): g_eq = (rho' + rho0) Theta(u), S_i = w_i (-u_z beta).
template <class P>
__device__ __forceinline__ void collide_g(float* k, const Macro& m, const Phys& ph)
{
    using LG = typename P::LG;
    const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const float rr = m.rho_p + ph.rho0;
    const float src = ph.c_lbe * (-m.uz * ph.beta);
    const float om = ph.omega_g;
    sfor<0, LG::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float keq = LG::w(i) * (m.rho_p + rr * hermite_P<LG, i>(m.ux, m.uy, m.uz, usq));
        k[i] = k[i] + om * (keq - k[i]) + LG::w(i) * src;
    });
}

}  // namespace lbm

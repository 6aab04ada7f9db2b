// Kernel templates of the library: the fused AA stream-and-collide step,
// initialisation, population/field transfer and the diagnostics reduction.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct StepArgs {
    void* f;          // QF * n3 elements, slot-major (f[i][z][y][x])
    void* g;          // QG * n3 elements
    Geometry geo;
    Phys ph;
};

// The fused AA update of one node: load the QF + QG populations (coalesced
// along x), moments, coupled rho'/u solve, f and g collisions, store.
template <class P, int FORCING, class T, bool ODD>
__device__ __forceinline__ void update_node(void* fv, void* gv, const Geometry& geo, const Phys& ph, int x,
                                            int y, int z)
{
    const NodeAddr a(geo, x, y, z);
    T* __restrict__ f = static_cast<T*>(fv);
    T* __restrict__ g = static_cast<T*>(gv);
    const uint32_t n3 = geo.n3;
    float h[P::QF], k[P::QG];
    load_node<typename P::LF, ODD, T>(f, n3, a, h);
    load_node<typename P::LG, ODD, T>(g, n3, a, k);
    const Macro m = node_macro<P>(h, k, ph);
    collide_f<P, FORCING>(h, m, ph);
    collide_g<P>(k, m, ph);
    const NodeAddr b(geo, (int)launder(x), (int)launder(y), (int)launder(z));
    store_node<typename P::LF, ODD, T>(f, n3, b, h);
    store_node<typename P::LG, ODD, T>(g, n3, b, k);
}

// One AA step for every node of one lattice.
template <class P, int FORCING, class T, bool ODD>
__global__ void __launch_bounds__(256) k_step(StepArgs args)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= args.geo.nx || y >= args.geo.ny) return;
    update_node<P, FORCING, T, ODD>(args.f, args.g, args.geo, args.ph, x, y, z);
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
};

struct BatchArgs {
    const BatchInstance* inst;
    const uint16_t* tile_inst;  // instance index of every tile
    uint32_t ntiles;
    int steps;                  // time steps of one persistent launch
    int odd0;                   // AA layout parity at the start
    unsigned* sync;             // grid barrier: arrivals, generation, error flag
    unsigned nblocks;           // blocks that must arrive at each barrier
    unsigned spin_limit;        // polls before a barrier wait gives up
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
    double amp;
    double rho0;
};

template <class L>
__device__ __forceinline__ void eq_dev_d(double rho_m1, double rho, double ux, double uy, double uz,
                                         double* out)
{
    const double c2 = L::cs2d;
    const double usq = ux * ux + uy * uy + uz * uz;
    sfor<0, L::kQ>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const double eu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
        const double Pi = eu / c2 + eu * eu / (2.0 * c2 * c2) - usq / (2.0 * c2);
        out[i] = L::wd(i) * (rho_m1 + rho * Pi);
    });
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
        double hf[P::QF], hg[P::QG];
        eq_dev_d<LF>(rho - 1.0, rho, ux, uy, uz, hf);
        // g_eq - w rho0 = w (rho' + (rho' + rho0) P)
        eq_dev_d<LG>(rp, rp + a.rho0, ux, uy, uz, hg);
        T* f = static_cast<T*>(a.f);
        T* g = static_cast<T*>(a.g);
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            double v = hf[i];
            if (a.xi_f) v += a.amp * LF::wd(i) * a.xi_f[(size_t)canon_code<LF>(i) * n3 + idx];
            st_pop<T>(f + (size_t)i * n3 + idx, (float)v);
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            double v = hg[i];
            if (a.xi_g) v += a.amp * LG::wd(i) * a.xi_g[(size_t)canon_code<LG>(i) * n3 + idx];
            st_pop<T>(g + (size_t)i * n3 + idx, (float)v);
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
    const double two_pi = 6.283185307179586476925286766559;
    const double dx = two_pi / a.geo.nx, dy = two_pi / a.geo.ny, dz = two_pi / a.geo.nz;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const double X = x * dx, Y = y * dy, Z = z * dz;
        double ux = a.U0 * sin(X) * cos(Y) * cos(Z);
        double uy = -a.U0 * cos(X) * sin(Y) * cos(Z);
        double uz = 0.0;
        if (a.noise != 0.0) {
            ux += a.noise * a.U0 * uniform_pm1(a.seed, idx);
            uy += a.noise * a.U0 * uniform_pm1(a.seed, (uint64_t)n3 + idx);
            uz += a.noise * a.U0 * uniform_pm1(a.seed, 2ull * n3 + idx);
        }
        double hf[P::QF], hg[P::QG];
        eq_dev_d<LF>(0.0, 1.0, ux, uy, uz, hf);
        eq_dev_d<LG>(0.0, a.rho0, ux, uy, uz, hg);
        T* f = static_cast<T*>(a.f);
        T* g = static_cast<T*>(a.g);
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(f + (size_t)i * n3 + idx, (float)hf[i]);
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(g + (size_t)i * n3 + idx, (float)hg[i]);
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
        const NodeAddr na(a.geo, x, y, z);
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
        const NodeAddr na(a.geo, x, y, z);
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
        sfor<0, P::QF>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(f + (size_t)i * n3 + idx, (float)(a.fout[(size_t)i * n3 + idx] - LF::wd(i)));
        });
        sfor<0, P::QG>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            st_pop<T>(g + (size_t)i * n3 + idx,
                      (float)(a.gout[(size_t)i * n3 + idx] - LG::wd(i) * a.rho0));
        });
    }
}

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
};

template <int NV, bool MAXLAST>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* out)
{
    __shared__ double sh[kDiagBlock / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    if (threadIdx.x < NV) {
        const int q = threadIdx.x;
        double acc = sh[0][q];
        for (int w = 1; w < kDiagBlock / 32; ++w) acc = (MAXLAST && q == NV - 1) ? fmax(acc, sh[w][q]) : acc + sh[w][q];
        out[q] = acc;
    }
}

template <class P, class T>
__global__ void __launch_bounds__(kDiagBlock) k_diag_moments(DiagArgs a)
{
    using LF = typename P::LF;
    const uint32_t n3 = a.geo.n3;
    double acc[kDiagPass1];
#pragma unroll
    for (int q = 0; q < kDiagPass1; ++q) acc[q] = 0.0;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<LF, true, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, true, T>(static_cast<const T*>(a.g), n3, na, k);
        } else {
            load_node<LF, false, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, false, T>(static_cast<const T*>(a.g), n3, na, k);
        }
        const Macro m = node_macro<P>(h, k, a.ph);
        // second moment of the deviations: M2 = sum e e h; Pi_neq = M2 - rho u u - drho cs^2 I.
        // node_macro left each opposite pair as (sum, difference); e e is the same
        // for e and -e, so a pair contributes e e (h_i + h_j), its stored sum.
        float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
        sfor<0, kPairs<LF>>([&](auto mc) {
            constexpr int i = 2 * decltype(mc)::value + 1;
            const float sp = h[i];
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
        const float dc = m.drho * LF::cs2;
        // S = s_scale / rho * (Pi_neq + (u F + F u) / 2), F = (0, 0, Fz)
        const float pxx = mxx - m.rho * m.ux * m.ux - dc;
        const float pyy = myy - m.rho * m.uy * m.uy - dc;
        const float pzz = mzz - m.rho * m.uz * m.uz - dc + m.uz * m.Fz;
        const float pxy = mxy - m.rho * m.ux * m.uy;
        const float pxz = mxz - m.rho * m.ux * m.uz + 0.5f * m.ux * m.Fz;
        const float pyz = myz - m.rho * m.uy * m.uz + 0.5f * m.uy * m.Fz;
        const float ss = pxx * pxx + pyy * pyy + pzz * pzz + 2.f * (pxy * pxy + pxz * pxz + pyz * pyz);
        const float sfac = a.s_scale * m.irho;
        const float usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
        acc[kDEk] += 0.5 * (double)usq;
        acc[kDEp] += (double)(a.ep_scale * m.rho_p * m.rho_p);
        acc[kDEpsK] += (double)(a.epsk_scale * sfac * sfac * ss);
        acc[kDDrho] += (double)m.drho;
        acc[kDA] += (double)m.a;
        acc[kDJx] += (double)m.jx;
        acc[kDJy] += (double)m.jy;
        acc[kDJz] += (double)m.jz;
        acc[kDUmax] = fmax(acc[kDUmax], (double)sqrtf(usq));
        if (a.fields) {
            a.fields[idx] = m.rho_p;
            a.fields[(size_t)n3 + idx] = m.ux;
            a.fields[2 * (size_t)n3 + idx] = m.uy;
            a.fields[3 * (size_t)n3 + idx] = m.uz;
        }
    }
    block_reduce_store<kDiagPass1, true>(acc, a.partials + (size_t)blockIdx.x * kDNumSlots);
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
    double acc[kDiagPass2] = {0.0, 0.0};
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3; idx += gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, idx, x, y, z);
        const NodeAddr na(a.geo, x, y, z);
        const uint32_t xp = na.off(1, 0, 0), xm = na.off(-1, 0, 0);
        const uint32_t yp = na.off(0, 1, 0), ym = na.off(0, -1, 0);
        const uint32_t zp = na.off(0, 0, 1), zm = na.off(0, 0, -1);
        const float gx = 0.5f * (rp[xp] - rp[xm]);
        const float gy = 0.5f * (rp[yp] - rp[ym]);
        const float gz = 0.5f * (rp[zp] - rp[zm]);
        const float wx = 0.5f * (uz[yp] - uz[ym]) - 0.5f * (uy[zp] - uy[zm]);
        const float wy = 0.5f * (ux[zp] - ux[zm]) - 0.5f * (uz[xp] - uz[xm]);
        const float wz = 0.5f * (uy[xp] - uy[xm]) - 0.5f * (ux[yp] - ux[ym]);
        acc[0] += (double)(a.epsp_scale * (gx * gx + gy * gy + gz * gz));
        acc[1] += (double)(a.nu * (wx * wx + wy * wy + wz * wz));
    }
    block_reduce_store<kDiagPass2, false>(acc, a.partials + (size_t)blockIdx.x * kDNumSlots + kDiagPass1);
}

// Final pass: one block adds the per-block partials in a fixed order.
__global__ void __launch_bounds__(kDiagBlock) k_diag_final(const double* partials, int nblocks, double* out)
{
    double acc[kDNumSlots];
#pragma unroll
    for (int q = 0; q < kDNumSlots; ++q) acc[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < kDNumSlots; ++q) {
            const double v = partials[(size_t)b * kDNumSlots + q];
            acc[q] = (q == kDUmax) ? fmax(acc[q], v) : acc[q] + v;
        }
    }
    __shared__ double sh[kDiagBlock / 32][kDNumSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDNumSlots; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, acc[q], o);
            acc[q] = (q == kDUmax) ? fmax(acc[q], t) : acc[q] + t;
        }
    }
    if (lane == 0)
        for (int q = 0; q < kDNumSlots; ++q) sh[wid][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < kDNumSlots) {
        const int q = threadIdx.x;
        double v = sh[0][q];
        for (int w = 1; w < kDiagBlock / 32; ++w) v = (q == kDUmax) ? fmax(v, sh[w][q]) : v + sh[w][q];
        out[q] = v;
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
        const NodeAddr na(a.geo, x, y, z);
        float h[P::QF], k[P::QG];
        if (a.odd) {
            load_node<typename P::LF, true, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, true, T>(static_cast<const T*>(a.g), n3, na, k);
        } else {
            load_node<typename P::LF, false, T>(static_cast<const T*>(a.f), n3, na, h);
            load_node<typename P::LG, false, T>(static_cast<const T*>(a.g), n3, na, k);
        }
        const Macro m = node_macro<P>(h, k, a.ph);
        a.rho[idx] = (double)m.rho;
        a.u[idx] = (double)m.ux;
        a.u[(size_t)n3 + idx] = (double)m.uy;
        a.u[2 * (size_t)n3 + idx] = (double)m.uz;
        a.rho_p[idx] = (double)m.rho_p;
    }
}

}  // namespace lbm

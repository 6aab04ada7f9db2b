// Host build of the library's per-node arithmetic (lbm_device.cuh is
// host-callable) that measures the rounding of the coupled rho' solve
// (Eqs. 7, 12, 16-18) against the same solve in FP64.
//
// A rounding that goes the same way on every node and every step compounds
// over a run; one that is unbiased averages out across the lattice. E_p is
// the mean of rho'^2 / 2 (Eq. 23), so a step changes it through
// sum rho' err; the statistic is that sum over sum rho'^2, the relative bias
// of rho' as E_p sees it, in units of 2^-23 (one FP32 ulp, relative). A
// negative value is a shrinkage of the scalar field, which lowers E_p step
// after step. Beside it: the same ratio for err^2 (its square root), the
// spread of the rounding.
//
// Usage: host_arith <pair 0: D3Q27xD3Q19, 1: D3Q19xD3Q7> <n> <Re> <Fr> <samples> <seed>
// Prints "<form> <bias> <spread>" for the FP32 form (node_macro) and the
// 16-bit short form (FastMoments).
#include "lbm_device.cuh"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

using namespace lbm;

namespace {

// SplitMix64 draws in [0, 1)
struct Rng {
    uint64_t s;
    double next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    double pm(double a) { return a * (2.0 * next() - 1.0); }
};

// Equilibrium deviations w (c + d P(u)) on lattice L, in FP64.
template <class L>
void eq(double c, double d, double ux, double uy, double uz, double* out)
{
    const double cs2 = 1.0 / L::inv_cs2, usq = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < L::kQ; ++i) {
        const double eu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
        out[i] = L::wd(i) * (c + d * (eu / cs2 + eu * eu / (2 * cs2 * cs2) - usq / (2 * cs2)));
    }
}

template <class P>
int run(int n, double Re, double Fr, long samples, uint64_t seed)
{
    using LF = typename P::LF;
    using LG = typename P::LG;
    constexpr int QF = P::QF, QG = P::QG;
    // the library's parameter mapping (Section 2.4, Eq. 19): U0 0.04, Pr 1,
    // G = N / 1024, beta = -N^2 rho0 / G, the printed scalar scheme
    const double U0 = 0.04, L = n / 6.283185307179586476925286766559;
    const double nu = U0 * L / Re, N = U0 / (Fr * L);
    const double tau_g = nu / (1.0 / LG::inv_cs2) + 0.5;
    Phys ph{};
    ph.G = (float)(N / 1024.0);
    ph.beta = (float)(-N * N / (N / 1024.0));
    ph.rho0 = 1.f;
    ph.kappa = (float)(0.5 * (1.0 - 1.0 / (2.0 * tau_g)) * (N * N / (N / 1024.0)));
    const double kap = ph.kappa, G = ph.G;
    Rng rng{seed};
    double sxe[2] = {0, 0}, se2[2] = {0, 0}, sx2 = 0;
    for (long s = 0; s < samples; ++s) {
        // a node of a stratified Taylor-Green state: rho near 1, |u| up to
        // U0, rho' over several binades of either sign
        const double drho = rng.pm(1e-3);
        const double ux = rng.pm(U0), uy = rng.pm(U0), uz = rng.pm(0.3 * U0);
        const double rp = (rng.next() < 0.5 ? -1.0 : 1.0) * std::pow(10.0, -3.0 + 4.0 * rng.next());
        double hf[27], hg[27];
        eq<LF>(drho, 1.0 + drho, ux, uy, uz, hf);
        eq<LG>(rp, rp + 1.0, ux, uy, uz, hg);
        float h[27], k[27];
        for (int i = 0; i < QF; ++i) h[i] = (float)(hf[i] + rng.pm(1e-6) * LF::wd(i));
        for (int i = 0; i < QG; ++i) k[i] = (float)(hg[i] + rng.pm(1e-6) * LG::wd(i));
        // FP64 solve from the same FP32 populations
        double d = 0, jz = 0, a = 0;
        for (int i = 0; i < QF; ++i) {
            d += h[i];
            jz += LF::ez(i) * (double)h[i];
        }
        for (int i = 0; i < QG; ++i) a += k[i];
        const double rho = 1.0 + d;
        const double exact = (a + kap * jz / rho) / (1.0 + kap * G / (2.0 * rho));
        float h1[27], k1[27], h2[27], k2[27];
        for (int i = 0; i < QF; ++i) h1[i] = h2[i] = h[i];
        for (int i = 0; i < QG; ++i) k1[i] = k2[i] = k[i];
        const Macro m1 = node_macro<P, true>(h1, k1, ph);
        const Macro m2 = node_macro<P, false>(h2, k2, ph);
        const double e1 = (double)m1.rho_p - exact, e2 = (double)m2.rho_p - exact;
        sx2 += exact * exact;
        sxe[0] += exact * e1;
        se2[0] += e1 * e1;
        sxe[1] += exact * e2;
        se2[1] += e2 * e2;
    }
    const double ulp = std::ldexp(1.0, -23);
    printf("fp32 %.6f %.6f\n", sxe[0] / sx2 / ulp, std::sqrt(se2[0] / sx2) / ulp);
    printf("short %.6f %.6f\n", sxe[1] / sx2 / ulp, std::sqrt(se2[1] / sx2) / ulp);
    return 0;
}

}  // namespace

int main(int argc, char** argv)
{
    if (argc < 7) {
        fprintf(stderr, "usage: host_arith pair n Re Fr samples seed\n");
        return 2;
    }
    const int pair = atoi(argv[1]), n = atoi(argv[2]);
    const double Re = atof(argv[3]), Fr = atof(argv[4]);
    const long samples = atol(argv[5]);
    const uint64_t seed = strtoull(argv[6], nullptr, 10);
    if (pair == 0) return run<Pair<27, 19>>(n, Re, Fr, samples, seed);
    if (pair == 1) return run<Pair<19, 7>>(n, Re, Fr, samples, seed);
    return 2;
}

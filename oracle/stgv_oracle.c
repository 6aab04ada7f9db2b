/*
 * stgv_oracle.c -- plain, slow FP64 CPU oracle of the double-distribution-
 * function (DDF) lattice Boltzmann update for the Boussinesq stratified
 * Taylor-Green vortex (paper: Section 2, Eqs. 5-18, Table A.1, Section 2.4).
 *
 * TEST INFRASTRUCTURE ONLY. The only code allowed to load this library is
 * tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py. The CUDA library shares no code, header, table or constant with
 * this file and neither one includes, links or loads the other.
 *
 * Layout: full populations f_i (not deviations), FP64, structure of arrays
 * f[i][z][y][x] with x fastest, two lattices and "pull" streaming. The
 * stencil tables are generated here by enumerating {-1,0,1}^3 and assigning
 * Table A.1's weight by |e|^2 (the GPU uses its own hand-written tables in a
 * different slot order; results are compared as fields or by velocity vector).
 *
 * One time step (paper order):
 *   1. moments rho = sum f (Eq. 6), j = sum e f (Eq. 7 first term), sigma = sum g;
 *   2. the coupled relations Eqs. 7, 12, 13, 16, 17, 18 (rho' needs u_z through
 *      R_i, u_z needs F, F needs rho') solved by fixed-point iteration to round-off;
 *   3. f collision, BGK (Eq. 8) with the equilibrium of Eq. 9 and the chosen
 *      forcing scheme (Guo, Shan-Chen velocity shift Eq. 10, EDM, HCZ);
 *   4. g collision, BGK (Eq. 14) toward g_eq = (rho' + rho0) Theta(u) (Eq. 15),
 *      plus the source S_i (Eqs. 11, 12);
 *   5. streaming f_i(x + e_i, t + 1) = f_i*(x, t) (Eqs. 5, 11), periodic.
 *
 * Readings taken where the paper is silent or inconsistent (listed in the
 * design notes as well):
 *   - Eq. 10 prints the Shan-Chen shift as tau_f F / (2 rho); with it the
 *     momentum gained per step is F/2, which contradicts Eq. 2. Default shift
 *     is the standard tau_f F / rho; params.sc_shift = 0.5 reproduces Eq. 10
 *     as printed.
 *   - Guo, EDM and HCZ are cited (Section 3.6) but not printed; the standard
 *     published forms are used (see collide_f below).
 *   - Eq. 11 adds S_i while Eq. 16 adds (1/2) sum R_i. Default follows the
 *     paper as printed (scalar_mode 0); scalar_mode 1 is the Chai-Shi
 *     consistent pair (add R_i in the LBE, (1/2) sum S_i in the moment).
 *   - The velocity entering Theta (Eq. 15) and S_i (Eq. 12) is the physical
 *     velocity of Eq. 7 in every forcing scheme. PARITY UNPINNED: no closed
 *     form separates this from using the shifted velocity under SC/EDM.
 *   - Initial populations are equilibria, f = f_eq(rho, u), g = g_eq(rho', u),
 *     optionally plus a seeded non-equilibrium perturbation. PARITY UNPINNED
 *     beyond the moment identities (the paper does not say).
 *   - Dissipation: eps_k from the non-equilibrium second moment (no finite
 *     differences), with the standard forcing correction of the strain rate;
 *     Eq. 25 (vorticity) and Eq. 26 (gradient of rho') are also evaluated
 *     with second-order central differences.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GUO 0
#define ORC_SC 1
#define ORC_EDM 2
#define ORC_HCZ 3

#define ORC_NDIAG 11
#define ORC_PI 3.14159265358979323846
#define ORC_G_OVER_N (1.0 / 1024.0)

typedef struct orc_params {
    int nx, ny, nz;
    int qf, qg;          /* momentum / scalar stencil sizes (7, 15, 19, 27) */
    int forcing;         /* ORC_GUO, ORC_SC, ORC_EDM, ORC_HCZ */
    int scalar_mode;     /* 0: Eqs. 11 and 16 as printed; 1: Chai-Shi pair */
    double tau_f;        /* Eq. 8: tau_f = nu / cs^2 + 1/2 */
    double tau_g;        /* Eq. 14: tau_g = D / cs^2 + 1/2 */
    double G;            /* gravitational acceleration, lattice units (Eq. 18) */
    double beta;         /* (d rho_b / d z)_LU, Eq. 13 */
    double rho0;         /* reference density (Eq. 3) */
    double sc_shift;     /* u_eq = j/rho + sc_shift * tau_f * F / rho */
} orc_params;

typedef struct orc_stencil {
    int q;
    int e[27][3];
    double w[27];
    double cs2;
} orc_stencil;

typedef struct orc_sim {
    orc_params p;
    orc_stencil sf, sg;
    size_t n3;
    double *f, *g;       /* current populations (post-stream, pre-collision) */
    double *ft, *gt;     /* post-collision scratch lattice */
    long long step;
} orc_sim;

/* ------------------------------------------------------------------------ */
/* Table A.1: D3Q7 (cs = 1/2), D3Q15, D3Q19, D3Q27 (cs = 1/sqrt 3).          */
/* Velocities grouped by |e|^2 = 0, 1, 2, 3; a group absent from a stencil  */
/* gets weight 0 and is dropped.                                            */
/* ------------------------------------------------------------------------ */
static int make_stencil(int q, orc_stencil* s)
{
    double wg[4] = {0, 0, 0, 0};
    double cs2;
    switch (q) {
    case 7:  cs2 = 1.0 / 4.0; wg[0] = 1.0 / 4.0; wg[1] = 1.0 / 8.0; break;
    case 15: cs2 = 1.0 / 3.0; wg[0] = 2.0 / 9.0; wg[1] = 1.0 / 9.0; wg[3] = 1.0 / 72.0; break;
    case 19: cs2 = 1.0 / 3.0; wg[0] = 1.0 / 3.0; wg[1] = 1.0 / 18.0; wg[2] = 1.0 / 36.0; break;
    case 27: cs2 = 1.0 / 3.0; wg[0] = 8.0 / 27.0; wg[1] = 2.0 / 27.0; wg[2] = 1.0 / 54.0;
             wg[3] = 1.0 / 216.0; break;
    default: return -1;
    }
    int k = 0;
    for (int ex = -1; ex <= 1; ++ex)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ez = -1; ez <= 1; ++ez) {
                int m = ex * ex + ey * ey + ez * ez;
                if (wg[m] == 0.0) continue;
                s->e[k][0] = ex; s->e[k][1] = ey; s->e[k][2] = ez;
                s->w[k] = wg[m];
                ++k;
            }
    s->q = k;
    s->cs2 = cs2;
    return (k == q) ? 0 : -1;
}

/* Eq. 9: second-order Hermite equilibrium on stencil st. */
static void equilibrium(const orc_stencil* st, double rho, const double u[3], double* feq)
{
    double c2 = st->cs2;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < st->q; ++i) {
        double eu = st->e[i][0] * u[0] + st->e[i][1] * u[1] + st->e[i][2] * u[2];
        feq[i] = rho * st->w[i] *
                 (1.0 + eu / c2 + (eu * eu) / (2.0 * c2 * c2) - usq / (2.0 * c2));
    }
}

/* Macroscopic state of one node (Eqs. 6, 7, 12, 16, 17, 18). */
typedef struct node_macro {
    double rho;      /* Eq. 6 */
    double j[3];     /* sum_i e_i f_i */
    double sigma;    /* sum_i g_i */
    double rho_p;    /* Eq. 16 */
    double F[3];     /* Eq. 18 */
    double u[3];     /* Eq. 7, physical velocity */
    double S[27];    /* Eq. 12, per scalar direction */
} node_macro;

static void macro_at(const orc_sim* s, size_t idx, node_macro* m)
{
    const orc_params* p = &s->p;
    const orc_stencil* sf = &s->sf;
    const orc_stencil* sg = &s->sg;
    m->rho = 0.0;
    m->j[0] = m->j[1] = m->j[2] = 0.0;
    for (int i = 0; i < sf->q; ++i) {
        double fi = s->f[(size_t)i * s->n3 + idx];
        m->rho += fi;
        m->j[0] += sf->e[i][0] * fi;
        m->j[1] += sf->e[i][1] * fi;
        m->j[2] += sf->e[i][2] * fi;
    }
    m->sigma = 0.0;
    for (int i = 0; i < sg->q; ++i) m->sigma += s->g[(size_t)i * s->n3 + idx];

    /* rho' appears on both sides of Eq. 16 (through R_i -> S_i -> u_z -> F).
     * Fixed-point iteration; the map is a contraction with factor
     * |(1/2)(1 - 1/(2 tau_g)) beta G / (2 rho)| << 1. */
    double rho_p = m->sigma - p->rho0;
    for (int it = 0; it < 200; ++it) {
        double Fz = -p->G * rho_p;                          /* Eq. 18 */
        double uz = m->j[2] / m->rho + Fz / (2.0 * m->rho); /* Eq. 7 */
        double sumS = 0.0, sumR = 0.0;
        for (int i = 0; i < sg->q; ++i) {
            double Si = sg->w[i] * (-uz * p->beta);         /* Eqs. 12, 13 */
            sumS += Si;
            sumR += (1.0 - 1.0 / (2.0 * p->tau_g)) * Si;    /* Eq. 17 */
        }
        double next;
        if (p->scalar_mode == 0)
            next = m->sigma + 0.5 * sumR - p->rho0;          /* Eq. 16 */
        else
            next = m->sigma + 0.5 * sumS - p->rho0;          /* Chai-Shi moment */
        double diff = fabs(next - rho_p);
        rho_p = next;
        if (diff <= 1e-16 * (1.0 + fabs(rho_p))) break;
    }
    m->rho_p = rho_p;
    m->F[0] = 0.0;
    m->F[1] = 0.0;
    m->F[2] = -p->G * rho_p;
    for (int a = 0; a < 3; ++a) m->u[a] = m->j[a] / m->rho + m->F[a] / (2.0 * m->rho);
    for (int i = 0; i < sg->q; ++i) m->S[i] = sg->w[i] * (-m->u[2] * p->beta);
}

/* Steps 3-4: collide node idx, writing post-collision values into ft/gt. */
static void collide_node(orc_sim* s, size_t idx)
{
    const orc_params* p = &s->p;
    const orc_stencil* sf = &s->sf;
    const orc_stencil* sg = &s->sg;
    node_macro m;
    macro_at(s, idx, &m);

    double f[27], feq[27], feq2[27], fout[27];
    for (int i = 0; i < sf->q; ++i) f[i] = s->f[(size_t)i * s->n3 + idx];
    double tf = p->tau_f;
    double c2 = sf->cs2;

    switch (p->forcing) {
    case ORC_GUO: {
        /* Guo, Zheng & Shi (2002): BGK toward f_eq(rho, u) with u of Eq. 7,
         * F_i = (1 - 1/(2 tau)) w_i [ (e_i - u)/cs^2 + (e_i.u) e_i / cs^4 ] . F */
        equilibrium(sf, m.rho, m.u, feq);
        for (int i = 0; i < sf->q; ++i) {
            double eu = sf->e[i][0] * m.u[0] + sf->e[i][1] * m.u[1] + sf->e[i][2] * m.u[2];
            double Fi = 0.0;
            for (int a = 0; a < 3; ++a)
                Fi += ((sf->e[i][a] - m.u[a]) / c2 + eu * sf->e[i][a] / (c2 * c2)) * m.F[a];
            Fi *= (1.0 - 1.0 / (2.0 * tf)) * sf->w[i];
            fout[i] = f[i] - (f[i] - feq[i]) / tf + Fi;
        }
        break;
    }
    case ORC_SC: {
        /* Shan-Chen (1993) velocity shift, Eq. 10: u_eq = j/rho + shift*tau F/rho */
        double ueq[3];
        for (int a = 0; a < 3; ++a) ueq[a] = m.j[a] / m.rho + p->sc_shift * tf * m.F[a] / m.rho;
        equilibrium(sf, m.rho, ueq, feq);
        for (int i = 0; i < sf->q; ++i) fout[i] = f[i] - (f[i] - feq[i]) / tf;
        break;
    }
    case ORC_EDM: {
        /* Exact difference method (Kupershtokh 2009): BGK toward f_eq(rho, j/rho)
         * plus f_eq(rho, j/rho + F/rho) - f_eq(rho, j/rho). */
        double u1[3], u2[3];
        for (int a = 0; a < 3; ++a) {
            u1[a] = m.j[a] / m.rho;
            u2[a] = u1[a] + m.F[a] / m.rho;
        }
        equilibrium(sf, m.rho, u1, feq);
        equilibrium(sf, m.rho, u2, feq2);
        for (int i = 0; i < sf->q; ++i) fout[i] = f[i] - (f[i] - feq[i]) / tf + (feq2[i] - feq[i]);
        break;
    }
    default: {
        /* HCZ (He-Shan-Doolen / He-Chen-Zhang): BGK toward f_eq(rho, u) plus
         * (1 - 1/(2 tau)) (e_i - u).F / (rho cs^2) f_eq_i(rho, u). */
        equilibrium(sf, m.rho, m.u, feq);
        for (int i = 0; i < sf->q; ++i) {
            double eF = 0.0;
            for (int a = 0; a < 3; ++a) eF += (sf->e[i][a] - m.u[a]) * m.F[a];
            double Fi = (1.0 - 1.0 / (2.0 * tf)) * eF / (m.rho * c2) * feq[i];
            fout[i] = f[i] - (f[i] - feq[i]) / tf + Fi;
        }
        break;
    }
    }
    for (int i = 0; i < sf->q; ++i) s->ft[(size_t)i * s->n3 + idx] = fout[i];

    /* Eqs. 11, 14, 15: g_eq = (rho' + rho0) Theta(u), Theta = f_eq / rho on the g stencil */
    double theta[27];
    equilibrium(sg, 1.0, m.u, theta);
    double c_lbe = (p->scalar_mode == 0) ? 1.0 : (1.0 - 1.0 / (2.0 * p->tau_g));
    for (int i = 0; i < sg->q; ++i) {
        double gi = s->g[(size_t)i * s->n3 + idx];
        double geq = (m.rho_p + p->rho0) * theta[i];
        s->gt[(size_t)i * s->n3 + idx] = gi - (gi - geq) / p->tau_g + c_lbe * m.S[i];
    }
}

static size_t wrap(long long v, int n)
{
    long long r = v % n;
    if (r < 0) r += n;
    return (size_t)r;
}

static size_t node_index(const orc_params* p, size_t x, size_t y, size_t z)
{
    return x + (size_t)p->nx * (y + (size_t)p->ny * z);
}

/* Step 5: pull streaming f_i(x) <- f_i*(x - e_i). */
static void stream_pull(orc_sim* s, const orc_stencil* st, const double* src, double* dst)
{
    const orc_params* p = &s->p;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t idx = node_index(p, x, y, z);
                for (int i = 0; i < st->q; ++i) {
                    size_t xs = wrap((long long)x - st->e[i][0], p->nx);
                    size_t ys = wrap((long long)y - st->e[i][1], p->ny);
                    size_t zs = wrap((long long)z - st->e[i][2], p->nz);
                    dst[(size_t)i * s->n3 + idx] = src[(size_t)i * s->n3 + node_index(p, xs, ys, zs)];
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Exported API                                                             */
/* ------------------------------------------------------------------------ */

int orc_stencil_info(int q, int* e, double* w, double* cs2)
{
    orc_stencil s;
    if (make_stencil(q, &s) != 0) return -1;
    for (int i = 0; i < s.q; ++i) {
        e[3 * i + 0] = s.e[i][0];
        e[3 * i + 1] = s.e[i][1];
        e[3 * i + 2] = s.e[i][2];
        w[i] = s.w[i];
    }
    *cs2 = s.cs2;
    return s.q;
}

int orc_equilibrium(int q, double rho, double ux, double uy, double uz, double* feq)
{
    orc_stencil s;
    if (make_stencil(q, &s) != 0) return -1;
    double u[3] = {ux, uy, uz};
    equilibrium(&s, rho, u, feq);
    return s.q;
}

/*
 * Section 2.4 and Eq. 19 -> lattice units. The box 2*pi holds n nodes, so the
 * reference length L = 1 is n / (2 pi) lattice spacings and the reference
 * velocity U = 1 is U0 lattice units. Re0 = U L / nu, Fr0 = U / (N L),
 * Sc = nu / D. Eq. 19 fixes only N^2 = -(G / rho0) d rho_b/dz; rho0 = 1 and
 * G = N / 1024, beta = -N^2 rho0 / G. The split matters only through the
 * compressible part of the scalar: the rho0 share of g_eq (Eq. 15) is
 * compressed by sound waves and G times that compression feeds them back
 * (growth rate ~ G / (2 cs)); a small G keeps this spurious acoustic growth
 * negligible over long runs while N, E_p (Eq. 23) and the Boussinesq limit are
 * unchanged.
 */
int orc_params_from_physics(orc_params* p, int n, int qf, int qg, int forcing,
                            double Re, double Fr, double Sc, double U0)
{
    orc_stencil sf, sg;
    if (n < 1 || Re <= 0.0 || Sc <= 0.0 || U0 <= 0.0 || !(Fr > 0.0)) return -1;
    if (make_stencil(qf, &sf) != 0 || make_stencil(qg, &sg) != 0) return -1;
    double L = n / (2.0 * ORC_PI);
    double nu = U0 * L / Re;
    double D = nu / Sc;
    double N = isinf(Fr) ? 0.0 : U0 / (Fr * L);
    memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = n;
    p->qf = qf;
    p->qg = qg;
    p->forcing = forcing;
    p->scalar_mode = 0;
    p->tau_f = nu / sf.cs2 + 0.5;
    p->tau_g = D / sg.cs2 + 0.5;
    p->rho0 = 1.0;
    p->G = ORC_G_OVER_N * N;
    p->beta = (N > 0.0) ? -N * N * p->rho0 / p->G : 0.0;
    p->sc_shift = 1.0;
    return 0;
}

orc_sim* orc_create(const orc_params* p)
{
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->forcing < 0 || p->forcing > 3) return NULL;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    if (make_stencil(p->qf, &s->sf) != 0 || make_stencil(p->qg, &s->sg) != 0) {
        free(s);
        return NULL;
    }
    s->n3 = (size_t)p->nx * p->ny * p->nz;
    s->f = (double*)calloc(s->n3 * s->sf.q, sizeof(double));
    s->ft = (double*)calloc(s->n3 * s->sf.q, sizeof(double));
    s->g = (double*)calloc(s->n3 * s->sg.q, sizeof(double));
    s->gt = (double*)calloc(s->n3 * s->sg.q, sizeof(double));
    if (!s->f || !s->ft || !s->g || !s->gt) {
        free(s->f); free(s->ft); free(s->g); free(s->gt); free(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->f); free(s->ft); free(s->g); free(s->gt);
    free(s);
}

long long orc_step_count(const orc_sim* s) { return s->step; }

/* Canonical code of a velocity e in {-1,0,1}^3, the index the seeded input
 * generator uses for its non-equilibrium perturbation arrays. */
static int velocity_code(const int e[3]) { return (e[0] + 1) * 9 + (e[1] + 1) * 3 + (e[2] + 1); }

/*
 * f = f_eq(rho, u) + amp * w_i * xi_f[code(e_i)],  g = g_eq(rho', u) + amp * w_i * xi_g[...]
 * rho, rho_p: n3 values; u: 3*n3 (ux block, uy block, uz block); xi_*: 27*n3 or NULL.
 */
int orc_init_fields(orc_sim* s, const double* rho, const double* u, const double* rho_p,
                    const double* xi_f, const double* xi_g, double amp)
{
    const orc_params* p = &s->p;
#pragma omp parallel for schedule(static)
    for (long long idx = 0; idx < (long long)s->n3; ++idx) {
        double uu[3] = {u[idx], u[s->n3 + idx], u[2 * s->n3 + idx]};
        double feq[27], theta[27];
        equilibrium(&s->sf, rho[idx], uu, feq);
        for (int i = 0; i < s->sf.q; ++i) {
            double v = feq[i];
            if (xi_f) v += amp * s->sf.w[i] * xi_f[(size_t)velocity_code(s->sf.e[i]) * s->n3 + idx];
            s->f[(size_t)i * s->n3 + idx] = v;
        }
        equilibrium(&s->sg, 1.0, uu, theta);
        for (int i = 0; i < s->sg.q; ++i) {
            double v = (rho_p[idx] + p->rho0) * theta[i];
            if (xi_g) v += amp * s->sg.w[i] * xi_g[(size_t)velocity_code(s->sg.e[i]) * s->n3 + idx];
            s->g[(size_t)i * s->n3 + idx] = v;
        }
    }
    s->step = 0;
    return 0;
}

int orc_set_populations(orc_sim* s, const double* f, const double* g)
{
    memcpy(s->f, f, sizeof(double) * s->n3 * s->sf.q);
    memcpy(s->g, g, sizeof(double) * s->n3 * s->sg.q);
    return 0;
}

int orc_get_populations(const orc_sim* s, double* f, double* g)
{
    memcpy(f, s->f, sizeof(double) * s->n3 * s->sf.q);
    memcpy(g, s->g, sizeof(double) * s->n3 * s->sg.q);
    return 0;
}

int orc_step(orc_sim* s, long long nsteps)
{
    const orc_params* p = &s->p;
    for (long long t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) collide_node(s, node_index(p, x, y, z));
        stream_pull(s, &s->sf, s->ft, s->f);
        stream_pull(s, &s->sg, s->gt, s->g);
        s->step += 1;
    }
    return 0;
}

/* Macroscopic fields of the current state: rho (Eq. 6), physical u (Eq. 7), rho' (Eq. 16). */
int orc_get_fields(const orc_sim* s, double* rho, double* u, double* rho_p)
{
#pragma omp parallel for schedule(static)
    for (long long idx = 0; idx < (long long)s->n3; ++idx) {
        node_macro m;
        macro_at(s, (size_t)idx, &m);
        if (rho) rho[idx] = m.rho;
        if (u) {
            u[idx] = m.u[0];
            u[s->n3 + idx] = m.u[1];
            u[2 * s->n3 + idx] = m.u[2];
        }
        if (rho_p) rho_p[idx] = m.rho_p;
    }
    return 0;
}

/*
 * Diagnostics of the current (post-stream, pre-collision) state, lattice units,
 * averages over the nx*ny*nz nodes:
 *   out[0]  E_k = < |u|^2 / 2 >                                  (Eq. 22)
 *   out[1]  E_p = < (G/N)^2 (rho'/rho0)^2 / 2 >                  (Eq. 23)
 *   out[2]  eps_k = 2 nu < S:S >, S from the non-equilibrium second moment:
 *           S = -[Pi_neq + (u F + F u)/2] / (2 rho cs^2 tau_f),
 *           Pi_neq = sum e e (f - f_eq(rho, u))
 *   out[3]  eps_p = D < (G/N)^2 |grad rho'|^2 / rho0^2 >          (Eq. 26, central differences)
 *   out[4]  eps_k(curl) = nu < |curl u|^2 >                       (Eq. 25, central differences)
 *   out[5]  sum_x sum_i f_i          out[6]  sum_x sum_i g_i
 *   out[7..9] sum_x sum_i e_i f_i    out[10] max_x |u|
 * Partial sums are taken per z plane, then added in plane order.
 */
int orc_diagnostics(const orc_sim* s, double* out)
{
    const orc_params* p = &s->p;
    const orc_stencil* sf = &s->sf;
    size_t n3 = s->n3;
    double* rp = (double*)malloc(sizeof(double) * n3);
    double* uf = (double*)malloc(sizeof(double) * 3 * n3);
    double* part = (double*)calloc((size_t)p->nz * 10, sizeof(double));
    if (!rp || !uf || !part) {
        free(rp); free(uf); free(part);
        return -1;
    }
    double nu = sf->cs2 * (p->tau_f - 0.5);
    double D = s->sg.cs2 * (p->tau_g - 0.5);
    double gn2 = (p->beta != 0.0) ? (-p->G * p->rho0 / p->beta) : 1.0; /* (G/N)^2 */

#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z) {
        double* acc = part + (size_t)z * 10;
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t idx = node_index(p, x, y, z);
                node_macro m;
                macro_at(s, idx, &m);
                rp[idx] = m.rho_p;
                uf[idx] = m.u[0];
                uf[n3 + idx] = m.u[1];
                uf[2 * n3 + idx] = m.u[2];
                double usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
                acc[0] += 0.5 * usq;
                acc[1] += 0.5 * gn2 * (m.rho_p / p->rho0) * (m.rho_p / p->rho0);
                double feq[27];
                equilibrium(sf, m.rho, m.u, feq);
                double Pi[3][3] = {{0}};
                double gsum = 0.0;
                for (int i = 0; i < sf->q; ++i) {
                    double fi = s->f[(size_t)i * n3 + idx];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) Pi[a][b] += sf->e[i][a] * sf->e[i][b] * (fi - feq[i]);
                    acc[2] += fi;
                }
                for (int i = 0; i < s->sg.q; ++i) gsum += s->g[(size_t)i * n3 + idx];
                acc[3] += gsum;
                double ss = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double Sab = -(Pi[a][b] + 0.5 * (m.u[a] * m.F[b] + m.F[a] * m.u[b])) /
                                     (2.0 * m.rho * sf->cs2 * p->tau_f);
                        ss += Sab * Sab;
                    }
                acc[4] += 2.0 * nu * ss;
                acc[5] += m.j[0];
                acc[6] += m.j[1];
                acc[7] += m.j[2];
                double um = sqrt(usq);
                if (um > acc[8]) acc[8] = um;
            }
    }
    double tot[10] = {0};
    for (int z = 0; z < p->nz; ++z) {
        for (int k = 0; k < 8; ++k) tot[k] += part[(size_t)z * 10 + k];
        if (part[(size_t)z * 10 + 8] > tot[8]) tot[8] = part[(size_t)z * 10 + 8];
        part[(size_t)z * 10 + 0] = 0.0;
        part[(size_t)z * 10 + 1] = 0.0;
    }

    /* Eqs. 25-26 with second-order central differences on the periodic grid. */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z) {
        double* acc = part + (size_t)z * 10;
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t xp = node_index(p, wrap(x + 1, p->nx), y, z), xm = node_index(p, wrap(x - 1, p->nx), y, z);
                size_t yp = node_index(p, x, wrap(y + 1, p->ny), z), ym = node_index(p, x, wrap(y - 1, p->ny), z);
                size_t zp = node_index(p, x, y, wrap(z + 1, p->nz)), zm = node_index(p, x, y, wrap(z - 1, p->nz));
                double gx = 0.5 * (rp[xp] - rp[xm]);
                double gy = 0.5 * (rp[yp] - rp[ym]);
                double gz = 0.5 * (rp[zp] - rp[zm]);
                acc[0] += D * gn2 * (gx * gx + gy * gy + gz * gz) / (p->rho0 * p->rho0);
                const double* ux = uf;
                const double* uy = uf + n3;
                const double* uz = uf + 2 * n3;
                double wx = 0.5 * (uz[yp] - uz[ym]) - 0.5 * (uy[zp] - uy[zm]);
                double wy = 0.5 * (ux[zp] - ux[zm]) - 0.5 * (uz[xp] - uz[xm]);
                double wz = 0.5 * (uy[xp] - uy[xm]) - 0.5 * (ux[yp] - ux[ym]);
                acc[1] += nu * (wx * wx + wy * wy + wz * wz);
            }
    }
    double epsp = 0.0, epsc = 0.0;
    for (int z = 0; z < p->nz; ++z) {
        epsp += part[(size_t)z * 10 + 0];
        epsc += part[(size_t)z * 10 + 1];
    }
    double inv = 1.0 / (double)n3;
    out[0] = tot[0] * inv;
    out[1] = tot[1] * inv;
    out[2] = tot[4] * inv;
    out[3] = epsp * inv;
    out[4] = epsc * inv;
    out[5] = tot[2];
    out[6] = tot[3];
    out[7] = tot[5];
    out[8] = tot[6];
    out[9] = tot[7];
    out[10] = tot[8];
    free(rp); free(uf); free(part);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_ndiag(void) { return ORC_NDIAG; }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }

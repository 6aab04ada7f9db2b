/*
 * lbm.h -- C ABI of the GB300 (sm_103a) double-distribution-function lattice
 * Boltzmann solver for the Boussinesq stratified Taylor-Green vortex.
 *
 * The operation behind this interface is the fused stream-and-collide update
 * of the paper's Section 2: momentum populations f_i on D3Q27 or D3Q19
 * (Eqs. 5-10), scalar populations g_i for the density perturbation rho' on
 * D3Q19 or D3Q7 (Eqs. 11-17), BGK relaxation (Eqs. 8, 14), the buoyancy force
 * F = (0, 0, -G rho') (Eq. 18) applied by the Guo source term, the Shan-Chen
 * velocity shift (Eq. 10), the exact difference method or the HCZ source term
 * (Section 3.6), the stencils of Table A.1, the Taylor-Green initial state of
 * Eq. 20 (Section 2.4) and the energy / dissipation diagnostics of Eqs. 22-26.
 *
 * Conventions.
 *  - Every function returns an int status: LBM_OK (0) or a negative LBM_E*
 *    code. On error, lbm_last_error() returns a message for the calling thread
 *    and the handle is left unchanged unless stated otherwise.
 *  - Lattice units throughout. Node (x, y, z) has linear index
 *    x + nx * (y + ny * z); host arrays are FP64, x fastest. A vector field is
 *    three consecutive blocks of nx*ny*nz values (u_x, then u_y, then u_z).
 *  - Populations per node are indexed in this library's slot order (see
 *    lbm_velocity_set): rest, 6 axis directions, 12 edges, 8 corners, with
 *    slots 2m-1 and 2m opposite.
 *  - Device work is enqueued on the handle's CUDA stream. lbm_step returns
 *    without waiting; functions that return host data wait for the stream.
 *  - Handles are opaque and owned by the library (lbm_destroy frees them).
 *    A handle is not thread-safe: one thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)        /* invalid argument */
#define LBM_ENOMEM (-2)        /* device or host allocation failed */
#define LBM_ECUDA (-3)         /* CUDA runtime error (message has the CUDA error string) */
#define LBM_ETIMEOUT (-4)      /* a bounded device wait ran out */
#define LBM_ENONFINITE (-5)    /* diagnostics found NaN or Inf (output still filled) */
#define LBM_EUNSUPPORTED (-6)  /* combination not compiled into this library */
#define LBM_ESTATE (-7)        /* call out of order (e.g. step before init) */

/* stencil pairs D3Q(m) x D3Q(n): m for f, n for g (Section 2.3) */
enum lbm_pair {
    LBM_D3Q27_D3Q19 = 0,
    LBM_D3Q19_D3Q7 = 1,
    LBM_D3Q27_D3Q27 = 2,
    LBM_D3Q19_D3Q19 = 3,
    LBM_D3Q19_D3Q15 = 4,
    LBM_D3Q15_D3Q7 = 5,
    LBM_D3Q7_D3Q27 = 6
};

/* forcing schemes (Section 3.6) */
enum lbm_forcing {
    LBM_GUO = 0,        /* Guo-Zheng-Shi discrete source term, u of Eq. 7 */
    LBM_SHAN_CHEN = 1,  /* velocity shift, Eq. 10 */
    LBM_EDM = 2,        /* exact difference method */
    LBM_HCZ = 3         /* He-Chen-Zhang source term */
};

/* population storage in HBM: FP32, or FP16/BF16 deviations f_i - w_i
 * (g_i - w_i rho0); the collision arithmetic is FP32 in every case */
enum lbm_storage { LBM_FP32 = 0, LBM_FP16_DEV = 1, LBM_BF16_DEV = 2 };

/* scalar source/moment pair (Eqs. 11, 16, 17) */
enum lbm_scalar_mode {
    LBM_SCALAR_PRINTED = 0,  /* LBE adds S_i, rho' = sum g + (1/2) sum R_i - rho0 (as printed) */
    LBM_SCALAR_CHAI_SHI = 1  /* LBE adds R_i, rho' = sum g + (1/2) sum S_i - rho0 */
};

/* Lattice-unit parameters. lbm_params_from_physics fills them from the
 * dimensionless numbers of Section 2.4. */
typedef struct lbm_params {
    int32_t nx, ny, nz;      /* lattice size, each >= 1, periodic */
    int32_t pair;            /* enum lbm_pair */
    int32_t forcing;         /* enum lbm_forcing */
    int32_t storage;         /* enum lbm_storage */
    int32_t scalar_mode;     /* enum lbm_scalar_mode */
    int32_t reserved;
    double tau_f;            /* Eq. 8: nu / cs^2 + 1/2, > 1/2 */
    double tau_g;            /* Eq. 14: D / cs^2 + 1/2, > 1/2 */
    double G;                /* gravity in lattice units (Eq. 18) */
    double beta;             /* (d rho_b / dz)_LU (Eqs. 12, 13) */
    double rho0;             /* reference density (Eqs. 3, 15) */
    double sc_shift;         /* Shan-Chen shift u_eq = j/rho + sc_shift tau_f F/rho;
                                1 standard, 0.5 = Eq. 10 as printed */
    double U0;               /* reference velocity, lattice units (reporting only) */
    double L;                /* reference length L = 1 in lattice spacings (reporting only) */
} lbm_params;

/* Diagnostics of the current state (post-stream, pre-collision), averages
 * over all nodes (Eqs. 22-26). The first block is in lattice units. The
 * second gives the same quantities in the paper's units (Section 2.4: the
 * reference velocity and length are 1, so the convective time is L / U0 time
 * steps), from the handle's U0 and L (lattice units): t = step U0 / L,
 * energies / U0^2, dissipation rates * L / U0^3. Those are NaN when U0 or L
 * is not positive (lattice parameters made without them). */
typedef struct lbm_diag {
    double Ek;          /* <|u|^2 / 2>, u of Eq. 7 (Eq. 22) */
    double Ep;          /* <(G/N)^2 (rho'/rho0)^2 / 2> (Eq. 23) */
    double eps_k;       /* 2 nu <S:S>, S from the non-equilibrium second moment of f */
    double eps_p;       /* D <(G/N)^2 |grad rho'|^2 / rho0^2>, central differences (Eq. 26) */
    double eps_k_curl;  /* nu <|curl u|^2>, central differences (Eq. 25) */
    double mass_f;      /* sum over nodes and slots of f_i */
    double mass_g;      /* sum over nodes and slots of g_i */
    double mom[3];      /* sum over nodes and slots of e_i f_i */
    double umax;        /* max |u| */
    int64_t step;       /* time steps taken since initialisation */
    /* paper units */
    double t;           /* step * U0 / L (convective times) */
    double Ek_phys;     /* Ek / U0^2 */
    double Ep_phys;     /* Ep / U0^2 */
    double eps_k_phys;  /* eps_k * L / U0^3 */
    double eps_p_phys;  /* eps_p * L / U0^3 */
    double eps_k_curl_phys;  /* eps_k_curl * L / U0^3 */
} lbm_diag;

typedef struct lbm_ctx* lbm_handle;

/* Message of the last failed call on this thread ("" if none). Never NULL. */
const char* lbm_last_error(void);

/* Library version string. */
const char* lbm_version(void);

/* Velocity set q in {7, 15, 19, 27} in this library's slot order:
 * e[3*i + a] (a = x, y, z), w[i] (Table A.1), *cs2. Arrays of 27 suffice.
 * Returns q, or LBM_EINVAL for another q. Any pointer may be NULL. */
int lbm_velocity_set(int q, int* e, double* w, double* cs2);

/* Section 2.4 and Eq. 19 -> lattice units for an n^3 box [0, 2 pi)^3
 * (n = nx; ny and nz are copied): L = nx / (2 pi), nu = U0 L / Re,
 * D = nu / Pr (Pr is the paper's Schmidt number Sc), tau_f = nu / cs^2 + 1/2,
 * tau_g = D / cs_g^2 + 1/2, N = U0 / (Fr L) (Fr may be +inf: unstratified),
 * rho0 = 1, G = N / 1024 and beta = -N^2 rho0 / G (Eq. 19 fixes only their
 * product), storage FP32, printed scalar pair, standard Shan-Chen shift.
 * Returns LBM_EINVAL for non-positive Re, Pr, U0, Fr or sizes. */
int lbm_params_from_physics(lbm_params* p, int nx, int ny, int nz, int pair, int forcing,
                            double Re, double Fr, double Pr, double U0);

/* Create a simulation from physical numbers (= lbm_params_from_physics +
 * lbm_create_params). The current CUDA device becomes the handle's device.
 * No device memory is allocated until lbm_attach or the first init call. */
int lbm_create(lbm_handle* out, int nx, int ny, int nz, int pair, int forcing,
               double Re, double Fr, double Pr, double U0);

/* Create a simulation from lattice-unit parameters (copied). LBM_EUNSUPPORTED
 * if the (pair, storage) kernels are not compiled into this library. */
int lbm_create_params(lbm_handle* out, const lbm_params* p);

/* Copy the handle's parameters out. */
int lbm_get_params(lbm_handle h, lbm_params* p);

/* Change the storage type (enum lbm_storage). Only before the first init
 * call or lbm_attach (LBM_ESTATE afterwards). */
int lbm_set_storage(lbm_handle h, int storage);

/* Enqueue all later device work on this cudaStream_t (not owned; NULL = the
 * legacy default stream, which also disables CUDA-graph replay). */
int lbm_set_stream(lbm_handle h, void* stream);

/* Bytes of the population store: (Q_f + Q_g) * nx*ny*nz * element size. */
int lbm_required_bytes(lbm_handle h, size_t* bytes);

/* Use caller-owned device memory (>= lbm_required_bytes, 256-byte aligned,
 * on the handle's device) as the population store; the caller keeps
 * ownership and must keep it alive until lbm_destroy. Must precede init.
 * Store layout: the Q_f f arrays, then the Q_g g arrays, each of nx*ny*nz
 * elements holding the deviations f_i - w_i and g_i - w_i rho0 (FP32, or
 * FP16 / BF16 per lbm_storage), z-major then y, one x-row contiguous. Within
 * a row node x sits at position x, except in 16-bit stores with even nx,
 * which keep the half-row order: position 2 x for x < nx/2 and
 * 2 (x - nx/2) + 1 otherwise, so that 32-bit word k of a row holds nodes k
 * and k + nx/2. After an odd number of steps the slots are in the swapped
 * AA arrangement; lbm_get_populations / lbm_set_populations read and write
 * node order in either case. */
int lbm_attach(lbm_handle h, void* device_ptr, size_t bytes);

/* Eq. 20 initial state (Section 2.4): u = U0 (sin x cos y cos z,
 * -cos x sin y cos z, 0) on x_i = 2 pi i / n, rho = 1, rho' = 0, plus
 * noise_amp * U0 * xi per component with xi uniform in [-1, 1) drawn from
 * SplitMix64(seed) at counter c = component * nx*ny*nz + node. Populations
 * are set to the equilibria f_eq(rho, u) (Eq. 9), g_eq(rho', u) (Eq. 15).
 * Requires nx = ny = nz (LBM_EINVAL otherwise). Resets the step counter. */
int lbm_init_tgv(lbm_handle h, uint64_t seed, double noise_amp);

/* Populations from host FP64 fields (not retained): rho[n3], u[3*n3],
 * rho_p[n3]; f = f_eq(rho, u) + amp w_i xi_f[code(e_i)][node],
 * g = g_eq(rho', u) + amp w_i xi_g[code(e_i)][node], where the optional
 * xi_f, xi_g are [27][n3] arrays indexed by code(e) = (ex+1)*9 + (ey+1)*3 +
 * (ez+1) (NULL: no perturbation). Returns once the host arrays have been
 * copied (they may then be reused); the initialisation completes in order on
 * the handle's stream. Resets the step counter. */
int lbm_init_fields(lbm_handle h, const double* rho, const double* u, const double* rho_p,
                    const double* xi_f, const double* xi_g, double amp);

/* Pipelined initialisation from host fields, for callers that start a new
 * state every few steps (ensembles, restarts from host data): the
 * host-to-device copies of the next state's fields overlap the current
 * steps. lbm_prefetch_fields enqueues the copies of rho[n3], u[3*n3],
 * rho_p[n3] (host FP64, pinned for the overlap) into one of two library
 * buffers on an internal copy stream and returns at once; the arrays must
 * stay unchanged until the matching lbm_init_prefetched (or lbm_synchronize)
 * returns. lbm_init_prefetched sets the populations from the last prefetch
 * as lbm_init_fields does without perturbation (f = f_eq(rho, u),
 * g = g_eq(rho', u)), in order on the handle's stream after the copies, and
 * resets the step counter. Errors: LBM_ESTATE for a second prefetch before
 * its init, or an init without a prefetch; LBM_ENOMEM if the two buffers
 * (10 * n3 doubles) cannot be allocated on the first prefetch. */
int lbm_prefetch_fields(lbm_handle h, const double* rho, const double* u, const double* rho_p);
int lbm_init_prefetched(lbm_handle h);

/* Advance nsteps >= 0 time steps (Eqs. 5, 11: collide, then stream) with
 * the in-place AA pattern; asynchronous on the handle's stream. */
int lbm_step(lbm_handle h, int64_t nsteps);

/* Block until the handle's stream (and its prefetch copies) are idle;
 * reports asynchronous CUDA errors. */
int lbm_synchronize(lbm_handle h);

/* Diagnostics of the current state into *out (waits for the stream).
 * LBM_ENONFINITE if any value is NaN/Inf (out is still written). */
int lbm_diagnostics(lbm_handle h, lbm_diag* out);

/* Fused diagnostics: the diagnostics of the current state (the same
 * quantities as lbm_diagnostics, Eqs. 22-26, with out->step = the step count
 * at entry), reduced by the first of nsteps >= 1 steps from the
 * post-stream, pre-collision populations that step loads anyway, followed by
 * the remaining nsteps - 1 steps. Returns when the diagnostics are on the
 * host; the steps may still run (asynchronous on the handle's stream).
 * The per-node sums are per step-kernel block instead of per diagnostics
 * block, so the results equal lbm_diagnostics' up to FP32 summation order;
 * with FP16/BF16 storage the node moments come from the step's short-form
 * FP32 arithmetic (~1e-8 relative difference).
 * Errors: LBM_EINVAL (nsteps < 1, null out), LBM_ESTATE (not initialised),
 * LBM_ENONFINITE as lbm_diagnostics. */
int lbm_step_diagnostics(lbm_handle h, int64_t nsteps, lbm_diag* out);

/* Macroscopic fields of the current state into host FP64 arrays: rho (Eq. 6),
 * physical u (Eq. 7, 3 blocks), rho' (Eq. 16). Any pointer may be NULL. */
int lbm_get_fields(lbm_handle h, double* rho, double* u, double* rho_p);

/* The same fields written into caller-owned device memory (FP64, on the
 * handle's device, the layout of lbm_get_fields; any pointer may be NULL),
 * for post-processing on the GPU (e.g. the kinetic-energy spectrum of
 * Section 3.5). Enqueued on the handle's stream; returns without waiting.
 * LBM_EINVAL for a pointer that is not device memory of that device. */
int lbm_get_fields_device(lbm_handle h, double* rho, double* u, double* rho_p);

/* Full populations (not deviations) of the current state in FP64, host
 * arrays f[Q_f][n3], g[Q_g][n3], slot order of lbm_velocity_set. */
int lbm_get_populations(lbm_handle h, double* f, double* g);

/* Full populations (FP64) of `count` sampled nodes of the current state:
 * nodes[k] is a linear node index (< nx*ny*nz, else LBM_EINVAL); outputs are
 * f[k * Q_f + i], g[k * Q_g + i] in this library's slot order. For
 * spot checks of large lattices without copying the whole store. */
int lbm_sample_populations(lbm_handle h, const int64_t* nodes, int64_t count, double* f, double* g);

/* Overwrite the populations from host FP64 arrays laid out as in
 * lbm_get_populations (checkpoint restore). The step counter is kept. */
int lbm_set_populations(lbm_handle h, const double* f, const double* g);

/* Time steps taken since the last init. */
int lbm_step_count(lbm_handle h, int64_t* step);

/* Diagnostics that allocate nothing: a variant of lbm_diagnostics for callers
 * that cannot call cudaMalloc or let a library do so, such as a host program
 * that hands all device memory to its own pool and forbids other
 * allocations, code that must not trigger the device-wide synchronisation a
 * cudaMalloc/cudaFree implies while other streams run, or a process close to
 * its memory limit. (The paper has no counterpart: it is an interface
 * convenience.)
 * Fills out->Ek, Ep, eps_k, mass_f, mass_g, mom, umax and step exactly as
 * lbm_diagnostics defines them (summed in a different block order, so equal
 * up to FP64 rounding); out->eps_p and out->eps_k_curl are set to NaN because
 * they need a field of nx*ny*nz values, which this variant does not have.
 * Scratch: one file-scope device array of 4096 x 11 doubles (~360 KB) that
 * every GPU loading this library holds until the process exits. It limits the
 * lattice to 4096 * 32768 = 134,217,728 nodes (512^3); larger lattices give
 * LBM_EINVAL. The array's device address is looked up (cudaGetSymbolAddress)
 * when a handle is created and, if that lookup failed, on the first call on
 * the device, so make that first call before any stream capture. A device
 * reset destroys every handle; handles created after it look the address up
 * again. The moment pass runs on at least 4 blocks per SM (as
 * lbm_diagnostics), at most one block per 256 nodes.
 * All calls share the array, which keeps the last call's contents: calls that
 * overlap on the GPU (several handles or threads, different streams) race and
 * must be serialised by the caller. Waits for the handle's stream. */
int lbm_diagnostics_noalloc(lbm_handle h, lbm_diag* out);

/* The 16-bit storage rule. FP16 or BF16 deviation storage (FP32 arithmetic)
 * serves a workload only while its energy and dissipation series (Eqs. 22-26:
 * E_k, E_p, eps_k, eps_p) stay within tol (0.01 in the precision target) of a
 * reference series of the same workload: the FP64 oracle where one can be
 * computed, else the FP32-storage run on the same GPU; otherwise FP32 storage
 * is the fallback. The comparison:
 *  - per quantity, max over samples |cand - ref| / max over samples |ref|
 *    (the series maximum as scale, since E_p and eps_p start at zero);
 *  - the total dissipation eps_k + eps_p at the two highest interior local
 *    maxima of the reference series (the double peak of Section 3.3), each
 *    relative to its own height (skipped where the reference has fewer
 *    peaks).
 * ref[count] and cand[count] are records of the same steps (LBM_EINVAL if a
 * step differs or a reference value is not finite); a non-finite candidate
 * value fails the rule. candidate_storage is an enum lbm_storage. Returns the
 * storage to use (candidate_storage if every deviation is <= tol, else
 * LBM_FP32), or a negative LBM_E* code; report (may be NULL) receives the
 * deviations. Host-only: no device work. */
typedef struct lbm_storage_report {
    double dev_Ek, dev_Ep, dev_eps_k, dev_eps_p;   /* max |cand - ref| / max |ref| */
    double dev_peak1, dev_peak2;   /* |cand - ref| / ref of eps_k + eps_p at the highest and the
                                      second-highest reference peak (NaN: no such peak) */
    int64_t step_peak1, step_peak2;   /* their steps (-1: no such peak) */
    int32_t selected;                 /* enum lbm_storage */
    int32_t pass;                     /* 1 if every deviation is <= tol */
} lbm_storage_report;

int lbm_storage_rule(const lbm_diag* ref, const lbm_diag* cand, int64_t count, int candidate_storage,
                     double tol, lbm_storage_report* report);

/* Launch shape of the step kernel (threads along x and y; bx * by <= 256,
 * bx a multiple of 32). With two nodes per thread (lbm_set_pairing) a
 * thread along x covers two nodes. Each AA parity has its own shape:
 * lbm_set_block sets both, lbm_get_block returns the even steps' shape (the
 * default odd-step shape of the D3Q27xD3Q19 two-nodes-per-thread kernel is
 * one row of 128 threads, its even-step shape 64 x 2). */
int lbm_set_block(lbm_handle h, int bx, int by);
int lbm_get_block(lbm_handle h, int* bx, int* by);

/* Time each candidate launch shape on this lattice (reps even+odd step pairs
 * each, every launch timed on its own with CUDA events) and keep the fastest
 * for each AA parity. The state is saved and restored, so the simulation is
 * unchanged. best_ms_per_step (the mean of the two parities' best) may be
 * NULL. */
int lbm_autotune(lbm_handle h, int reps, double* best_ms_per_step);

/* For FP16/BF16 storage and even nx the step kernel can update two nodes
 * per thread: nodes k and k + nx/2 of a row, which the half-row order of the
 * store (see lbm_attach) keeps in one 32-bit word, so that every slot of
 * both AA steps moves as one aligned word; the per-node arithmetic is the
 * one-node kernel's.
 * mode: LBM_PAIRING_OFF (one node per thread), LBM_PAIRING_ALL (the default:
 * two nodes per thread at both AA parities), LBM_PAIRING_EVEN (two nodes on
 * even steps, one node on odd steps).
 * Ignored for FP32 storage and odd nx. Resets the launch shape to its
 * default. Error: LBM_EINVAL for another mode. */
enum lbm_pairing { LBM_PAIRING_OFF = 0, LBM_PAIRING_ALL = 1, LBM_PAIRING_EVEN = 2 };
int lbm_set_pairing(lbm_handle h, int mode);

/* Tile staging (FP16/BF16 storage, nx a multiple of 64; off by default):
 * the step kernel is persistent and warp-specialised. For each tile of W
 * nodes of an x-row (W = 256, 128 or 64, the largest dividing nx) a producer
 * warp issues one bulk asynchronous copy (cp.async.bulk, completion on an
 * mbarrier) per slot row into a ring of shared-memory stages; W / 64 consumer
 * warps, two nodes per thread, load their words from a stage, hand it back
 * (a second mbarrier per stage) and update; the per-node arithmetic and the
 * stores are those of the two-nodes-per-thread kernel (Eqs. 5-18 as in
 * lbm_step). enable = 0 returns to the kernels selected by lbm_set_pairing.
 * Every wait on a copy or a stage is bounded; a wait that runs out makes the
 * next lbm_synchronize return LBM_ETIMEOUT (the lattice state is then not
 * valid). */
int lbm_set_tile_staging(lbm_handle h, int enable);

/* *width = the tile width the staged kernel uses for this lattice, or 0 if
 * the step runs without tile staging (FP32 storage, nx not a multiple of 64,
 * staging disabled, or no store yet). */
int lbm_uses_tile_staging(lbm_handle h, int* width);

/* Test hook for the bounded waits of tile staging: with extra_tx_bytes > 0
 * each consumer warp also waits, after the copies of its first tile have
 * landed, on a barrier of its own that expects extra_tx_bytes which no copy
 * delivers, so that wait runs out; every wait polls at most spin_limit times.
 * A warp whose wait ran out raises the error flag and stops; the producer
 * warp, whose wait for the stages to be handed back then runs out too, stops
 * issuing and waits for its bulk copies still in flight with a fixed limit of
 * its own (about 0.3-1 s, independent of spin_limit) before it exits, so no
 * copy writes shared memory after the block has ended. (0, 1 << 22) restores
 * normal operation. Errors: LBM_EINVAL for spin_limit = 0 or
 * extra_tx_bytes >= 2^20. */
int lbm_set_stage_test(lbm_handle h, unsigned extra_tx_bytes, unsigned spin_limit);

/* ---- z-slab decomposition (one lattice over several GPUs) ----------------
 * A lattice of global size nx * ny * NZ split along z over R ranks: each
 * rank's handle is a lattice of nx * ny * (nz_r + 2) planes, plane 0 and
 * plane nz_r + 1 being ghost copies of the planes just below and above its
 * own planes 1 .. nz_r (periodic: rank 0's lower neighbour is rank R - 1).
 * Initialise each slab with its own planes and the two neighbouring ones
 * (lbm_init_fields or lbm_set_populations with the global field's planes
 * z_r - 1 .. z_r + nz_r). The even AA step is local to a node; the odd step
 * (Eqs. 5, 11 in the in-place pattern) reads the slots opposite to e_z = +-1
 * from the neighbouring planes and writes slots e_z = +-1 into them, so the
 * boundary planes reach into the ghost planes at odd steps only. Around every
 * odd step (lbm_step one step at a time; lbm_step_count even before it) the
 * ranks exchange two halo buffers each way:
 *   phase 0, before the step: the e_z = +1 slots of plane 1 go to the lower
 *     neighbour's upper ghost, the e_z = -1 slots of plane nz_r to the upper
 *     neighbour's lower ghost;
 *   phase 1, after the step: the e_z = -1 slots written into the lower ghost
 *     go back to the lower neighbour's plane nz_r, the e_z = +1 slots written
 *     into the upper ghost to the upper neighbour's plane 1.
 * lbm_halo_pack(phase) fills to_lower / to_upper; lbm_halo_unpack(phase)
 * takes what the lower neighbour sent as its to_upper (from_lower) and what
 * the upper neighbour sent as its to_lower (from_upper). With one rank the
 * slab is its own neighbour (from_lower = its to_upper). The exchange itself
 * (NCCL send/recv, or copies between devices) is the caller's.
 * After an odd step count the store keeps a node's populations at neighbour
 * locations (the AA layout), so reading a slab then (lbm_diagnostics,
 * lbm_get_fields, lbm_get_populations) needs the neighbours' current slots in
 * the ghost planes: a phase-0 exchange first (harmless to repeat before the
 * next odd step). After an even step count every read is local.
 * In slab mode the step kernels update planes 1 .. nz - 2 only;
 * lbm_diagnostics reduces the own planes (averages over them: combine ranks
 * by node count) and returns eps_p and eps_k_curl as NaN (their central
 * differences would need neighbour fields); lbm_step_diagnostics,
 * lbm_diagnostics_noalloc, lbm_init_tgv and tile staging are not available. */

/* enable = 1: planes 0 and nz - 1 are ghost planes (nz >= 3, else
 * LBM_EINVAL); 0: an ordinary periodic lattice. */
int lbm_set_slab(lbm_handle h, int enable);

/* Bytes of one halo buffer: (number of f slots with e_z = +1 + number of g
 * slots with e_z = +1) * nx * ny * element size (D3Q27xD3Q19: 9 + 5 planes). */
int lbm_halo_bytes(lbm_handle h, size_t* bytes);

/* Device buffers (lbm_halo_bytes each, on the handle's device). Enqueued on
 * the handle's stream (device-to-device copies, one per slot and plane);
 * return without waiting. LBM_ESTATE without slab mode or store; LBM_EINVAL
 * for another phase, or a buffer that is null or not device memory of the
 * handle's device. */
int lbm_halo_pack(lbm_handle h, int phase, void* to_lower, void* to_upper);
int lbm_halo_unpack(lbm_handle h, int phase, const void* from_lower, const void* from_upper);

/* Enable (1, default) or disable (0) CUDA-graph replay in lbm_step. */
int lbm_set_graphs(lbm_handle h, int enable);

/* Free the handle and every library-owned device buffer. NULL is allowed. */
int lbm_destroy(lbm_handle h);

/* ---- Batched instances -------------------------------------------------
 * A parameter sweep of the paper's kind (Sections 3.2-3.6: stencil pairs,
 * forcing schemes, Froude numbers, resolutions) as many independent periodic
 * lattices. Three drivers:
 *  - persistent (default): one launch advances every instance by
 *    `steps_per_launch` steps. Each step's work is a list of tiles (runs of
 *    consecutive nodes of one instance); blocks claim tiles from one queue in
 *    step order, and a tile of step s starts once its own instance has
 *    finished step s - 1 (a per-instance completion count), so instances never
 *    wait for each other and there is no grid-wide barrier. Every wait is
 *    bounded. The launch is replayed from a CUDA graph;
 *  - per instance: each instance advanced by its own single-lattice step
 *    kernel (its own launch shape), replayed from a CUDA graph of 64 steps in
 *    which every instance's chain of steps is its own branch (up to 128
 *    branches, largest instances first; instances share no memory, so the
 *    branches overlap and fill each other's tails);
 *  - per step: one launch per (pair, forcing) variant over that variant's
 *    tiles, replayed the same way with one branch per variant.
 * Instances may differ in size, pair (D3Q27xD3Q19, D3Q19xD3Q7), forcing and
 * parameters; storage is FP32. Each instance's arithmetic is the
 * single-lattice update's (bit for bit in the per-instance driver, which runs
 * the single-lattice kernels). */
typedef struct lbm_batch_ctx* lbm_batch;

enum lbm_batch_mode { LBM_BATCH_PERSISTENT = 0, LBM_BATCH_PER_STEP = 1, LBM_BATCH_INSTANCES = 2 };

/* Create `count` (1..65535) instances from lattice parameters (copied) and
 * allocate their stores on the current device. LBM_EUNSUPPORTED for a
 * storage other than FP32 or a pair other than the two above. */
int lbm_batch_create(lbm_batch* out, const lbm_params* params, int count);

/* Number of instances. */
int lbm_batch_count(lbm_batch b, int* count);

/* Handle of instance i (owned by the batch: never lbm_destroy it). Use it
 * for lbm_get_fields, lbm_get_populations, lbm_sample_populations or
 * lbm_diagnostics of that instance; lbm_step on it advances it alone. */
int lbm_batch_instance(lbm_batch b, int i, lbm_handle* h);

/* Stream for all batch work (not owned; NULL disables graph replay). */
int lbm_batch_set_stream(lbm_batch b, void* stream);

/* LBM_BATCH_PERSISTENT (default; steps_per_launch steps per persistent
 * launch, default 100; at most 320 instances, whose descriptors travel in the
 * launch's parameter block: LBM_EUNSUPPORTED beyond, and such batches start
 * in LBM_BATCH_PER_STEP), LBM_BATCH_PER_STEP (one launch per variant and
 * step, replayed from a CUDA graph of 64 steps) or LBM_BATCH_INSTANCES (each
 * instance's own step kernel, one graph branch per instance). */
int lbm_batch_set_mode(lbm_batch b, int mode, int steps_per_launch);

/* Tile shape of the per-step driver: bx in {16, 32, 64, 128} nodes along x,
 * by along y, bx*by a multiple of 32 and <= 256 (default 32 x 8). */
int lbm_batch_set_block(lbm_batch b, int bx, int by);

/* Nodes per tile of the persistent driver: a multiple of 256 in
 * [256, 65536] (default 2048; 256-thread blocks, nodes / 256 per thread). */
int lbm_batch_set_flow_nodes(lbm_batch b, int nodes);
int lbm_batch_get_flow_nodes(lbm_batch b, int* nodes);

/* Current per-step tile shape, mode and grid size (blocks of the persistent
 * launch, or tiles for per-step launches). Pointers may be NULL. */
int lbm_batch_get_config(lbm_batch b, int* bx, int* by, int* mode, int* grid);

/* lbm_init_tgv on every instance (same seed and noise amplitude). */
int lbm_batch_init_tgv(lbm_batch b, uint64_t seed, double noise_amp);

/* Advance every instance by nsteps >= 0 steps, asynchronously. */
int lbm_batch_step(lbm_batch b, int64_t nsteps);

/* Wait for the batch stream. LBM_ETIMEOUT if a dependency wait of a
 * persistent launch ran out (the kernel then ended early and the instances'
 * state is undefined); the flag is cleared. */
int lbm_batch_synchronize(lbm_batch b);

/* lbm_diagnostics of every instance into out[count] (waits; LBM_ETIMEOUT as
 * lbm_batch_synchronize; LBM_ENONFINITE if any instance has NaN/Inf). */
int lbm_batch_diagnostics(lbm_batch b, lbm_diag* out);

/* Time the drivers and keep the fastest: every per-step tile shape, the
 * persistent driver with 1024, 2048, 4096 and 8192 nodes per tile, and the
 * per-instance driver after lbm_autotune of every instance's launch shape;
 * for each candidate one warm-up span, then reps spans timed with CUDA
 * events, a span being one 64-step graph (per-step and per-instance drivers)
 * or one persistent launch of steps_per_launch steps. The instances' state is
 * saved and restored. best_ms_per_step may be NULL. */
int lbm_batch_autotune(lbm_batch b, int reps, double* best_ms_per_step);

/* Test hook for the timeout path of the persistent driver: every
 * dependency wait expects `extra_completions` more completed tiles than
 * exist (so with extra_completions > 0 the first wait of a launch's second
 * step cannot complete) and gives up after `spin_limit` polls (defaults 0 and
 * 4194304). */
int lbm_batch_set_barrier_test(lbm_batch b, unsigned extra_completions, unsigned spin_limit);

/* Split a sweep of independent instances over nranks processes, one GPU
 * each, with no communication on the data path: every rank computes the same
 * owner table and creates a batch of the instances it owns. Longest
 * processing time first: instances in decreasing order of bytes per step
 * ((Q_f + Q_g) * nx*ny*nz * element size; ties by lower index), each to the
 * rank with the fewest bytes so far (ties: lower rank). owner[count]
 * receives each instance's rank; *imbalance (may be NULL) the largest rank's
 * bytes over the mean. Host-only: no device work. LBM_EINVAL for bad
 * arguments or parameters. */
int lbm_batch_partition(const lbm_params* params, int count, int nranks, int32_t* owner, double* imbalance);

/* Free the batch, its instances and their stores. NULL is allowed. */
int lbm_batch_destroy(lbm_batch b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */

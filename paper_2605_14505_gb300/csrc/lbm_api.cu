// C ABI (include/lbm.h): handle management, parameter mapping, launches,
// CUDA-graph replay of the AA step pair, diagnostics, autotuning.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"
#include "lbm_stage.cuh"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);     \
    } while (0)

struct PairInfo {
    int qf, qg;
};

bool pair_info(int pair, PairInfo* out)
{
    static const PairInfo t[7] = {{27, 19}, {19, 7}, {27, 27}, {19, 19}, {19, 15}, {15, 7}, {7, 27}};
    if (pair < 0 || pair > 6) return false;
    *out = t[pair];
    return true;
}

double cs2_of(int q) { return q == 7 ? 0.25 : 1.0 / 3.0; }

size_t elem_size(int storage) { return storage == LBM_FP32 ? 4 : 2; }

constexpr int kGraphSteps = 64;   // even number: the graph starts and ends in natural layout

// Looks up (again) the device address of the allocation-free diagnostics
// scratch on `device`, which must be current; defined with the array below.
void static_scratch_refresh(int device);

}  // namespace

struct lbm_ctx {
    lbm_params p{};
    PairInfo q{};
    Geometry geo{};
    Phys ph{};
    const KernelSet* ks = nullptr;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* store = nullptr;
    size_t store_bytes = 0;
    bool own_store = false;
    bool initialized = false;
    int64_t step = 0;
    int odd = 0;           // layout parity of the store
    int bx = 0, by = 0;      // launch shape of the even AA steps
    int bxo = 0, byo = 0;    // and of the odd ones
    int pairing = LBM_PAIRING_ALL;   // two nodes per thread (16-bit storage, even nx)
    bool tile_staging = false;        // bulk-copy staged kernel where it applies
    bool slab = false;                // z-slab: planes 0 and nz - 1 are ghost planes (lbm_set_slab)
    int stage_grid = 0;               // persistent grid of the staged kernel (0: not derived yet)
    int* d_err = nullptr;             // device flag raised by a bounded wait that ran out
    uint32_t stage_spin = 1u << 22;   // mbarrier polls per wait
    uint32_t stage_extra_tx = 0;      // test hook: bytes a barrier of their own expects and no copy delivers
    // diagnostics scratch
    float* diag_fields = nullptr;
    double* diag_partials = nullptr;
    int diag_rows = 0;                 // rows of kDNumSlots the partials hold
    cudaEvent_t diag_event = nullptr;  // diagnostics copied to the host
    double* diag_out = nullptr;
    double* diag_host = nullptr;   // pinned
    int diag_blocks = 0;
    // host<->device staging
    double* staging = nullptr;
    size_t staging_bytes = 0;
    cudaEvent_t copy_event = nullptr;   // host->device copies of lbm_init_fields done
    // lbm_prefetch_fields / lbm_init_prefetched: two device buffers of the
    // five FP64 fields, filled on a copy stream while the lattice steps
    double* pre[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pre_done[2] = {nullptr, nullptr};   // copies into pre[b] complete
    cudaEvent_t pre_free[2] = {nullptr, nullptr};   // the init that read pre[b] complete
    bool pre_free_recorded[2] = {false, false};
    int pre_next = 0;     // buffer the next prefetch fills
    int pre_ready = -1;   // buffer holding a prefetch not yet used, or -1
    // CUDA graph of kGraphSteps steps starting from the natural layout
    bool graphs = true;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
};

namespace {

void derive_phys(lbm_ctx* h)
{
    const lbm_params& p = h->p;
    Phys& ph = h->ph;
    ph.delta_f = (float)((2.0 * p.tau_f - 1.0) / p.tau_f);
    ph.delta_g = (float)((2.0 * p.tau_g - 1.0) / p.tau_g);
    ph.G = (float)p.G;
    ph.beta = (float)p.beta;
    ph.rho0 = (float)p.rho0;
    const double c_mom = (p.scalar_mode == LBM_SCALAR_PRINTED) ? 0.5 * (1.0 - 1.0 / (2.0 * p.tau_g)) : 0.5;
    const double c_lbe = (p.scalar_mode == LBM_SCALAR_PRINTED) ? 1.0 : 1.0 - 1.0 / (2.0 * p.tau_g);
    ph.kappa = (float)(c_mom * -p.beta);
    ph.c_lbe = (float)c_lbe;
    ph.guo_pref = (float)(1.0 - 1.0 / (2.0 * p.tau_f));
    ph.guo_tau = (float)(p.tau_f - 0.5);
    ph.sc_tau = (float)(p.sc_shift * p.tau_f);
    h->geo.nx = p.nx;
    h->geo.ny = p.ny;
    h->geo.nz = p.nz;
    h->geo.n3 = (uint32_t)((size_t)p.nx * p.ny * p.nz);
}

// Tile width of the staged kernel (a multiple of 64 that divides nx), or 0
// where it does not apply: FP32 storage, nx not a multiple of 64, or a store
// not 16-byte aligned (bulk copies need 16-byte aligned rows).
int stage_width(const lbm_ctx* h)
{
    if (!h->tile_staging || h->slab || h->ks->staged[h->p.forcing][0] == nullptr || h->store == nullptr) return 0;
    if (reinterpret_cast<uintptr_t>(h->store) % 16 != 0) return 0;
    const int nx = h->p.nx;
    return nx % 256 == 0 ? 256 : nx % 128 == 0 ? 128 : nx % 64 == 0 ? 64 : 0;
}

bool uses_pairs(const lbm_ctx* h, int odd)
{
    const bool wanted = h->pairing == LBM_PAIRING_ALL || (h->pairing == LBM_PAIRING_EVEN && !odd);
    return wanted && h->ks->step2[h->p.forcing][0] != nullptr && (h->p.nx % 2) == 0;
}

// Default launch shape of one AA parity, from per-parity sweeps of the
// candidate shapes at 256^3: the two-nodes-per-thread kernel runs best in
// 128-thread blocks of 64 x 2, except on the odd steps of D3Q27xD3Q19, where
// one row of 128 is faster (FP16 0.462 against 0.465 ms, BF16 0.462 against
// 0.467 ms); the one-node kernels in one row of 256 threads on even steps
// and on the odd steps of the pairs with 38 to 46 populations per node, one
// row of 128 on the odd steps of the smaller pairs (D3Q19xD3Q7 0.515 / 0.528
// ms, D3Q19xD3Q19 0.751 / 0.768 ms, against 0.520 / 0.528 and 0.758 / 0.776
// as 128 on both), and for D3Q27xD3Q27 (two 128-register blocks per SM) one
// row of 64 on even steps and 128 on odd steps (1.058 / 1.096 ms against
// 1.072 / 1.155 ms as 256).
void pick_block(const lbm_ctx* h, int odd, int& bx, int& by)
{
    const bool pairs = uses_pairs(h, odd);
    const int xunits = pairs ? h->p.nx / 2 : h->p.nx;
    const int qsum = h->q.qf + h->q.qg;
    const bool big = qsum >= 46;
    const int threads = pairs ? 128 : qsum > 46 ? (odd ? 128 : 64) : (odd && qsum <= 34) ? 128 : 256;
    const int want = pairs ? ((odd && big) ? 128 : 64) : threads;
    bx = 32;
    while (bx * 2 <= want && bx * 2 <= xunits) bx *= 2;
    by = threads / bx;
    while (by > 1 && by / 2 >= h->p.ny) by /= 2;
}

void default_block(lbm_ctx* h)
{
    pick_block(h, 0, h->bx, h->by);
    pick_block(h, 1, h->bxo, h->byo);
}

dim3 step_block(const lbm_ctx* h, int odd)
{
    return odd ? dim3((unsigned)h->bxo, (unsigned)h->byo) : dim3((unsigned)h->bx, (unsigned)h->by);
}

void drop_graph(lbm_ctx* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
}

int ensure_store(lbm_ctx* h)
{
    if (h->store) return LBM_OK;
    size_t bytes = (size_t)(h->q.qf + h->q.qg) * h->geo.n3 * elem_size(h->p.storage);
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "cudaMalloc of %zu bytes for the population store failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    h->store = ptr;
    h->store_bytes = bytes;
    h->own_store = true;
    return LBM_OK;
}

void* f_ptr(lbm_ctx* h) { return h->store; }
void* g_ptr(lbm_ctx* h)
{
    return static_cast<char*>(h->store) + (size_t)h->q.qf * h->geo.n3 * elem_size(h->p.storage);
}

int ensure_staging(lbm_ctx* h, size_t bytes)
{
    if (!h->copy_event && cudaEventCreateWithFlags(&h->copy_event, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "event creation failed");
    }
    if (h->staging_bytes >= bytes) return LBM_OK;
    if (h->staging) cudaFree(h->staging);
    h->staging = nullptr;
    h->staging_bytes = 0;
    cudaError_t e = cudaMalloc(&h->staging, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->staging = nullptr;
        return fail(LBM_ENOMEM, "cudaMalloc of %zu staging bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    h->staging_bytes = bytes;
    return LBM_OK;
}

// Diagnostics scratch: FP32 fields for pass 2, per-block partials (at least
// `rows` rows), the totals, a pinned host copy and its completion event.
int ensure_diag(lbm_ctx* h, int rows = 0)
{
    if (!h->diag_fields) {
        h->diag_blocks = 4 * (h->num_sms > 0 ? h->num_sms : 132);
        size_t fbytes = 4 * (size_t)h->geo.n3 * sizeof(float);
        if (cudaMalloc(&h->diag_fields, fbytes) != cudaSuccess ||
            cudaMalloc(&h->diag_out, 16 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&h->diag_host, 16 * sizeof(double)) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->diag_event, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ENOMEM, "diagnostics scratch allocation failed");
        }
    }
    const int need = rows > h->diag_blocks ? rows : h->diag_blocks;
    if (h->diag_rows < need) {
        if (h->diag_partials) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->diag_partials);
            h->diag_partials = nullptr;
            h->diag_rows = 0;
        }
        if (cudaMalloc(&h->diag_partials, (size_t)need * kDNumSlots * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ENOMEM, "diagnostics partials allocation failed");
        }
        h->diag_rows = need;
    }
    return LBM_OK;
}

// DiagArgs of the current state (scales of Eqs. 22-26 from the parameters).
DiagArgs diag_args(lbm_ctx* h)
{
    const lbm_params& p = h->p;
    const double cs2f = cs2_of(h->q.qf), cs2g = cs2_of(h->q.qg);
    const double gn2 = (p.beta != 0.0) ? (-p.G * p.rho0 / p.beta) : 1.0;
    const double nu = cs2f * (p.tau_f - 0.5), D = cs2g * (p.tau_g - 0.5);
    DiagArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.odd = h->odd;
    a.ep_scale = (float)(0.5 * gn2 / (p.rho0 * p.rho0));
    a.epsk_scale = (float)(2.0 * nu);
    a.s_scale = (float)(-1.0 / (2.0 * cs2f * p.tau_f));
    a.epsp_scale = (float)(D * gn2 / (p.rho0 * p.rho0));
    a.nu = (float)nu;
    a.fields = h->diag_fields;
    a.partials = h->diag_partials;
    const uint32_t plane = (uint32_t)p.nx * (uint32_t)p.ny;
    a.idx0 = h->slab ? plane : 0u;
    a.idx1 = h->slab ? h->geo.n3 - plane : h->geo.n3;
    return a;
}

// Nodes the diagnostics cover: every node, or a z-slab's own planes.
double owned_nodes(const lbm_ctx* h)
{
    const double plane = (double)h->p.nx * (double)h->p.ny;
    return h->slab ? (double)h->geo.n3 - 2.0 * plane : (double)h->geo.n3;
}

// The paper-unit block of a record (Section 2.4: U = L = 1, so one
// convective time is L / U0 steps): t = step U0 / L, energies / U0^2,
// dissipation rates * L / U0^3; NaN without a positive U0 and L.
void fill_phys(const lbm_params& p, lbm_diag* out)
{
    const bool ok = p.U0 > 0.0 && p.L > 0.0 && std::isfinite(p.U0) && std::isfinite(p.L);
    const double nan = std::numeric_limits<double>::quiet_NaN();
    const double e = ok ? 1.0 / (p.U0 * p.U0) : nan;
    const double r = ok ? p.L / (p.U0 * p.U0 * p.U0) : nan;
    out->t = ok ? (double)out->step * p.U0 / p.L : nan;
    out->Ek_phys = out->Ek * e;
    out->Ep_phys = out->Ep * e;
    out->eps_k_phys = out->eps_k * r;
    out->eps_p_phys = out->eps_p * r;
    out->eps_k_curl_phys = out->eps_k_curl * r;
}

// Totals (diag_host) -> lbm_diag of the state at `step`.
int fill_diag(const lbm_ctx* h, int64_t step, lbm_diag* out)
{
    const double* s = h->diag_host;
    const double nodes = owned_nodes(h);
    const double inv = 1.0 / nodes;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    out->Ek = s[kDEk] * inv;
    out->Ep = s[kDEp] * inv;
    out->eps_k = s[kDEpsK] * inv;
    // a z-slab has no neighbour fields for the central differences
    out->eps_p = h->slab ? nan : s[kDEpsP] * inv;
    out->eps_k_curl = h->slab ? nan : s[kDEpsKCurl] * inv;
    out->mass_f = nodes + s[kDDrho];
    out->mass_g = nodes * h->p.rho0 + s[kDA];
    out->mom[0] = s[kDJx];
    out->mom[1] = s[kDJy];
    out->mom[2] = s[kDJz];
    out->umax = s[kDUmax];
    out->step = step;
    fill_phys(h->p, out);
    const int checked = h->slab ? kDiagPass1 : kDNumSlots;
    for (int q = 0; q < checked; ++q)
        if (!std::isfinite(s[q])) return fail(LBM_ENONFINITE, "non-finite diagnostics at step %lld", (long long)step);
    return LBM_OK;
}

dim3 step_grid(const lbm_ctx* h, int odd)
{
    const int xunits = uses_pairs(h, odd) ? h->p.nx / 2 : h->p.nx;
    const dim3 b = step_block(h, odd);
    return dim3((unsigned)((xunits + (int)b.x - 1) / (int)b.x), (unsigned)((h->p.ny + (int)b.y - 1) / (int)b.y),
                (unsigned)h->p.nz);
}

cudaError_t launch_staged(lbm_ctx* h, int odd, int W, cudaStream_t s)
{
    const void* k = h->ks->staged[h->p.forcing][odd];
    const size_t smem = stage_smem_bytes(h->q.qf + h->q.qg, W);
    StageArgs a{};
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.W = W;
    a.ntx = h->p.nx / W;
    a.ntiles = (uint32_t)a.ntx * (uint32_t)h->p.ny * (uint32_t)h->p.nz;
    a.err = h->d_err;
    a.spin_limit = h->stage_spin;
    a.extra_tx = h->stage_extra_tx;
    if (h->stage_grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(h->ks->staged[h->p.forcing][odd ^ 1],
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, stage_threads(W), smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        const size_t cap = (size_t)(h->num_sms > 0 ? h->num_sms : 1) * (size_t)occ;
        h->stage_grid = (int)(a.ntiles < cap ? a.ntiles : cap);
    }
    void* args[] = {&a};
    return cudaLaunchKernel(k, dim3((unsigned)h->stage_grid), dim3((unsigned)stage_threads(W)), args, smem, s);
}

cudaError_t launch_step(lbm_ctx* h, int odd, cudaStream_t s)
{
    const int W = stage_width(h);
    if (W > 0) return launch_staged(h, odd, W, s);
    StepArgs a{};
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    // a z-slab updates its own planes 1 .. nz - 2; the ghost planes are only
    // read and written by the boundary planes' odd steps (never wrapped)
    a.z0 = h->slab ? 1 : 0;
    dim3 grid = step_grid(h, odd);
    if (h->slab) grid.z = (unsigned)(h->p.nz - 2);
    void* args[] = {&a};
    const void* k = uses_pairs(h, odd) ? h->ks->step2[h->p.forcing][odd] : h->ks->step[h->p.forcing][odd];
    return cudaLaunchKernel(k, grid, step_block(h, odd), args, 0, s);
}

int flat_grid(const lbm_ctx* h)
{
    size_t blocks = ((size_t)h->geo.n3 + 255) / 256;
    size_t cap = (size_t)(h->num_sms > 0 ? h->num_sms : 132) * 16;
    return (int)(blocks < cap ? blocks : cap);
}

int check_handle(lbm_ctx* h)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return LBM_OK;
}

int validate_params(const lbm_params* p, PairInfo* q)
{
    if (!p) return fail(LBM_EINVAL, "null parameters");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_EINVAL, "lattice sizes must be >= 1");
    size_t n3 = (size_t)p->nx * p->ny * p->nz;
    if (n3 > 0x7fffffffull) return fail(LBM_EINVAL, "nx*ny*nz = %zu exceeds 2^31 - 1 nodes", n3);
    if (p->nz > 65535) return fail(LBM_EINVAL, "nz must be <= 65535");
    if (!pair_info(p->pair, q)) return fail(LBM_EINVAL, "unknown stencil pair %d", p->pair);
    if ((size_t)(q->qf > q->qg ? q->qf : q->qg) * n3 > 0xffffffffull)
        return fail(LBM_EINVAL, "Q * nx*ny*nz = %zu exceeds the 32-bit element offsets of the store",
                    (size_t)(q->qf > q->qg ? q->qf : q->qg) * n3);
    if (p->forcing < 0 || p->forcing > 3) return fail(LBM_EINVAL, "unknown forcing scheme %d", p->forcing);
    if (p->storage < 0 || p->storage > 2) return fail(LBM_EINVAL, "unknown storage %d", p->storage);
    if (p->scalar_mode < 0 || p->scalar_mode > 1) return fail(LBM_EINVAL, "unknown scalar mode %d", p->scalar_mode);
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5) || !std::isfinite(p->tau_f) || !std::isfinite(p->tau_g))
        return fail(LBM_EINVAL, "relaxation times must be finite and > 1/2 (tau_f=%g, tau_g=%g)", p->tau_f,
                    p->tau_g);
    if (!std::isfinite(p->G) || !std::isfinite(p->beta) || !std::isfinite(p->rho0) || !std::isfinite(p->sc_shift))
        return fail(LBM_EINVAL, "non-finite physical parameter");
    return LBM_OK;
}

int after_init(lbm_ctx* h)
{
    h->initialized = true;
    h->step = 0;
    h->odd = 0;
    return LBM_OK;
}

// Slots of velocity set q (this library's order) whose e_z equals sign,
// into slots[] (may be null); returns their number.
int halo_slots(int q, int sign, int* slots)
{
    auto pick = [&](auto lat) {
        using L = decltype(lat);
        int n = 0;
        for (int i = 0; i < L::kQ; ++i)
            if (L::ez(i) == sign) {
                if (slots) slots[n] = i;
                ++n;
            }
        return n;
    };
    switch (q) {
    case 7: return pick(Lattice<7>{});
    case 15: return pick(Lattice<15>{});
    case 19: return pick(Lattice<19>{});
    default: return pick(Lattice<27>{});
    }
}

// LBM_OK if p is device memory of the handle's device (the halo copies are
// device-to-device).
int check_device_buffer(const lbm_ctx* h, const void* p)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice || attr.device != h->device) {
        cudaGetLastError();
        return fail(LBM_EINVAL, "halo buffers must be device memory on the handle's device");
    }
    return LBM_OK;
}

// Halo buffer <-> plane z of the store: the f slots with e_z = sign, then the
// g slots with e_z = sign, nx*ny elements each (one contiguous run per slot
// and plane in the store). pack = store -> buffer.
int halo_copy(lbm_ctx* h, int z, int sign, void* buf, bool pack)
{
    const size_t es = elem_size(h->p.storage);
    const size_t plane = (size_t)h->p.nx * (size_t)h->p.ny * es;
    int slots[27];
    char* b = static_cast<char*>(buf);
    for (int part = 0; part < 2; ++part) {
        const int q = part ? h->q.qg : h->q.qf;
        char* base = static_cast<char*>(part ? g_ptr(h) : f_ptr(h));
        const int n = halo_slots(q, sign, slots);
        for (int k = 0; k < n; ++k) {
            char* at = base + ((size_t)slots[k] * h->geo.n3) * es + (size_t)z * plane;
            LBM_CUDA(cudaMemcpyAsync(pack ? b : at, pack ? at : b, plane, cudaMemcpyDeviceToDevice, h->stream),
                     "halo copy");
            b += plane;
        }
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

const char* lbm_version(void) { return "paper_2605_14505_gb300 lbm 0.1 (sm_103a)"; }

int lbm_velocity_set(int q, int* e, double* w, double* cs2)
{
    auto fill = [&](auto lat) {
        using L = decltype(lat);
        for (int i = 0; i < L::kQ; ++i) {
            if (e) {
                e[3 * i + 0] = L::ex(i);
                e[3 * i + 1] = L::ey(i);
                e[3 * i + 2] = L::ez(i);
            }
            if (w) w[i] = L::wd(i);
        }
        if (cs2) *cs2 = L::cs2d;
        return L::kQ;
    };
    switch (q) {
    case 7: return fill(Lattice<7>{});
    case 15: return fill(Lattice<15>{});
    case 19: return fill(Lattice<19>{});
    case 27: return fill(Lattice<27>{});
    default: return fail(LBM_EINVAL, "unknown velocity set Q%d", q);
    }
}

int lbm_params_from_physics(lbm_params* p, int nx, int ny, int nz, int pair, int forcing, double Re,
                            double Fr, double Pr, double U0)
{
    PairInfo q;
    if (!p) return fail(LBM_EINVAL, "null parameters");
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "lattice sizes must be >= 1");
    if (!pair_info(pair, &q)) return fail(LBM_EINVAL, "unknown stencil pair %d", pair);
    if (!(Re > 0) || !(Pr > 0) || !(U0 > 0) || !(Fr > 0) || std::isnan(Fr))
        return fail(LBM_EINVAL, "Re, Fr, Pr and U0 must be positive");
    std::memset(p, 0, sizeof(*p));
    const double two_pi = 6.283185307179586476925286766559;
    const double L = nx / two_pi;
    const double nu = U0 * L / Re;
    const double D = nu / Pr;
    const double N = std::isinf(Fr) ? 0.0 : U0 / (Fr * L);
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->pair = pair;
    p->forcing = forcing;
    p->storage = LBM_FP32;
    p->scalar_mode = LBM_SCALAR_PRINTED;
    p->tau_f = nu / cs2_of(q.qf) + 0.5;
    p->tau_g = D / cs2_of(q.qg) + 0.5;
    p->rho0 = 1.0;
    p->G = N / 1024.0;
    p->beta = N > 0 ? -N * N * p->rho0 / p->G : 0.0;
    p->sc_shift = 1.0;
    p->U0 = U0;
    p->L = L;
    return LBM_OK;
}

int lbm_create_params(lbm_handle* out, const lbm_params* p)
{
    if (!out) return fail(LBM_EINVAL, "null output handle");
    *out = nullptr;
    PairInfo q;
    int rc = validate_params(p, &q);
    if (rc) return rc;
    const KernelSet* ks = kernel_set(p->pair, p->storage);
    if (!ks) return fail(LBM_EUNSUPPORTED, "stencil pair %d with storage %d is not compiled in", p->pair, p->storage);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    lbm_ctx* h = new (std::nothrow) lbm_ctx();
    if (!h) return fail(LBM_ENOMEM, "host allocation failed");
    h->p = *p;
    h->q = q;
    h->ks = ks;
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    // a device reset ends every handle, so looking the scratch address up
    // again here keeps the cached one valid for every handle in use
    static_scratch_refresh(dev);
    derive_phys(h);
    default_block(h);
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaStreamCreate");
    }
    h->own_stream = true;
    if (cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess || cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (h->d_err) cudaFree(h->d_err);
        cudaStreamDestroy(h->stream);
        delete h;
        return fail(LBM_ENOMEM, "device error-flag allocation failed");
    }
    *out = h;
    return LBM_OK;
}

int lbm_create(lbm_handle* out, int nx, int ny, int nz, int pair, int forcing, double Re, double Fr, double Pr,
               double U0)
{
    lbm_params p;
    int rc = lbm_params_from_physics(&p, nx, ny, nz, pair, forcing, Re, Fr, Pr, U0);
    if (rc) return rc;
    return lbm_create_params(out, &p);
}

int lbm_get_params(lbm_handle h, lbm_params* p)
{
    if (!h || !p) return fail(LBM_EINVAL, "null argument");
    *p = h->p;
    return LBM_OK;
}

int lbm_set_storage(lbm_handle h, int storage)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (h->store) return fail(LBM_ESTATE, "storage can only change before the store exists");
    if (storage < 0 || storage > 2) return fail(LBM_EINVAL, "unknown storage %d", storage);
    const KernelSet* ks = kernel_set(h->p.pair, storage);
    if (!ks) return fail(LBM_EUNSUPPORTED, "storage %d is not compiled in for pair %d", storage, h->p.pair);
    h->p.storage = storage;
    h->ks = ks;
    h->stage_grid = 0;
    default_block(h);
    drop_graph(h);
    return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void* stream)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->own_stream) {
        cudaStreamSynchronize(h->stream);
        cudaStreamDestroy(h->stream);
    }
    h->stream = static_cast<cudaStream_t>(stream);
    h->own_stream = false;
    return LBM_OK;
}

int lbm_required_bytes(lbm_handle h, size_t* bytes)
{
    if (!h || !bytes) return fail(LBM_EINVAL, "null argument");
    *bytes = (size_t)(h->q.qf + h->q.qg) * h->geo.n3 * elem_size(h->p.storage);
    return LBM_OK;
}

int lbm_attach(lbm_handle h, void* device_ptr, size_t bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->store) return fail(LBM_ESTATE, "a population store is already in place");
    size_t need;
    lbm_required_bytes(h, &need);
    if (!device_ptr) return fail(LBM_EINVAL, "null device pointer");
    if (bytes < need) return fail(LBM_EINVAL, "store of %zu bytes is smaller than the %zu required", bytes, need);
    if (reinterpret_cast<uintptr_t>(device_ptr) % 256 != 0) return fail(LBM_EINVAL, "store must be 256-byte aligned");
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, device_ptr);
    if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice || attr.device != h->device) {
        cudaGetLastError();
        return fail(LBM_EINVAL, "store must be device memory on the handle's device");
    }
    h->store = device_ptr;
    h->store_bytes = bytes;
    h->own_store = false;
    return LBM_OK;
}

int lbm_init_tgv(lbm_handle h, uint64_t seed, double noise_amp)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->slab) return fail(LBM_EINVAL, "a z-slab is initialised from the global field's planes (lbm_init_fields "
                                         "or lbm_set_populations), not by lbm_init_tgv");
    if (h->p.nx != h->p.ny || h->p.nx != h->p.nz) return fail(LBM_EINVAL, "the Taylor-Green box needs nx = ny = nz");
    if (!std::isfinite(noise_amp)) return fail(LBM_EINVAL, "non-finite noise amplitude");
    if ((rc = ensure_store(h))) return rc;
    // sin and cos of x_i = 2 pi i / n for the kernel, in the staging buffer
    const int n = h->p.nx;
    std::vector<double> trig(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double x = 6.283185307179586476925286766559 * i / n;
        trig[i] = std::sin(x);
        trig[n + i] = std::cos(x);
    }
    if ((rc = ensure_staging(h, trig.size() * sizeof(double)))) return rc;
    LBM_CUDA(cudaMemcpyAsync(h->staging, trig.data(), trig.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream),
             "copy trig table");
    LBM_CUDA(cudaEventRecord(h->copy_event, h->stream), "init_tgv event");
    TgvArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.trig = h->staging;
    a.U0 = h->p.U0;
    a.noise = noise_amp;
    a.seed = seed;
    a.rho0 = h->p.rho0;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->init_tgv, dim3(flat_grid(h)), dim3(256), args, 0, h->stream), "init_tgv launch");
    LBM_CUDA(cudaEventSynchronize(h->copy_event), "init_tgv");   // the table's host copy may go
    return after_init(h);
}

int lbm_init_fields(lbm_handle h, const double* rho, const double* u, const double* rho_p, const double* xi_f,
                    const double* xi_g, double amp)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !u || !rho_p) return fail(LBM_EINVAL, "rho, u and rho_p are required");
    if ((rc = ensure_store(h))) return rc;
    const size_t n3 = h->geo.n3;
    size_t ndoubles = 5 * n3 + (xi_f ? 27 * n3 : 0) + (xi_g ? 27 * n3 : 0);
    if ((rc = ensure_staging(h, ndoubles * sizeof(double)))) return rc;
    double* d = h->staging;
    LBM_CUDA(cudaMemcpyAsync(d, rho, n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy rho");
    LBM_CUDA(cudaMemcpyAsync(d + n3, u, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy u");
    LBM_CUDA(cudaMemcpyAsync(d + 4 * n3, rho_p, n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy rho_p");
    double* dxf = nullptr;
    double* dxg = nullptr;
    size_t off = 5 * n3;
    if (xi_f) {
        dxf = d + off;
        off += 27 * n3;
        LBM_CUDA(cudaMemcpyAsync(dxf, xi_f, 27 * n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy xi_f");
    }
    if (xi_g) {
        dxg = d + off;
        LBM_CUDA(cudaMemcpyAsync(dxg, xi_g, 27 * n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy xi_g");
    }
    InitArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.rho = d;
    a.u = d + n3;
    a.rho_p = d + 4 * n3;
    a.xi_f = dxf;
    a.xi_g = dxg;
    a.amp_f = (float)amp;
    a.rho0 = h->p.rho0;
    void* args[] = {&a};
    // the host arrays may be reused once the copies are done; the
    // initialisation itself completes in stream order
    LBM_CUDA(cudaEventRecord(h->copy_event, h->stream), "init_fields event");
    LBM_CUDA(cudaLaunchKernel(h->ks->init_fields, dim3(flat_grid(h)), dim3(256), args, 0, h->stream),
             "init_fields launch");
    LBM_CUDA(cudaEventSynchronize(h->copy_event), "init_fields");
    return after_init(h);
}

int lbm_prefetch_fields(lbm_handle h, const double* rho, const double* u, const double* rho_p)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !u || !rho_p) return fail(LBM_EINVAL, "rho, u and rho_p are required");
    if (h->pre_ready >= 0) return fail(LBM_ESTATE, "a prefetch is already waiting for lbm_init_prefetched");
    const size_t n3 = h->geo.n3;
    if (!h->copy_stream) {
        if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ECUDA, "copy stream creation failed");
        }
        for (int b = 0; b < 2; ++b) {
            if (cudaEventCreateWithFlags(&h->pre_done[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->pre_free[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaMalloc(&h->pre[b], 5 * n3 * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                return fail(LBM_ENOMEM, "prefetch buffer allocation failed");
            }
        }
    }
    const int b = h->pre_next;
    if (h->pre_free_recorded[b])
        LBM_CUDA(cudaStreamWaitEvent(h->copy_stream, h->pre_free[b], 0), "prefetch wait");
    double* d = h->pre[b];
    LBM_CUDA(cudaMemcpyAsync(d, rho, n3 * sizeof(double), cudaMemcpyHostToDevice, h->copy_stream), "prefetch rho");
    LBM_CUDA(cudaMemcpyAsync(d + n3, u, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, h->copy_stream), "prefetch u");
    LBM_CUDA(cudaMemcpyAsync(d + 4 * n3, rho_p, n3 * sizeof(double), cudaMemcpyHostToDevice, h->copy_stream),
             "prefetch rho_p");
    LBM_CUDA(cudaEventRecord(h->pre_done[b], h->copy_stream), "prefetch event");
    h->pre_ready = b;
    h->pre_next = b ^ 1;
    return LBM_OK;
}

int lbm_init_prefetched(lbm_handle h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->pre_ready < 0) return fail(LBM_ESTATE, "lbm_init_prefetched without a prefetch");
    if ((rc = ensure_store(h))) return rc;
    const int b = h->pre_ready;
    const size_t n3 = h->geo.n3;
    LBM_CUDA(cudaStreamWaitEvent(h->stream, h->pre_done[b], 0), "init wait");
    InitArgs a{};
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.rho = h->pre[b];
    a.u = h->pre[b] + n3;
    a.rho_p = h->pre[b] + 4 * n3;
    a.rho0 = h->p.rho0;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->init_fields, dim3(flat_grid(h)), dim3(256), args, 0, h->stream),
             "init_prefetched launch");
    LBM_CUDA(cudaEventRecord(h->pre_free[b], h->stream), "init event");
    h->pre_free_recorded[b] = true;
    h->pre_ready = -1;
    // the caller's host arrays of this prefetch may be reused from here on
    LBM_CUDA(cudaEventSynchronize(h->pre_done[b]), "prefetch copies");
    return after_init(h);
}

int lbm_step(lbm_handle h, int64_t nsteps)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    if (!h->initialized) return fail(LBM_ESTATE, "lbm_step before initialisation");
    while (nsteps > 0) {
        if (h->graphs && h->stream != nullptr && h->odd == 0 && nsteps >= kGraphSteps) {
            if (!h->graph) {
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) e = launch_step(h, s & 1, h->stream);
                    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    h->graph = nullptr;
                    h->graphs = false;  // fall back to eager launches
                    continue;
                }
            }
            LBM_CUDA(cudaGraphLaunch(h->graph, h->stream), "graph launch");
            h->step += kGraphSteps;
            nsteps -= kGraphSteps;
            continue;
        }
        LBM_CUDA(launch_step(h, h->odd, h->stream), "step launch");
        h->odd ^= 1;
        h->step += 1;
        nsteps -= 1;
    }
    return LBM_OK;
}

int lbm_synchronize(lbm_handle h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (h->copy_stream) LBM_CUDA(cudaStreamSynchronize(h->copy_stream), "copy stream synchronize");
    int err = 0;
    LBM_CUDA(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
    if (err) {
        LBM_CUDA(cudaMemset(h->d_err, 0, sizeof(int)), "error flag reset");
        return fail(LBM_ETIMEOUT, "a shared-memory staging wait of the step kernel ran out; the lattice state "
                                  "is not valid");
    }
    return LBM_OK;
}

int lbm_diagnostics(lbm_handle h, lbm_diag* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBM_EINVAL, "null output");
    if (!h->initialized) return fail(LBM_ESTATE, "diagnostics before initialisation");
    if ((rc = ensure_diag(h))) return rc;
    DiagArgs a = diag_args(h);
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->diag_moments, dim3(h->diag_blocks), dim3(kDiagBlock), args, 0, h->stream),
             "diag pass 1");
    if (!h->slab)
        LBM_CUDA(cudaLaunchKernel(diag_gradients_kernel(), dim3(h->diag_blocks), dim3(kDiagBlock), args, 0, h->stream),
                 "diag pass 2");
    const double* pp = h->diag_partials;
    int nb = h->diag_blocks;
    int nb2 = h->slab ? 0 : h->diag_blocks;
    double* dout = h->diag_out;
    void* fargs[] = {&pp, &nb, &nb2, &dout};
    LBM_CUDA(cudaLaunchKernel(diag_final_kernel(), dim3(1), dim3(kDiagBlock), fargs, 0, h->stream), "diag pass 3");
    LBM_CUDA(cudaMemcpyAsync(h->diag_host, h->diag_out, kDNumSlots * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "diag copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "diagnostics");
    return fill_diag(h, h->step, out);
}

int lbm_step_diagnostics(lbm_handle h, int64_t nsteps, lbm_diag* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBM_EINVAL, "null output");
    if (nsteps < 1) return fail(LBM_EINVAL, "lbm_step_diagnostics needs at least one step");
    if (!h->initialized) return fail(LBM_ESTATE, "lbm_step_diagnostics before initialisation");
    if (h->slab) return fail(LBM_EUNSUPPORTED, "a z-slab steps with lbm_step and reports with lbm_diagnostics");
    const int odd = h->odd;
    const bool pairs = uses_pairs(h, odd);
    const dim3 grid = step_grid(h, odd);
    const int rows = (int)(grid.x * grid.y * grid.z);
    const int level1 = h->num_sms > 0 ? h->num_sms : 132;   // first-level rows of the final pass
    if ((rc = ensure_diag(h, rows + level1))) return rc;
    const DiagArgs da = diag_args(h);
    StepArgs a{};
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.dg = DiagSink{da.ep_scale, da.epsk_scale, da.s_scale, h->diag_fields, h->diag_partials};
    void* args[] = {&a};
    const void* k = pairs ? h->ks->step2_diag[h->p.forcing][odd] : h->ks->step_diag[h->p.forcing][odd];
    LBM_CUDA(cudaLaunchKernel(k, grid, step_block(h, odd), args, 0, h->stream), "diagnosing step");
    const int64_t step0 = h->step;
    h->odd ^= 1;
    h->step += 1;
    DiagArgs g = da;
    void* gargs[] = {&g};
    LBM_CUDA(cudaLaunchKernel(diag_gradients_kernel(), dim3(h->diag_blocks), dim3(kDiagBlock), gargs, 0, h->stream),
             "diag pass 2");
    // pass 3 in two levels: `level1` blocks each sum a contiguous range of the
    // step blocks' rows (and of the pass-2 rows) into one row, then one block
    const double* pp = h->diag_partials;
    int nb1 = rows, nb2 = h->diag_blocks;
    double* mid = h->diag_partials + (size_t)rows * kDNumSlots;
    void* l1args[] = {&pp, &nb1, &nb2, &mid};
    LBM_CUDA(cudaLaunchKernel(diag_final_kernel(), dim3(level1), dim3(kDiagBlock), l1args, 0, h->stream),
             "diag pass 3a");
    const double* pm = mid;
    int nl = level1;
    double* dout = h->diag_out;
    void* fargs[] = {&pm, &nl, &nl, &dout};
    LBM_CUDA(cudaLaunchKernel(diag_final_kernel(), dim3(1), dim3(kDiagBlock), fargs, 0, h->stream), "diag pass 3b");
    LBM_CUDA(cudaMemcpyAsync(h->diag_host, h->diag_out, kDNumSlots * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "diag copy");
    LBM_CUDA(cudaEventRecord(h->diag_event, h->stream), "diag event");
    if ((rc = lbm_step(h, nsteps - 1))) return rc;
    LBM_CUDA(cudaEventSynchronize(h->diag_event), "diagnostics");
    return fill_diag(h, step0, out);
}

int lbm_get_fields(lbm_handle h, double* rho, double* u, double* rho_p)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->initialized) return fail(LBM_ESTATE, "fields requested before initialisation");
    const size_t n3 = h->geo.n3;
    if ((rc = ensure_staging(h, 5 * n3 * sizeof(double)))) return rc;
    FieldArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.odd = h->odd;
    a.rho = h->staging;
    a.u = h->staging + n3;
    a.rho_p = h->staging + 4 * n3;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->get_fields, dim3(flat_grid(h)), dim3(256), args, 0, h->stream), "get_fields");
    if (rho) LBM_CUDA(cudaMemcpyAsync(rho, a.rho, n3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy rho");
    if (u) LBM_CUDA(cudaMemcpyAsync(u, a.u, 3 * n3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy u");
    if (rho_p)
        LBM_CUDA(cudaMemcpyAsync(rho_p, a.rho_p, n3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy rho_p");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "get_fields");
    return LBM_OK;
}

int lbm_get_fields_device(lbm_handle h, double* rho, double* u, double* rho_p)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->initialized) return fail(LBM_ESTATE, "fields requested before initialisation");
    double* outs[3] = {rho, u, rho_p};
    for (double* p : outs) {
        if (!p) continue;
        cudaPointerAttributes attr;
        cudaError_t e = cudaPointerGetAttributes(&attr, p);
        if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice || attr.device != h->device) {
            cudaGetLastError();
            return fail(LBM_EINVAL, "field outputs must be device memory on the handle's device");
        }
    }
    FieldArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.odd = h->odd;
    a.rho = rho;
    a.u = u;
    a.rho_p = rho_p;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->get_fields, dim3(flat_grid(h)), dim3(256), args, 0, h->stream),
             "get_fields_device");
    return LBM_OK;
}

int lbm_get_populations(lbm_handle h, double* f, double* g)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !g) return fail(LBM_EINVAL, "null output");
    if (!h->initialized) return fail(LBM_ESTATE, "populations requested before initialisation");
    const size_t n3 = h->geo.n3;
    const size_t nq = (size_t)h->q.qf + h->q.qg;
    if ((rc = ensure_staging(h, nq * n3 * sizeof(double)))) return rc;
    PopArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.fout = h->staging;
    a.gout = h->staging + (size_t)h->q.qf * n3;
    a.rho0 = h->p.rho0;
    a.odd = h->odd;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->get_pops, dim3(flat_grid(h)), dim3(256), args, 0, h->stream), "get_pops");
    LBM_CUDA(cudaMemcpyAsync(f, a.fout, (size_t)h->q.qf * n3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "copy f");
    LBM_CUDA(cudaMemcpyAsync(g, a.gout, (size_t)h->q.qg * n3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "copy g");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "get_populations");
    return LBM_OK;
}

int lbm_sample_populations(lbm_handle h, const int64_t* nodes, int64_t count, double* f, double* g)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!nodes || !f || !g))) return fail(LBM_EINVAL, "invalid sample arguments");
    if (!h->initialized) return fail(LBM_ESTATE, "populations requested before initialisation");
    if (count == 0) return LBM_OK;
    for (int64_t s = 0; s < count; ++s)
        if (nodes[s] < 0 || nodes[s] >= (int64_t)h->geo.n3)
            return fail(LBM_EINVAL, "node index %lld out of range", (long long)nodes[s]);
    const size_t nq = (size_t)h->q.qf + h->q.qg;
    const size_t bytes = (size_t)count * (nq * sizeof(double) + sizeof(int64_t));
    if ((rc = ensure_staging(h, bytes))) return rc;
    SampleArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.fout = h->staging;
    a.gout = h->staging + (size_t)count * h->q.qf;
    int64_t* dnodes = reinterpret_cast<int64_t*>(h->staging + (size_t)count * nq);
    a.nodes = dnodes;
    a.count = count;
    a.rho0 = h->p.rho0;
    a.odd = h->odd;
    LBM_CUDA(cudaMemcpyAsync(dnodes, nodes, (size_t)count * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream),
             "copy nodes");
    void* args[] = {&a};
    const unsigned blocks = (unsigned)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
    LBM_CUDA(cudaLaunchKernel(h->ks->sample_pops, dim3(blocks), dim3(256), args, 0, h->stream), "sample_pops");
    LBM_CUDA(cudaMemcpyAsync(f, a.fout, (size_t)count * h->q.qf * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "copy f");
    LBM_CUDA(cudaMemcpyAsync(g, a.gout, (size_t)count * h->q.qg * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "copy g");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "sample_populations");
    return LBM_OK;
}

int lbm_set_populations(lbm_handle h, const double* f, const double* g)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !g) return fail(LBM_EINVAL, "null input");
    if ((rc = ensure_store(h))) return rc;
    const size_t n3 = h->geo.n3;
    const size_t nq = (size_t)h->q.qf + h->q.qg;
    if ((rc = ensure_staging(h, nq * n3 * sizeof(double)))) return rc;
    PopArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.fout = h->staging;
    a.gout = h->staging + (size_t)h->q.qf * n3;
    a.rho0 = h->p.rho0;
    a.odd = 0;
    LBM_CUDA(cudaMemcpyAsync(a.fout, f, (size_t)h->q.qf * n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream),
             "copy f");
    LBM_CUDA(cudaMemcpyAsync(a.gout, g, (size_t)h->q.qg * n3 * sizeof(double), cudaMemcpyHostToDevice, h->stream),
             "copy g");
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->set_pops, dim3(flat_grid(h)), dim3(256), args, 0, h->stream), "set_pops");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "set_populations");
    h->initialized = true;
    h->odd = 0;
    return LBM_OK;
}

int lbm_step_count(lbm_handle h, int64_t* step)
{
    if (!h || !step) return fail(LBM_EINVAL, "null argument");
    *step = h->step;
    return LBM_OK;
}

int lbm_set_block(lbm_handle h, int bx, int by)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 256)
        return fail(LBM_EINVAL, "block (%d, %d): bx must be a positive multiple of 32 and bx*by <= 256", bx, by);
    h->bx = h->bxo = bx;
    h->by = h->byo = by;
    drop_graph(h);
    return LBM_OK;
}

int lbm_get_block(lbm_handle h, int* bx, int* by)
{
    if (!h || !bx || !by) return fail(LBM_EINVAL, "null argument");
    *bx = h->bx;
    *by = h->by;
    return LBM_OK;
}

int lbm_autotune(lbm_handle h, int reps, double* best_ms_per_step)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->initialized) return fail(LBM_ESTATE, "autotune needs an initialised state");
    if (reps < 1) return fail(LBM_EINVAL, "reps must be >= 1");
    static const int cand[][2] = {{32, 1}, {32, 2}, {32, 4}, {32, 8}, {64, 1}, {64, 2}, {64, 4},
                                  {128, 1}, {128, 2}, {256, 1}};
    void* backup = nullptr;
    size_t bytes = (size_t)(h->q.qf + h->q.qg) * h->geo.n3 * elem_size(h->p.storage);
    LBM_CUDA(cudaMalloc(&backup, bytes), "autotune backup allocation");
    // one event between consecutive launches, so that each launch is timed
    // on its own and the two AA parities get their own best shape
    std::vector<cudaEvent_t> ev(2 * (size_t)reps + 1, nullptr);
    for (cudaEvent_t& e : ev) cudaEventCreate(&e);
    cudaMemcpyAsync(backup, h->store, bytes, cudaMemcpyDeviceToDevice, h->stream);
    const int save_bx = h->bx, save_by = h->by, save_bxo = h->bxo, save_byo = h->byo, save_odd = h->odd;
    double best[2] = {1e300, 1e300};
    int bbx[2] = {save_bx, save_bxo}, bby[2] = {save_by, save_byo};
    cudaError_t err = cudaSuccess;
    for (const auto& c : cand) {
        if (c[0] > 32 && c[0] / 2 >= h->p.nx) continue;  // wider than the row
        if (c[1] > 1 && (c[1] / 2) >= h->p.ny) continue;
        h->bx = h->bxo = c[0];
        h->by = h->byo = c[1];
        // warm-up pair, then timed pairs
        for (int s = 0; s < 2 && err == cudaSuccess; ++s) err = launch_step(h, (save_odd + s) & 1, h->stream);
        if (err == cudaSuccess) err = cudaEventRecord(ev[0], h->stream);
        for (int s = 0; s < 2 * reps && err == cudaSuccess; ++s) {
            err = launch_step(h, (save_odd + s) & 1, h->stream);
            if (err == cudaSuccess) err = cudaEventRecord(ev[s + 1], h->stream);
        }
        if (err == cudaSuccess) err = cudaEventSynchronize(ev[2 * reps]);
        if (err != cudaSuccess) break;
        double t[2] = {0.0, 0.0};
        for (int s = 0; s < 2 * reps; ++s) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
            t[(save_odd + s) & 1] += ms / reps;
        }
        for (int par = 0; par < 2; ++par)
            if (t[par] < best[par]) {
                best[par] = t[par];
                bbx[par] = c[0];
                bby[par] = c[1];
            }
    }
    cudaMemcpyAsync(h->store, backup, bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaFree(backup);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    h->odd = save_odd;
    if (err != cudaSuccess) {
        h->bx = save_bx;
        h->by = save_by;
        h->bxo = save_bxo;
        h->byo = save_byo;
        return cuda_fail(err, "autotune");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "autotune restore");
    h->bx = bbx[0];
    h->by = bby[0];
    h->bxo = bbx[1];
    h->byo = bby[1];
    drop_graph(h);
    if (best_ms_per_step) *best_ms_per_step = 0.5 * (best[0] + best[1]);
    return LBM_OK;
}

int lbm_set_pairing(lbm_handle h, int mode)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (mode < LBM_PAIRING_OFF || mode > LBM_PAIRING_EVEN) return fail(LBM_EINVAL, "pairing mode must be 0, 1 or 2");
    h->pairing = mode;
    default_block(h);
    drop_graph(h);
    return LBM_OK;
}

int lbm_set_tile_staging(lbm_handle h, int enable)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    h->tile_staging = enable != 0;
    h->stage_grid = 0;
    drop_graph(h);
    return LBM_OK;
}

int lbm_uses_tile_staging(lbm_handle h, int* width)
{
    if (!h || !width) return fail(LBM_EINVAL, "null argument");
    *width = stage_width(h);
    return LBM_OK;
}

int lbm_set_stage_test(lbm_handle h, unsigned extra_tx_bytes, unsigned spin_limit)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (spin_limit == 0) return fail(LBM_EINVAL, "spin_limit must be positive");
    if (extra_tx_bytes >= (1u << 20)) return fail(LBM_EINVAL, "extra_tx_bytes must be below 2^20 (mbarrier tx count)");
    h->stage_extra_tx = extra_tx_bytes;
    h->stage_spin = spin_limit;
    drop_graph(h);
    return LBM_OK;
}

int lbm_set_slab(lbm_handle h, int enable)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (enable && h->p.nz < 3) return fail(LBM_EINVAL, "a z-slab needs nz >= 3 (two ghost planes and one of its own)");
    h->slab = enable != 0;
    h->stage_grid = 0;
    drop_graph(h);
    return LBM_OK;
}

int lbm_halo_bytes(lbm_handle h, size_t* bytes)
{
    if (!h || !bytes) return fail(LBM_EINVAL, "null argument");
    *bytes = (size_t)(halo_slots(h->q.qf, 1, nullptr) + halo_slots(h->q.qg, 1, nullptr)) * (size_t)h->p.nx *
             (size_t)h->p.ny * elem_size(h->p.storage);
    return LBM_OK;
}

int lbm_halo_pack(lbm_handle h, int phase, void* to_lower, void* to_upper)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->slab) return fail(LBM_ESTATE, "halo exchange without lbm_set_slab");
    if (!h->store) return fail(LBM_ESTATE, "halo exchange before the store exists");
    if (phase != 0 && phase != 1) return fail(LBM_EINVAL, "phase must be 0 (before an odd step) or 1 (after it)");
    if (!to_lower || !to_upper) return fail(LBM_EINVAL, "null buffer");
    if ((rc = check_device_buffer(h, to_lower)) || (rc = check_device_buffer(h, to_upper))) return rc;
    const int top = h->p.nz - 1;
    // phase 0: own boundary planes (plane 1: e_z = +1 slots; plane nz-2: e_z = -1)
    // phase 1: ghost planes (plane 0: e_z = -1 slots; plane nz-1: e_z = +1)
    if ((rc = halo_copy(h, phase ? 0 : 1, phase ? -1 : +1, to_lower, true))) return rc;
    return halo_copy(h, phase ? top : top - 1, phase ? +1 : -1, to_upper, true);
}

int lbm_halo_unpack(lbm_handle h, int phase, const void* from_lower, const void* from_upper)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->slab) return fail(LBM_ESTATE, "halo exchange without lbm_set_slab");
    if (!h->store) return fail(LBM_ESTATE, "halo exchange before the store exists");
    if (phase != 0 && phase != 1) return fail(LBM_EINVAL, "phase must be 0 (before an odd step) or 1 (after it)");
    if (!from_lower || !from_upper) return fail(LBM_EINVAL, "null buffer");
    if ((rc = check_device_buffer(h, from_lower)) || (rc = check_device_buffer(h, from_upper))) return rc;
    const int top = h->p.nz - 1;
    // phase 0: into the ghost planes (plane 0: e_z = -1 slots; plane nz-1: e_z = +1)
    // phase 1: into the own boundary planes (plane 1: e_z = +1; plane nz-2: e_z = -1)
    if ((rc = halo_copy(h, phase ? 1 : 0, phase ? +1 : -1, const_cast<void*>(from_lower), false))) return rc;
    return halo_copy(h, phase ? top - 1 : top, phase ? -1 : +1, const_cast<void*>(from_upper), false);
}

int lbm_set_graphs(lbm_handle h, int enable)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    h->graphs = enable != 0;
    if (!h->graphs) drop_graph(h);
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free diagnostics: the block partials of the moment pass and the
// final sums live in this file-scope device array instead of cudaMalloc'ed
// scratch. Host code cannot use the array's name as a device address, so the
// address is looked up with the device current and cached per device: when a
// handle is created (lbm_create_params) and, if still missing, on the first
// allocation-free call. A device reset destroys every handle, and the handles
// made after it look the address up again when they are created.
// ---------------------------------------------------------------------------
namespace {
constexpr int kStaticMaxBlocks = 4096;
constexpr uint32_t kStaticNodesPerBlock = 32768;
constexpr size_t kStaticOutOffset = (size_t)kStaticMaxBlocks * kDNumSlots;
constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_addr[kStaticMaxDevices] = {};
}  // namespace

static __device__ __align__(256) double g_static_scratch[kStaticOutOffset + 16];

namespace {
void static_scratch_refresh(int device)
{
    if (device < 0 || device >= kStaticMaxDevices) return;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_static_mutex);
    g_static_addr[device] = (e == cudaSuccess) ? static_cast<double*>(p) : nullptr;
}

int static_scratch_address(int device, double** out)
{
    if (device < 0 || device >= kStaticMaxDevices) return fail(LBM_EUNSUPPORTED, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the static diagnostics scratch");
        g_static_addr[device] = static_cast<double*>(p);
    }
    *out = g_static_addr[device];
    return LBM_OK;
}
}  // namespace

extern "C" {

int lbm_diagnostics_noalloc(lbm_handle h, lbm_diag* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBM_EINVAL, "null output");
    const uint32_t n3 = h->geo.n3;
    const uint32_t min_blocks = (n3 + kStaticNodesPerBlock - 1) / kStaticNodesPerBlock;
    if (min_blocks > (uint32_t)kStaticMaxBlocks)
        return fail(LBM_EINVAL,
                    "lattice of %u nodes exceeds the static diagnostics scratch (at most %u nodes); "
                    "use lbm_diagnostics",
                    n3, (unsigned)kStaticMaxBlocks * kStaticNodesPerBlock);
    if (!h->initialized) return fail(LBM_ESTATE, "diagnostics before initialisation");
    if (h->slab) return fail(LBM_EUNSUPPORTED, "allocation-free diagnostics of a z-slab (use lbm_diagnostics)");
    double* scratch = nullptr;
    if ((rc = static_scratch_address(h->device, &scratch))) return rc;
    // the moment pass strides over the lattice, so the grid fills the GPU
    // (4 blocks per SM, as lbm_diagnostics) whatever the node count, within
    // the array's rows and without blocks that get no node
    const uint32_t sms = (uint32_t)(h->num_sms > 0 ? h->num_sms : 132);
    const uint32_t busy = std::min(4 * sms, (n3 + kDiagBlock - 1) / (uint32_t)kDiagBlock);
    const uint32_t blocks = std::min((uint32_t)kStaticMaxBlocks, std::max(min_blocks, busy));
    const lbm_params& p = h->p;
    const double cs2f = cs2_of(h->q.qf);
    const double gn2 = (p.beta != 0.0) ? (-p.G * p.rho0 / p.beta) : 1.0;
    const double nu = cs2f * (p.tau_f - 0.5);
    DiagArgs a;
    a.f = f_ptr(h);
    a.g = g_ptr(h);
    a.geo = h->geo;
    a.ph = h->ph;
    a.odd = h->odd;
    a.ep_scale = (float)(0.5 * gn2 / (p.rho0 * p.rho0));
    a.epsk_scale = (float)(2.0 * nu);
    a.s_scale = (float)(-1.0 / (2.0 * cs2f * p.tau_f));
    a.epsp_scale = 0.f;
    a.nu = (float)nu;
    a.fields = nullptr;      // no field scratch: the central-difference pass is skipped
    a.partials = scratch;    // every block overwrites its own record, nothing needs clearing
    a.idx0 = 0;
    a.idx1 = n3;
    void* args[] = {&a};
    LBM_CUDA(cudaLaunchKernel(h->ks->diag_moments, dim3(blocks), dim3(kDiagBlock), args, 0, h->stream),
             "static diag pass 1");
    const double* pp = scratch;
    int nb = (int)blocks;
    int nb2 = 0;   // no pass 2 here
    double* dout = scratch + kStaticOutOffset;
    void* fargs[] = {&pp, &nb, &nb2, &dout};
    LBM_CUDA(cudaLaunchKernel(diag_final_kernel(), dim3(1), dim3(kDiagBlock), fargs, 0, h->stream),
             "static diag pass 2");
    double s[kDNumSlots];
    LBM_CUDA(cudaMemcpyAsync(s, dout, sizeof(s), cudaMemcpyDeviceToHost, h->stream), "static diag copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "static diagnostics");
    const double inv = 1.0 / (double)n3;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    out->Ek = s[kDEk] * inv;
    out->Ep = s[kDEp] * inv;
    out->eps_k = s[kDEpsK] * inv;
    out->eps_p = nan;
    out->eps_k_curl = nan;
    out->mass_f = (double)n3 + s[kDDrho];
    out->mass_g = (double)n3 * p.rho0 + s[kDA];
    out->mom[0] = s[kDJx];
    out->mom[1] = s[kDJy];
    out->mom[2] = s[kDJz];
    out->umax = s[kDUmax];
    out->step = h->step;
    fill_phys(p, out);
    for (int q = 0; q < kDiagPass1; ++q)
        if (!std::isfinite(s[q])) return fail(LBM_ENONFINITE, "non-finite diagnostics at step %lld", (long long)h->step);
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    if (!h) return LBM_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->own_store && h->store) cudaFree(h->store);
    if (h->staging) cudaFree(h->staging);
    if (h->diag_fields) cudaFree(h->diag_fields);
    if (h->diag_partials) cudaFree(h->diag_partials);
    if (h->diag_out) cudaFree(h->diag_out);
    if (h->diag_host) cudaFreeHost(h->diag_host);
    if (h->diag_event) cudaEventDestroy(h->diag_event);
    if (h->copy_event) cudaEventDestroy(h->copy_event);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    for (int b = 0; b < 2; ++b) {
        if (h->pre[b]) cudaFree(h->pre[b]);
        if (h->pre_done[b]) cudaEventDestroy(h->pre_done[b]);
        if (h->pre_free[b]) cudaEventDestroy(h->pre_free[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->d_err) cudaFree(h->d_err);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched instances: many independent lattices advanced by one launch.
// ---------------------------------------------------------------------------
struct lbm_batch_ctx {
    std::vector<lbm_ctx*> inst;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BatchInstance* d_inst = nullptr;
    uint16_t* d_tile = nullptr;
    unsigned* d_sync = nullptr;
    uint32_t ntiles = 0;
    uint32_t vbeg[8] = {}, vend[8] = {};   // tiles of each (pair, forcing) variant
    // per-variant streams and events: the captured graph runs each variant's
    // chain of steps as its own branch (variants share no instance)
    cudaStream_t vstream[8] = {};
    cudaEvent_t vjoin[8] = {};
    cudaEvent_t vfork = nullptr;
    // per-instance driver: chain c runs instances chain_of[c] in order, each
    // with its own single-lattice step kernel; streams and join events are
    // created on first use
    std::vector<std::vector<int>> chain_of;
    std::vector<cudaStream_t> cstream;
    std::vector<cudaEvent_t> cjoin;
    int bx = 32, by = 8;
    int mode = LBM_BATCH_PERSISTENT;
    int chunk = 100;
    int persistent_grid = 0;
    unsigned spin_limit = 1u << 22;   // ~0.3-1 s of polling at 64 ns naps
    unsigned extra_dep = 0;           // test hook: completions a dependency wait expects that never come
    // persistent driver: one step's tile list, its tile size, the queue and
    // completion counters, the kernel variant and its graphs (one per parity)
    uint16_t* d_flow_inst = nullptr;
    unsigned* d_flow = nullptr;
    uint32_t flow_tiles = 0;
    uint32_t flow_nodes = 2048;
    bool guo_sc_only = false;
    FlowArgs* flow_args = nullptr;   // the persistent launch's parameter block (descriptors by value)
    cudaGraphExec_t pgraph[2] = {nullptr, nullptr};
    int pgraph_steps[2] = {0, 0};
    bool initialized = false;
    int64_t step = 0;
    int odd = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

constexpr int kBatchGraphSteps = 64;
constexpr int kMaxChains = 128;   // graph branches of the per-instance driver

void batch_drop_graph(lbm_batch_ctx* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (int k = 0; k < 2; ++k) {
        if (b->pgraph[k]) cudaGraphExecDestroy(b->pgraph[k]);
        b->pgraph[k] = nullptr;
        b->pgraph_steps[k] = 0;
    }
}

int batch_build_tiles(lbm_batch_ctx* b)
{
    std::vector<BatchInstance> hi(b->inst.size());
    std::vector<uint16_t> tiles;
    uint32_t t0 = 0;
    // tiles listed variant by variant, so that each per-variant launch covers one range
    std::vector<size_t> order(b->inst.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) {
        return 4 * b->inst[a]->p.pair + b->inst[a]->p.forcing < 4 * b->inst[c]->p.pair + b->inst[c]->p.forcing;
    });
    for (int v = 0; v < 8; ++v) b->vbeg[v] = b->vend[v] = 0;
    for (size_t i : order) {
        lbm_ctx* h = b->inst[i];
        BatchInstance& I = hi[i];
        I.f = f_ptr(h);
        I.g = g_ptr(h);
        I.geo = h->geo;
        I.ph = h->ph;
        I.variant = 4 * h->p.pair + h->p.forcing;
        I.tx = (uint32_t)((h->p.nx + b->bx - 1) / b->bx);
        I.ty = (uint32_t)((h->p.ny + b->by - 1) / b->by);
        I.tile0 = t0;
        const uint64_t n = (uint64_t)I.tx * I.ty * (uint64_t)h->p.nz;
        if ((uint64_t)t0 + n > 0xffffffffull) return fail(LBM_EINVAL, "batch tile count exceeds 2^32");
        tiles.insert(tiles.end(), (size_t)n, (uint16_t)i);
        const int v = I.variant;
        if (b->vend[v] == b->vbeg[v]) b->vbeg[v] = t0;
        t0 += (uint32_t)n;
        b->vend[v] = t0;
    }
    b->ntiles = t0;
    // persistent driver: runs of flow_nodes consecutive nodes, instances with
    // the most bytes per step first
    std::vector<size_t> big(b->inst.size());
    for (size_t i = 0; i < big.size(); ++i) big[i] = i;
    std::stable_sort(big.begin(), big.end(),
                     [&](size_t a, size_t c) { return b->inst[a]->store_bytes > b->inst[c]->store_bytes; });
    std::vector<uint16_t> flow;
    b->guo_sc_only = true;
    for (size_t i : big) {
        BatchInstance& I = hi[i];
        I.flow0 = (uint32_t)flow.size();
        I.nflow = (I.geo.n3 + b->flow_nodes - 1) / b->flow_nodes;
        flow.insert(flow.end(), (size_t)I.nflow, (uint16_t)i);
        if (b->inst[i]->p.forcing != LBM_GUO && b->inst[i]->p.forcing != LBM_SHAN_CHEN) b->guo_sc_only = false;
    }
    if (flow.size() > 0x7fffffffull) return fail(LBM_EINVAL, "batch tile count exceeds 2^31");
    b->flow_tiles = (uint32_t)flow.size();
    if (hi.size() <= (size_t)kFlowMaxInst) {
        if (!b->flow_args) b->flow_args = new (std::nothrow) FlowArgs();
        if (!b->flow_args) return fail(LBM_ENOMEM, "host allocation failed");
        for (size_t i = 0; i < hi.size(); ++i) b->flow_args->inst[i] = hi[i];
    }
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_tile) cudaFree(b->d_tile);
    if (b->d_flow_inst) cudaFree(b->d_flow_inst);
    if (b->d_flow) cudaFree(b->d_flow);
    b->d_inst = nullptr;
    b->d_tile = nullptr;
    b->d_flow_inst = nullptr;
    b->d_flow = nullptr;
    if (cudaMalloc(&b->d_inst, hi.size() * sizeof(BatchInstance)) != cudaSuccess ||
        cudaMalloc(&b->d_tile, tiles.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&b->d_flow_inst, flow.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&b->d_flow, (1 + hi.size()) * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "batch descriptor allocation failed");
    }
    LBM_CUDA(cudaMemcpy(b->d_inst, hi.data(), hi.size() * sizeof(BatchInstance), cudaMemcpyHostToDevice),
             "copy batch descriptors");
    LBM_CUDA(cudaMemcpy(b->d_tile, tiles.data(), tiles.size() * sizeof(uint16_t), cudaMemcpyHostToDevice),
             "copy batch tiles");
    LBM_CUDA(cudaMemcpy(b->d_flow_inst, flow.data(), flow.size() * sizeof(uint16_t), cudaMemcpyHostToDevice),
             "copy batch tile list");
    int per_sm = 0;
    LBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_flow_kernel(b->guo_sc_only), 256, 0),
             "batch occupancy");
    if (per_sm < 1) return fail(LBM_EUNSUPPORTED, "persistent batch kernel does not fit on an SM");
    b->persistent_grid = per_sm * b->num_sms;
    batch_drop_graph(b);
    return LBM_OK;
}

BatchArgs batch_args(const lbm_batch_ctx* b, int steps, int odd0, unsigned grid)
{
    BatchArgs a;
    a.inst = b->d_inst;
    a.tile_inst = b->d_tile;
    a.ntiles = b->ntiles;
    a.tile_begin = 0;
    a.tile_end = b->ntiles;
    a.steps = steps;
    a.odd0 = odd0;
    a.sync = b->d_sync;
    a.spin_limit = b->spin_limit;
    a.flow_inst = b->d_flow_inst;
    a.flow_tiles = b->flow_tiles;
    a.flow_nodes = b->flow_nodes;
    a.flow = b->d_flow;
    a.extra_dep = b->extra_dep;
    (void)grid;
    return a;
}

cudaError_t batch_launch_variant(lbm_batch_ctx* b, int v, int odd, cudaStream_t s)
{
    const uint32_t n = b->vend[v] - b->vbeg[v];
    if (n == 0) return cudaSuccess;
    // one tile per block: the block scheduler then overlaps the descriptor
    // loads that start every tile (measured 2 % faster than a strided loop)
    const unsigned grid = (unsigned)n;
    BatchArgs a = batch_args(b, 1, odd, grid);
    a.tile_begin = b->vbeg[v];
    a.tile_end = b->vend[v];
    void* args[] = {&a};
    return cudaLaunchKernel(batch_variant_kernel(v, odd), dim3(grid), dim3(b->bx, b->by), args, 0, s);
}

cudaError_t batch_launch_step(lbm_batch_ctx* b, int odd, cudaStream_t s)
{
    for (int v = 0; v < 8; ++v) {
        cudaError_t e = batch_launch_variant(b, v, odd, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Per-instance driver: instances sorted by bytes per step, largest first,
// dealt round-robin to min(count, kMaxChains) chains, so that the longest
// chains start first and the chains carry similar work.
cudaError_t batch_ensure_chains(lbm_batch_ctx* b)
{
    if (!b->chain_of.empty()) return cudaSuccess;
    const int n = (int)b->inst.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto bytes = [&](int i) { return b->inst[i]->store_bytes; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return bytes(a) > bytes(c); });
    const int nc = n < kMaxChains ? n : kMaxChains;
    b->chain_of.assign(nc, {});
    for (int k = 0; k < n; ++k) b->chain_of[k % nc].push_back(order[k]);
    b->cstream.assign(nc, nullptr);
    b->cjoin.assign(nc, nullptr);
    for (int c = 0; c < nc; ++c) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cstream[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cjoin[c], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Per-instance driver: nsteps steps of every instance, each by lbm_step on
// its chain's stream (the instance's own 64-step graph replays, eager steps
// outside them), the chains forked from and joined back to b->stream.
int batch_step_instances(lbm_batch_ctx* b, int64_t nsteps)
{
    LBM_CUDA(batch_ensure_chains(b), "batch chain streams");
    LBM_CUDA(cudaEventRecord(b->vfork, b->stream), "batch fork");
    for (size_t c = 0; c < b->chain_of.size(); ++c) {
        LBM_CUDA(cudaStreamWaitEvent(b->cstream[c], b->vfork, 0), "batch fork wait");
        for (int i : b->chain_of[c]) {
            lbm_ctx* h = b->inst[i];
            h->stream = b->cstream[c];
            const int rc = lbm_step(h, nsteps);
            h->stream = b->stream;
            if (rc) return rc;
        }
        LBM_CUDA(cudaEventRecord(b->cjoin[c], b->cstream[c]), "batch join");
        LBM_CUDA(cudaStreamWaitEvent(b->stream, b->cjoin[c], 0), "batch join wait");
    }
    return LBM_OK;
}

// Records `steps` steps (from the natural layout) into the capture running on
// b->stream: each variant's chain on its own stream, forked from and joined
// back to b->stream.
cudaError_t batch_capture_steps(lbm_batch_ctx* b, int steps)
{
    cudaError_t e = cudaEventRecord(b->vfork, b->stream);
    for (int v = 0; v < 8 && e == cudaSuccess; ++v) {
        if (b->vend[v] == b->vbeg[v]) continue;
        e = cudaStreamWaitEvent(b->vstream[v], b->vfork, 0);
        for (int s = 0; s < steps && e == cudaSuccess; ++s) e = batch_launch_variant(b, v, s & 1, b->vstream[v]);
        if (e == cudaSuccess) e = cudaEventRecord(b->vjoin[v], b->vstream[v]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->vjoin[v], 0);
    }
    return e;
}

// One persistent launch of `steps` steps: clear the queue and completion
// counters, then the kernel (a plain launch: see lbm_batch.cu).
cudaError_t batch_launch_persistent(lbm_batch_ctx* b, int steps, int odd, cudaStream_t s)
{
    const unsigned grid = (unsigned)b->persistent_grid;
    // the descriptors travel in the parameter block (b->flow_args, filled by
    // batch_build_tiles); the launch copies it
    FlowArgs& fa = *b->flow_args;
    fa.a = batch_args(b, steps, odd, grid);
    cudaError_t e = cudaMemsetAsync(b->d_flow, 0, (1 + b->inst.size()) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&fa};
    return cudaLaunchKernel(batch_flow_kernel(b->guo_sc_only), dim3(grid), dim3(256), args, 0, s);
}

// The same launch replayed from a CUDA graph (one per starting parity).
cudaError_t batch_persistent_graph(lbm_batch_ctx* b, int steps, int odd)
{
    if (!b->pgraph[odd] || b->pgraph_steps[odd] != steps) {
        if (b->pgraph[odd]) cudaGraphExecDestroy(b->pgraph[odd]);
        b->pgraph[odd] = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = batch_launch_persistent(b, steps, odd, b->stream);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->pgraph[odd], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        b->pgraph_steps[odd] = steps;
    }
    return cudaGraphLaunch(b->pgraph[odd], b->stream);
}

void batch_sync_instances(lbm_batch_ctx* b)
{
    for (lbm_ctx* h : b->inst) {
        h->step = b->step;
        h->odd = b->odd;
        h->initialized = b->initialized;
    }
}

int batch_check(lbm_batch_ctx* b)
{
    if (!b) return fail(LBM_EINVAL, "null batch");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch* out, const lbm_params* params, int count)
{
    if (!out) return fail(LBM_EINVAL, "null output");
    *out = nullptr;
    if (!params || count < 1 || count > 65535) return fail(LBM_EINVAL, "count must be in [1, 65535]");
    for (int i = 0; i < count; ++i) {
        if (params[i].storage != LBM_FP32)
            return fail(LBM_EUNSUPPORTED, "batched instances use FP32 storage (instance %d)", i);
        if (params[i].pair != LBM_D3Q27_D3Q19 && params[i].pair != LBM_D3Q19_D3Q7)
            return fail(LBM_EUNSUPPORTED, "batched instances use D3Q27xD3Q19 or D3Q19xD3Q7 (instance %d)", i);
    }
    lbm_batch_ctx* b = new (std::nothrow) lbm_batch_ctx();
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    int rc = LBM_OK;
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(LBM_ECUDA, "stream creation failed");
    }
    b->own_stream = true;
    bool streams_ok = cudaEventCreateWithFlags(&b->vfork, cudaEventDisableTiming) == cudaSuccess;
    for (int v = 0; v < 8 && streams_ok; ++v) {
        streams_ok = cudaStreamCreateWithFlags(&b->vstream[v], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&b->vjoin[v], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!streams_ok) {
        cudaGetLastError();
        rc = fail(LBM_ECUDA, "batch stream or event creation failed");
    }
    for (int i = 0; i < count && rc == LBM_OK; ++i) {
        lbm_handle h = nullptr;
        rc = lbm_create_params(&h, &params[i]);
        if (rc) break;
        b->inst.push_back(h);
        if ((rc = lbm_set_stream(h, b->stream))) break;
        if ((rc = ensure_store(h))) break;
    }
    if (rc == LBM_OK && (cudaMalloc(&b->d_sync, 4 * sizeof(unsigned)) != cudaSuccess ||
                         cudaMemset(b->d_sync, 0, 4 * sizeof(unsigned)) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail(LBM_ENOMEM, "batch barrier allocation failed");
    }
    if (rc == LBM_OK) rc = batch_build_tiles(b);
    if (rc == LBM_OK && b->inst.size() > (size_t)kFlowMaxInst) b->mode = LBM_BATCH_PER_STEP;
    if (rc) {
        std::string msg = g_last_error;
        lbm_batch_destroy(b);
        g_last_error = msg;
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_count(lbm_batch b, int* count)
{
    if (!b || !count) return fail(LBM_EINVAL, "null argument");
    *count = (int)b->inst.size();
    return LBM_OK;
}

int lbm_batch_instance(lbm_batch b, int i, lbm_handle* h)
{
    if (!b || !h) return fail(LBM_EINVAL, "null argument");
    if (i < 0 || i >= (int)b->inst.size()) return fail(LBM_EINVAL, "instance %d out of range", i);
    *h = b->inst[i];
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch b, void* stream)
{
    int rc = batch_check(b);
    if (rc) return rc;
    if (b->own_stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    b->stream = static_cast<cudaStream_t>(stream);
    b->own_stream = false;
    for (lbm_ctx* h : b->inst) h->stream = b->stream;
    batch_drop_graph(b);
    return LBM_OK;
}

int lbm_batch_set_mode(lbm_batch b, int mode, int steps_per_launch)
{
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (mode != LBM_BATCH_PERSISTENT && mode != LBM_BATCH_PER_STEP && mode != LBM_BATCH_INSTANCES)
        return fail(LBM_EINVAL, "unknown mode %d", mode);
    if (steps_per_launch < 1) return fail(LBM_EINVAL, "steps per launch must be >= 1");
    if (mode == LBM_BATCH_PERSISTENT && b->inst.size() > (size_t)kFlowMaxInst)
        return fail(LBM_EUNSUPPORTED, "the persistent driver takes at most %d instances (batch has %zu)", kFlowMaxInst,
                    b->inst.size());
    if (mode != b->mode) batch_drop_graph(b);   // the graph holds one driver's launches
    b->mode = mode;
    b->chunk = steps_per_launch;
    return LBM_OK;
}

int lbm_batch_set_block(lbm_batch b, int bx, int by)
{
    int rc = batch_check(b);
    if (rc) return rc;
    if (!(bx == 16 || bx == 32 || bx == 64 || bx == 128) || by < 1 || bx * by > 256 || (bx * by) % 32 != 0)
        return fail(LBM_EINVAL, "batch block (%d, %d): bx in {16, 32, 64, 128}, bx*by a multiple of 32 <= 256", bx, by);
    b->bx = bx;
    b->by = by;
    return batch_build_tiles(b);
}

int lbm_batch_get_config(lbm_batch b, int* bx, int* by, int* mode, int* grid)
{
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (bx) *bx = b->bx;
    if (by) *by = b->by;
    if (mode) *mode = b->mode;
    if (grid) *grid = b->mode == LBM_BATCH_PERSISTENT ? b->persistent_grid : (int)b->ntiles;   // tiles: also per instance
    return LBM_OK;
}

int lbm_batch_init_tgv(lbm_batch b, uint64_t seed, double noise_amp)
{
    int rc = batch_check(b);
    if (rc) return rc;
    for (lbm_ctx* h : b->inst)
        if ((rc = lbm_init_tgv(h, seed, noise_amp))) return rc;
    b->initialized = true;
    b->step = 0;
    b->odd = 0;
    batch_sync_instances(b);
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int64_t nsteps)
{
    int rc = batch_check(b);
    if (rc) return rc;
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    if (!b->initialized) return fail(LBM_ESTATE, "batch step before initialisation");
    if (b->mode == LBM_BATCH_INSTANCES && nsteps > 0) {
        // no stream: every instance in turn on the legacy stream
        if (b->stream == nullptr) {
            for (lbm_ctx* h : b->inst)
                if ((rc = lbm_step(h, nsteps))) return rc;
        } else if ((rc = batch_step_instances(b, nsteps))) {
            return rc;
        }
        b->odd ^= (int)(nsteps & 1);
        b->step += nsteps;
        nsteps = 0;
    }
    while (nsteps > 0) {
        if (b->mode == LBM_BATCH_PERSISTENT) {
            // queue positions are 32-bit: steps * tiles per step (plus the
            // grid's claims past the end) must stay below 2^32
            const int64_t kmax = (int64_t)((0xffffffffull - 2ull * (uint64_t)b->persistent_grid) / b->flow_tiles);
            const int64_t chunk = std::min<int64_t>(b->chunk, std::max<int64_t>(kmax, 1));
            const int k = (int)(nsteps < chunk ? nsteps : chunk);
            if (b->stream != nullptr && k == chunk)
                LBM_CUDA(batch_persistent_graph(b, k, b->odd), "persistent batch graph");
            else
                LBM_CUDA(batch_launch_persistent(b, k, b->odd, b->stream), "persistent batch launch");
            b->odd ^= (k & 1);
            b->step += k;
            nsteps -= k;
            continue;
        }
        if (b->stream != nullptr && b->odd == 0 && nsteps >= kBatchGraphSteps) {
            if (!b->graph) {
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    e = batch_capture_steps(b, kBatchGraphSteps);
                    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
            }
            LBM_CUDA(cudaGraphLaunch(b->graph, b->stream), "batch graph launch");
            b->step += kBatchGraphSteps;
            nsteps -= kBatchGraphSteps;
            continue;
        }
        LBM_CUDA(batch_launch_step(b, b->odd, b->stream), "batch step launch");
        b->odd ^= 1;
        b->step += 1;
        nsteps -= 1;
    }
    batch_sync_instances(b);
    return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch b)
{
    int rc = batch_check(b);
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
    unsigned flags[4];
    LBM_CUDA(cudaMemcpy(flags, b->d_sync, sizeof(flags), cudaMemcpyDeviceToHost), "read barrier state");
    if (flags[2] != 0u) {
        cudaMemset(b->d_sync, 0, 4 * sizeof(unsigned));
        return fail(LBM_ETIMEOUT, "a dependency wait of the persistent batch kernel ran out; "
                                  "the state of the batch is undefined");
    }
    return LBM_OK;
}

int lbm_batch_diagnostics(lbm_batch b, lbm_diag* out)
{
    int rc = lbm_batch_synchronize(b);
    if (rc) return rc;
    if (!out) return fail(LBM_EINVAL, "null output");
    int worst = LBM_OK;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        rc = lbm_diagnostics(b->inst[i], &out[i]);
        if (rc == LBM_ENONFINITE) worst = rc;
        else if (rc) return rc;
    }
    return worst;
}

int lbm_batch_autotune(lbm_batch b, int reps, double* best_ms_per_step)
{
    int rc = batch_check(b);
    if (rc) return rc;
    if (!b->initialized) return fail(LBM_ESTATE, "autotune needs an initialised batch");
    if (reps < 1) return fail(LBM_EINVAL, "reps must be >= 1");
    if ((rc = lbm_batch_synchronize(b))) return rc;
    std::vector<void*> backup(b->inst.size(), nullptr);
    for (size_t i = 0; i < b->inst.size(); ++i) {
        if (cudaMalloc(&backup[i], b->inst[i]->store_bytes) != cudaSuccess) {
            cudaGetLastError();
            for (void* p : backup) if (p) cudaFree(p);
            return fail(LBM_ENOMEM, "autotune backup allocation failed");
        }
        cudaMemcpyAsync(backup[i], b->inst[i]->store, b->inst[i]->store_bytes, cudaMemcpyDeviceToDevice, b->stream);
    }
    static const int cand[][2] = {{16, 8}, {32, 2}, {32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1}, {128, 2}};
    static const int flow_cand[] = {1024, 2048, 4096, 8192};
    const int save_bx = b->bx, save_by = b->by, save_mode = b->mode, save_odd = b->odd;
    const uint32_t save_flow = b->flow_nodes;
    const int64_t save_step = b->step;
    double best = 1e300;
    int bbx = save_bx, bby = save_by, bmode = save_mode;
    uint32_t bflow = save_flow;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one candidate as lbm_batch_step runs it: a warm-up span (which also
    // builds the graphs), then `reps` spans timed with events; a span is one
    // 64-step graph (per-step and per-instance drivers) or one persistent launch
    auto time_mode = [&](int mode, double* per) {
        b->mode = mode;
        const int64_t span = (mode == LBM_BATCH_PERSISTENT) ? b->chunk : kBatchGraphSteps;
        int r = lbm_batch_step(b, span);
        if (r) return r;
        cudaEventRecord(e0, b->stream);
        r = lbm_batch_step(b, span * (int64_t)reps);
        cudaEventRecord(e1, b->stream);
        if (r) return r;
        if ((r = lbm_batch_synchronize(b))) return r;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *per = ms / (double)(span * reps);
        return LBM_OK;
    };
    for (const auto& c : cand) {
        b->bx = c[0];
        b->by = c[1];
        if ((rc = batch_build_tiles(b))) break;
        double per = 0.0;
        if ((rc = time_mode(LBM_BATCH_PER_STEP, &per))) break;
        if (per < best) {
            best = per;
            bbx = c[0];
            bby = c[1];
            bmode = LBM_BATCH_PER_STEP;
        }
    }
    b->bx = save_bx;
    b->by = save_by;
    const bool flow_ok = b->inst.size() <= (size_t)kFlowMaxInst;
    for (size_t k = 0; flow_ok && k < sizeof(flow_cand) / sizeof(flow_cand[0]) && rc == LBM_OK; ++k) {
        b->flow_nodes = (uint32_t)flow_cand[k];
        if ((rc = batch_build_tiles(b))) break;
        double per = 0.0;
        if ((rc = time_mode(LBM_BATCH_PERSISTENT, &per))) break;
        if (per < best) {
            best = per;
            bbx = save_bx;
            bby = save_by;
            bflow = b->flow_nodes;
            bmode = LBM_BATCH_PERSISTENT;
        }
    }
    b->flow_nodes = save_flow;
    if (rc == LBM_OK) {
        // per-instance driver: every instance's own launch shape, then whole
        // 64-step graphs of all chains
        batch_sync_instances(b);
        for (lbm_ctx* h : b->inst)
            if ((rc = lbm_autotune(h, reps, nullptr))) break;
        b->mode = LBM_BATCH_INSTANCES;
        batch_drop_graph(b);
        if (rc == LBM_OK) rc = lbm_batch_step(b, kBatchGraphSteps);   // warm-up, builds the graph
        if (rc == LBM_OK) {
            cudaEventRecord(e0, b->stream);
            rc = lbm_batch_step(b, kBatchGraphSteps * (int64_t)reps);
            cudaEventRecord(e1, b->stream);
        }
        if (rc == LBM_OK) rc = lbm_batch_synchronize(b);
        if (rc == LBM_OK) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / (double)(kBatchGraphSteps * reps);
            if (per < best) {
                best = per;
                bbx = b->bx;
                bby = b->by;
                bflow = b->flow_nodes;
                bmode = LBM_BATCH_INSTANCES;
            }
        }
    }
    for (size_t i = 0; i < b->inst.size(); ++i) {
        cudaMemcpyAsync(b->inst[i]->store, backup[i], b->inst[i]->store_bytes, cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    for (void* p : backup) cudaFree(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->odd = save_odd;
    b->step = save_step;
    b->bx = bbx;
    b->by = bby;
    b->flow_nodes = bflow;
    b->mode = bmode;
    int rc2 = batch_build_tiles(b);
    batch_sync_instances(b);
    if (rc) return rc;
    if (rc2) return rc2;
    if (best_ms_per_step) *best_ms_per_step = best;
    return LBM_OK;
}

int lbm_batch_set_barrier_test(lbm_batch b, unsigned extra_completions, unsigned spin_limit)
{
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (spin_limit < 1) return fail(LBM_EINVAL, "spin limit must be >= 1");
    b->extra_dep = extra_completions;
    b->spin_limit = spin_limit;
    batch_drop_graph(b);
    return LBM_OK;
}

int lbm_batch_partition(const lbm_params* params, int count, int nranks, int32_t* owner, double* imbalance)
{
    if (!params || !owner || count < 1 || count > 65535 || nranks < 1)
        return fail(LBM_EINVAL, "lbm_batch_partition: null argument, count outside [1, 65535] or nranks < 1");
    std::vector<double> bytes(count);
    for (int i = 0; i < count; ++i) {
        PairInfo q;
        int rc = validate_params(&params[i], &q);
        if (rc) return rc;
        bytes[i] = (double)(q.qf + q.qg) * (double)params[i].nx * params[i].ny * params[i].nz *
                   (double)elem_size(params[i].storage);
    }
    // longest first (ties: lower index first), each to the least-loaded rank (ties: lower rank)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return bytes[a] > bytes[c]; });
    std::vector<double> load(nranks, 0.0);
    for (int i : order) {
        int r = 0;
        for (int k = 1; k < nranks; ++k)
            if (load[k] < load[r]) r = k;
        owner[i] = r;
        load[r] += bytes[i];
    }
    if (imbalance) {
        double total = 0.0, mx = 0.0;
        for (double l : load) {
            total += l;
            mx = std::max(mx, l);
        }
        *imbalance = mx / (total / nranks);
    }
    return LBM_OK;
}

int lbm_batch_set_flow_nodes(lbm_batch b, int nodes)
{
    int rc = batch_check(b);
    if (rc) return rc;
    if (nodes < 256 || nodes > 65536 || nodes % 256 != 0)
        return fail(LBM_EINVAL, "nodes per tile must be a multiple of 256 in [256, 65536] (got %d)", nodes);
    b->flow_nodes = (uint32_t)nodes;
    return batch_build_tiles(b);
}

int lbm_batch_get_flow_nodes(lbm_batch b, int* nodes)
{
    if (!b || !nodes) return fail(LBM_EINVAL, "null argument");
    *nodes = (int)b->flow_nodes;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b)
{
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (lbm_ctx* h : b->inst) {
        h->stream = nullptr;
        h->own_stream = false;
        lbm_destroy(h);
    }
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_tile) cudaFree(b->d_tile);
    if (b->d_flow_inst) cudaFree(b->d_flow_inst);
    if (b->d_flow) cudaFree(b->d_flow);
    delete b->flow_args;
    if (b->d_sync) cudaFree(b->d_sync);
    for (int v = 0; v < 8; ++v) {
        if (b->vstream[v]) cudaStreamDestroy(b->vstream[v]);
        if (b->vjoin[v]) cudaEventDestroy(b->vjoin[v]);
    }
    if (b->vfork) cudaEventDestroy(b->vfork);
    for (cudaStream_t cs : b->cstream)
        if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t ce : b->cjoin)
        if (ce) cudaEventDestroy(ce);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The 16-bit storage rule (host logic on a few numbers per sample).
// ---------------------------------------------------------------------------
namespace {

// max_s |c_s - r_s| / max_s |r_s| of one diagnostics quantity; +inf when the
// candidate is not finite, 0 for an all-zero reference matched exactly.
template <class Get>
double series_dev(const lbm_diag* ref, const lbm_diag* cand, int64_t count, Get get)
{
    double scale = 0.0, worst = 0.0;
    for (int64_t s = 0; s < count; ++s) {
        const double r = get(ref[s]), c = get(cand[s]);
        if (!std::isfinite(c)) return std::numeric_limits<double>::infinity();
        scale = std::max(scale, std::fabs(r));
        worst = std::max(worst, std::fabs(c - r));
    }
    if (scale > 0.0) return worst / scale;
    return worst > 0.0 ? std::numeric_limits<double>::infinity() : 0.0;
}

}  // namespace

extern "C" {

int lbm_storage_rule(const lbm_diag* ref, const lbm_diag* cand, int64_t count, int candidate_storage, double tol,
                     lbm_storage_report* report)
{
    if (!ref || !cand || count < 1) return fail(LBM_EINVAL, "lbm_storage_rule needs two series of >= 1 samples");
    if (candidate_storage < LBM_FP32 || candidate_storage > LBM_BF16_DEV)
        return fail(LBM_EINVAL, "unknown storage %d", candidate_storage);
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(LBM_EINVAL, "tol must be finite and > 0");
    for (int64_t s = 0; s < count; ++s) {
        if (ref[s].step != cand[s].step)
            return fail(LBM_EINVAL, "sample %lld: reference step %lld, candidate step %lld", (long long)s,
                        (long long)ref[s].step, (long long)cand[s].step);
        if (!std::isfinite(ref[s].Ek) || !std::isfinite(ref[s].Ep) || !std::isfinite(ref[s].eps_k) ||
            !std::isfinite(ref[s].eps_p))
            return fail(LBM_EINVAL, "reference sample %lld is not finite", (long long)s);
    }
    lbm_storage_report r{};
    r.dev_Ek = series_dev(ref, cand, count, [](const lbm_diag& d) { return d.Ek; });
    r.dev_Ep = series_dev(ref, cand, count, [](const lbm_diag& d) { return d.Ep; });
    r.dev_eps_k = series_dev(ref, cand, count, [](const lbm_diag& d) { return d.eps_k; });
    r.dev_eps_p = series_dev(ref, cand, count, [](const lbm_diag& d) { return d.eps_p; });
    // the two highest interior local maxima of the reference eps_k + eps_p
    auto eps = [](const lbm_diag& d) { return d.eps_k + d.eps_p; };
    int64_t p1 = -1, p2 = -1;
    for (int64_t s = 1; s + 1 < count; ++s) {
        const double e = eps(ref[s]);
        if (!(e > eps(ref[s - 1]) && e >= eps(ref[s + 1]))) continue;
        if (p1 < 0 || e > eps(ref[p1])) {
            p2 = p1;
            p1 = s;
        } else if (p2 < 0 || e > eps(ref[p2])) {
            p2 = s;
        }
    }
    const double nan = std::numeric_limits<double>::quiet_NaN();
    auto peak_dev = [&](int64_t s) {
        if (s < 0) return nan;
        const double c = eps(cand[s]);
        if (!std::isfinite(c)) return std::numeric_limits<double>::infinity();
        return std::fabs(c - eps(ref[s])) / std::fabs(eps(ref[s]));
    };
    r.dev_peak1 = peak_dev(p1);
    r.dev_peak2 = peak_dev(p2);
    r.step_peak1 = p1 < 0 ? -1 : ref[p1].step;
    r.step_peak2 = p2 < 0 ? -1 : ref[p2].step;
    bool pass = r.dev_Ek <= tol && r.dev_Ep <= tol && r.dev_eps_k <= tol && r.dev_eps_p <= tol;
    if (p1 >= 0) pass = pass && r.dev_peak1 <= tol;
    if (p2 >= 0) pass = pass && r.dev_peak2 <= tol;
    r.pass = pass ? 1 : 0;
    r.selected = pass ? candidate_storage : LBM_FP32;
    if (report) *report = r;
    return r.selected;
}

}  // extern "C"

// Kernel tables, one per (stencil pair, storage type); each instantiation file
// defines one. Entries are kernel function pointers launched with
// cudaLaunchKernel by the C ABI in lbm_api.cu.
#pragma once

namespace lbm {

struct KernelSet {
    int qf, qg;
    const void* step[4][2];   // [forcing][odd]
    const void* step2[4][2];  // two nodes per thread (16-bit storage, even nx), or null
    const void* staged[4][2]; // two nodes per thread, bulk-copy staged tiles (16-bit storage), or null
    const void* step_diag[4][2];   // step that also reduces the diagnostics of its input state
    const void* step2_diag[4][2];  // the same for the two-nodes-per-thread kernel, or null
    const void* init_fields;
    const void* init_tgv;
    const void* get_pops;
    const void* set_pops;
    const void* diag_moments;
    const void* get_fields;
    const void* sample_pops;
};

// pair: 0 = D3Q27xD3Q19, 1 = D3Q19xD3Q7, 2 = D3Q27xD3Q27, 3 = D3Q19xD3Q19,
//       4 = D3Q19xD3Q15, 5 = D3Q15xD3Q7, 6 = D3Q7xD3Q27
// storage: 0 = FP32, 1 = FP16 deviation, 2 = BF16 deviation
// Returns null for a combination that is not compiled in.
const KernelSet* kernel_set(int pair, int storage);

const void* diag_gradients_kernel();
const void* diag_final_kernel();

// Batched update (FP32 storage, D3Q27xD3Q19 and D3Q19xD3Q7, all forcings).
const void* batch_variant_kernel(int variant, int odd);   // variant = 4 * pair + forcing
const void* batch_flow_kernel(bool guo_sc_only);   // persistent driver

}  // namespace lbm

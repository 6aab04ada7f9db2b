// Lookup of the compiled kernel tables, and the two non-templated
// diagnostics kernels (compiled here only).
#define LBM_REDUCTION_KERNELS
#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"

namespace lbm {

const KernelSet* kernels_q27q19_f32();
const KernelSet* kernels_q27q19_f16();
const KernelSet* kernels_q27q19_bf16();
const KernelSet* kernels_q19q7_f32();
const KernelSet* kernels_q19q7_f16();
const KernelSet* kernels_q19q7_bf16();
const KernelSet* kernels_q27q27_f32();
const KernelSet* kernels_q19q19_f32();
const KernelSet* kernels_q19q15_f32();
const KernelSet* kernels_q15q7_f32();
const KernelSet* kernels_q7q27_f32();
const KernelSet* kernels_q27q27_f16();
const KernelSet* kernels_q19q19_f16();
const KernelSet* kernels_q19q15_f16();
const KernelSet* kernels_q15q7_f16();
const KernelSet* kernels_q7q27_f16();

const KernelSet* kernel_set(int pair, int storage)
{
    if (storage < 0 || storage > 2) return nullptr;
    switch (pair) {
    case 0: return storage == 0 ? kernels_q27q19_f32() : storage == 1 ? kernels_q27q19_f16() : kernels_q27q19_bf16();
    case 1: return storage == 0 ? kernels_q19q7_f32() : storage == 1 ? kernels_q19q7_f16() : kernels_q19q7_bf16();
    // the paper's other pairs (Sections 3.2-3.3), FP32 and FP16 storage (the
    // 16-bit storage rule keeps FP16; BF16 misses it on the headline pair)
    case 2: return storage == 0 ? kernels_q27q27_f32() : storage == 1 ? kernels_q27q27_f16() : nullptr;
    case 3: return storage == 0 ? kernels_q19q19_f32() : storage == 1 ? kernels_q19q19_f16() : nullptr;
    case 4: return storage == 0 ? kernels_q19q15_f32() : storage == 1 ? kernels_q19q15_f16() : nullptr;
    case 5: return storage == 0 ? kernels_q15q7_f32() : storage == 1 ? kernels_q15q7_f16() : nullptr;
    case 6: return storage == 0 ? kernels_q7q27_f32() : storage == 1 ? kernels_q7q27_f16() : nullptr;
    default: return nullptr;
    }
}

const void* diag_gradients_kernel() { return (const void*)k_diag_gradients; }
const void* diag_final_kernel() { return (const void*)k_diag_final; }

}  // namespace lbm

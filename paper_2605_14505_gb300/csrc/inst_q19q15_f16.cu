// Kernel table: D3Q19 x D3Q15, f16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q19q15_f16, 19, 15, __half)

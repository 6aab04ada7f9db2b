// Kernel table: D3Q19 x D3Q15, f32 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q19q15_f32, 19, 15, float)

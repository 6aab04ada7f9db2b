// Kernel table: D3Q15 x D3Q7, f32 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q15q7_f32, 15, 7, float)

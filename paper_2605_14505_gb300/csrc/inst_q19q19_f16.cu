// Kernel table: D3Q19 x D3Q19, f16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q19q19_f16, 19, 19, __half)

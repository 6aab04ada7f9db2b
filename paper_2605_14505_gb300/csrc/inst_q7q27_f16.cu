// Kernel table: D3Q7 x D3Q27, f16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q7q27_f16, 7, 27, __half)

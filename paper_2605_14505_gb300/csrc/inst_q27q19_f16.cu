// Kernel table: D3Q27 x D3Q19, f16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q27q19_f16, 27, 19, __half)

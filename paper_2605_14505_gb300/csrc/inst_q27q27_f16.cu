// Kernel table: D3Q27 x D3Q27, f16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q27q27_f16, 27, 27, __half)

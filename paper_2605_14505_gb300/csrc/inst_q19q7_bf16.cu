// Kernel table: D3Q19 x D3Q7, bf16 storage.
#include "lbm_inst.cuh"
LBM_DEFINE_KERNEL_SET(kernels_q19q7_bf16, 19, 7, __nv_bfloat16)

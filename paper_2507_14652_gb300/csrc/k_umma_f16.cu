// k_umma_f16.cu -- the tensor-core engines of k_umma.cu with fp16 GEMM operands
// (HMC_PREC_FP16): the same kernels compiled with the 16-bit type set to __half.
#define HMC_F16 1
#include "k_umma.cu"

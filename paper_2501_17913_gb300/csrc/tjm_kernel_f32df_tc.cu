// Instantiation of the persistent trajectory kernel with the tcgen05
// contraction path: contractions in float, factorizations in double-float (FP64 emulated on the FP32 pipes).
#define TJM_TENSOR_CORES 1
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32df_tc, float, df64)

// Instantiation of the persistent trajectory kernel with the tcgen05
// contraction path: contractions and factorizations in float.
#define TJM_TENSOR_CORES 1
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32d32_tc, float, float)

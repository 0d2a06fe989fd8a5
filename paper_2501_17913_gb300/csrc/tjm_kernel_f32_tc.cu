// Instantiation of the persistent trajectory kernel with the tcgen05
// contraction path: contractions in float, factorizations in double.
#define TJM_TENSOR_CORES 1
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32_tc, float, double)

// Instantiation of the persistent trajectory kernel on the CUDA cores:
// contractions and factorizations in float.
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32d32, float, float)

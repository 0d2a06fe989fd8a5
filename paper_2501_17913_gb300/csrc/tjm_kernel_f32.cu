// Instantiation of the persistent trajectory kernel on the CUDA cores:
// contractions in float, factorizations in double.
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32, float, double)

// Instantiation of the persistent trajectory kernel on the CUDA cores:
// contractions in double, factorizations in double.
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f64, double, double)

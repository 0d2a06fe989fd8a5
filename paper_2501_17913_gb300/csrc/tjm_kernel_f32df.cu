// Instantiation of the persistent trajectory kernel on the CUDA cores:
// contractions in float, factorizations in double-float (FP64 emulated on the FP32 pipes).
#include "tjm_kernel_inst.cuh"

TJM_DEFINE_LAUNCH(f32df, float, df64)

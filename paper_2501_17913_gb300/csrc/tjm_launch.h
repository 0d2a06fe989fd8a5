// Launchers of the persistent trajectory kernel, one per precision pair and,
// for FP32 contractions, one more with the tcgen05 path (suffix _tc); each
// lives in its own translation unit so the instantiations compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "tjm_types.h"

namespace tjm {

#define TJM_DECLARE_LAUNCH(NAME)                                                                              \
  cudaError_t launch_##NAME(cudaStream_t s, SlotDev* const* order, int n, int* next, int max_steps, int ctas, \
                            char* scratch, long long stride, ScratchDims dims, long long tc_min_work);                               \
  int occupancy_##NAME(int use_tc);

TJM_DECLARE_LAUNCH(f64)
TJM_DECLARE_LAUNCH(f32)
TJM_DECLARE_LAUNCH(f32d32)
TJM_DECLARE_LAUNCH(f32df)
TJM_DECLARE_LAUNCH(f32_tc)
TJM_DECLARE_LAUNCH(f32d32_tc)
TJM_DECLARE_LAUNCH(f32df_tc)

}  // namespace tjm

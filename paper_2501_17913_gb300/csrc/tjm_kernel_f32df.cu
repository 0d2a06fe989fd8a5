// Instantiation of the persistent trajectory kernel: contractions in float,
// factorizations in double-float (FP64 emulated on the FP32 pipes).
#include "tjm_kernels.cuh"
#include "tjm_launch.h"

namespace tjm {

cudaError_t launch_f32df(cudaStream_t s, SlotDev* const* order, int n, int* next, int max_steps, int ctas,
                        char* scratch, long long stride, ScratchDims dims, long long tc_min_work) {
  auto kern = advance_kernel<float, df64>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<float, df64>(true));
  if (e != cudaSuccess) return e;
  kern<<<ctas, TJM_THREADS, smem_bytes<float, df64>(tc_min_work > 0), s>>>(order, n, next, max_steps, scratch, stride,
                                                                        dims, tc_min_work);
  return cudaGetLastError();
}

int occupancy_f32df(int use_tc) {
  int per_sm = 0;
  cudaFuncSetAttribute(advance_kernel<float, df64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem_bytes<float, df64>(true));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advance_kernel<float, df64>, TJM_THREADS,
                                                smem_bytes<float, df64>(use_tc != 0));
  return per_sm;
}

}  // namespace tjm

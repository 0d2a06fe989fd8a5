// Instantiation of the persistent trajectory kernel: contractions in double,
// factorizations in double.
#include "tjm_kernels.cuh"
#include "tjm_launch.h"

namespace tjm {

cudaError_t launch_f64(cudaStream_t s, SlotDev* const* order, int n, int* next, int max_steps, int ctas,
                        char* scratch, long long stride, ScratchDims dims, long long tc_min_work) {
  auto kern = advance_kernel<double, double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<double, double>(true));
  if (e != cudaSuccess) return e;
  kern<<<ctas, TJM_THREADS, smem_bytes<double, double>(tc_min_work > 0), s>>>(order, n, next, max_steps, scratch, stride,
                                                                        dims, tc_min_work);
  return cudaGetLastError();
}

int occupancy_f64(int use_tc) {
  int per_sm = 0;
  cudaFuncSetAttribute(advance_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem_bytes<double, double>(true));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advance_kernel<double, double>, TJM_THREADS,
                                                smem_bytes<double, double>(use_tc != 0));
  return per_sm;
}

}  // namespace tjm

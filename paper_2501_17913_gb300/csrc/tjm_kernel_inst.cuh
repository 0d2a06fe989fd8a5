// Launcher and occupancy query of one instantiation of the persistent
// trajectory kernel.  Each translation unit that expands TJM_DEFINE_LAUNCH
// compiles one precision pair, with (TJM_TENSOR_CORES = 1) or without the
// tcgen05 contraction path, so the instantiations compile in parallel.
#pragma once
#include "tjm_kernels.cuh"
#include "tjm_launch.h"

#define TJM_DEFINE_LAUNCH(NAME, TC, TD)                                                                              \
  namespace tjm {                                                                                                    \
  cudaError_t launch_##NAME(cudaStream_t s, SlotDev* const* order, int n, int* next, int max_steps, int ctas,        \
                            char* scratch, long long stride, ScratchDims dims, long long tc_min_work) {              \
    auto kern = advance_kernel<TC, TD>;                                                                              \
    const bool tc = TJM_TENSOR_CORES && tc_min_work > 0;                                                             \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<TC, TD>(tc)); \
    if (e != cudaSuccess) return e;                                                                                  \
    kern<<<ctas, TJM_THREADS, smem_bytes<TC, TD>(tc), s>>>(order, n, next, max_steps, scratch, stride, dims,         \
                                                             tc ? tc_min_work : 0);                                  \
    return cudaGetLastError();                                                                                       \
  }                                                                                                                  \
  int occupancy_##NAME(int use_tc) {                                                                                 \
    int per_sm = 0;                                                                                                  \
    const bool tc = TJM_TENSOR_CORES && use_tc;                                                                      \
    if (cudaFuncSetAttribute(advance_kernel<TC, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,                    \
                             smem_bytes<TC, TD>(tc)) != cudaSuccess)                                                 \
      return 0;                                                                                                      \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advance_kernel<TC, TD>, TJM_THREADS,                  \
                                                      smem_bytes<TC, TD>(tc)) != cudaSuccess)                        \
      return 0;                                                                                                      \
    return per_sm;                                                                                                   \
  }                                                                                                                  \
  }

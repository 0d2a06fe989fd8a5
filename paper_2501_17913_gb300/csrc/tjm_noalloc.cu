// tjm_svd_noalloc: the one-CTA Jacobi SVD with its workspace in a file-scope
// device array instead of memory obtained from cudaMalloc.
//
// Some callers cannot let a library allocate device memory: applications that
// hand all device memory to their own pool or arena allocator and forbid any
// other allocation, and latency-sensitive loops that must not pay for
// cudaMalloc/cudaFree (cudaFree synchronises the whole device and stalls every
// other stream).  For them this entry point takes device pointers for its
// inputs and outputs and uses only the static workspace below.
#include <cuda_runtime.h>

#include <mutex>

#include "tjm.h"
#include "tjm_svd_call.cuh"

namespace {

constexpr int kMaxDim = TJM_NOALLOC_MAX_DIM;
// workspace of the largest problem (a 128 x 128 work matrix, 16-byte complex
// elements for FP64 and double-float, 8 for FP32), laid out and sized by the
// same function as every other standalone SVD call, plus the permutation ints
constexpr size_t kWorkBytes = (tjm::svd_call_slots(kMaxDim, kMaxDim) * 16 + 255) / 256 * 256;
constexpr size_t kIntBytes = (size_t)2 * kMaxDim * sizeof(int);
constexpr size_t kScratchBytes = kWorkBytes + kIntBytes;
static_assert(kWorkBytes >= tjm::svd_call_slots(kMaxDim, kMaxDim) * 16, "workspace holds the largest call");

// Held by every GPU that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_svd_scratch[kScratchBytes];

// Device address of g_svd_scratch per device ordinal, looked up once per device.
std::mutex g_mu;
void* g_addr[64] = {nullptr};

template <class T>
__global__ void __launch_bounds__(TJM_THREADS, 1)
svd_noalloc_kernel(int m, int n, const tjm::cx<double>* A, tjm::cx<double>* U, double* S, tjm::cx<double>* V,
                   tjm::cx<T>* ws, int* iw) {
  __shared__ double red[TJM_WARPS * 64];
  // nothing in the workspace has to be cleared between calls: every entry the
  // factorization reads is written first within the call
  tjm::svd_call_body<T>(m, n, A, U, S, V, ws, iw, red);
}

}  // namespace

extern "C" tjm_status tjm_svd_noalloc(int double_precision, int m, int n, const double* A, double* U, double* S,
                                      double* V, void* stream) {
  if (m < 1 || n < 1 || !A || !U || !S || !V || double_precision < 0 || double_precision > 2) return TJM_EINVAL;
  if (m > kMaxDim || n > kMaxDim) return TJM_EINVAL;   // the static workspace holds at most 128 x 128
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TJM_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // g_svd_scratch names a host-side stand-in in host code; the kernel needs
      // the device address, fetched with this device current
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_svd_scratch) != cudaSuccess || !p) return TJM_ECUDA;
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  unsigned char* scratch = reinterpret_cast<unsigned char*>(base);
  int* iw = reinterpret_cast<int*>(scratch + kWorkBytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const auto* dA = reinterpret_cast<const tjm::cx<double>*>(A);
  auto* dU = reinterpret_cast<tjm::cx<double>*>(U);
  auto* dV = reinterpret_cast<tjm::cx<double>*>(V);
  // An error the caller left pending is not ours to consume: report it
  // without launching and leave it in place.
  if (cudaPeekAtLastError() != cudaSuccess) return TJM_ECUDA;
  if (double_precision == 2)
    svd_noalloc_kernel<tjm::df64><<<1, TJM_THREADS, 0, st>>>(m, n, dA, dU, S, dV,
                                                             reinterpret_cast<tjm::cx<tjm::df64>*>(scratch), iw);
  else if (double_precision)
    svd_noalloc_kernel<double><<<1, TJM_THREADS, 0, st>>>(m, n, dA, dU, S, dV,
                                                           reinterpret_cast<tjm::cx<double>*>(scratch), iw);
  else
    svd_noalloc_kernel<float><<<1, TJM_THREADS, 0, st>>>(m, n, dA, dU, S, dV,
                                                          reinterpret_cast<tjm::cx<float>*>(scratch), iw);
  // nothing was pending before the launch, so an error now is the launch's own
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return TJM_ECUDA;
  }
  return TJM_OK;
}

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
#include "tjm_linalg.cuh"

namespace {

constexpr int kMaxDim = TJM_NOALLOC_MAX_DIM;
// workspace of the largest problem (FP64): work matrix, U, V, the rotation
// accumulator with its singular-value tail, the singular values, and the
// permutation ints -- identical to the per-call layout of the SVD self test
constexpr size_t kComplexSlots = (size_t)2 * kMaxDim * kMaxDim + 2 * kMaxDim * kMaxDim + 4 * kMaxDim + 8;
constexpr size_t kWorkBytes = kComplexSlots * 16;
constexpr size_t kIntBytes = (size_t)2 * kMaxDim * sizeof(int);
constexpr size_t kScratchBytes = kWorkBytes + kIntBytes;

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
  const bool tr = m < n;
  const int mm = tr ? n : m, nn = tr ? m : n;
  tjm::cx<T>* a = ws;
  tjm::cx<T>* u = a + mm * nn;
  tjm::cx<T>* v = u + mm * nn;
  tjm::cx<T>* vw = v + nn * nn;
  T* s = reinterpret_cast<T*>(vw + nn * nn + 2 * nn);
  // every workspace entry the factorization reads is written here or inside
  // blk_svd_jacobi first, so nothing has to be cleared between calls
  for (int e = threadIdx.x; e < mm * nn; e += TJM_THREADS) {
    const int i = e % mm, j = e / mm;
    a[e] = tr ? tjm::cvt<T>(tjm::conj(A[j * n + i])) : tjm::cvt<T>(A[i * n + j]);
  }
  __syncthreads();
  tjm::blk_svd_jacobi<T>(mm, nn, a, u, s, v, vw, reinterpret_cast<T*>(vw + nn * nn), iw, red, true);
  __syncthreads();
  for (int e = threadIdx.x; e < m * nn; e += TJM_THREADS) {
    const int i = e / nn, j = e % nn;
    U[e] = tjm::cvt<double>(tr ? v[j * nn + i] : u[j * mm + i]);
  }
  for (int e = threadIdx.x; e < n * nn; e += TJM_THREADS) {
    const int i = e / nn, j = e % nn;
    V[e] = tjm::cvt<double>(tr ? u[j * mm + i] : v[j * nn + i]);
  }
  for (int e = threadIdx.x; e < nn; e += TJM_THREADS) S[e] = (double)s[e];
}

}  // namespace

extern "C" tjm_status tjm_svd_noalloc(int double_precision, int m, int n, const double* A, double* U, double* S,
                                      double* V, void* stream) {
  if (m < 1 || n < 1 || !A || !U || !S || !V) return TJM_EINVAL;
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
  if (double_precision)
    svd_noalloc_kernel<double><<<1, TJM_THREADS, 0, st>>>(m, n, dA, dU, S, dV,
                                                           reinterpret_cast<tjm::cx<double>*>(scratch), iw);
  else
    svd_noalloc_kernel<float><<<1, TJM_THREADS, 0, st>>>(m, n, dA, dU, S, dV,
                                                          reinterpret_cast<tjm::cx<float>*>(scratch), iw);
  return cudaGetLastError() == cudaSuccess ? TJM_OK : TJM_ECUDA;
}

// Kernel-level entry points for testing the CTA building blocks in isolation:
// Householder QR, one-sided Jacobi SVD, the Lanczos tridiagonal exponential
// and the Philox stream.  Each runs one CTA on one small problem.
#include <cuda_runtime.h>

#include <vector>

#include "tjm.h"
#include "tjm_linalg.cuh"

namespace tjm {

template <class T>
__global__ void __launch_bounds__(TJM_THREADS, 1)
qr_test_kernel(int m, int n, const cx<double>* A, cx<double>* Q, cx<double>* R, cx<T>* ws) {
  __shared__ double red[TJM_WARPS * 64];
  const int k = m < n ? m : n;
  cx<T>* a = ws;
  cx<T>* q = a + m * n;
  cx<T>* r = q + m * k;
  cx<T>* rd = r + k * n;
  T* tau = reinterpret_cast<T*>(rd + k);
  for (int e = threadIdx.x; e < m * n; e += TJM_THREADS) {
    const int i = e % m, j = e / m;          // column-major work, row-major input
    a[e] = cvt<T>(A[i * n + j]);
  }
  __syncthreads();
  blk_qr<T>(m, n, a, q, r, rd, tau, red);
  __syncthreads();
  for (int e = threadIdx.x; e < m * k; e += TJM_THREADS) {
    const int i = e / k, j = e % k;
    Q[e] = cvt<double>(q[j * m + i]);
  }
  for (int e = threadIdx.x; e < k * n; e += TJM_THREADS) {
    const int i = e / n, j = e % n;
    R[e] = cvt<double>(r[j * k + i]);
  }
}

template <class T>
__global__ void __launch_bounds__(TJM_THREADS, 1)
svd_test_kernel(int m, int n, const cx<double>* A, cx<double>* U, double* S, cx<double>* V, cx<T>* ws, int* iw) {
  __shared__ double red[TJM_WARPS * 64];
  const bool tr = m < n;
  const int mm = tr ? n : m, nn = tr ? m : n;
  cx<T>* a = ws;
  cx<T>* u = a + mm * nn;
  cx<T>* v = u + mm * nn;
  cx<T>* vw = v + nn * nn;
  T* s = reinterpret_cast<T*>(vw + nn * nn + 2 * nn);
  for (int e = threadIdx.x; e < mm * nn; e += TJM_THREADS) {
    const int i = e % mm, j = e / mm;
    a[e] = tr ? cvt<T>(conj(A[j * n + i])) : cvt<T>(A[i * n + j]);
  }
  __syncthreads();
  blk_svd_jacobi<T>(mm, nn, a, u, s, v, vw, reinterpret_cast<T*>(vw + nn * nn), iw, red, true);
  __syncthreads();
  // A = Uw S Vw^H (or its adjoint): return U (m x nn), V (n x nn) row-major
  for (int e = threadIdx.x; e < m * nn; e += TJM_THREADS) {
    const int i = e / nn, j = e % nn;
    U[e] = cvt<double>(tr ? v[j * nn + i] : u[j * mm + i]);
  }
  for (int e = threadIdx.x; e < n * nn; e += TJM_THREADS) {
    const int i = e / nn, j = e % nn;
    V[e] = cvt<double>(tr ? u[j * mm + i] : v[j * nn + i]);
  }
  for (int e = threadIdx.x; e < nn; e += TJM_THREADS) S[e] = (double)s[e];
}

__global__ void expm_test_kernel(int k, const double* alpha, const double* beta, double theta, cx<double>* c) {
  if (threadIdx.x < 32) warp_expm_tridiag(k, alpha, beta, theta, c);
}

__global__ void philox_test_kernel(int n, unsigned long long seed, const unsigned long long* traj,
                                   const unsigned* step, const unsigned* branch, double* u1, double* u2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tjm_uniforms(seed, traj[i], step[i], branch[i], u1 + i, u2 + i);
}

}  // namespace tjm

namespace {

struct Dev {
  std::vector<void*> ptrs;
  ~Dev() { for (void* p : ptrs) cudaFree(p); }
  template <class T> T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return reinterpret_cast<T*>(p);
  }
};

tjm_status finish() {
  const cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? TJM_OK : TJM_ECUDA;
}

}  // namespace

extern "C" {

tjm_status tjm_selftest_qr(int double_precision, int m, int n, const double* A, double* Q, double* R) {
  if (m < 1 || n < 1 || m > 256 || n > 256 || !A || !Q || !R) return TJM_EINVAL;
  const int k = m < n ? m : n;
  Dev d;
  auto* dA = d.get<tjm::cx<double>>(m * n);
  auto* dQ = d.get<tjm::cx<double>>(m * k);
  auto* dR = d.get<tjm::cx<double>>(k * n);
  char* ws = d.get<char>((size_t)(m * n + m * k + k * n + 2 * k + 8) * 16);
  if (!dA || !dQ || !dR || !ws) return TJM_ENOMEM;
  if (cudaMemcpy(dA, A, (size_t)m * n * 16, cudaMemcpyHostToDevice) != cudaSuccess) return TJM_ECUDA;
  if (double_precision)
    tjm::qr_test_kernel<double><<<1, TJM_THREADS>>>(m, n, dA, dQ, dR, reinterpret_cast<tjm::cx<double>*>(ws));
  else
    tjm::qr_test_kernel<float><<<1, TJM_THREADS>>>(m, n, dA, dQ, dR, reinterpret_cast<tjm::cx<float>*>(ws));
  if (finish()) return TJM_ECUDA;
  cudaMemcpy(Q, dQ, (size_t)m * k * 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(R, dR, (size_t)k * n * 16, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

tjm_status tjm_selftest_svd(int double_precision, int m, int n, const double* A, double* U, double* S, double* V) {
  if (m < 1 || n < 1 || m > 256 || n > 256 || !A || !U || !S || !V) return TJM_EINVAL;
  const int mm = m > n ? m : n, nn = m < n ? m : n;
  Dev d;
  auto* dA = d.get<tjm::cx<double>>(m * n);
  auto* dU = d.get<tjm::cx<double>>(m * nn);
  auto* dV = d.get<tjm::cx<double>>(n * nn);
  auto* dS = d.get<double>(nn);
  char* ws = d.get<char>((size_t)(2 * mm * nn + 2 * nn * nn + 4 * nn + 8) * 16);
  int* iw = d.get<int>(2 * nn);
  if (!dA || !dU || !dV || !dS || !ws || !iw) return TJM_ENOMEM;
  if (cudaMemcpy(dA, A, (size_t)m * n * 16, cudaMemcpyHostToDevice) != cudaSuccess) return TJM_ECUDA;
  if (double_precision)
    tjm::svd_test_kernel<double><<<1, TJM_THREADS>>>(m, n, dA, dU, dS, dV, reinterpret_cast<tjm::cx<double>*>(ws), iw);
  else
    tjm::svd_test_kernel<float><<<1, TJM_THREADS>>>(m, n, dA, dU, dS, dV, reinterpret_cast<tjm::cx<float>*>(ws), iw);
  if (finish()) return TJM_ECUDA;
  cudaMemcpy(U, dU, (size_t)m * nn * 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(V, dV, (size_t)n * nn * 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(S, dS, (size_t)nn * 8, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

tjm_status tjm_selftest_expm_tridiag(int k, const double* alpha, const double* beta, double theta, double* c) {
  if (k < 1 || k > 32 || !alpha || !c || (k > 1 && !beta)) return TJM_EINVAL;
  Dev d;
  double* da = d.get<double>(32);
  double* db = d.get<double>(32);
  auto* dc = d.get<tjm::cx<double>>(32);
  if (!da || !db || !dc) return TJM_ENOMEM;
  cudaMemcpy(da, alpha, k * 8, cudaMemcpyHostToDevice);
  if (k > 1) cudaMemcpy(db, beta, (k - 1) * 8, cudaMemcpyHostToDevice);
  tjm::expm_test_kernel<<<1, 32>>>(k, da, db, theta, dc);
  if (finish()) return TJM_ECUDA;
  cudaMemcpy(c, dc, (size_t)k * 16, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

tjm_status tjm_selftest_philox(uint64_t seed, const uint64_t* traj, const uint32_t* step, const uint32_t* branch, int n,
                               double* u1, double* u2) {
  if (n < 1 || !traj || !step || !branch || !u1 || !u2) return TJM_EINVAL;
  Dev d;
  auto* dt = d.get<unsigned long long>(n);
  auto* ds = d.get<unsigned>(n);
  auto* db = d.get<unsigned>(n);
  double* d1 = d.get<double>(n);
  double* d2 = d.get<double>(n);
  if (!dt || !ds || !db || !d1 || !d2) return TJM_ENOMEM;
  cudaMemcpy(dt, traj, (size_t)n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(ds, step, (size_t)n * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(db, branch, (size_t)n * 4, cudaMemcpyHostToDevice);
  tjm::philox_test_kernel<<<(n + 127) / 128, 128>>>(n, seed, dt, ds, db, d1, d2);
  if (finish()) return TJM_ECUDA;
  cudaMemcpy(u1, d1, (size_t)n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(u2, d2, (size_t)n * 8, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

}  // extern "C"

// Kernel-level entry points for testing the CTA building blocks in isolation:
// Householder QR, one-sided Jacobi SVD, the Lanczos tridiagonal exponential
// and the Philox stream.  Each runs one CTA on one small problem.
#include <cuda_runtime.h>

#include <vector>

#include "tjm.h"
#include "tjm_linalg.cuh"
#include "tjm_svd_call.cuh"
#include "tjm_tc.cuh"

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
  svd_call_body<T>(m, n, A, U, S, V, ws, iw, red);
}

// C = op(A) op(B) on the tensor cores, one CTA.  A is given row-major M x K,
// B row-major K x N (complex double, converted to float); a_cm / b_kc store
// them column-major (A's i index contiguous) / K-contiguous first, so both
// operand access patterns of the GEMM are exercised.
__global__ void __launch_bounds__(TJM_THREADS, 1)
tc_cgemm_test_kernel(int M, int N, int K, int ca, int cb, int a_cm, int b_kc, const cx<double>* A,
                     const cx<double>* B, cx<double>* C, cx<float>* fa, cx<float>* fb, cx<float>* fc, int* ok) {
  extern __shared__ __align__(1024) char dsm[];
  __shared__ tc::Ctl ctl;
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  for (int e = threadIdx.x; e < M * K; e += TJM_THREADS) {
    const int i = e / K, k = e % K;
    fa[a_cm ? k * M + i : e] = cvt<float>(A[e]);
  }
  for (int e = threadIdx.x; e < K * N; e += TJM_THREADS) {
    const int k = e / N, j = e % N;
    fb[b_kc ? j * K + k : e] = cvt<float>(B[e]);
  }
  __syncthreads();
  tc::cta_setup(&ctl, 1);
  tc::TcA ta = {};
  ta.p = fa; ta.si = a_cm ? 1 : K; ta.sk = a_cm ? M : 1; ta.conj = ca;
  tc::TcB tb = {};
  tb.p = fb; tb.sk = b_kc ? 1 : N; tb.sj = b_kc ? K : 1; tb.conj = cb;
  const bool good = tc::cgemm(&ctl, M, N, K, mk(1.f, 0.f), ta, tb, fc, N, 1, false, smem);
  tc::cta_teardown(&ctl);
  for (int e = threadIdx.x; e < M * N; e += TJM_THREADS) C[e] = cvt<double>(fc[e]);
  if (threadIdx.x == 0) *ok = good ? 1 : 0;
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
  if (double_precision == 2)
    tjm::qr_test_kernel<tjm::df64><<<1, TJM_THREADS>>>(m, n, dA, dQ, dR, reinterpret_cast<tjm::cx<tjm::df64>*>(ws));
  else if (double_precision)
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
  char* ws = d.get<char>(tjm::svd_call_slots(mm, nn) * 16);
  int* iw = d.get<int>(2 * nn);
  if (!dA || !dU || !dV || !dS || !ws || !iw) return TJM_ENOMEM;
  if (cudaMemcpy(dA, A, (size_t)m * n * 16, cudaMemcpyHostToDevice) != cudaSuccess) return TJM_ECUDA;
  if (double_precision == 2)
    tjm::svd_test_kernel<tjm::df64><<<1, TJM_THREADS>>>(m, n, dA, dU, dS, dV,
                                                        reinterpret_cast<tjm::cx<tjm::df64>*>(ws), iw);
  else if (double_precision)
    tjm::svd_test_kernel<double><<<1, TJM_THREADS>>>(m, n, dA, dU, dS, dV, reinterpret_cast<tjm::cx<double>*>(ws), iw);
  else
    tjm::svd_test_kernel<float><<<1, TJM_THREADS>>>(m, n, dA, dU, dS, dV, reinterpret_cast<tjm::cx<float>*>(ws), iw);
  if (finish()) return TJM_ECUDA;
  cudaMemcpy(U, dU, (size_t)m * nn * 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(V, dV, (size_t)n * nn * 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(S, dS, (size_t)nn * 8, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

tjm_status tjm_selftest_tc_cgemm(int M, int N, int K, int conj_a, int conj_b, int a_col_major, int b_k_contig,
                                 const double* A, const double* B, double* C) {
  if (M < 1 || N < 1 || K < 1 || M > 1024 || N > 1024 || K > 1024 || !A || !B || !C) return TJM_EINVAL;
  Dev d;
  auto* dA = d.get<tjm::cx<double>>((size_t)M * K);
  auto* dB = d.get<tjm::cx<double>>((size_t)K * N);
  auto* dC = d.get<tjm::cx<double>>((size_t)M * N);
  auto* fa = d.get<tjm::cx<float>>((size_t)M * K);
  auto* fb = d.get<tjm::cx<float>>((size_t)K * N);
  auto* fc = d.get<tjm::cx<float>>((size_t)M * N);
  int* ok = d.get<int>(1);
  if (!dA || !dB || !dC || !fa || !fb || !fc || !ok) return TJM_ENOMEM;
  if (cudaMemcpy(dA, A, (size_t)M * K * 16, cudaMemcpyHostToDevice) != cudaSuccess) return TJM_ECUDA;
  if (cudaMemcpy(dB, B, (size_t)K * N * 16, cudaMemcpyHostToDevice) != cudaSuccess) return TJM_ECUDA;
  const int smem = tjm::tc::kSmemBytes + 1024;
  if (cudaFuncSetAttribute(tjm::tc_cgemm_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return TJM_ECUDA;
  tjm::tc_cgemm_test_kernel<<<1, TJM_THREADS, smem>>>(M, N, K, conj_a, conj_b, a_col_major, b_k_contig, dA, dB, dC,
                                                     fa, fb, fc, ok);
  if (finish()) return TJM_ECUDA;
  int h = 0;
  cudaMemcpy(&h, ok, sizeof h, cudaMemcpyDeviceToHost);
  cudaMemcpy(C, dC, (size_t)M * N * 16, cudaMemcpyDeviceToHost);
  return h ? TJM_OK : TJM_ETIMEOUT;
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

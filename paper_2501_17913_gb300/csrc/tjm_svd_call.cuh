// One standalone SVD call on one CTA: the body shared by the allocating self
// test (tjm_selftest_svd) and the allocation-free entry point
// (tjm_svd_noalloc), with the workspace layout both size from one function.
#pragma once
#include <stddef.h>

#include "tjm_linalg.cuh"

namespace tjm {

// Workspace of one call in complex elements of the factorization precision,
// for a work matrix of mm x nn (mm >= nn): the work matrix, U (mm x nn),
// V (nn x nn), the rotation accumulator (nn x nn) followed by 2 nn slots of
// unsorted singular values, the sorted singular values (nn reals), and 8
// slots of slack.
__host__ __device__ constexpr size_t svd_call_slots(int mm, int nn) {
  return (size_t)2 * mm * nn + (size_t)2 * nn * nn + (size_t)4 * nn + 8;
}

// A is m x n, row-major complex double; U (m x nn), V (n x nn) row-major, S
// (nn) descending, A = U diag(S) V^H, nn = min(m, n).  ws holds
// svd_call_slots(max(m, n), nn) complex T; iw holds 2 nn ints.  Every
// workspace entry read is written first, here or inside blk_svd_jacobi.
template <class T>
__device__ void svd_call_body(int m, int n, const cx<double>* A, cx<double>* U, double* S, cx<double>* V, cx<T>* ws,
                              int* iw, double* red) {
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
  // the work matrix was A or A^H: return U (m x nn) and V (n x nn) of A
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

}  // namespace tjm

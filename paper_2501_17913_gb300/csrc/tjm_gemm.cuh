// CTA-wide complex GEMM on CUDA cores with arbitrary operand strides.
//
//   C(i, j) = alpha * sum_k A(i, k) B(k, j)  [+ C(i, j) if accumulate]
//
// A(i, k) = a.p[i * a.si + k * a.sk] (conjugated if a.conj), B likewise, so
// every contraction of the effective-Hamiltonian networks is one call with no
// explicit transposes.  64 x 64 output tiles, 16-deep K slices staged in shared
// memory with a register prefetch of the next slice; each thread owns a 4 x 4
// block of complex accumulators in the working precision.
#pragma once
#include "tjm_common.cuh"

namespace tjm {

template <class T> struct MatA { const cx<T>* p; long long si, sk; int conj; };
template <class T> struct MatB { const cx<T>* p; long long sk, sj; int conj; };

template <class T> __host__ __device__ inline MatA<T> matA(const cx<T>* p, long long si, long long sk, int cj = 0) {
  MatA<T> m; m.p = p; m.si = si; m.sk = sk; m.conj = cj; return m;
}
template <class T> __host__ __device__ inline MatB<T> matB(const cx<T>* p, long long sk, long long sj, int cj = 0) {
  MatB<T> m; m.p = p; m.sk = sk; m.sj = sj; m.conj = cj; return m;
}

constexpr int GB_M = 64, GB_N = 64, GB_K = 16;
template <class T> constexpr int gemm_smem_bytes() { return 2 * GB_K * GB_M * (int)sizeof(cx<T>); }

// Batched: for b < batch, operands offset by (sa, sb, sc) elements.
template <class T>
__device__ __noinline__ void blk_gemm_batched(int batch, int M, int N, int K, cx<T> alpha, MatA<T> A, long long sa, MatB<T> B,
                                 long long sb, cx<T>* C, long long sci, long long scj, long long sc, bool accumulate,
                                 char* smem) {
  cx<T>* As = reinterpret_cast<cx<T>*>(smem);          // [GB_K][GB_M]
  cx<T>* Bs = As + GB_K * GB_M;                          // [GB_K][GB_N]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tm = (M + GB_M - 1) / GB_M, tn = (N + GB_N - 1) / GB_N;
  const int ntile = batch * tm * tn;
  const int nk = (K + GB_K - 1) / GB_K;
  const bool a_kfast = (A.sk == 1);
  const bool b_jfast = (B.sj == 1) || (B.sk != 1);
  if (M <= 0 || N <= 0) return;
  for (int t = 0; t < ntile; ++t) {
    const int b = t / (tm * tn), r0 = t % (tm * tn);
    const int i0 = (r0 / tn) * GB_M, j0 = (r0 % tn) * GB_N;
    const cx<T>* Ap = A.p + b * sa;
    const cx<T>* Bp = B.p + b * sb;
    cx<T> acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = czero<T>();
    cx<T> ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + TJM_THREADS * q;
        int ii, kk;
        if (a_kfast) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
        const int i = i0 + ii, k = k0 + kk;
        cx<T> v = czero<T>();
        if (i < M && k < K) { v = Ap[i * A.si + k * A.sk]; if (A.conj) v.y = -v.y; }
        ra[q] = v;
        int jj, kb;
        if (b_jfast) { jj = e & 63; kb = e >> 6; } else { kb = e & 15; jj = e >> 4; }
        const int j = j0 + jj, kq = k0 + kb;
        cx<T> u = czero<T>();
        if (j < N && kq < K) { u = Bp[kq * B.sk + j * B.sj]; if (B.conj) u.y = -u.y; }
        rb[q] = u;
      }
    };
    auto store = [&]() {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + TJM_THREADS * q;
        int ii, kk;
        if (a_kfast) { kk = e & 15; ii = e >> 4; } else { ii = e & 63; kk = e >> 6; }
        As[kk * GB_M + ii] = ra[q];
        int jj, kb;
        if (b_jfast) { jj = e & 63; kb = e >> 6; } else { kb = e & 15; jj = e >> 4; }
        Bs[kb * GB_N + jj] = rb[q];
      }
    };
    load(0);
    for (int ks = 0; ks < nk; ++ks) {
      __syncthreads();
      store();
      __syncthreads();
      if (ks + 1 < nk) load((ks + 1) * GB_K);
#pragma unroll 4
      for (int kk = 0; kk < GB_K; ++kk) {
        cx<T> a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk * GB_M + ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[kk * GB_N + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], bb[c]);
      }
    }
    cx<T>* Cp = C + b * sc;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + ty + 16 * r;
      if (i >= M) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + tx + 16 * c;
        if (j >= N) continue;
        cx<T> v = alpha * acc[r][c];
        cx<T>* dst = Cp + i * sci + j * scj;
        if (accumulate) v = v + *dst;
        *dst = v;
      }
    }
  }
  __syncthreads();
}

template <class T>
__device__ __forceinline__ void blk_gemm(int M, int N, int K, MatA<T> A, MatB<T> B, cx<T>* C, long long sci,
                                         long long scj, char* smem, cx<T> alpha = mk((T)1, (T)0),
                                         bool accumulate = false) {
  blk_gemm_batched<T>(1, M, N, K, alpha, A, 0, B, 0, C, sci, scj, 0, accumulate, smem);
}

// out[p][o][q] = sum_i Wm[o][i] in[p][i][q] -- the small MPO contraction
// between the two big GEMMs of an effective-Hamiltonian application.
// Wm (O x I, complex double, row-major) is staged in shared memory in the
// working precision; zero entries of the MPO are skipped.
template <class T>
__device__ __noinline__ void blk_wapply(int P, int O, int I, int Q, const cx<double>* Wm, const cx<T>* in, long long sip,
                           long long sii, cx<T>* out, long long sop, long long soo, char* smem) {
  cx<T>* Ws = reinterpret_cast<cx<T>*>(smem);
  __syncthreads();
  for (int e = threadIdx.x; e < O * I; e += TJM_THREADS) Ws[e] = cvt<T>(Wm[e]);
  __syncthreads();
  const long long tot = (long long)P * Q;
  for (long long e = threadIdx.x; e < tot; e += TJM_THREADS) {
    const int p = (int)(e / Q), q = (int)(e % Q);
    const cx<T>* src = in + p * sip + q;
    cx<T>* dst = out + p * sop + q;
    for (int o = 0; o < O; ++o) {
      cx<T> acc = czero<T>();
      const cx<T>* wr = Ws + o * I;
      for (int i = 0; i < I; ++i) {
        const cx<T> w = wr[i];
        if (w.x != (T)0 || w.y != (T)0) cfma(acc, w, src[i * sii]);
      }
      dst[o * soo] = acc;
    }
  }
  __syncthreads();
}

}  // namespace tjm

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
#include "tjm_tc.cuh"

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
// bytes of shared memory reserved for GEMM staging (two 16-deep tiles of 64 complex doubles)
constexpr int kSmemGemm = 32768;
template <class T> constexpr int gemm_smem_bytes() { return 2 * GB_K * GB_M * (int)sizeof(cx<T>); }

// A operand formed on the fly from an MPO block in row-sparse form (see
// blk_wgemm): A(i, k) = sum_z val[z] t1[x * sip + col[z] * chr + b] over the
// entries z of MPO row o = t * Dr + v, with i = x * dd + t and k = v * chr + b.
template <class T> struct WaArgs {
  const cx<T>* val; const int* col; const int* rp;
  const cx<T>* t1; int sip, dd, Dr, chr;
};

// One layout variant: AK = A's k index is contiguous (else its i index),
// BJ = B's j index is contiguous (else its k index); TM x TM output tiles
// (TM = 64 or 32), each thread owning (TM/16) x (TM/16) complex accumulators.
// Each thread loads TM/16 elements of A and of B per 16-deep slice; their tile
// coordinates are fixed per thread, so the loads need no per-element index
// arithmetic.
template <class T, bool AK, bool BJ, int TM, bool WA = false>
__device__ __noinline__ void gemm_core(int batch, int M, int N, int K, cx<T> alpha, const cx<T>* __restrict__ A,
                                       int sai, int sak, int ca, long long sa, const cx<T>* __restrict__ B, int sbk,
                                       int sbj, int cb, long long sb, cx<T>* C, int sci, int scj, long long sc,
                                       bool accumulate, char* smem, WaArgs<T> wa = WaArgs<T>{}) {
  constexpr int NQ = TM / 16;              // loads and accumulator rows / columns per thread
  constexpr int KS = TJM_THREADS / TM;     // k rows covered per load round in the i- / j-contiguous layouts
  cx<T>* As = reinterpret_cast<cx<T>*>(smem);          // [GB_K][TM]
  cx<T>* Bs = As + GB_K * TM;                            // [GB_K][TM]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a_i = AK ? (tid >> 4) : (tid % TM);          // + 16 q   (AK)
  const int a_k = AK ? (tid & 15) : (tid / TM);          // + KS q   (!AK)
  const int b_j = BJ ? (tid % TM) : (tid >> 4);          // + 16 q   (!BJ)
  const int b_k = BJ ? (tid / TM) : (tid & 15);          // + KS q   (BJ)
  const int tm = (M + TM - 1) / TM, tn = (N + TM - 1) / TM;
  const int ntile = batch * tm * tn;
  const int nk = (K + GB_K - 1) / GB_K;
  const T sga = ca ? (T)-1 : (T)1, sgb = cb ? (T)-1 : (T)1;
  for (int t = 0; t < ntile; ++t) {
    const int bt = t / (tm * tn), r0 = t % (tm * tn);
    const int i0 = (r0 / tn) * TM, j0 = (r0 % tn) * TM;
    const cx<T>* Ap = A + bt * sa;
    const cx<T>* Bp = B + bt * sb;
    cx<T> acc[NQ][NQ];
#pragma unroll
    for (int r = 0; r < NQ; ++r)
#pragma unroll
      for (int c = 0; c < NQ; ++c) acc[r][c] = czero<T>();
    cx<T> ra[NQ], rb[NQ];
    auto load = [&](int k0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i = i0 + a_i + (AK ? 16 * q : 0), k = k0 + a_k + (AK ? 0 : KS * q);
        cx<T> v = czero<T>();
        if constexpr (WA) {
          if (i < M && k < K) {
            const int x = i / wa.dd, t = i - x * wa.dd;
            const int vv = k / wa.chr, b = k - vv * wa.chr;
            const int o = t * wa.Dr + vv;
            const cx<T>* src = wa.t1 + (long long)x * wa.sip + b;
            const int z1 = wa.rp[o + 1];
            for (int z = wa.rp[o]; z < z1; ++z) cfma(v, wa.val[z], src[wa.col[z] * wa.chr]);
          }
        } else {
          if (i < M && k < K) v = Ap[i * sai + k * sak];
          v.y *= sga;
        }
        ra[q] = v;
        const int j = j0 + b_j + (BJ ? 0 : 16 * q), kb = k0 + b_k + (BJ ? KS * q : 0);
        cx<T> u = czero<T>();
        if (j < N && kb < K) u = Bp[kb * sbk + j * sbj];
        u.y *= sgb;
        rb[q] = u;
      }
    };
    load(0);
    for (int ks = 0; ks < nk; ++ks) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        As[(a_k + (AK ? 0 : KS * q)) * TM + a_i + (AK ? 16 * q : 0)] = ra[q];
        Bs[(b_k + (BJ ? KS * q : 0)) * TM + b_j + (BJ ? 0 : 16 * q)] = rb[q];
      }
      __syncthreads();
      if (ks + 1 < nk) load((ks + 1) * GB_K);
#pragma unroll 4
      for (int kk = 0; kk < GB_K; ++kk) {
        cx<T> av[NQ], bv[NQ];
#pragma unroll
        for (int r = 0; r < NQ; ++r) av[r] = As[kk * TM + ty + 16 * r];
#pragma unroll
        for (int c = 0; c < NQ; ++c) bv[c] = Bs[kk * TM + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < NQ; ++r)
#pragma unroll
          for (int c = 0; c < NQ; ++c) cfma(acc[r][c], av[r], bv[c]);
      }
    }
    cx<T>* Cp = C + bt * sc;
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
      const int i = i0 + ty + 16 * r;
      if (i >= M) continue;
#pragma unroll
      for (int c = 0; c < NQ; ++c) {
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

// Tile choice.  gemm_tile_rule == 0: always 64 x 64 tiles.  == 1: 32 x 32
// tiles when either output dimension is at most 32 (small bonds, chain ends),
// where a 64 x 64 tile would leave most of its threads without an output.
// The rule is a per-launch setting (see the kernel), picked by the host-side
// autotuner from timed launches.
__shared__ int gemm_tile_rule;

// Tensor-core state of the CTA (tjm_tc.cuh).  When enabled, every FP32 GEMM of
// at least tc_ctl.min_work complex multiply-adds runs on the tensor cores;
// smaller ones (chain ends, tiny bonds) stay on the CUDA cores, where one
// 128-row MMA tile would be mostly padding.
__shared__ tc::Ctl tc_ctl;

// TJM_TENSOR_CORES (per translation unit) decides whether the kernels built
// there carry the tcgen05 path at all.  A kernel image that holds any tcgen05
// instruction is granted a single resident CTA per SM (measured on GB300 with
// the occupancy API: the same 128-register, 256-thread trajectory kernel
// reports two without them), so the CUDA-core instantiations are compiled
// without it and the tensor-core ones live in translation units of their own.
#ifndef TJM_TENSOR_CORES
#define TJM_TENSOR_CORES 0
#endif

__device__ __forceinline__ bool use_tc(long long work) {
#if TJM_TENSOR_CORES
  return tc_ctl.enabled && work >= tc_ctl.min_work;
#else
  (void)work;
  return false;
#endif
}

template <class T, bool AK, bool BJ>
__device__ __forceinline__ void gemm_layout(int batch, int M, int N, int K, cx<T> alpha, const cx<T>* A, int sai,
                                            int sak, int ca, long long sa, const cx<T>* B, int sbk, int sbj, int cb,
                                            long long sb, cx<T>* C, int sci, int scj, long long sc, bool accumulate,
                                            char* smem) {
  if (gemm_tile_rule == 1 && (M <= 32 || N <= 32))
    gemm_core<T, AK, BJ, 32>(batch, M, N, K, alpha, A, sai, sak, ca, sa, B, sbk, sbj, cb, sb, C, sci, scj, sc,
                             accumulate, smem);
  else
    gemm_core<T, AK, BJ, 64>(batch, M, N, K, alpha, A, sai, sak, ca, sa, B, sbk, sbj, cb, sb, C, sci, scj, sc,
                             accumulate, smem);
}

// Batched: for b < batch, operands offset by (sa, sb, sc) elements.
template <class T>
__device__ __forceinline__ void blk_gemm_batched(int batch, int M, int N, int K, cx<T> alpha, MatA<T> A,
                                                 long long sa, MatB<T> B, long long sb, cx<T>* C, long long sci,
                                                 long long scj, long long sc, bool accumulate, char* smem) {
  if (M <= 0 || N <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (K > 0 && use_tc((long long)M * N * K)) {
      tc::TcA ta = {};
      ta.si = A.si; ta.sk = A.sk; ta.conj = A.conj;
      tc::TcB tb = {};
      tb.sk = B.sk; tb.sj = B.sj; tb.conj = B.conj;
      for (int b = 0; b < batch; ++b) {
        ta.p = A.p + b * sa;
        tb.p = B.p + b * sb;
        tc::cgemm(&tc_ctl, M, N, K, alpha, ta, tb, C + b * sc, sci, scj, accumulate, smem);
      }
      return;
    }
  }
  const bool ak = A.sk == 1;
  const bool bj = (B.sj == 1) || (B.sk != 1);
  if (ak && bj)
    gemm_layout<T, true, true>(batch, M, N, K, alpha, A.p, (int)A.si, (int)A.sk, A.conj, sa, B.p, (int)B.sk,
                               (int)B.sj, B.conj, sb, C, (int)sci, (int)scj, sc, accumulate, smem);
  else if (ak)
    gemm_layout<T, true, false>(batch, M, N, K, alpha, A.p, (int)A.si, (int)A.sk, A.conj, sa, B.p, (int)B.sk,
                                (int)B.sj, B.conj, sb, C, (int)sci, (int)scj, sc, accumulate, smem);
  else if (bj)
    gemm_layout<T, false, true>(batch, M, N, K, alpha, A.p, (int)A.si, (int)A.sk, A.conj, sa, B.p, (int)B.sk,
                                (int)B.sj, B.conj, sb, C, (int)sci, (int)scj, sc, accumulate, smem);
  else
    gemm_layout<T, false, false>(batch, M, N, K, alpha, A.p, (int)A.si, (int)A.sk, A.conj, sa, B.p, (int)B.sk,
                                 (int)B.sj, B.conj, sb, C, (int)sci, (int)scj, sc, accumulate, smem);
}

template <class T>
__device__ __forceinline__ void blk_gemm(int M, int N, int K, MatA<T> A, MatB<T> B, cx<T>* C, long long sci,
                                         long long scj, char* smem, cx<T> alpha = mk((T)1, (T)0),
                                         bool accumulate = false) {
  blk_gemm_batched<T>(1, M, N, K, alpha, A, 0, B, 0, C, sci, scj, 0, accumulate, smem);
}

// out[p][o][q] = sum_i Wm[o][i] in[p][i][q] -- the small MPO contraction
// between the two big GEMMs of an effective-Hamiltonian application.
// Wm (O x I <= 32 x 32, complex double, row-major) is compressed by warp 0
// into a row-sparse list in shared memory (the MPO is mostly zeros), then
// every thread handles (p, q) pairs reading only the inputs that matter.
//
// A scalar `shift` can be added on nsh diagonal entries (o, i) =
// (so0 + t * so_step, si0 + t * si_step), t < nsh: this is how a constant
// times the identity rides on an MPO's on-site channel.
// Row-sparse form of Wm (+ the shift entries) in shared memory at csr:
// val [O * I], col [O * I], rp [O + 1].  Ends with a barrier.
template <class T>
__device__ __forceinline__ void wcsr_build(int O, int I, const cx<double>* Wm, char* csr, double shift, int nsh,
                                           int so0, int so_step, int si0, int si_step) {
  cx<T>* val = reinterpret_cast<cx<T>*>(csr);
  int* col = reinterpret_cast<int*>(val + O * I);
  int* rp = col + O * I;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int o = threadIdx.x;
    int ish = -1;                       // column of this row's shift entry, if any
    if (shift != 0.0 && o >= so0 && (o - so0) % so_step == 0 && (o - so0) / so_step < nsh)
      ish = si0 + ((o - so0) / so_step) * si_step;
    int cnt = 0;
    if (o < O)
      for (int i = 0; i < I; ++i) {
        cx<double> w = Wm[o * I + i];
        if (i == ish) w.x += shift;
        cnt += (w.x != 0.0 || w.y != 0.0);
      }
    int incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (o >= d) incl += v;
    }
    const int start = incl - cnt;
    if (o < O) {
      rp[o] = start;
      if (o == O - 1) rp[O] = incl;
      int pos = start;
      for (int i = 0; i < I; ++i) {
        cx<double> w = Wm[o * I + i];
        if (i == ish) w.x += shift;
        if (w.x != 0.0 || w.y != 0.0) { val[pos] = cvt<T>(w); col[pos] = i; ++pos; }
      }
    }
  }
  __syncthreads();
}

template <class T>
__device__ __noinline__ void blk_wapply(int P, int O, int I, int Q, const cx<double>* Wm, const cx<T>* __restrict__ in,
                                        long long sip, long long sii, cx<T>* __restrict__ out, long long sop, long long soo,
                                        char* smem, double shift = 0.0, int nsh = 0, int so0 = 0, int so_step = 1,
                                        int si0 = 0, int si_step = 1) {
  const cx<T>* val = reinterpret_cast<const cx<T>*>(smem);
  const int* col = reinterpret_cast<const int*>(val + O * I);
  const int* rp = col + O * I;
  wcsr_build<T>(O, I, Wm, smem, shift, nsh, so0, so_step, si0, si_step);
  const long long tot = (long long)P * Q;
  for (long long e = threadIdx.x; e < tot; e += TJM_THREADS) {
    const int p = (int)(e / Q), q = (int)(e % Q);
    const cx<T>* src = in + p * sip + q;
    cx<T>* dst = out + p * sop + q;
    for (int o = 0; o < O; ++o) {
      cx<T> acc = czero<T>();
      const int e1 = rp[o + 1];
      for (int z = rp[o]; z < e1; ++z) cfma(acc, val[z], src[col[z] * sii]);
      dst[o * soo] = acc;
    }
  }
  __syncthreads();
}

// y[(x t)][j] = sum_(v b) [sum_(w s) Wm[(t v)][(w s)] t1[x][(w s)][b]] R[(v b)][j]
// for x < P, t < dd, j < chr: the MPO contraction and the second GEMM of an
// effective-Hamiltonian application in one pass.  The MPO block is applied
// while G3's A tile is loaded, so the (P dd) x (Dr chr) intermediate is never
// written.  FP32 only: the row-sparse MPO sits in shared memory above the
// GEMM staging tiles (16 KB of the 32 KB GEMM area).
template <class T>
__device__ __noinline__ void blk_wgemm(int P, int dd, int Dr, int I, int chr, const cx<double>* Wm,
                                       const cx<T>* __restrict__ t1, const cx<T>* R, cx<T>* y, char* smem,
                                       char* csr_global, double shift, int nsh, int so0, int so_step, int si0,
                                       int si_step) {
  static_assert(sizeof(T) == 4, "fused MPO GEMM is for FP32 contractions");
  const int O = dd * Dr;
  if (use_tc((long long)P * dd * chr * Dr * chr)) {
    // the tensor cores own the shared staging area: the row-sparse block goes to global scratch (L1-resident)
    wcsr_build<T>(O, I, Wm, csr_global, shift, nsh, so0, so_step, si0, si_step);
    tc::TcA ta = {};
    ta.fused = 1;
    ta.val = reinterpret_cast<const cx<float>*>(csr_global);
    ta.col = reinterpret_cast<const int*>(ta.val + O * I);
    ta.rp = ta.col + O * I;
    ta.t1 = t1; ta.sip = I * chr; ta.dd = dd; ta.Dr = Dr; ta.chr = chr;
    tc::TcB tb = {};
    tb.p = R; tb.sk = chr; tb.sj = 1;
    tc::cgemm(&tc_ctl, P * dd, chr, Dr * chr, mk(1.f, 0.f), ta, tb, y, chr, 1, false, smem);
    return;
  }
  char* csr = smem + 2 * GB_K * 64 * (int)sizeof(cx<T>);
  wcsr_build<T>(O, I, Wm, csr, shift, nsh, so0, so_step, si0, si_step);
  WaArgs<T> wa;
  wa.val = reinterpret_cast<const cx<T>*>(csr);
  wa.col = reinterpret_cast<const int*>(wa.val + O * I);
  wa.rp = wa.col + O * I;
  wa.t1 = t1; wa.sip = I * chr; wa.dd = dd; wa.Dr = Dr; wa.chr = chr;
  const int M = P * dd, N = chr, K = Dr * chr;
  const cx<T> one = mk((T)1, (T)0);
  if (gemm_tile_rule == 1 && (M <= 32 || N <= 32))
    gemm_core<T, true, true, 32, true>(1, M, N, K, one, nullptr, 0, 1, 0, 0, R, chr, 1, 0, 0, y, chr, 1, 0, false,
                                       smem, wa);
  else
    gemm_core<T, true, true, 64, true>(1, M, N, K, one, nullptr, 0, 1, 0, 0, R, chr, 1, 0, 0, y, chr, 1, 0, false,
                                       smem, wa);
}

}  // namespace tjm

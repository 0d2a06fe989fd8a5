// Common device building blocks of the batched tensor-jump-method kernels:
// complex arithmetic, block-wide reductions, the Philox4x32-10 generator and
// plain vector operations.  Every function whose name starts with blk_ is
// called by ALL threads of a CTA (it may contain __syncthreads()).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tjm_df64.cuh"

#ifndef TJM_THREADS
#define TJM_THREADS 256
#endif
#define TJM_WARPS (TJM_THREADS / 32)

namespace tjm {

// ------------------------------------------------------------------ complex
template <class T> struct __align__(2 * sizeof(T)) cx { T x, y; };
typedef cx<float> cf;
typedef cx<double> cd;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <class T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.x, s * a.y); }
template <class T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.x, -a.y); }
template <class T> __host__ __device__ __forceinline__ T norm2(cx<T> a) { return a.x * a.x + a.y * a.y; }
// a += b * c
template <class T> __device__ __forceinline__ void cfma(cx<T>& a, cx<T> b, cx<T> c) {
  a.x = fma(b.x, c.x, a.x); a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y); a.y = fma(b.y, c.x, a.y);
}
// a += conj(b) * c
template <class T> __device__ __forceinline__ void cfma_cj(cx<T>& a, cx<T> b, cx<T> c) {
  a.x = fma(b.x, c.x, a.x); a.x = fma(b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y); a.y = fma(-b.y, c.x, a.y);
}
// double-float complex arithmetic with fused real parts (tjm_df64.cuh: df_dot2, df_fma2)
__host__ __device__ __forceinline__ cx<df64> operator*(cx<df64> a, cx<df64> b) {
  return mk(df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x));
}
__device__ __forceinline__ void cfma(cx<df64>& a, cx<df64> b, cx<df64> c) {
  a.x = df_fma2(a.x, b.x, c.x, -b.y, c.y);
  a.y = df_fma2(a.y, b.x, c.y, b.y, c.x);
}
__device__ __forceinline__ void cfma_cj(cx<df64>& a, cx<df64> b, cx<df64> c) {
  a.x = df_fma2(a.x, b.x, c.x, b.y, c.y);
  a.y = df_fma2(a.y, b.x, c.y, -b.y, c.x);
}
__host__ __device__ __forceinline__ df64 norm2(cx<df64> a) { return df_dot2(a.x, a.x, a.y, a.y); }
// c x + s y for real c, s and complex x, y (a plane rotation's column update)
template <class T> __device__ __forceinline__ cx<T> rot_comb(T c, cx<T> x, T s, cx<T> y) { return c * x + s * y; }
__device__ __forceinline__ cx<df64> rot_comb(df64 c, cx<df64> x, df64 s, cx<df64> y) {
  return mk(df_dot2(c, x.x, s, y.x), df_dot2(c, x.y, s, y.y));
}
template <class To, class Ti> __device__ __forceinline__ cx<To> cvt(cx<Ti> a) { return mk((To)a.x, (To)a.y); }
template <class T> __device__ __forceinline__ cx<T> czero() { return mk((T)0, (T)0); }

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Compensated warp sum of FP32 values: each lane carries (hi, lo) with
// hi + lo exact; partner pairs are added with Knuth's TwoSum (the rounding
// error of hi1 + hi2 recovered exactly) and the low parts summed on top
// (Dekker's double-length addition).  The result is the sum correctly rounded
// up to a few units of 2^-48 -- the accuracy of an FP64 reduction at the cost
// of FP32 instructions, which GB300 issues 64x faster than FP64.
struct f2s { float hi, lo; };
__device__ __forceinline__ f2s df_add(f2s a, f2s b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ void warp_sum_df2(float& v0, float& v1) {
  f2s a = {v0, 0.f}, b = {v1, 0.f};
  for (int o = 16; o > 0; o >>= 1) {
    a = df_add(a, {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
    b = df_add(b, {__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o)});
  }
  v0 = a.hi + a.lo; v1 = b.hi + b.lo;
}
// Accurate warp sums in the factorization precision: FP64 shuffles for
// double, compensated FP32 for float.
__device__ __forceinline__ void warp_sum_acc2(double& v0, double& v1) { v0 = warp_sum(v0); v1 = warp_sum(v1); }
__device__ __forceinline__ void warp_sum_acc2(float& v0, float& v1) { warp_sum_df2(v0, v1); }

// Sums over an aligned group of 8 lanes (mask m = exactly those lanes).
template <class T> __device__ __forceinline__ T grp8_sum(T v, unsigned m) {
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}
__device__ __forceinline__ void grp8_sum_acc2(double& v0, double& v1, unsigned m) {
  v0 = grp8_sum(v0, m);
  v1 = grp8_sum(v1, m);
}
// compensated (see warp_sum_df2) for FP32
__device__ __forceinline__ void grp8_sum_acc2(float& v0, float& v1, unsigned m) {
  f2s a = {v0, 0.f}, b = {v1, 0.f};
  for (int o = 4; o > 0; o >>= 1) {
    a = df_add(a, {__shfl_xor_sync(m, a.hi, o), __shfl_xor_sync(m, a.lo, o)});
    b = df_add(b, {__shfl_xor_sync(m, b.hi, o), __shfl_xor_sync(m, b.lo, o)});
  }
  v0 = a.hi + a.lo; v1 = b.hi + b.lo;
}

// double-float versions: both words are shuffled, partners added with the
// accurate double-word adder
__device__ __forceinline__ df64 grp8_sum(df64 v, unsigned m) {
  for (int o = 4; o > 0; o >>= 1) v = v + shfl_xor_df(m, v, o);
  return v;
}
__device__ __forceinline__ void grp8_sum_acc2(df64& v0, df64& v1, unsigned m) {
  v0 = grp8_sum(v0, m);
  v1 = grp8_sum(v1, m);
}
__device__ __forceinline__ df64 warp_sum(df64 v) {
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor_df(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of one double per thread over the CTA; every thread gets the result.
// red must hold TJM_WARPS doubles of shared memory.
__device__ __forceinline__ double blk_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < TJM_WARPS; ++i) s += red[i];
  return s;
}

// As blk_sum in FP32, for sums of non-negative terms (no cancellation, so FP32
// is accurate to a few ulps and no FP64 instruction is needed).
__device__ __forceinline__ float blk_sumf(float v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* rf = reinterpret_cast<float*>(red);
  __syncthreads();
  if (lane == 0) rf[w] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < TJM_WARPS; ++i) s += rf[i];
  return s;
}
__device__ __forceinline__ double blk_sum_pos(double v, double* red) { return blk_sum(v, red); }
__device__ __forceinline__ float blk_sum_pos(float v, double* red) { return blk_sumf(v, red); }

// Several sums at once: partial[j] for j < n (n <= 64); results land in out[j]
// (shared memory) after the call.  red needs n * TJM_WARPS doubles.
__device__ __forceinline__ void blk_sums_finish(int n, double* red, double* out) {
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += TJM_THREADS) {
    double s = 0.0;
    for (int w = 0; w < TJM_WARPS; ++w) s += red[j * TJM_WARPS + w];
    out[j] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): two 32x32->64-bit multiplies per round, xor with the other counter
// words and the key, Weyl key schedule; ten rounds.
struct u32x4 { uint32_t v[4]; };
__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c.v[0];
    const uint64_t p1 = (uint64_t)M1 * c.v[2];
    u32x4 n;
    n.v[0] = (uint32_t)(p1 >> 32) ^ c.v[1] ^ k0;
    n.v[1] = (uint32_t)p1;
    n.v[2] = (uint32_t)(p0 >> 32) ^ c.v[3] ^ k1;
    n.v[3] = (uint32_t)p0;
    c = n;
  }
  return c;
}
// 53-bit uniform in [0, 1) from two words.
__host__ __device__ inline double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}
// (u1, u2) of one trajectory, one step, one branch (0 = main, 1 = sampling).
__host__ __device__ inline void tjm_uniforms(uint64_t seed, uint64_t traj, uint32_t step, uint32_t branch,
                                             double* u1, double* u2) {
  u32x4 c;
  c.v[0] = (uint32_t)traj; c.v[1] = (uint32_t)(traj >> 32); c.v[2] = step; c.v[3] = branch;
  const u32x4 x = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  *u1 = u53(x.v[0], x.v[1]);
  *u2 = u53(x.v[2], x.v[3]);
}

// ------------------------------------------------------------------ vectors (global memory)
template <class T> __device__ void blk_copy(cx<T>* dst, const cx<T>* src, int n) {
  for (int i = threadIdx.x; i < n; i += TJM_THREADS) dst[i] = src[i];
}
template <class T> __device__ void blk_scale(cx<T>* x, int n, cx<double> s) {
  const cx<T> st = mk((T)s.x, (T)s.y);
  for (int i = threadIdx.x; i < n; i += TJM_THREADS) x[i] = st * x[i];
}
// ||x||^2 with per-thread partial sums in the working precision, combined in FP64.
template <class T> __device__ double blk_nrm2sq(const cx<T>* x, int n, double* red) {
  T acc = 0;
  for (int i = threadIdx.x; i < n; i += TJM_THREADS) { const cx<T> v = x[i]; acc = fma(v.x, v.x, acc); acc = fma(v.y, v.y, acc); }
  return blk_sum((double)acc, red);
}
template <> __device__ inline double blk_nrm2sq<float>(const cf* x, int n, double* red) {
  // Kahan-compensated FP32 partials: the norm feeds the jump decision
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < n; i += TJM_THREADS) {
    const cf v = x[i];
    const float t = fmaf(v.x, v.x, v.y * v.y);
    const float y = t - c;
    const float u = s + y;
    c = (u - s) - y;
    s = u;
  }
  return blk_sum((double)s - (double)c, red);
}

}  // namespace tjm

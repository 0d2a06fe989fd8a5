// CTA-wide complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C(i, j) = alpha * sum_k A(i, k) B(k, j)  [+ C(i, j) if accumulate]
//
// The effective-Hamiltonian and environment contractions of the TDVP sweep
// (paper Fig. 2: L . W . A . R) are complex GEMMs whose operands are FP32.
// They run here as real GEMMs on the tensor pipe:
//   * complex -> real ("4M" in planar form): A and B are staged as separate
//     real and imaginary planes, and the two accumulators of tensor memory
//     receive C_re = A_re B_re - A_im B_im (the second product with the MMA's
//     negate-A bit) and C_im = A_re B_im + A_im B_re;
//   * FP32 accuracy from TF32 inputs ("3xTF32"): x = hi + lo with hi = x
//     rounded to TF32 and lo the FP32 remainder, and A B = Ahi Bhi + Ahi Blo +
//     Alo Bhi up to the dropped Alo Blo (2^-22 relative) -- three MMAs per
//     real product, twelve per k-step, accumulating in FP32 in tensor memory.
// One thread issues tcgen05.mma (kind::tf32, M = 128, N <= 128, K = 8) from
// shared-memory operand tiles in the K-major no-swizzle core-matrix layout;
// the accumulators (128 lanes x 2N FP32 columns) live in tensor memory and
// are read back with tcgen05.ld.  Operand tiles pass through registers on
// their way to shared memory because every element is split (hi / lo) and
// de-interleaved, which a bulk tensor copy cannot do; the global loads of the
// next K chunk are issued before the current one is written, and three
// stages let the loads of one chunk overlap the MMAs of the previous ones,
// ordered by mbarriers that tcgen05.commit arrives on.  Every mbarrier wait
// is bounded: on timeout the CTA records the failure, stops issuing MMAs and
// the caller marks the trajectory failed.
#pragma once
#include <stdint.h>

#include "tjm_common.cuh"

namespace tjm {
namespace tc {

// ------------------------------------------------------------------ geometry
constexpr int kM = 128;                         // MMA rows (TMEM lanes)
constexpr int kNc = 128;                        // max complex columns per tile (re + im: 256 TMEM columns)
constexpr int kKc = 8;                          // complex K per stage: one MMA k-step of 8 TF32
constexpr int kKq = kKc / 4;                    // core matrices (4 TF32 wide) along K per stage
constexpr int kPlaneA = kM * kKc * 4;           // one A plane (re or im, hi or lo)
constexpr int kPlaneB = kNc * kKc * 4;          // one B plane
constexpr int kStageBytes = 4 * kPlaneA + 4 * kPlaneB;
constexpr int kStages = 3;
constexpr int kSmemBytes = kStages * kStageBytes;   // 96 KB of operand staging
constexpr int kTmemCols = 256;

// Byte offset of real element (row, k) in a K-major, no-swizzle operand plane:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (the
// descriptor's leading-dimension offset), 8-row groups kKq * 128 B apart (its
// stride-dimension offset).
__device__ __forceinline__ int core_off(int row, int k) {
  return ((((row >> 3) * kKq) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2);
}
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = kKq * 128;

// Per-CTA control block in static shared memory.
struct Ctl {
  uint64_t bar[kStages];         // MMA-completion barriers, one per stage
  uint32_t issued[kStages];      // commits made on each barrier
  uint32_t waited[kStages];      // completions consumed on each barrier
  uint32_t tmem;                 // TMEM base address of this CTA's accumulator
  int failed;                    // a bounded wait ran out: no further MMAs
  int enabled;                   // FP32 contractions go to the tensor cores
  long long min_work;            // ... from this many complex multiply-adds on
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation: one full warp, power-of-two column count >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), the sm_100-family version bits (46..47 = 1), no base
// offset, relative leading-dimension mode, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}
// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), negate A (bit 13), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28, dense.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool neg_a = false) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: thread j of the warp gets lane
// (32 * (warp % 4) + j) of the addressed TMEM rows.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x -> (hi, lo): hi = x rounded to TF32 (kept in an FP32 container), lo = x - hi exactly.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// ------------------------------------------------------------------ setup / teardown
// Called by all threads of the CTA at kernel start (after ctl is zeroed is not
// required: this writes every field).  Warp 0 allocates the accumulator.
__device__ __forceinline__ void cta_setup(Ctl* ctl, int enabled, long long min_work = 16384) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->bar[s], 1);
      ctl->issued[s] = 0;
      ctl->waited[s] = 0;
    }
    ctl->failed = 0;
    ctl->enabled = enabled;
    ctl->min_work = min_work;
    fence_barrier_init();
  }
  if (enabled && threadIdx.x < 32) tmem_alloc(&ctl->tmem, kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}
__device__ __forceinline__ void cta_teardown(Ctl* ctl) {
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (ctl->enabled && threadIdx.x < 32) tmem_dealloc(ctl->tmem, kTmemCols);
}

// Wait (all threads) for the next completion of stage barrier s; bounded.
// Returns false, uniformly across the CTA, if any thread ran out of patience.
__device__ __forceinline__ bool stage_wait(Ctl* ctl, int s) {
  const uint32_t par = ctl->waited[s] & 1u;
  bool ok = false;
  for (long long it = 0; it < (1LL << 24); ++it) {
    if (mbar_try_wait(&ctl->bar[s], par)) { ok = true; break; }
  }
  const int bad = __syncthreads_or(!ok);
  if (threadIdx.x == 0) {
    ctl->waited[s] += 1;
    if (bad) ctl->failed = 1;
  }
  __syncthreads();
  return !bad;
}

// ------------------------------------------------------------------ the GEMM
// Operand access: A(i, k) = a[i * sai + k * sak] (conj if ca), B(k, j) =
// b[k * sbk + j * sbj] (conj if cb); the W-fused variant forms A on the fly
// from an MPO block in row-sparse form (see WaArgs in tjm_gemm.cuh).
struct TcA {
  const cx<float>* p; long long si, sk; int conj;
  // W-fused: A(i, k) = sum_z val[z] t1[x * sip + col[z] * chr + b], row o = t * Dr + v of the MPO block,
  // i = x * dd + t, k = v * chr + b
  const cx<float>* val; const int* col; const int* rp; const cx<float>* t1; int sip, dd, Dr, chr;
  int fused;
};
struct TcB { const cx<float>* p; long long sk, sj; int conj; };

__device__ __forceinline__ cx<float> tc_loadA(const TcA& a, int M, int K, int i, int k) {
  cx<float> v = czero<float>();
  if (i >= M || k >= K) return v;
  if (a.fused) {
    const int x = i / a.dd, t = i - x * a.dd;
    const int vv = k / a.chr, b = k - vv * a.chr;
    const int o = t * a.Dr + vv;
    const cx<float>* src = a.t1 + (long long)x * a.sip + b;
    const int z1 = a.rp[o + 1];
    for (int z = a.rp[o]; z < z1; ++z) cfma(v, a.val[z], src[a.col[z] * a.chr]);
    return v;
  }
  v = a.p[i * a.si + k * a.sk];
  if (a.conj) v.y = -v.y;
  return v;
}
__device__ __forceinline__ cx<float> tc_loadB(const TcB& b, int K, int N, int k, int j) {
  cx<float> v = czero<float>();
  if (k >= K || j >= N) return v;
  v = b.p[k * b.sk + j * b.sj];
  if (b.conj) v.y = -v.y;
  return v;
}

// C = alpha A B (+ C).  M, N, K > 0; C(i, j) at c[i * sci + j * scj].  All
// threads of the CTA call it; smem is the 96 KB staging area (16-byte
// aligned).  Returns false if a wait timed out (results are then undefined).
static __device__ __noinline__ bool cgemm(Ctl* ctl, int M, int N, int K, cx<float> alpha, TcA A, TcB B, cx<float>* C,
                                          long long sci, long long scj, bool accumulate, char* smem) {
  if (ctl->failed) return false;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool a_kc = A.fused || A.sk == 1 || A.si != 1;     // A's k index is the contiguous one
  const bool b_kc = !(B.sj == 1 || B.sk != 1);              // B's k index is the contiguous one
  // each thread stages one row of A and one row of B, 4 consecutive k of the 8 in a chunk
  const int ra = a_kc ? (tid >> 1) : (tid & 127), qa = a_kc ? (tid & 1) : (tid >> 7);
  const int rb = b_kc ? (tid >> 1) : (tid & 127), qb = b_kc ? (tid & 1) : (tid >> 7);
  const int nk = (K + kKc - 1) / kKc;
  const int ntile_n = (N + kNc - 1) / kNc;
  const uint32_t sbase = saddr(smem);
  for (int i0 = 0; i0 < M; i0 += kM) {
    for (int tn = 0; tn < ntile_n; ++tn) {
      const int j0 = tn * kNc;
      const int nt = N - j0 < kNc ? N - j0 : kNc;      // complex columns of this tile
      const int ntp = (nt + 15) & ~15;                   // padded to the M = 128 MMA's N granularity
      const uint32_t idesc = idesc_tf32(kM, ntp), idesc_neg = idesc_tf32(kM, ntp, true);
      const uint32_t t_re = ctl->tmem, t_im = ctl->tmem + (uint32_t)ntp;
      cx<float> xa[4], xb[4];
      auto fetch = [&](int kc) {
        const int k0 = kc * kKc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xa[q] = tc_loadA(A, M, K, i0 + ra, k0 + 4 * qa + q);
          xb[q] = rb < ntp ? tc_loadB(B, K, N, k0 + 4 * qb + q, j0 + rb) : czero<float>();
        }
      };
      fetch(0);
      for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % kStages;
        cx<float> ca[4], cb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { ca[q] = xa[q]; cb[q] = xb[q]; }
        if (kc + 1 < nk) fetch(kc + 1);        // in flight while this chunk is split and written
        if (kc >= kStages && !stage_wait(ctl, st)) return false;
        char* sp = smem + st * kStageBytes;
        {
          float4 rh, rl, ih, il;
          split_tf32(ca[0].x, rh.x, rl.x); split_tf32(ca[1].x, rh.y, rl.y);
          split_tf32(ca[2].x, rh.z, rl.z); split_tf32(ca[3].x, rh.w, rl.w);
          split_tf32(ca[0].y, ih.x, il.x); split_tf32(ca[1].y, ih.y, il.y);
          split_tf32(ca[2].y, ih.z, il.z); split_tf32(ca[3].y, ih.w, il.w);
          const int o = core_off(ra, 4 * qa);
          *reinterpret_cast<float4*>(sp + o) = rh;
          *reinterpret_cast<float4*>(sp + kPlaneA + o) = rl;
          *reinterpret_cast<float4*>(sp + 2 * kPlaneA + o) = ih;
          *reinterpret_cast<float4*>(sp + 3 * kPlaneA + o) = il;
        }
        if (rb < ntp) {
          float4 rh, rl, ih, il;
          split_tf32(cb[0].x, rh.x, rl.x); split_tf32(cb[1].x, rh.y, rl.y);
          split_tf32(cb[2].x, rh.z, rl.z); split_tf32(cb[3].x, rh.w, rl.w);
          split_tf32(cb[0].y, ih.x, il.x); split_tf32(cb[1].y, ih.y, il.y);
          split_tf32(cb[2].y, ih.z, il.z); split_tf32(cb[3].y, ih.w, il.w);
          const int o = core_off(rb, 4 * qb);
          char* sb = sp + 4 * kPlaneA;
          *reinterpret_cast<float4*>(sb + o) = rh;
          *reinterpret_cast<float4*>(sb + kPlaneB + o) = rl;
          *reinterpret_cast<float4*>(sb + 2 * kPlaneB + o) = ih;
          *reinterpret_cast<float4*>(sb + 3 * kPlaneB + o) = il;
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          fence_after_sync();
          const uint32_t a0 = sbase + st * kStageBytes;
          const uint64_t are_h = sdesc(a0, kLBO, kSBO), are_l = sdesc(a0 + kPlaneA, kLBO, kSBO);
          const uint64_t aim_h = sdesc(a0 + 2 * kPlaneA, kLBO, kSBO), aim_l = sdesc(a0 + 3 * kPlaneA, kLBO, kSBO);
          const uint32_t b0 = a0 + 4 * kPlaneA;
          const uint64_t bre_h = sdesc(b0, kLBO, kSBO), bre_l = sdesc(b0 + kPlaneB, kLBO, kSBO);
          const uint64_t bim_h = sdesc(b0 + 2 * kPlaneB, kLBO, kSBO), bim_l = sdesc(b0 + 3 * kPlaneB, kLBO, kSBO);
          const uint32_t acc0 = kc > 0 ? 1u : 0u;
          // C_re += A_re B_re - A_im B_im   (small terms first)
          mma_tf32(t_re, are_l, bre_h, idesc, acc0);
          mma_tf32(t_re, are_h, bre_l, idesc, 1u);
          mma_tf32(t_re, are_h, bre_h, idesc, 1u);
          mma_tf32(t_re, aim_l, bim_h, idesc_neg, 1u);
          mma_tf32(t_re, aim_h, bim_l, idesc_neg, 1u);
          mma_tf32(t_re, aim_h, bim_h, idesc_neg, 1u);
          // C_im += A_re B_im + A_im B_re
          mma_tf32(t_im, are_l, bim_h, idesc, acc0);
          mma_tf32(t_im, are_h, bim_l, idesc, 1u);
          mma_tf32(t_im, are_h, bim_h, idesc, 1u);
          mma_tf32(t_im, aim_l, bre_h, idesc, 1u);
          mma_tf32(t_im, aim_h, bre_l, idesc, 1u);
          mma_tf32(t_im, aim_h, bre_h, idesc, 1u);
          mma_commit(&ctl->bar[st]);
          ctl->issued[st] += 1;
        }
        __syncthreads();
      }
      // drain: every commit of this tile completed (they complete in order)
      for (int s2 = 0; s2 < kStages; ++s2)
        while (ctl->waited[s2] < ctl->issued[s2])
          if (!stage_wait(ctl, s2)) return false;
      fence_after_sync();
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows), complex columns [64 (w / 4), + 64)
      const int row = i0 + 32 * (warp & 3) + lane;
      const int half = warp >> 2;
      const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
      for (int c0 = half * (kNc / 2); c0 < ntp && c0 < (half + 1) * (kNc / 2); c0 += 16) {
        float vr[16], vi[16];
        tmem_ld16(t_re + lane_off + (uint32_t)c0, vr);
        tmem_ld16(t_im + lane_off + (uint32_t)c0, vi);
        tmem_wait_ld();
        if (row < M) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int j = j0 + c0 + e;
            if (j < j0 + nt) {
              cx<float> r = mk(alpha.x * vr[e] - alpha.y * vi[e], alpha.x * vi[e] + alpha.y * vr[e]);
              cx<float>* dst = C + row * sci + j * scj;
              if (accumulate) r = r + *dst;
              *dst = r;
            }
          }
        }
      }
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
    }
  }
  return true;
}

}  // namespace tc
}  // namespace tjm

// CTA-wide complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C(i, j) = alpha * sum_k A(i, k) B(k, j)  [+ C(i, j) if accumulate]
//
// The effective-Hamiltonian and environment contractions of the TDVP sweep
// (paper Fig. 2: L . W . A . R) are complex GEMMs whose operands are FP32.
// They run here as real GEMMs on the tensor pipe:
//   * complex -> real ("4M" split in one product): the interleaved complex A
//     (M x K) is the real matrix [a_re a_im ...] of M x 2K; B is expanded to
//     the real 2K x 2N matrix of 2x2 blocks [[b_re, b_im], [-b_im, b_re]], so
//     the real product is C interleaved (M x 2N);
//   * FP32 accuracy from TF32 inputs ("3xTF32"): x = hi + lo with hi = x
//     rounded to TF32 and lo the FP32 remainder, and A B = Ahi Bhi + Ahi Blo +
//     Alo Bhi up to the dropped Alo Blo (2^-22 relative) -- three MMAs per
//     k-step accumulating in FP32 in tensor memory.
// One thread issues tcgen05.mma (kind::tf32, M = 128, N <= 256, K = 8) from
// shared-memory operand tiles in the K-major no-swizzle core-matrix layout;
// the accumulator (128 lanes x N FP32 columns) lives in tensor memory and is
// read back with tcgen05.ld.  Operand tiles pass through registers on their
// way to shared memory because every element is split (hi / lo) and B is
// expanded, which a bulk tensor copy cannot do; two stages let the loads of
// one K chunk overlap the MMAs of the previous one, ordered by mbarriers that
// tcgen05.commit arrives on.  Every mbarrier wait is bounded: on timeout the
// CTA records the failure, stops issuing MMAs and the caller marks the
// trajectory failed.
#pragma once
#include <stdint.h>

#include "tjm_common.cuh"

namespace tjm {
namespace tc {

// ------------------------------------------------------------------ geometry
constexpr int kM = 128;                         // MMA rows (TMEM lanes)
constexpr int kNr = 256;                        // max real columns per tile (TMEM columns)
constexpr int kKc = 8;                          // complex K per stage
constexpr int kKr = 2 * kKc;                    // real K per stage (two MMAs of K = 8)
constexpr int kKq = kKr / 4;                    // core matrices (4 TF32 wide) along K per stage
constexpr int kABytes = kM * kKr * 4;           // one A tile (hi or lo)
constexpr int kBBytes = kNr * kKr * 4;          // one B tile (hi or lo)
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr int kStages = 2;
constexpr int kSmemBytes = kStages * kStageBytes;   // 96 KB of operand staging
constexpr int kTmemCols = 256;

// Byte offset of real element (row, kr) in a K-major, no-swizzle operand tile:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (the
// descriptor's leading-dimension offset), 8-row groups kKq * 128 B apart (its
// stride-dimension offset).
__device__ __forceinline__ int core_off(int row, int kr) {
  return ((((row >> 3) * kKq) + (kr >> 2)) << 7) + ((row & 7) << 4) + ((kr & 3) << 2);
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
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28, dense, no negation.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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
__device__ __forceinline__ void cta_setup(Ctl* ctl, int enabled) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->bar[s], 1);
      ctl->issued[s] = 0;
      ctl->waited[s] = 0;
    }
    ctl->failed = 0;
    ctl->enabled = enabled;
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
  const bool b_nc = B.sj == 1 || B.sk != 1;                 // B's j index is the contiguous one
  const int nk = (K + kKc - 1) / kKc;
  const int ntile_n = (N + kNr / 2 - 1) / (kNr / 2);
  const uint32_t sbase = saddr(smem);
  for (int i0 = 0; i0 < M; i0 += kM) {
    for (int tn = 0; tn < ntile_n; ++tn) {
      const int j0 = tn * (kNr / 2);
      const int nt = N - j0 < kNr / 2 ? N - j0 : kNr / 2;     // complex columns of this tile
      const int ntp = (nt + 7) & ~7;                             // padded to the MMA's N granularity
      const uint32_t idesc = idesc_tf32(kM, 2 * ntp);
      for (int kc = 0; kc < nk; ++kc) {
        const int k0 = kc * kKc;
        const int st = kc & 1;
        // global -> registers first, so the loads are in flight while we wait for the stage
        cx<float> ra[4], rb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ia = a_kc ? (tid >> 1) : ((tid & 31) * 4 + q);
          const int ka = a_kc ? ((tid & 1) * 4 + q) : (tid >> 5);
          ra[q] = tc_loadA(A, M, K, i0 + ia, k0 + ka);
          const int kb = b_nc ? (tid >> 5) : ((tid & 1) * 4 + q);
          const int jb = b_nc ? ((tid & 31) * 4 + q) : (tid >> 1);
          rb[q] = jb < ntp ? tc_loadB(B, K, N, k0 + kb, j0 + jb) : czero<float>();
        }
        if (kc >= kStages && !stage_wait(ctl, st)) return false;
        char* sA = smem + st * kStageBytes;
        char* sAl = sA + kABytes;
        char* sB = sAl + kABytes;
        char* sBl = sB + kBBytes;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ia = a_kc ? (tid >> 1) : ((tid & 31) * 4 + q);
          const int ka = a_kc ? ((tid & 1) * 4 + q) : (tid >> 5);
          float2 h, l;
          split_tf32(ra[q].x, h.x, l.x);
          split_tf32(ra[q].y, h.y, l.y);
          const int oa = core_off(ia, 2 * ka);
          *reinterpret_cast<float2*>(sA + oa) = h;
          *reinterpret_cast<float2*>(sAl + oa) = l;
          const int kb = b_nc ? (tid >> 5) : ((tid & 1) * 4 + q);
          const int jb = b_nc ? ((tid & 31) * 4 + q) : (tid >> 1);
          if (jb < ntp) {
            float brh, brl, bih, bil;
            split_tf32(rb[q].x, brh, brl);
            split_tf32(rb[q].y, bih, bil);
            // rows 2j (real part of C) and 2j+1 (imaginary part), columns 2k (times a_re), 2k+1 (times a_im)
            const int o0 = core_off(2 * jb, 2 * kb), o1 = core_off(2 * jb + 1, 2 * kb);
            *reinterpret_cast<float2*>(sB + o0) = make_float2(brh, -bih);
            *reinterpret_cast<float2*>(sB + o1) = make_float2(bih, brh);
            *reinterpret_cast<float2*>(sBl + o0) = make_float2(brl, -bil);
            *reinterpret_cast<float2*>(sBl + o1) = make_float2(bil, brl);
          }
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          fence_after_sync();
          const uint32_t a_hi = sbase + st * kStageBytes, a_lo = a_hi + kABytes;
          const uint32_t b_hi = a_lo + kABytes, b_lo = b_hi + kBBytes;
#pragma unroll
          for (int s = 0; s < kKr / 8; ++s) {
            const uint32_t ko = s * 2 * 128;     // two core matrices (8 TF32) per MMA k-step
            const uint32_t acc0 = (kc > 0 || s > 0) ? 1u : 0u;
            mma_tf32(ctl->tmem, sdesc(a_lo + ko, kLBO, kSBO), sdesc(b_hi + ko, kLBO, kSBO), idesc, acc0);
            mma_tf32(ctl->tmem, sdesc(a_hi + ko, kLBO, kSBO), sdesc(b_lo + ko, kLBO, kSBO), idesc, 1u);
            mma_tf32(ctl->tmem, sdesc(a_hi + ko, kLBO, kSBO), sdesc(b_hi + ko, kLBO, kSBO), idesc, 1u);
          }
          mma_commit(&ctl->bar[st]);
          ctl->issued[st] += 1;
        }
        __syncthreads();
      }
      // drain: every commit of this tile completed (they complete in order)
      for (int s = 0; s < kStages; ++s)
        while (ctl->waited[s] < ctl->issued[s])
          if (!stage_wait(ctl, s)) return false;
      fence_after_sync();
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows), column half w / 4
      const int row = i0 + 32 * (warp & 3) + lane;
      const int half = warp >> 2;
      for (int c0 = half * (kNr / 2); c0 < 2 * ntp && c0 < (half + 1) * (kNr / 2); c0 += 16) {
        float v[16];
        tmem_ld16(ctl->tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
        tmem_wait_ld();
        if (row < M) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = j0 + c0 / 2 + e;
            if (j < j0 + nt) {
              cx<float> r = mk(alpha.x * v[2 * e] - alpha.y * v[2 * e + 1], alpha.x * v[2 * e + 1] + alpha.y * v[2 * e]);
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

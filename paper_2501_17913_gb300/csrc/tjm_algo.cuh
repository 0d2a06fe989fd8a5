// The tensor jump method for one trajectory, executed by one CTA.
//
// Everything here is block-level (all threads call every function).  The
// contraction precision is Tc (complex float or double: site tensors,
// environments, Krylov vectors, GEMMs); the decomposition precision is Td
// (QR / SVD workspaces).  Reductions that decide anything -- norms, dp, jump
// weights, Lanczos coefficients, expectation values -- are accumulated in FP64.
//
// Paper: arXiv:2501.17913, Sec. "Tensor jump method" (Eqs. TimeEvolutionFunctions,
// SimulationStep), Sec. "Dynamic TDVP", Sec. "Dissipative contraction",
// Sec. "Stochastic jump process", Sec. "Algorithm".
#pragma once
#include "tjm_common.cuh"
#include "tjm_gemm.cuh"
#include "tjm_linalg.cuh"
#include "tjm_types.h"

namespace tjm {

constexpr int kD = 2;   // physical dimension (spin-1/2 chains)

// ------------------------------------------------------------------ views
template <class Tc> struct Mps {
  cx<Tc>* base;
  long long cap;    // elements per site slot
  int* chi;         // bond dimensions [L + 1]
  __device__ cx<Tc>* site(int l) const { return base + (long long)l * cap; }
};

template <class Tc, class Td> struct Ctx {
  const ProbDev* P;
  SlotDev* S;
  Mps<Tc> mps;           // the sampling MPS Phi of this trajectory
  Mps<Tc> xmps;          // copy used by the sampling layer
  cx<Tc>* envL;          // [L + 1][cap_env]
  cx<Tc>* envR;
  long long cap_env;
  // per-CTA scratch
  cx<Tc>* krylov; cx<Tc>* w; cx<Tc>* t1; cx<Tc>* t2; cx<Tc>* theta; cx<Tc>* tmp; cx<Tc>* bond;
  cx<Tc>* E; cx<Tc>* F;
  cx<Td>* da; cx<Td>* du; cx<Td>* dv; cx<Td>* dvw; cx<Td>* drd; Td* dtau; Td* ds; int* iw;
  cx<double>* G;         // [L][4] per-site reduced 2x2 blocks
  cx<double>* G2;        // [L][16] reduced 4x4 blocks of sites (l, l+1) where a two-site observable starts
  double* wts;           // jump weights
  char* wcsr;            // row-sparse MPO block of a fused tensor-core matvec
  // shared memory
  char* gsm; double* red; double* sc;
  char* fsm;             // factorization workspace in shared memory (nullptr if none)
  int fsm_bytes;         // its size
  char* fsv;             // shared scratch for unsorted singular values (fsm_bytes > 0 only)
  __device__ cx<Tc>* Lenv(int b) const { return envL + (long long)b * cap_env; }
  __device__ cx<Tc>* Renv(int b) const { return envR + (long long)b * cap_env; }
};

// Phase timer: every wrapped statement ends in a CTA-wide barrier, so thread
// 0's clock64() interval is the CTA's time in that phase.
#define TJM_TIMED(c, ph, stmt)                                                   \
  do {                                                                           \
    const long long _t0 = clock64();                                             \
    stmt;                                                                        \
    if (threadIdx.x == 0) (c).S->stats.cyc[ph] += (unsigned long long)(clock64() - _t0); \
  } while (0)

// Energy shift per site: H - eshift * sum_i I_i has its expectation value near
// zero, so the FP32 sums of the environment contractions stay small.  A
// constant shift only multiplies every local exponential by a phase.
template <class Tc, class Td>
__device__ __forceinline__ double site_shift(const Ctx<Tc, Td>& c) {
  return c.P->shift_ok ? -c.S->eshift : 0.0;
}

// Work counters (thread 0 only; one CTA owns a slot).
template <class Tc, class Td>
__device__ __forceinline__ void count_contract(const Ctx<Tc, Td>& c, double cmacs) {
  if (threadIdx.x == 0) c.S->stats.flops_contract += 8.0 * cmacs;
}
template <class Tc, class Td>
__device__ __forceinline__ void count_decomp(const Ctx<Tc, Td>& c, double cmacs) {
  if (threadIdx.x == 0) c.S->stats.flops_decomp += 8.0 * cmacs;
}

// ------------------------------------------------------------------ site-local operator
// M[a][t][b] <- sum_s op[t][s] M[a][s][b]   (op: 2x2 complex double, row-major)
template <class Tc>
__device__ void blk_site_op(cx<Tc>* M, int chl, int chr, const cx<double>* op, cx<double> scale) {
  const cx<Tc> o00 = cvt<Tc>(scale * op[0]), o01 = cvt<Tc>(scale * op[1]);
  const cx<Tc> o10 = cvt<Tc>(scale * op[2]), o11 = cvt<Tc>(scale * op[3]);
  for (int e = threadIdx.x; e < chl * chr; e += TJM_THREADS) {
    const int a = e / chr, b = e % chr;
    cx<Tc>* p0 = M + (long long)(a * kD) * chr + b;
    cx<Tc>* p1 = p0 + chr;
    const cx<Tc> x0 = *p0, x1 = *p1;
    cx<Tc> y0 = czero<Tc>(), y1 = czero<Tc>();
    cfma(y0, o00, x0); cfma(y0, o01, x1);
    cfma(y1, o10, x0); cfma(y1, o11, x1);
    *p0 = y0; *p1 = y1;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ effective Hamiltonians
// FP32 contractions on the CUDA cores fuse the MPO block into the second GEMM's operand loads; on
// the tensor cores (and in FP64) T2 = W T1 is formed first, so that the GEMM streams a plain operand.
template <class Tc>
__device__ __forceinline__ bool fused_matvec() {
  if constexpr (sizeof(Tc) == 4) return !tc_ctl.enabled;
  return false;
}

// One site l: y[x][t][y'] = sum Lenv[l][x,w,a] W_l[w,v,t,s] M[a,s,b] Renv[l+1][v,b,y']
template <class Tc, class Td>
__device__ __noinline__ void heff1(const Ctx<Tc, Td>& c, int l, const cx<Tc>* x, cx<Tc>* y) {
  const int chl = c.mps.chi[l], chr = c.mps.chi[l + 1];
  const int Dl = c.P->Dbond[l], Dr = c.P->Dbond[l + 1];
  // G1: T1[(x w), (s b)] = L[(x w), a] M[a, (s b)]
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * Dl, kD * chr, chl, matA(c.Lenv(l), chl, 1), matB(x, kD * chr, 1), c.t1, kD * chr, 1, c.gsm));
  if (fused_matvec<Tc>()) {
    if constexpr (sizeof(Tc) == 4)
      TJM_TIMED(c, PH_GEMM, blk_wgemm<Tc>(chl, kD, Dr, Dl * kD, chr, c.P->Wm1 + c.P->Wm1_off[l], c.t1, c.Renv(l + 1),
                                          y, c.gsm, c.wcsr, site_shift(c), kD, Dr - 1, Dr, 0, 1));
  } else {
    // G2: T2[x][(t v)][b] = sum_(w s) Wm1[(t v)][(w s)] T1[x][(w s)][b]
    TJM_TIMED(c, PH_WAPPLY, blk_wapply<Tc>(chl, kD * Dr, Dl * kD, chr, c.P->Wm1 + c.P->Wm1_off[l], c.t1, (long long)Dl * kD * chr, chr, c.t2,
                   (long long)kD * Dr * chr, chr, c.gsm, site_shift(c), kD, Dr - 1, Dr, 0, 1));
    // G3: y[(x t), y'] = T2[(x t), (v b)] R[(v b), y']
    TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * kD, chr, Dr * chr, matA(c.t2, (long long)Dr * chr, 1), matB(c.Renv(l + 1), chr, 1), y, chr, 1,
                 c.gsm));
  }
  count_contract(c, (double)chl * Dl * kD * chr * chl + (double)chl * chr * kD * Dr * Dl * kD +
                        (double)chl * kD * chr * Dr * chr);
}

// Two sites (l, l+1) on theta[a][s1][s2][b]
template <class Tc, class Td>
__device__ __noinline__ void heff2(const Ctx<Tc, Td>& c, int l, int chl, int chr, const cx<Tc>* x, cx<Tc>* y) {
  const int Dl = c.P->Dbond[l], Dr = c.P->Dbond[l + 2];
  const int d2 = kD * kD;
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * Dl, d2 * chr, chl, matA(c.Lenv(l), chl, 1), matB(x, d2 * chr, 1), c.t1, d2 * chr, 1, c.gsm));
  if (fused_matvec<Tc>()) {
    if constexpr (sizeof(Tc) == 4)
      TJM_TIMED(c, PH_GEMM, blk_wgemm<Tc>(chl, d2, Dr, Dl * d2, chr, c.P->W12 + c.P->W12_off[l], c.t1, c.Renv(l + 2),
                                          y, c.gsm, c.wcsr, 2.0 * site_shift(c), d2, Dr - 1, Dr, 0, 1));
  } else {
    TJM_TIMED(c, PH_WAPPLY, blk_wapply<Tc>(chl, d2 * Dr, Dl * d2, chr, c.P->W12 + c.P->W12_off[l], c.t1, (long long)Dl * d2 * chr, chr, c.t2,
                   (long long)d2 * Dr * chr, chr, c.gsm, 2.0 * site_shift(c), d2, Dr - 1, Dr, 0, 1));
    TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * d2, chr, Dr * chr, matA(c.t2, (long long)Dr * chr, 1), matB(c.Renv(l + 2), chr, 1), y, chr, 1,
                 c.gsm));
  }
  count_contract(c, (double)chl * Dl * d2 * chr * chl + (double)chl * chr * d2 * Dr * Dl * d2 +
                        (double)chl * d2 * chr * Dr * chr);
}

// Bond b (between sites b-1 and b): y[x][y'] = sum Lenv[b][x,w,a] C[a,b'] Renv[b][w,b',y']
template <class Tc, class Td>
__device__ __noinline__ void heff0(const Ctx<Tc, Td>& c, int b, int chl, int chr, const cx<Tc>* x, cx<Tc>* y) {
  const int D = c.P->Dbond[b];
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * D, chr, chl, matA(c.Lenv(b), chl, 1), matB(x, chr, 1), c.t1, chr, 1, c.gsm));
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl, chr, D * chr, matA(c.t1, (long long)D * chr, 1), matB(c.Renv(b), chr, 1), y, chr, 1, c.gsm));
  count_contract(c, (double)chl * D * chr * chl + (double)chl * chr * D * chr);
}

// Lenv[l+1][y][v][b] = sum conj(A[x,t,y]) Lenv[l][x,w,a] W[w,v,t,s] A[a,s,b]
template <class Tc, class Td>
__device__ __noinline__ void env_left(const Ctx<Tc, Td>& c, int l) {
  const int chl = c.mps.chi[l], chr = c.mps.chi[l + 1];
  const int Dl = c.P->Dbond[l], Dr = c.P->Dbond[l + 1];
  const cx<Tc>* A = c.mps.site(l);
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * Dl, kD * chr, chl, matA(c.Lenv(l), chl, 1), matB(A, kD * chr, 1), c.t1, kD * chr, 1, c.gsm));
  TJM_TIMED(c, PH_WAPPLY, blk_wapply<Tc>(chl, kD * Dr, Dl * kD, chr, c.P->Wm1 + c.P->Wm1_off[l], c.t1, (long long)Dl * kD * chr, chr, c.t2,
                 (long long)kD * Dr * chr, chr, c.gsm, site_shift(c), kD, Dr - 1, Dr, 0, 1));
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chr, Dr * chr, chl * kD, matA(A, 1, chr, 1), matB(c.t2, (long long)Dr * chr, 1), c.Lenv(l + 1),
               (long long)Dr * chr, 1, c.gsm));
  count_contract(c, (double)chl * Dl * kD * chr * chl + (double)chl * chr * kD * Dr * Dl * kD +
                        (double)chr * Dr * chr * chl * kD);
}

// Renv[l][w][a][x] = sum B[a,s,b] W[w,v,t,s] Renv[l+1][v,b,y] conj(B[x,t,y])
template <class Tc, class Td>
__device__ __noinline__ void env_right(const Ctx<Tc, Td>& c, int l) {
  const int chl = c.mps.chi[l], chr = c.mps.chi[l + 1];
  const int Dl = c.P->Dbond[l], Dr = c.P->Dbond[l + 1];
  const cx<Tc>* B = c.mps.site(l);
  // S1[(a s)][v][y] = B[(a s), b] R_v[b, y]
  TJM_TIMED(c, PH_GEMM, blk_gemm_batched<Tc>(Dr, chl * kD, chr, chr, mk((Tc)1, (Tc)0), matA(B, chr, 1), 0,
                       matB(c.Renv(l + 1), chr, 1), (long long)chr * chr, c.t1, (long long)Dr * chr, 1, chr, false,
                       c.gsm));
  // S2[a][(w t)][y] = sum_(s v) WmR[(w t)][(s v)] S1[a][(s v)][y]
  TJM_TIMED(c, PH_WAPPLY, blk_wapply<Tc>(chl, Dl * kD, kD * Dr, chr, c.P->WmR + c.P->WmR_off[l], c.t1, (long long)kD * Dr * chr, chr, c.t2,
                 (long long)Dl * kD * chr, chr, c.gsm, site_shift(c), kD, 0, 1, Dr - 1, Dr));
  // Rnew[w][a][x] = S2[a][w][(t y)] conj(B[x][(t y)])
  TJM_TIMED(c, PH_GEMM, blk_gemm_batched<Tc>(Dl, chl, chl, kD * chr, mk((Tc)1, (Tc)0), matA(c.t2, (long long)Dl * kD * chr, 1), kD * chr,
                       matB(B, 1, kD * chr, 1), 0, c.Renv(l), chl, 1, (long long)chl * chl, false, c.gsm));
  count_contract(c, (double)Dr * chl * kD * chr * chr + (double)chl * chr * Dl * kD * kD * Dr +
                        (double)Dl * chl * chl * kD * chr);
}

template <class Tc, class Td>
__device__ void build_right_envs(const Ctx<Tc, Td>& c) {
  const int L = c.P->L;
  if (threadIdx.x == 0) { c.Renv(L)[0] = mk((Tc)1, (Tc)0); c.Lenv(0)[0] = mk((Tc)1, (Tc)0); }
  __syncthreads();
  for (int l = L - 1; l >= 1; --l) env_right(c, l);
  if (threadIdx.x == 0) atomicAdd(&c.S->stats.env_updates, (unsigned long long)(L - 1));
  if (!c.P->shift_ok) return;
  // <H - shift> of the right-canonical state from site 0 and its environment;
  // the energy per site becomes the shift of the next environments
  const int n0 = c.mps.chi[0] * kD * c.mps.chi[1];
  heff1(c, 0, c.mps.site(0), c.w);
  double e = 0.0, nn = 0.0;
  for (int i = threadIdx.x; i < n0; i += TJM_THREADS) {
    const cx<Tc> a = c.mps.site(0)[i], b = c.w[i];
    e += (double)a.x * b.x + (double)a.y * b.y;
    nn += (double)a.x * a.x + (double)a.y * a.y;
  }
  e = blk_sum(e, c.red);
  nn = blk_sum(nn, c.red + 16);
  if (threadIdx.x == 0 && nn > 0.0 && e == e) c.S->eshift += e / nn / L;
  __syncthreads();
}

// ------------------------------------------------------------------ Lanczos exponential
// v <- exp(i theta H) v with H given by `kind` (1: one site l, 2: two sites l,l+1,
// 0: bond l).  Stopping rule: |beta_k [exp(i theta T_k) e_1]_k| < tol or kmax
// matvecs.  Full re-orthogonalisation: the three-term recurrence followed by
// one classical Gram-Schmidt pass over the whole basis, coefficients in FP64.
// Returns the number of matvecs.
template <class Tc, class Td>
__device__ __noinline__ int lanczos(const Ctx<Tc, Td>& c, int kind, int l, int chl, int chr, cx<Tc>* v, int n, double theta) {
  const int kmax = c.P->krylov_max;
  const double tol = c.P->krylov_tol;
  double* alpha = c.sc;            // [kmax]
  double* beta = c.sc + 64;        // [kmax]
  cx<double>* cf = reinterpret_cast<cx<double>*>(c.sc + 128);   // [kmax]
  double* hh = c.sc + 256;         // [2 * kmax] re/im of CGS coefficients
  const double b0 = sqrt(blk_nrm2sq(v, n, c.red));
  if (!(b0 > 0.0)) return 0;
  {
    const Tc f = (Tc)(1.0 / b0);
    for (int i = threadIdx.x; i < n; i += TJM_THREADS) c.krylov[i] = f * v[i];
  }
  __syncthreads();
  int k = 0;
  for (;; ++k) {
    const cx<Tc>* vk = c.krylov + (long long)k * n;
    TJM_TIMED(c, PH_MATVEC, {
      if (kind == 1) heff1(c, l, vk, c.w);
      else if (kind == 2) heff2(c, l, chl, chr, vk, c.w);
      else heff0(c, l, chl, chr, vk, c.w);
    });
    // Three-term recurrence, then one classical Gram-Schmidt pass against
    // the whole basis (the recurrence acts as the first orthogonalisation
    // pass).  (1) w -= beta_{k-1} v_{k-1} while forming alpha = <v_k, w>;
    // (2) w -= alpha v_k while forming all coefficients h_j = <v_j, w> in
    // chunks of 8 basis vectors; (3) w -= sum_j h_j v_j while forming ||w||^2.
    // Coefficients are reduced in FP64; alpha_k = alpha + Re h_k.
    const int nb = k + 1;
    // w and the basis are distinct buffers: say so, so loads of later
    // elements may be issued ahead of the stores to w
    cx<Tc>* __restrict__ wv = c.w;
    const cx<Tc>* __restrict__ kb = c.krylov;
    const cx<Tc>* __restrict__ vk0 = kb + (long long)k * n;
    double al_k;
    {
      const cx<Tc>* __restrict__ vkm = kb + (long long)(k > 0 ? k - 1 : 0) * n;
      const Tc bm = k > 0 ? (Tc)beta[k - 1] : (Tc)0;
      Tc ax = 0;
#pragma unroll 2
      for (int i = threadIdx.x; i < n; i += TJM_THREADS) {
        cx<Tc> t = wv[i];
        if (k > 0) { t.x -= bm * vkm[i].x; t.y -= bm * vkm[i].y; }
        wv[i] = t;
        const cx<Tc> v = vk0[i];
        ax = fma(v.x, t.x, fma(v.y, t.y, ax));
      }
      // <v_k, w> is real for Hermitian H up to rounding; what is left of it
      // is removed with h_k below
      al_k = blk_sum((double)ax, c.red);
      __syncthreads();   // red is reused for the coefficients
    }
    {
      const Tc a0 = (Tc)al_k;
      for (int j0 = 0; j0 < nb; j0 += 8) {
        const int jn = nb - j0 < 8 ? nb - j0 : 8;
        cx<Tc> acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = czero<Tc>();
#pragma unroll 2
        for (int i = threadIdx.x; i < n; i += TJM_THREADS) {
          cx<Tc> wi = wv[i];
          if (j0 == 0) {   // each thread updates, then rereads, only its own entries
            const cx<Tc> v = vk0[i];
            wi.x -= a0 * v.x;
            wi.y -= a0 * v.y;
            wv[i] = wi;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < jn) cfma_cj(acc[q], kb[(long long)(j0 + q) * n + i], wi);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < jn) {
            const double ax = warp_sum((double)acc[q].x), ay = warp_sum((double)acc[q].y);
            if ((threadIdx.x & 31) == 0) {
              c.red[(2 * (j0 + q)) * TJM_WARPS + (threadIdx.x >> 5)] = ax;
              c.red[(2 * (j0 + q) + 1) * TJM_WARPS + (threadIdx.x >> 5)] = ay;
            }
          }
        }
      }
    }
    blk_sums_finish(2 * nb, c.red, hh);
    al_k += hh[2 * k];
    double wn2;
    {
      // coefficients converted once (FP64 -> working precision), not per element
      cx<Tc>* hw = reinterpret_cast<cx<Tc>*>(c.red);
      for (int j = threadIdx.x; j < nb; j += TJM_THREADS) hw[j] = mk((Tc)hh[2 * j], (Tc)hh[2 * j + 1]);
      __syncthreads();
      Tc n2 = 0;
#pragma unroll 2
      for (int i = threadIdx.x; i < n; i += TJM_THREADS) {
        cx<Tc> t = wv[i];
#pragma unroll 4
        for (int j = 0; j < nb; ++j) t = t - hw[j] * kb[(long long)j * n + i];
        wv[i] = t;
        n2 = fma(t.x, t.x, n2);
        n2 = fma(t.y, t.y, n2);
      }
      wn2 = blk_sum((double)n2, c.red + 64);
    }
    if (threadIdx.x == 0) alpha[k] = al_k;
    __syncthreads();
    const double bk = sqrt(wn2);
    TJM_TIMED(c, PH_EXPM, {
      if (threadIdx.x < 32) warp_expm_tridiag(k + 1, alpha, beta, theta, cf);
      __syncthreads();
    });
    const bool stop = !(bk * sqrt(norm2(cf[k])) >= tol) || (k == kmax - 1);
    if (stop) break;
    if (threadIdx.x == 0) beta[k] = bk;
    {
      const Tc f = (Tc)(1.0 / bk);
      cx<Tc>* vn = c.krylov + (long long)(k + 1) * n;
      for (int i = threadIdx.x; i < n; i += TJM_THREADS) vn[i] = f * c.w[i];
    }
    __syncthreads();
  }
  const int nk = k + 1;
  cx<Tc>* cw = reinterpret_cast<cx<Tc>*>(c.red);
  for (int j = threadIdx.x; j < nk; j += TJM_THREADS) cw[j] = mk((Tc)(b0 * cf[j].x), (Tc)(b0 * cf[j].y));
  __syncthreads();
#pragma unroll 2
  for (int i = threadIdx.x; i < n; i += TJM_THREADS) {
    cx<Tc> acc = czero<Tc>();
    for (int j = 0; j < nk; ++j) cfma(acc, cw[j], c.krylov[(long long)j * n + i]);
    v[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* ctr = kind == 1 ? &c.S->stats.mv_heff1 : (kind == 2 ? &c.S->stats.mv_heff2 : &c.S->stats.mv_heff0);
    atomicAdd(ctr, (unsigned long long)nk);
    if (k == kmax - 1) atomicAdd(&c.S->stats.krylov_capped, 1ull);
  }
  return nk;
}

// ------------------------------------------------------------------ factorizations on site tensors
// QR of the (rows x cols) matrix whose (i, j) element is src[i*si + j*sj]
// (conjugated if cj), in the factorization precision Td.  The thin Q (rows x k,
// column-major) is formed in place in the workspace -- shared memory when the
// matrix fits there, else the global buffer c.da -- and returned through *Q;
// R (k x cols, column-major) is left in c.dv.  Returns k = min(rows, cols).
template <class Tc, class Td>
__device__ __noinline__ int qr_of(const Ctx<Tc, Td>& c, int rows, int cols, const cx<Tc>* src, long long si,
                                  long long sj, bool cj, const cx<Td>** Q) {
  const bool in_smem = (long long)c.fsm_bytes >= (long long)rows * cols * (long long)sizeof(cx<Td>);
  cx<Td>* a = in_smem ? reinterpret_cast<cx<Td>*>(c.fsm) : c.da;
  for (long long e = threadIdx.x; e < (long long)rows * cols; e += TJM_THREADS) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    cx<Tc> x = src[i * si + j * sj];
    if (cj) x.y = -x.y;
    a[e] = cvt<Td>(x);
  }
  __syncthreads();
  TJM_TIMED(c, PH_QR, {
    blk_qr<Td>(rows, cols, a, a, c.dv, c.drd, c.dtau, c.red);
    __syncthreads();
  });
  {
    const double k = rows < cols ? rows : cols;
    // Householder factorization and explicit thin Q: 2 (m n^2 - n^3/3) complex multiply-adds each way
    count_decomp(c, 4.0 * ((double)rows * cols * k - k * k * k / 3.0));
  }
  *Q = a;
  return rows < cols ? rows : cols;
}

// Move the centre right: M_l = Q R, M_l <- Q; R (k x chr_old) is left in c.bond
// (row-major, Tc).  Updates chi[l+1] = k.
template <class Tc, class Td>
__device__ int qr_right(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int l) {
  const int chl = m.chi[l], chr = m.chi[l + 1];
  const int rows = chl * kD;
  cx<Tc>* M = m.site(l);
  const cx<Td>* Q;
  const int k = qr_of(c, rows, chr, M, chr, 1, false, &Q);
  for (long long e = threadIdx.x; e < (long long)rows * k; e += TJM_THREADS) {
    const int i = (int)(e / k), j = (int)(e % k);
    M[e] = cvt<Tc>(Q[(long long)j * rows + i]);
  }
  for (long long e = threadIdx.x; e < (long long)k * chr; e += TJM_THREADS) {
    const int i = (int)(e / chr), j = (int)(e % chr);
    c.bond[e] = cvt<Tc>(c.dv[(long long)j * k + i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) m.chi[l + 1] = k;
  __syncthreads();
  return k;
}

// Move the centre left: M_l = C Q with Q right-orthonormal (QR of M_l^H);
// M_l <- Q; C (chl_old x k) left in c.bond (row-major).  Updates chi[l] = k.
template <class Tc, class Td>
__device__ int rq_left(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int l) {
  const int chl = m.chi[l], chr = m.chi[l + 1];
  const int cols = kD * chr;
  cx<Tc>* M = m.site(l);
  // A = M^H : (cols x chl), A(i, j) = conj(M[j][i])
  const cx<Td>* Q;
  const int k = qr_of(c, cols, chl, M, 1, cols, true, &Q);
  // new M = Q^H : (k x cols)
  for (long long e = threadIdx.x; e < (long long)k * cols; e += TJM_THREADS) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    M[e] = cvt<Tc>(conj(Q[(long long)i * cols + j]));
  }
  // C = R^H : (chl x k), R is (k x chl) column-major in dv
  for (long long e = threadIdx.x; e < (long long)chl * k; e += TJM_THREADS) {
    const int i = (int)(e / k), j = (int)(e % k);
    c.bond[e] = cvt<Tc>(conj(c.dv[(long long)i * k + j]));
  }
  __syncthreads();
  if (threadIdx.x == 0) m.chi[l] = k;
  __syncthreads();
  return k;
}

// M_{l+1} <- C M_{l+1}, C = c.bond (k x chi_old), chi[l+1] already k.
template <class Tc, class Td>
__device__ void absorb_right(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int l, int chi_old) {
  const int k = m.chi[l + 1], chn = m.chi[l + 2];
  cx<Tc>* M = m.site(l + 1);
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(k, kD * chn, chi_old, matA(c.bond, chi_old, 1), matB(M, kD * chn, 1), c.tmp, kD * chn, 1, c.gsm));
  blk_copy(M, c.tmp, k * kD * chn);
  __syncthreads();
}

// M_{l-1} <- M_{l-1} C, C = c.bond (chi_old x k), chi[l] already k.
template <class Tc, class Td>
__device__ void absorb_left(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int l, int chi_old) {
  const int k = m.chi[l], chp = m.chi[l - 1];
  cx<Tc>* M = m.site(l - 1);
  TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chp * kD, k, chi_old, matA(M, chi_old, 1), matB(c.bond, k, 1), c.tmp, k, 1, c.gsm));
  blk_copy(M, c.tmp, chp * kD * k);
  __syncthreads();
}

// Truncation rank from the sorted singular values in c.ds (n of them):
// smallest r >= 1 with sum_{i>=r} s_i^2 <= eps * sum_i s_i^2, capped at cap;
// exact mode keeps everything.
template <class Tc, class Td>
__device__ int trunc_rank(const Ctx<Tc, Td>& c, int n) {
  __shared__ int r_sh;
  if (threadIdx.x == 0) {
    int r = n;
    if (!c.P->exact) {
      double tot = 0.0;
      for (int i = 0; i < n; ++i) tot += (double)c.ds[i] * (double)c.ds[i];
      double tail = 0.0;
      for (int i = n - 1; i >= 1; --i) {
        const double w = (double)c.ds[i] * (double)c.ds[i];
        if (tail + w <= c.P->trunc_eps * tot) { tail += w; r = i; } else break;
      }
      if (r > c.P->chi_max) r = c.P->chi_max;
      if (r < 1) r = 1;
    }
    r_sh = r;
  }
  __syncthreads();
  const int r = r_sh;
  __syncthreads();
  return r;
}

// SVD of the (m x n) matrix src[i*si + j*sj]: on exit U (m x nn) in c.du,
// V (n x nn) in c.dv (both column-major, Td), s in c.ds (descending), with
// nn = min(m, n) and src = U diag(s) V^H.
template <class Tc, class Td>
__device__ __noinline__ int svd_of(const Ctx<Tc, Td>& c, int m, int n, const cx<Tc>* src, long long si, long long sj) {
  const bool tr = m < n;
  const int mm = tr ? n : m, nn = tr ? m : n;
  // work matrix (mm x nn): A or A^H, in shared memory when it fits (the GEMM
  // staging area then holds the rotation accumulator)
  const bool in_smem = (long long)c.fsm_bytes >= (long long)mm * nn * (long long)sizeof(cx<Td>) &&
                       (long long)nn * nn * (long long)sizeof(cx<Td>) <= kSmemGemm;
  cx<Td>* a = in_smem ? reinterpret_cast<cx<Td>*>(c.fsm) : c.da;
  cx<Td>* vw = in_smem ? reinterpret_cast<cx<Td>*>(c.gsm) : c.dvw;
  Td* sv = in_smem ? reinterpret_cast<Td*>(c.fsv) : reinterpret_cast<Td*>(c.dvw + (long long)nn * nn);
  for (long long e = threadIdx.x; e < (long long)mm * nn; e += TJM_THREADS) {
    const int i = (int)(e % mm), j = (int)(e / mm);
    cx<Tc> x = tr ? conj(src[j * si + i * sj]) : src[i * si + j * sj];
    a[e] = cvt<Td>(x);
  }
  __syncthreads();
  // on the work matrix: Wk = Uw diag(s) Vw^H; Uw -> du (mm x nn), Vw -> dv (nn x nn)
  int sweeps = 0;
  TJM_TIMED(c, PH_SVD, sweeps = blk_svd_jacobi<Td>(mm, nn, a, c.du, c.ds, c.dv, vw, sv, c.iw, c.red, c.P->exact != 0));
  // per sweep and pair: three column dot products and two column rotations (A and V)
  count_decomp(c, (double)(sweeps + 1) * 0.5 * nn * (nn - 1) * (3.0 * mm + 2.0 * (mm + nn)));
  if (tr) {
    // A = (Wk)^H = Vw diag(s) Uw^H : U = Vw (m x nn), V = Uw (n x nn); swap buffers by copy
    for (long long e = threadIdx.x; e < (long long)mm * nn; e += TJM_THREADS) c.da[e] = c.du[e];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)nn * nn; e += TJM_THREADS) c.du[e] = c.dv[e];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)mm * nn; e += TJM_THREADS) c.dv[e] = c.da[e];
    __syncthreads();
  }
  return nn;
}

// ------------------------------------------------------------------ dynamic TDVP U[dt]
// L->R then R->L half sweep with tau = dt/2 each; per bond: two-site update
// if chi < chi_max, else one-site.  Forward updates exp(-i H tau), backward
// exp(+i H tau).  Pre/post: centre at 0, sites 1..L-1 right-canonical, Renv valid.
template <class Tc, class Td>
__device__ __noinline__ void tdvp_sweep(const Ctx<Tc, Td>& c, double tau) {
  const ProbDev* P = c.P;
  const int L = P->L;
  const Mps<Tc>& m = c.mps;
  bool last_two = false;
  for (int l = 0; l < L - 1; ++l) {
    const int chl = m.chi[l], chb = m.chi[l + 1], chr = m.chi[l + 2];
    if (chb < P->chi_max) {
      // theta = M_l M_{l+1}  -> (chl*d) x (d*chr)
      blk_gemm<Tc>(chl * kD, kD * chr, chb, matA(m.site(l), chb, 1), matB(m.site(l + 1), kD * chr, 1), c.theta,
                   kD * chr, 1, c.gsm);
      const int n = chl * kD * kD * chr;
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 2, l, chl, chr, c.theta, n, -tau));
      const int nn = svd_of(c, chl * kD, kD * chr, c.theta, kD * chr, 1);
      const int r = trunc_rank(c, nn);
      cx<Tc>* A = m.site(l);
      cx<Tc>* B = m.site(l + 1);
      const int rows = chl * kD, cols = kD * chr;
      for (long long e = threadIdx.x; e < (long long)rows * r; e += TJM_THREADS) {
        const int i = (int)(e / r), j = (int)(e % r);
        A[e] = cvt<Tc>(c.du[(long long)j * rows + i]);
      }
      for (long long e = threadIdx.x; e < (long long)r * cols; e += TJM_THREADS) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        B[e] = cvt<Tc>((Td)c.ds[i] * conj(c.dv[(long long)i * cols + j]));
      }
      __syncthreads();
      if (threadIdx.x == 0) m.chi[l + 1] = r;
      __syncthreads();
      env_left(c, l);
      if (l + 1 < L - 1) TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, l + 1, 0, 0, m.site(l + 1), r * kD * chr, +tau));
      last_two = true;
    } else {
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, l, 0, 0, m.site(l), chl * kD * chb, -tau));
      const int k = qr_right(c, m, l);
      env_left(c, l);
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 0, l + 1, k, chb, c.bond, k * chb, +tau));
      absorb_right(c, m, l, chb);
      last_two = false;
    }
  }
  if (!last_two) TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, L - 1, 0, 0, m.site(L - 1), m.chi[L - 1] * kD * m.chi[L], -tau));
  last_two = false;
  for (int l = L - 1; l >= 1; --l) {
    const int chl = m.chi[l - 1], chb = m.chi[l], chr = m.chi[l + 1];
    if (chb < P->chi_max) {
      blk_gemm<Tc>(chl * kD, kD * chr, chb, matA(m.site(l - 1), chb, 1), matB(m.site(l), kD * chr, 1), c.theta,
                   kD * chr, 1, c.gsm);
      const int n = chl * kD * kD * chr;
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 2, l - 1, chl, chr, c.theta, n, -tau));
      const int nn = svd_of(c, chl * kD, kD * chr, c.theta, kD * chr, 1);
      const int r = trunc_rank(c, nn);
      cx<Tc>* A = m.site(l - 1);
      cx<Tc>* B = m.site(l);
      const int rows = chl * kD, cols = kD * chr;
      for (long long e = threadIdx.x; e < (long long)r * cols; e += TJM_THREADS) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        B[e] = cvt<Tc>(conj(c.dv[(long long)i * cols + j]));
      }
      for (long long e = threadIdx.x; e < (long long)rows * r; e += TJM_THREADS) {
        const int i = (int)(e / r), j = (int)(e % r);
        A[e] = cvt<Tc>((Td)c.ds[j] * c.du[(long long)j * rows + i]);
      }
      __syncthreads();
      if (threadIdx.x == 0) m.chi[l] = r;
      __syncthreads();
      env_right(c, l);
      if (l - 1 > 0) TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, l - 1, 0, 0, m.site(l - 1), chl * kD * r, +tau));
      last_two = true;
    } else {
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, l, 0, 0, m.site(l), chb * kD * chr, -tau));
      const int k = rq_left(c, m, l);
      env_right(c, l);
      TJM_TIMED(c, PH_LANCZOS, lanczos(c, 0, l, chb, k, c.bond, chb * k, +tau));
      absorb_left(c, m, l, chb);
      last_two = false;
    }
  }
  if (!last_two) TJM_TIMED(c, PH_LANCZOS, lanczos(c, 1, 0, 0, 0, m.site(0), m.chi[0] * kD * m.chi[1], -tau));
  if (threadIdx.x == 0) atomicAdd(&c.S->stats.env_updates, (unsigned long long)(2 * (L - 1)));
}

// ------------------------------------------------------------------ local 2x2 blocks
// For a state with centre at site 0 and sites 1..L-1 right-canonical:
// G[l][t][s] = sum conj(M_l[a',t,b]) E_l[a',a] M_l[a,s,b] with E_l the left
// transfer matrix of sites 0..l-1 (E_0 = 1).  Then <psi|O_l|psi> =
// sum_ts O[t][s] G[l][t][s] and <psi|psi> = G[l][0][0] + G[l][1][1].
//
// With two_site, also G2[l][(t1 t2)][(s1 s2)] = sum conj(Th[a',t1,t2,b]) (E_l Th)[a',s1,s2,b] for the
// sites l flagged in site_has2, Th = M_l M_{l+1} (sites l+2.. are right-canonical), so that
// <psi|O_{l,l+1}|psi> = sum O[(t1 t2)][(s1 s2)] G2[l][(t1 t2)][(s1 s2)].
template <class Tc, class Td>
__device__ __noinline__ void local_blocks(const Ctx<Tc, Td>& c, const Mps<Tc>& m, bool two_site = false) {
  const int L = c.P->L;
  if (threadIdx.x == 0) c.E[0] = mk((Tc)1, (Tc)0);
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    const int chl = m.chi[l], chr = m.chi[l + 1];
    const cx<Tc>* M = m.site(l);
    // F[a'][(s b)] = E[a'][a] M[a][(s b)]
    TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl, kD * chr, chl, matA(c.E, chl, 1), matB(M, kD * chr, 1), c.F, kD * chr, 1, c.gsm));
    // G[t][s] = sum_(a' b) conj(M[a'][t][b]) F[a'][s][b]
    cx<Tc> g[4] = {czero<Tc>(), czero<Tc>(), czero<Tc>(), czero<Tc>()};
    for (int e = threadIdx.x; e < chl * chr; e += TJM_THREADS) {
      const int a = e / chr, b = e % chr;
      const cx<Tc> m0 = M[(a * kD) * chr + b], m1 = M[(a * kD + 1) * chr + b];
      const cx<Tc> f0 = c.F[(a * kD) * chr + b], f1 = c.F[(a * kD + 1) * chr + b];
      cfma_cj(g[0], m0, f0); cfma_cj(g[1], m0, f1); cfma_cj(g[2], m1, f0); cfma_cj(g[3], m1, f1);
    }
    for (int q = 0; q < 4; ++q) {
      const double gx = warp_sum((double)g[q].x), gy = warp_sum((double)g[q].y);
      if ((threadIdx.x & 31) == 0) {
        c.red[(2 * q) * TJM_WARPS + (threadIdx.x >> 5)] = gx;
        c.red[(2 * q + 1) * TJM_WARPS + (threadIdx.x >> 5)] = gy;
      }
    }
    blk_sums_finish(8, c.red, c.sc + 448);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4; ++q) c.G[(long long)l * 4 + q] = mk(c.sc[448 + 2 * q], c.sc[448 + 2 * q + 1]);
    if (two_site && l + 1 < L && c.P->site_has2[l]) {
      const int chm = m.chi[l + 1], chn = m.chi[l + 2];
      const cx<Tc>* N = m.site(l + 1);
      // Th[(a s1), (s2 b)] = M_l[(a s1), c] M_{l+1}[c, (s2 b)];  T[a', (s1 s2 b)] = E[a', a] Th[a, (s1 s2 b)]
      TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl * kD, kD * chn, chm, matA(M, chm, 1), matB(N, kD * chn, 1), c.theta,
                                         kD * chn, 1, c.gsm));
      TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chl, kD * kD * chn, chl, matA(c.E, chl, 1), matB(c.theta, kD * kD * chn, 1),
                                         c.tmp, kD * kD * chn, 1, c.gsm));
      cx<Tc> h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) h[q] = czero<Tc>();
      for (int e = threadIdx.x; e < chl * chn; e += TJM_THREADS) {
        const int a = e / chn, b = e % chn;
        cx<Tc> th[4], tt[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          th[p] = c.theta[((long long)a * 4 + p) * chn + b];
          tt[p] = c.tmp[((long long)a * 4 + p) * chn + b];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) cfma_cj(h[p * 4 + q], th[p], tt[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const double hx = warp_sum((double)h[q].x), hy = warp_sum((double)h[q].y);
        if ((threadIdx.x & 31) == 0) {
          c.red[(2 * q) * TJM_WARPS + (threadIdx.x >> 5)] = hx;
          c.red[(2 * q + 1) * TJM_WARPS + (threadIdx.x >> 5)] = hy;
        }
      }
      blk_sums_finish(32, c.red, c.sc + 448);
      if (threadIdx.x < 16)
        c.G2[(long long)l * 16 + threadIdx.x] = mk(c.sc[448 + 2 * threadIdx.x], c.sc[448 + 2 * threadIdx.x + 1]);
      __syncthreads();
    }
    // E'[b'][b] = sum_(a' s) conj(M[a'][s][b']) F[a'][s][b]
    if (l + 1 < L)
      TJM_TIMED(c, PH_GEMM, blk_gemm<Tc>(chr, chr, chl * kD, matA(M, 1, chr, 1), matB(c.F, chr, 1), c.E, chr, 1, c.gsm));
    __syncthreads();
  }
}

template <class Tc, class Td>
__device__ void measure(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int row) {
  const ProbDev* P = c.P;
  local_blocks(c, m, P->n_obs2 > 0);
  double* out = c.S->out + (long long)row * P->n_cols;
  for (int o = threadIdx.x; o < P->n_obs; o += TJM_THREADS) {
    const int l = P->osite[o];
    const cx<double>* op = P->oop + 4 * o;
    const cx<double>* g = c.G + 4 * (long long)l;
    cx<double> v = czero<double>();
    for (int q = 0; q < 4; ++q) cfma(v, op[q], g[q]);
    out[o] = v.x / (g[0].x + g[3].x);
  }
  for (int o = threadIdx.x; o < P->n_obs2; o += TJM_THREADS) {
    const int l = P->osite2[o];
    const cx<double>* op = P->oop2 + 16 * o;
    const cx<double>* g2 = c.G2 + 16 * (long long)l;
    const cx<double>* g = c.G + 4 * (long long)l;
    cx<double> v = czero<double>();
    for (int q = 0; q < 16; ++q) cfma(v, op[q], g2[q]);
    out[P->n_obs + o] = v.x / (g[0].x + g[3].x);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ projection error
// eps = ||(I - P) H psi|| of 1TDVP at the normalised state m (Sec. "Error measures"), for an MPO with
// nearest-neighbour terms, where the two-site tangent projector P2 already reproduces H psi:
//   eps^2 = ||P2 H psi||^2 - ||P1 H psi||^2
//         = sum_l ||H2_l Theta_l||^2 - sum_{0<l<L-1} ||H1_l A_l||^2 - sum_l ||H1_l A_l||^2 + sum_l ||H0_l C_l||^2
// with A_l the centre tensor, C_l the bond matrix and Theta_l = A_l B_{l+1} of the mixed-canonical form
// centred at l (the tangent projectors are sums of orthogonal parts, so their squared norms add).  One
// left-to-right sweep with QR steps; m must be right-canonical with its centre at site 0 and is left
// left-canonical (same state).  Uses the trajectory's environment arrays; the shifted MPO (H - E I) has
// the same projection error, since psi lies in the tangent space, and keeps the sums small.
template <class Tc, class Td>
__device__ __noinline__ double projection_error(const Ctx<Tc, Td>& c0, const Mps<Tc>& m) {
  Ctx<Tc, Td> c = c0;
  c.mps = m;
  const int L = c.P->L;
  if (threadIdx.x == 0) { c.Renv(L)[0] = mk((Tc)1, (Tc)0); c.Lenv(0)[0] = mk((Tc)1, (Tc)0); }
  __syncthreads();
  for (int l = L - 1; l >= 1; --l) env_right(c, l);
  double s1 = 0.0, s1i = 0.0, s2 = 0.0, s0 = 0.0;
  for (int l = 0; l < L; ++l) {
    const int chl = m.chi[l], chr = m.chi[l + 1];
    heff1(c, l, m.site(l), c.w);
    const double n1 = blk_nrm2sq(c.w, chl * kD * chr, c.red);
    s1 += n1;
    if (l > 0 && l < L - 1) s1i += n1;
    if (l + 1 < L) {
      const int chn = m.chi[l + 2];
      blk_gemm<Tc>(chl * kD, kD * chn, chr, matA(m.site(l), chr, 1), matB(m.site(l + 1), kD * chn, 1), c.theta,
                   kD * chn, 1, c.gsm);
      heff2(c, l, chl, chn, c.theta, c.w);
      s2 += blk_nrm2sq(c.w, chl * kD * kD * chn, c.red);
      const int k = qr_right(c, m, l);
      env_left(c, l);
      heff0(c, l + 1, k, chr, c.bond, c.w);
      s0 += blk_nrm2sq(c.w, k * chr, c.red);
      absorb_right(c, m, l, chr);
    }
  }
  const double e2 = s2 - s1i - s1 + s0;
  return e2 > 0.0 ? sqrt(e2) : 0.0;
}

// ------------------------------------------------------------------ dissipation + jump
// Phi <- J_eps(D[tau] Phi) for the MPS m (Sec. "Dissipative contraction",
// Sec. "Stochastic jump process"); same readings as the oracle:
// D during a right-to-left RQ sweep (centre -> 0, dp = 1 - ||M_0||^2);
// jump iff u1 < dp; weights gamma_m <L_m^dag L_m>; smallest m (site-major)
// with u2 * sum(w) < cumsum; sqrt(gamma) L_m applied; QR sweep to the right,
// then right-to-left SVD sweep truncating every bond; normalise.
// Returns false on a numerical failure (non-positive or non-finite norm).
template <class Tc, class Td>
__device__ __noinline__ bool dissipate_jump(const Ctx<Tc, Td>& c, const Mps<Tc>& m, const cx<double>* Dops, double u1, double u2) {
  const ProbDev* P = c.P;
  const int L = P->L;
  for (int l = L - 1; l >= 0; --l) {
    blk_site_op(m.site(l), m.chi[l], m.chi[l + 1], Dops + 4 * l, mk(1.0, 0.0));
    if (l > 0) {
      const int chold = m.chi[l];
      rq_left(c, m, l);
      absorb_left(c, m, l, chold);
    }
  }
  const double n2 = blk_nrm2sq(m.site(0), m.chi[0] * kD * m.chi[1], c.red);
  if (!(n2 > 0.0) || !(n2 < 1e300)) return false;
  const double dp = 1.0 - n2;
  if (threadIdx.x == 0) {
    const double mg = fabs(u1 - dp);
    double* mm1 = &c.S->stats.min_margin1;
    if (mg < *mm1) *mm1 = mg;
  }
  if (!(u1 < dp)) {
    blk_scale(m.site(0), m.chi[0] * kD * m.chi[1], mk(1.0 / sqrt(n2), 0.0));
    __syncthreads();
    return true;
  }
  // weights from the local 2x2 blocks of the current (centre-0) state
  local_blocks(c, m);
  __shared__ int pick_sh;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int j = 0; j < P->n_jumps; ++j) {
      const cx<double>* g = c.G + 4 * (long long)P->jsite[j];
      const cx<double>* q = P->jLdL + 4 * j;
      cx<double> v = czero<double>();
      for (int t = 0; t < 4; ++t) cfma(v, q[t], g[t]);
      c.wts[j] = P->jgamma[j] * v.x;
      tot += c.wts[j];
    }
    const double target = u2 * tot;
    double cum = 0.0, mg = 1e300;
    int pick = P->n_jumps - 1;
    bool found = false;
    for (int j = 0; j < P->n_jumps; ++j) {
      cum += c.wts[j];
      mg = fmin(mg, fabs(target - cum));
      if (!found && target < cum) { pick = j; found = true; }
    }
    mg /= tot;
    if (mg < c.S->stats.min_margin2) c.S->stats.min_margin2 = mg;
    c.S->stats.jumps += 1;
    pick_sh = pick;
  }
  __syncthreads();
  const int pk = pick_sh;
  const int s = P->jsite[pk];
  blk_site_op(m.site(s), m.chi[s], m.chi[s + 1], P->jop + 4 * pk, mk(sqrt(P->jgamma[pk]), 0.0));
  for (int l = 0; l < L - 1; ++l) {
    const int chold = m.chi[l + 1];
    qr_right(c, m, l);
    absorb_right(c, m, l, chold);
  }
  for (int l = L - 1; l >= 1; --l) {
    const int chl = m.chi[l], chr = m.chi[l + 1];
    const int cols = kD * chr;
    cx<Tc>* M = m.site(l);
    const int nn = svd_of(c, chl, cols, M, cols, 1);
    const int r = trunc_rank(c, nn);
    // M_l <- V^H[:r] (r x cols); bond = U[:, :r] diag(s) (chl x r)
    for (long long e = threadIdx.x; e < (long long)r * cols; e += TJM_THREADS) {
      const int i = (int)(e / cols), j = (int)(e % cols);
      M[e] = cvt<Tc>(conj(c.dv[(long long)i * cols + j]));
    }
    for (long long e = threadIdx.x; e < (long long)chl * r; e += TJM_THREADS) {
      const int i = (int)(e / r), j = (int)(e % r);
      c.bond[e] = cvt<Tc>((Td)c.ds[j] * c.du[(long long)j * chl + i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) m.chi[l] = r;
    __syncthreads();
    absorb_left(c, m, l, chl);
  }
  const double n0 = blk_nrm2sq(m.site(0), m.chi[0] * kD * m.chi[1], c.red);
  if (!(n0 > 0.0) || !(n0 < 1e300)) return false;
  blk_scale(m.site(0), m.chi[0] * kD * m.chi[1], mk(1.0 / sqrt(n0), 0.0));
  __syncthreads();
  return true;
}

}  // namespace tjm

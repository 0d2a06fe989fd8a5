// The persistent trajectory kernel: each CTA repeatedly takes the next slot
// (one trajectory) from an atomic counter and advances it through the tensor
// jump method's time steps (Sec. "Algorithm"):
//   Phi_0 = J(D[dt/2] Psi(0));  for j >= 1:  X = U[dt] Phi_{j-1},
//   Psi(j dt) = J'(D[dt/2] X) measured on a copy (branch 1),
//   Phi_j = J(D[dt] X) (branch 0) while j < n.
#pragma once
#include "tjm_algo.cuh"

// CTAs per SM the register allocation must allow (2: at most 128 registers per thread).
#ifndef TJM_MIN_BLOCKS
#define TJM_MIN_BLOCKS 2
#endif

namespace tjm {

// Byte offsets of the per-CTA scratch; the same arithmetic runs on the host
// (to size the allocation) and on the device (to carve it).
struct ScratchMap {
  long long krylov, w, t1, t2, theta, tmp, bond, E, F, xsites, xchi;
  long long da, du, dv, dvw, drd, dtau, ds, iw, G, G2, wts, wcsr, total;
};

__host__ __device__ inline long long align256(long long x) { return (x + 255) & ~255LL; }

// row-sparse MPO block of a fused matvec when the tensor cores own the shared
// staging area: values (<= 32 x 32 complex), columns and row pointers
constexpr long long kWcsrBytes = 32 * 32 * 16 + 32 * 32 * 4 + 33 * 4;

__host__ __device__ inline ScratchMap scratch_map(const ScratchDims& d, int szc, int szd) {
  // szc / szd: bytes of one complex element in the contraction / decomposition precision
  ScratchMap m;
  const long long chi = d.chi_cap, n2 = 4 * chi * chi, cap_site = 2 * chi * chi, mm = 2 * chi;
  long long o = 0;
  auto take = [&](long long bytes) { const long long r = o; o = align256(o + bytes); return r; };
  m.krylov = take((long long)d.kmax * n2 * szc);
  m.w = take(n2 * szc);
  m.t1 = take(chi * d.Dmax * 4 * chi * szc);
  m.t2 = take(chi * d.Dmax * 4 * chi * szc);
  m.theta = take(n2 * szc);
  m.tmp = take(n2 * szc);
  m.bond = take(chi * chi * szc);
  m.E = take(chi * chi * szc);
  m.F = take(2 * chi * chi * szc);
  m.xsites = take((long long)d.Lmax * cap_site * szc);
  m.xchi = take((long long)(d.Lmax + 1) * 4);
  m.da = take(mm * mm * szd);
  m.du = take(mm * mm * szd);
  m.dv = take(mm * mm * szd);
  m.dvw = take((mm * mm + 2 * mm) * szd);
  m.drd = take(mm * szd);
  m.dtau = take(mm * szd);
  m.ds = take(mm * szd);
  m.iw = take(2 * mm * 4);
  m.G = take((long long)d.Lmax * 4 * 16);
  m.G2 = take((long long)d.Lmax * 16 * 16);
  m.wts = take((long long)(d.jmax + 1) * 8);
  m.wcsr = take(kWcsrBytes);
  m.total = o;
  return m;
}

// Dynamic shared memory, in this order: reduction scratch (4 KB), scalars
// (4 KB), the CUDA-core GEMM staging area (32 KB) and, for FP32 contractions,
// 64 KB more plus 1 KB of singular values.  The 96 KB from the GEMM staging
// area on are the tensor cores' operand stages when they run the
// contractions; the 64 KB part is also the factorization workspace of an
// FP32 QR / SVD (up to 128 x 64 complex), which never runs while a GEMM is in
// flight.  FP64 contractions use the first 40 KB only and leave the rest of
// the SM's L1 to cache their global workspaces.
constexpr int kSmemRedOff = 0;
constexpr int kSmemGsmOff = 8192;
constexpr int kSmemFsmOff = kSmemGsmOff + kSmemGemm;
constexpr int kFsmBytes = 65536;
constexpr int kSmemFsvOff = kSmemFsmOff + kFsmBytes;
static_assert(kSmemFsvOff - kSmemGsmOff >= tc::kSmemBytes, "tensor-core stages fit the GEMM and factorization areas");
// Dynamic shared memory of a launch: the 96 KB tensor-core / FP32-factorization area only when it
// is used, so that an FP64 / double-float factorization launch on the CUDA cores leaves the rest
// of the SM's L1 to cache its global workspace.
template <class Tc, class Td> constexpr int smem_bytes(bool use_tc) {
  return (sizeof(Tc) == 4 && (use_tc || sizeof(Td) == 4)) ? kSmemFsvOff + 1024 : kSmemFsmOff;
}

template <class Tc, class Td>
__device__ void make_ctx(Ctx<Tc, Td>& c, SlotDev* S, char* scr, const ScratchDims& dims, char* smem) {
  const ScratchMap mp = scratch_map(dims, (int)sizeof(cx<Tc>), (int)sizeof(cx<Td>));
  c.P = S->prob;
  c.S = S;
  c.mps.base = reinterpret_cast<cx<Tc>*>(S->sites);
  c.mps.cap = S->cap_site;
  c.mps.chi = S->chi;
  c.xmps.base = reinterpret_cast<cx<Tc>*>(scr + mp.xsites);
  c.xmps.cap = S->cap_site;
  c.xmps.chi = reinterpret_cast<int*>(scr + mp.xchi);
  c.envL = reinterpret_cast<cx<Tc>*>(S->envL);
  c.envR = reinterpret_cast<cx<Tc>*>(S->envR);
  c.cap_env = S->cap_env;
  c.krylov = reinterpret_cast<cx<Tc>*>(scr + mp.krylov);
  c.w = reinterpret_cast<cx<Tc>*>(scr + mp.w);
  c.t1 = reinterpret_cast<cx<Tc>*>(scr + mp.t1);
  c.t2 = reinterpret_cast<cx<Tc>*>(scr + mp.t2);
  c.theta = reinterpret_cast<cx<Tc>*>(scr + mp.theta);
  c.tmp = reinterpret_cast<cx<Tc>*>(scr + mp.tmp);
  c.bond = reinterpret_cast<cx<Tc>*>(scr + mp.bond);
  c.E = reinterpret_cast<cx<Tc>*>(scr + mp.E);
  c.F = reinterpret_cast<cx<Tc>*>(scr + mp.F);
  c.da = reinterpret_cast<cx<Td>*>(scr + mp.da);
  c.du = reinterpret_cast<cx<Td>*>(scr + mp.du);
  c.dv = reinterpret_cast<cx<Td>*>(scr + mp.dv);
  c.dvw = reinterpret_cast<cx<Td>*>(scr + mp.dvw);
  c.drd = reinterpret_cast<cx<Td>*>(scr + mp.drd);
  c.dtau = reinterpret_cast<Td*>(scr + mp.dtau);
  c.ds = reinterpret_cast<Td*>(scr + mp.ds);
  c.iw = reinterpret_cast<int*>(scr + mp.iw);
  c.G = reinterpret_cast<cx<double>*>(scr + mp.G);
  c.G2 = reinterpret_cast<cx<double>*>(scr + mp.G2);
  c.wts = reinterpret_cast<double*>(scr + mp.wts);
  c.wcsr = scr + mp.wcsr;
  c.gsm = smem + kSmemGsmOff;
  c.red = reinterpret_cast<double*>(smem + kSmemRedOff);
  c.sc = c.red + 512;
  if (sizeof(Td) == 4) {
    c.fsm = smem + kSmemFsmOff;
    c.fsm_bytes = kFsmBytes;
    c.fsv = smem + kSmemFsvOff;
  } else {
    c.fsm = nullptr;
    c.fsm_bytes = 0;
    c.fsv = nullptr;
  }
}

template <class Tc, class Td>
__device__ void copy_mps(const Ctx<Tc, Td>& c, const Mps<Tc>& dst, const Mps<Tc>& src) {
  const int L = c.P->L;
  for (int l = threadIdx.x; l <= L; l += TJM_THREADS) dst.chi[l] = src.chi[l];
  for (int l = 0; l < L; ++l) {
    const int n = src.chi[l] * kD * src.chi[l + 1];
    blk_copy(dst.site(l), src.site(l), n);
  }
  __syncthreads();
}

// Bring the MPS held in the slot to right-canonical form with the centre at
// site 0 (RQ sweep) and normalise it.
template <class Tc, class Td>
__device__ bool canonicalise(const Ctx<Tc, Td>& c) {
  const int L = c.P->L;
  const Mps<Tc>& m = c.mps;
  for (int l = L - 1; l >= 1; --l) {
    const int chold = m.chi[l];
    rq_left(c, m, l);
    absorb_left(c, m, l, chold);
  }
  const double n2 = blk_nrm2sq(m.site(0), m.chi[0] * kD * m.chi[1], c.red);
  if (!(n2 > 0.0) || !(n2 < 1e300)) return false;
  blk_scale(m.site(0), m.chi[0] * kD * m.chi[1], mk(1.0 / sqrt(n2), 0.0));
  __syncthreads();
  return true;
}

// Observables of the state m into output row `row`, then, if requested, the
// projection error of 1TDVP at m in the row's last column.  The error sweep
// changes the gauge, so it runs on the sampling copy (made here when m is the
// trajectory's own state) after the observables are taken.
template <class Tc, class Td>
__device__ void measure_row(const Ctx<Tc, Td>& c, const Mps<Tc>& m, int row) {
  measure(c, m, row);
  if (!c.P->proj_err) return;
  const Mps<Tc>* pm = &m;
  if (m.base == c.mps.base) {
    copy_mps(c, c.xmps, c.mps);
    pm = &c.xmps;
  }
  double eps;
  TJM_TIMED(c, PH_MEASURE, eps = projection_error(c, *pm));
  if (threadIdx.x == 0) c.S->out[(long long)row * c.P->n_cols + c.P->n_cols - 1] = eps;
  __syncthreads();
}

// Load the initial MPS, then canonicalise it.
template <class Tc, class Td>
__device__ bool init_state(const Ctx<Tc, Td>& c) {
  const int L = c.P->L;
  const Mps<Tc>& m = c.mps;
  for (int l = threadIdx.x; l <= L; l += TJM_THREADS) m.chi[l] = c.S->init_chi[l];
  __syncthreads();
  long long off = 0;
  for (int l = 0; l < L; ++l) {
    const int n = m.chi[l] * kD * m.chi[l + 1];
    cx<Tc>* dst = m.site(l);
    for (int i = threadIdx.x; i < n; i += TJM_THREADS) dst[i] = cvt<Tc>(c.S->init[off + i]);
    off += n;
  }
  __syncthreads();
  return canonicalise(c);
}

// The sampling layer and the main-branch jump of step j (Eq. SimulationStep):
// measure J'(D[dt/2] X) on a copy if j is an output step, then
// Phi_j = J(D[dt] X) while j < n.  X is the slot's MPS on entry.
//
// First-order baseline (trotter_order 1): Phi_j = J(D[dt] X) for every j, and
// Psi(j dt) = Phi_j is measured directly.
template <class Tc, class Td>
__device__ bool finish_step(const Ctx<Tc, Td>& c, int j, bool sample) {
  const ProbDev* P = c.P;
  SlotDev* S = c.S;
  bool ok = true;
  if (P->trotter_order == 1) {
    double u1, u2;
    tjm_uniforms(S->seed, S->traj_id, (uint32_t)j, 0, &u1, &u2);
    TJM_TIMED(c, PH_DJ, ok = dissipate_jump(c, c.mps, P->Dfull, u1, u2));
    if (ok && sample && P->sample_row[j] >= 0) TJM_TIMED(c, PH_MEASURE, measure_row(c, c.mps, P->sample_row[j]));
    if (ok && j < P->n_steps) TJM_TIMED(c, PH_ENVBUILD, build_right_envs(c));
    return ok;
  }
  if (sample && P->sample_row[j] >= 0) {
    copy_mps(c, c.xmps, c.mps);
    double u1, u2;
    tjm_uniforms(S->seed, S->traj_id, (uint32_t)j, 1, &u1, &u2);
    TJM_TIMED(c, PH_DJ, ok = dissipate_jump(c, c.xmps, P->Dhalf, u1, u2));
    if (ok) TJM_TIMED(c, PH_MEASURE, measure_row(c, c.xmps, P->sample_row[j]));
  }
  if (ok && j < P->n_steps) {
    double u1, u2;
    tjm_uniforms(S->seed, S->traj_id, (uint32_t)j, 0, &u1, &u2);
    TJM_TIMED(c, PH_DJ, ok = dissipate_jump(c, c.mps, P->Dfull, u1, u2));
    if (ok) TJM_TIMED(c, PH_ENVBUILD, build_right_envs(c));
  }
  return ok;
}

// max_steps >= 0: advance by up to max_steps whole time steps.
// max_steps == -1: apply only U[dt] of the next step (X = U Phi).
// max_steps == -2: apply only the main-branch D[dt] and J of a step whose
//                  U[dt] was applied by a -1 call (no sampling layer).
template <class Tc, class Td>
__device__ void run_slot(SlotDev* S, int max_steps, char* scr, const ScratchDims& dims, char* smem) {
  Ctx<Tc, Td> c;
  make_ctx(c, S, scr, dims, smem);
  const ProbDev* P = c.P;
  if (S->status != 0) return;
  if (threadIdx.x == 0) gemm_tile_rule = P->gemm_rule;
  __syncthreads();
  int step = S->step;
  int flags = S->flags;
  bool ok = true;
  if (step < 0) {
    const long long t_init = clock64();
    ok = init_state(c);
    if (ok && P->sample_row[0] >= 0) measure_row(c, c.mps, P->sample_row[0]);
    if (ok && P->n_steps > 0) {
      if (P->trotter_order != 1) {      // F_0 = J(D[dt/2] .) of the Strang-split method
        double u1, u2;
        tjm_uniforms(S->seed, S->traj_id, 0, 0, &u1, &u2);
        ok = dissipate_jump(c, c.mps, P->Dhalf, u1, u2);
      }
      if (ok) build_right_envs(c);
    }
    step = 0;
    flags = 0;
    if (threadIdx.x == 0) S->stats.cyc[PH_INIT] += (unsigned long long)(clock64() - t_init);
  } else if (flags & 1) {
    ok = canonicalise(c);
    if (ok) build_right_envs(c);
    flags &= ~1;
  }
  if (ok && max_steps == -1 && !(flags & 2) && step < P->n_steps) {
    TJM_TIMED(c, PH_TDVP, tdvp_sweep(c, 0.5 * P->dt));
    flags |= 2;
  } else if (ok && max_steps == -2 && (flags & 2)) {
    ok = finish_step(c, step + 1, false);
    step += 1;
    flags &= ~2;
  } else if (ok && max_steps >= 0) {
    int done = 0;
    if ((flags & 2) && done < max_steps) {
      ok = finish_step(c, step + 1, true);
      step += 1;
      flags &= ~2;
      ++done;
    }
    while (ok && step < P->n_steps && done < max_steps) {
      const int j = step + 1;
      TJM_TIMED(c, PH_TDVP, tdvp_sweep(c, 0.5 * P->dt));
      ok = finish_step(c, j, true);
      step = j;
      ++done;
    }
  }
  __syncthreads();
  if (tc_ctl.failed) ok = false;     // a bounded tensor-core wait ran out: results are not trustworthy
  if (threadIdx.x == 0) {
    S->step = step;
    S->flags = flags;
    if (!ok) S->status = 3;
  }
  __syncthreads();
}

// Built with TJM_TENSOR_CORES = 1 and tc_min_work > 0: FP32 contractions of at
// least that many complex multiply-adds run on the tensor cores (tcgen05) and
// the CTA holds its tensor-memory accumulator for the whole persistent launch;
// FP64 contractions never do.  kTensorCores keeps the two builds' kernels
// apart by name; the tensor-core build runs one CTA per SM anyway, so it is
// not held to the two-CTA register budget.
template <class Tc, class Td, int kTensorCores = TJM_TENSOR_CORES>
__global__ void __launch_bounds__(TJM_THREADS, kTensorCores ? 1 : TJM_MIN_BLOCKS)
advance_kernel(SlotDev* const* order, int n_slots, int* next, int max_steps, char* scratch, long long stride,
               ScratchDims dims, long long tc_min_work) {
  extern __shared__ __align__(TJM_TENSOR_CORES ? 1024 : 16) char smem[];
  __shared__ int sid;
  char* scr = scratch + (long long)blockIdx.x * stride;
#if TJM_TENSOR_CORES
  tc::cta_setup(&tc_ctl, sizeof(Tc) == 4 && tc_min_work > 0, tc_min_work);
#else
  if (threadIdx.x == 0) {
    tc_ctl.enabled = 0;
    tc_ctl.failed = 0;
    tc_ctl.min_work = 0;
  }
  __syncthreads();
#endif
  for (;;) {
    if (threadIdx.x == 0) sid = atomicAdd(next, 1);
    __syncthreads();
    const int s = sid;
    __syncthreads();
    if (s >= n_slots) break;
    run_slot<Tc, Td>(order[s], max_steps, scr, dims, smem);
  }
#if TJM_TENSOR_CORES
  tc::cta_teardown(&tc_ctl);
#endif
}

}  // namespace tjm

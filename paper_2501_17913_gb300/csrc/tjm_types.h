// Device-side descriptors shared by the host runtime and the kernels.
// Plain C layout: every pointer is a device pointer.
#pragma once
#include <stdint.h>

namespace tjm {

template <class T> struct cx;

// One problem: H as an MPO, the jump operators, dt, chi_max, truncation,
// observables and the output schedule (TJM Sec. "Initialization").
struct ProbDev {
  int L, chi_max, exact, krylov_max;
  int shift_ok;        // MPO in finite-state form: a constant can ride on the on-site channel
  int gemm_rule;       // GEMM tile rule of this run's slots (0: 64x64 tiles; 1: 32x32 for small outputs)
  int n_jumps, n_obs, n_steps, n_samples;
  double dt, trunc_eps, krylov_tol;
  const int* Dbond;                       // [L + 1] MPO bond dimensions
  const cx<double>* Wm1; const long long* Wm1_off;   // per site: [(t v)][(w s)]
  const cx<double>* WmR; const long long* WmR_off;   // per site: [(w t)][(s v)]
  const cx<double>* W12; const long long* W12_off;   // per bond l: [(t1 t2 v)][(w s1 s2)]
  const cx<double>* Dhalf;                // [L][4]  D_l[dt/2]
  const cx<double>* Dfull;                // [L][4]  D_l[dt]
  const int* jsite;                       // [n_jumps], site-major order
  const cx<double>* jop;                  // [n_jumps][4]
  const cx<double>* jLdL;                 // [n_jumps][4]  L^dag L
  const double* jgamma;                   // [n_jumps]
  const int* osite;                       // [n_obs]
  const cx<double>* oop;                  // [n_obs][4]
  const int* sample_row;                  // [n_steps + 1] -> output row or -1
  // two-site observables on (osite2, osite2 + 1), written after the one-site ones in each output row
  int n_obs2;
  const int* osite2;                      // [n_obs2]
  const cx<double>* oop2;                 // [n_obs2][16], row (t1 t2), column (s1 s2)
  const int* site_has2;                   // [L]: 1 if some two-site observable starts at the site
  int trotter_order;                      // 2: the Strang-split TJM; 1: the first-order baseline
  int proj_err;                           // 1: the last output column is the 1TDVP projection error
  int n_cols;                             // output columns: n_obs + n_obs2 + proj_err
};

struct SlotStats {
  unsigned long long mv_heff1, mv_heff2, mv_heff0, env_updates, krylov_capped, jumps;
  double min_margin1, min_margin2;
  double flops_contract;   // real flops of the tensor contractions (8 per complex multiply-add)
  double flops_decomp;     // real flops of the QR / SVD factorizations (Jacobi: per rotation applied)
  unsigned long long cyc[12];   // SM cycles by phase, see tjm_phase
};

// Phases timed with clock64() by thread 0 of the CTA owning a slot.
enum tjm_phase {
  PH_GEMM = 0, PH_WAPPLY = 1, PH_LANCZOS = 2, PH_QR = 3, PH_SVD = 4, PH_DJ = 5, PH_MEASURE = 6, PH_TDVP = 7,
  PH_ENVBUILD = 8, PH_EXPM = 9, PH_MATVEC = 10, PH_INIT = 11
};

// One trajectory.
struct SlotDev {
  const ProbDev* prob;
  unsigned long long traj_id, seed;
  int step;            // -1: not started; j: F_0..F_j done (Phi_j held)
  int status;          // 0 ok, 3 numeric failure
  int chi_cap;
  int flags;           // bit 0: state loaded from outside (canonicalise, rebuild envs)
                       // bit 1: U[dt] of step+1 applied, X held (phase-wise stepping)
  double eshift;       // energy per site subtracted from H (a global phase; keeps FP32 sums small)
  void* sites;         // [L][cap_site] complex Tc
  int* chi;            // [L + 1]
  void* envL;          // [L + 1][cap_env]
  void* envR;          // [L + 1][cap_env]
  long long cap_site, cap_env;
  double* out;         // [n_samples][n_obs]
  const cx<double>* init;   // initial MPS, packed site tensors
  const int* init_chi;      // [L + 1]
  SlotStats stats;
};

// Per-CTA scratch sizing (elements); identical arithmetic on host and device.
struct ScratchDims {
  int chi_cap, Dmax, kmax, Lmax, jmax;
};

}  // namespace tjm

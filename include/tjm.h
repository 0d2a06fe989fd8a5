/*
 * tjm.h -- C ABI of the batched tensor-jump-method library for GB300 (sm_103a).
 *
 * The library simulates Lindblad dynamics (arXiv:2501.17913, Eq. Lindblad)
 * by many independent Monte-Carlo wave-function trajectories, each held as a
 * matrix product state and advanced by the tensor jump method (TJM): the
 * dissipative contraction D (Sec. "Dissipative contraction"), the stochastic
 * jump process J (Sec. "Stochastic jump process") and the dynamic one-/two-
 * site TDVP U (Sec. "Dynamic TDVP"), in the Strang order of Eq.
 * TimeEvolutionFunctions with the sampling MPS of Eq. SimulationStep.  All
 * trajectories of a run advance together on one GPU.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) pairs of doubles, row-major.
 *   - Physical dimension d = 2 (spin-1/2 chains); other d give TJM_EINVAL.
 *   - All pointers are HOST pointers.  Inputs are copied during the call; the
 *     caller keeps ownership of every buffer it passes.  The library owns all
 *     device memory and releases it in tjm_run_free / tjm_destroy.
 *   - Every call returns a tjm_status and never aborts the process; the text
 *     of the last error of a context is available from tjm_last_error.
 *   - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef TJM_H
#define TJM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tjm_ctx tjm_ctx;
typedef int tjm_status;

enum {
  TJM_OK = 0,
  TJM_EINVAL = 1,     /* invalid argument (sizes, shapes, times off the dt grid, ...) */
  TJM_ENOMEM = 2,     /* device memory exhausted */
  TJM_ENUMERIC = 3,   /* at least one trajectory hit a non-finite or zero norm */
  TJM_ETIMEOUT = 4,   /* a bounded wait gave up (tjm_wait) */
  TJM_EBUSY = 5,      /* the run is still executing (tjm_poll) */
  TJM_EINTERNAL = 6,  /* library bug or inconsistent state */
  TJM_ECUDA = 7       /* a CUDA runtime call failed; see tjm_last_error */
};

/* Arithmetic of the GPU path (the precision plan: contractions in FP32, the
 * QR/SVD truncations, norms, jump probabilities and Lanczos coefficients in
 * FP64).
 *   FP64        everything in double (the plain FP64 baseline).
 *   FP32        tensor contractions and Krylov vectors in complex FP32 with
 *               FP32 accumulation; QR and SVD in native FP64; norms, jump
 *               weights, Lanczos coefficients and expectation values
 *               accumulated in FP64.
 *   FP32_DEC32  as FP32 but QR and SVD in FP32, in shared memory, with
 *               compensated FP32 reductions in the Jacobi SVD and a
 *               Gram-Schmidt pass that keeps the factors orthonormal to FP32
 *               working precision (a stated-error mode).
 *   FP32_DF64   (default) as FP32 with QR and SVD in emulated FP64:
 *               double-float numbers (pairs of FP32 carrying a 48-bit
 *               significand) on the FP32 pipes.  GB300 executes 2 native FP64
 *               FMAs per clock per SM against 128 FP32 FMAs; the emulation
 *               gives the FP64 factorizations about 3x the native rate with
 *               results equal to native FP64 to ~1e-11 relative. */
enum { TJM_PREC_FP64 = 0, TJM_PREC_FP32 = 1, TJM_PREC_FP32_DEC32 = 2, TJM_PREC_FP32_DF64 = 3 };

/* Hamiltonian H0 as a matrix product operator (Methods, Sec. "Matrix product
 * (density) operators"; Sec. "Initialization" item 2).  D[0..L] are the MPO
 * bond dimensions with D[0] = D[L] = 1, D[b] <= 8.  W packs the site tensors
 * one after the other; site l is [D[l]][D[l+1]][d][d] with the first physical
 * index the output (bra) index:  H0 = sum prod_l W_l[w_l][w_{l+1}][t_l][s_l] |t><s|. */
typedef struct {
  int L;
  int d;
  const int* D;
  const double* W;
} tjm_mpo;

/* A single-site jump operator L_m acting on `site` with coupling rate gamma_m
 * (Eq. Lindblad; Sec. "Initialization" item 3).  op is 2x2, row-major. */
typedef struct {
  int site;
  double rate;
  double op[8];
} tjm_jump;

/* A single-site observable O on `site` (Eq. TJMExpVal); the library returns
 * Re <Psi|O|Psi> per trajectory. */
typedef struct {
  int site;
  double op[8];
} tjm_observable;

/* A two-site observable O on (site, site + 1), e.g. the nearest-neighbour
 * correlator X (x) X of Fig. 4b: 4 x 4 complex, row-major, row index
 * (t1 t2) and column index (s1 s2) with `site` the more significant.  The
 * library returns Re <Psi|O|Psi> per trajectory. */
typedef struct {
  int site;
  double op[32];
} tjm_observable2;

/* Initial state Psi(0) (Sec. "Initialization" item 1). */
enum { TJM_STATE_ZERO = 0, TJM_STATE_PRODUCT = 1, TJM_STATE_PRODUCT_PER_TRAJ = 2, TJM_STATE_MPS = 3 };
typedef struct {
  int kind;
  /* PRODUCT: [L][d] complex, one state for all trajectories.
   * PRODUCT_PER_TRAJ: [n_traj][L][d] complex.
   * MPS: packed site tensors, site l is [chi[l]][d][chi[l+1]] complex. */
  const double* data;
  const int* chi;     /* MPS only: bond dimensions [L + 1], chi[0] = chi[L] = 1 */
} tjm_state;

typedef struct {
  int precision;        /* TJM_PREC_*; default TJM_PREC_FP32_DF64 */
  int krylov_max;       /* Lanczos iterations per exponential, <= 30; default 30 */
  double krylov_tol;    /* Lanczos a-posteriori error tolerance; default 1e-12 (FP64) / 1e-7 (FP32) */
  int exact_full_bond;  /* 1: pad product states to full bond dimension, never truncate */
  int device;           /* CUDA device ordinal; default 0 */
  int max_ctas;         /* 0: one resident wave of CTAs; else an upper bound */
  int energy_shift;     /* 1 (default): evolve with H - E*I, E the trajectory's energy at the start of
                         * each step, when H is in finite-state form (identity strings in the first
                         * and last MPO channels).  A constant shift only changes the global phase,
                         * so observables are unchanged; it keeps the FP32 environment sums near
                         * zero instead of near the extensive energy.  0: evolve with H as given. */
  int tile_rule;        /* initial GEMM tile rule of new runs (see tjm_run_set_tile_rule); default 0 */
  int tensor_cores;     /* 0 (default): every contraction runs on the CUDA cores (FMA, round-to-nearest
                         * accumulation).  1: FP32 contractions of at least tc_min_work complex
                         * multiply-adds run on the tensor cores (tcgen05, TF32 inputs split hi + lo,
                         * "3xTF32", FP32 accumulation in tensor memory).  Measured on GB300: that
                         * accumulation truncates (a sum of 320 positive products comes out low by about
                         * 3e-6 relative, the CUDA-core sum is unbiased), which a trajectory whose jump
                         * draw falls near a threshold turns into an O(1) difference from its FP64
                         * trajectory; and a kernel that holds the tcgen05 path is resident at one CTA per
                         * SM instead of two, which made it slower on the trajectory workloads measured.
                         * FP64 contractions always use the CUDA cores. */
  int trotter_order;    /* 2 (default): the Strang-split TJM with its sampling layer (Sec. "Higher-order
                         * Trotterization", Eq. SimulationStep).  1: the first-order baseline the paper
                         * compares with (Fig. 4a, dotted): Phi_j = J(D[dt] U[dt] Phi_{j-1}) from
                         * Phi_0 = Psi(0), and Psi(j dt) = Phi_j is measured directly. */
  int projection_error; /* 1: every output row gets one more column, the projection error of 1TDVP
                         * ||(I - P) H |Psi>|| at the measured state (Sec. "Error measures"), computed by
                         * a diagnostic sweep that uses the two-site tangent space (exact for MPOs with
                         * nearest-neighbour terms).  Default 0. */
  int64_t tc_min_work;  /* with tensor_cores: the smallest GEMM, in complex multiply-adds, that goes to the
                         * tensor cores (smaller ones stay on the CUDA cores); 0 = 16384 */
} tjm_options;

/* Fill opts with the defaults above. */
void tjm_default_options(tjm_options* opts);

/* tjm_create -- define one TJM problem (Sec. "Initialization" items 2-6).
 *   H        Hamiltonian MPO (L >= 2).
 *   jumps    n_jumps single-site jump operators with rates >= 0 (may be 0 jumps).
 *   dt       time step > 0;  chi_max >= 1 maximum bond dimension (<= 64);
 *   trunc_eps relative discarded weight allowed per SVD truncation (>= 0).
 *   opts     may be NULL for the defaults.
 * The dissipators D_l[dt/2], D_l[dt] of Eq. DissipativeMPO and the MPO layouts
 * used by the kernels are prepared here and copied to the device.
 * On success *out owns the context; release it with tjm_destroy. */
tjm_status tjm_create(tjm_ctx** out, const tjm_mpo* H, const tjm_jump* jumps, int n_jumps, double dt, int chi_max,
                      double trunc_eps, const tjm_options* opts);

/* tjm_run -- start N = n_traj trajectories with global ids
 * first_traj .. first_traj + n_traj - 1, from psi0, recording the n_obs
 * observables at the n_times times (strictly increasing multiples of dt,
 * including 0 if wanted; T = times[n_times-1] sets n = T/dt steps).
 * Trajectory i draws its random numbers from Philox4x32-10 with
 * key = seed and counter = (global id, step, branch), so results do not depend
 * on how trajectories are batched or sharded.  Asynchronous: returns after the
 * launch.  *run_id identifies the run for the calls below. */
tjm_status tjm_run(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                   const tjm_observable* obs, int n_obs, const double* times, int n_times, int64_t* run_id);

/* tjm_run_prepare -- as tjm_run but launches nothing: allocates and uploads
 * the run so that tjm_run_advance can move it forward step by step. */
tjm_status tjm_run_prepare(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                           const tjm_observable* obs, int n_obs, const double* times, int n_times, int64_t* run_id);

/* tjm_run_prepare2 / tjm_run2 -- as tjm_run_prepare / tjm_run with two-site
 * observables as well: every output row holds the n_obs one-site values
 * followed by the n_obs2 two-site values (results then have n_obs + n_obs2
 * columns in tjm_result).  A two-site observable needs site + 1 < L. */
tjm_status tjm_run_prepare2(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                            const tjm_observable* obs, int n_obs, const tjm_observable2* obs2, int n_obs2,
                            const double* times, int n_times, int64_t* run_id);
tjm_status tjm_run2(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                    const tjm_observable* obs, int n_obs, const tjm_observable2* obs2, int n_obs2, const double* times,
                    int n_times, int64_t* run_id);

/* tjm_run_advance -- launch one persistent kernel that moves every trajectory
 * of the run forward by at most max_steps time steps (the first call also
 * performs the initialisation and F_0).  Asynchronous.
 * max_steps = -1 applies only U[dt] of the next step; max_steps = -2 then
 * applies only that step's main-branch D[dt] and J (no sampling layer):
 * phase-wise stepping for inspecting the sub-steps with tjm_run_get_state. */
tjm_status tjm_run_advance(tjm_ctx* ctx, int64_t run_id, int max_steps);

/* tjm_run_group_advance -- one persistent kernel over the trajectories of
 * several runs (possibly of different contexts on the same device), each
 * moved forward by at most max_steps steps.  Work is ordered by estimated
 * cost (largest first).  Launched on the stream of ctxs[0]; asynchronous (the
 * work list lives in ctxs[0] and is refilled in stream order). */
tjm_status tjm_run_group_advance(tjm_ctx* const* ctxs, const int64_t* run_ids, int n_runs, int max_steps);

/* tjm_scratch_bytes -- device bytes of the per-CTA scratch that a launch of
 * this context's precision holds for trajectories of up to chi_cap and L
 * sites (all resident CTAs together); it is allocated at the first launch
 * that needs it and kept by the context.  For admission control by memory. */
tjm_status tjm_scratch_bytes(const tjm_ctx* ctx, int chi_cap, int L, int64_t* bytes);

/* tjm_resident_ctas -- CTAs (trajectories in flight) of one launch of this context: the resident wave
 * the occupancy of its kernel allows on this device, before the max_ctas cap (two per SM for the
 * CUDA-core builds, one per SM for the tensor-core build).  0 for a null context. */
int tjm_resident_ctas(const tjm_ctx* ctx);

/* tjm_poll -- TJM_OK if the run's device work has finished, TJM_EBUSY if not. */
tjm_status tjm_poll(tjm_ctx* ctx, int64_t run_id);

/* tjm_wait -- bounded host wait for the run's device work (its last launch):
 * TJM_OK once finished, TJM_ETIMEOUT if it is still executing after timeout_s
 * seconds (the work continues; wait or poll again later).  No device code
 * waits on anything, so this host wait is the only wait that needs a bound.
 * TJM_EINVAL for a negative timeout or an unknown run. */
tjm_status tjm_wait(tjm_ctx* ctx, int64_t run_id, double timeout_s);

/* tjm_result -- wait for the run and copy results.
 *   mean, sem  [n_times][n_obs]: trajectory average and standard error of the
 *              mean (Eq. TJMExpVal), may be NULL.
 *   per_traj   [n_traj][n_times][n_obs], may be NULL.
 * Returns TJM_ENUMERIC (results still copied) if any trajectory failed
 * numerically; tjm_run_stats reports how many. */
tjm_status tjm_result(tjm_ctx* ctx, int64_t run_id, double* mean, double* sem, double* per_traj);

typedef struct {
  int64_t n_traj, steps_done_min, steps_done_max, failed;
  uint64_t matvec_one_site, matvec_two_site, matvec_bond, env_updates, krylov_capped, jumps;
  double min_margin_jump, min_margin_pick;   /* closest |u - threshold| over all jump decisions */
  int64_t final_bond_sum;                    /* sum over trajectories and bonds of the bond dimension */
  int64_t final_bond_max;
  double flops_contract;                     /* real flops of all tensor contractions (8 per complex MAC) */
  double flops_decomp;                       /* real flops of the QR / SVD factorizations */
  uint64_t cycles[12];                       /* SM cycles summed over trajectories, by phase: GEMM, MPO
                                                contraction, Lanczos, QR, SVD, dissipation+jump, measurement,
                                                TDVP sweep, environment build, Krylov exponential, matvec
                                                inside Lanczos, initialisation */
} tjm_stats;

/* tjm_run_stats -- work counters of a run (waits for the run). */
tjm_status tjm_run_stats(tjm_ctx* ctx, int64_t run_id, tjm_stats* out);

/* tjm_run_margins -- per-trajectory smallest distance between a uniform and
 * its decision threshold (jump / pick), [n_traj] each; may be NULL. */
tjm_status tjm_run_margins(tjm_ctx* ctx, int64_t run_id, double* margin_jump, double* margin_pick);

/* tjm_run_bonds -- current bond dimensions of every trajectory of the run,
 * [n_traj][L + 1] ints (waits for the run). */
tjm_status tjm_run_bonds(tjm_ctx* ctx, int64_t run_id, int* chi);

/* tjm_run_get_state -- copy trajectory `traj` (0-based within the run) of a
 * run: its completed step count, bond dimensions chi [L + 1] and site tensors
 * packed as in tjm_state (site l is [chi[l]][d][chi[l+1]] complex; data must
 * hold sum_l chi[l]*d*chi[l+1] complex numbers, at most L*d*64*64).  The
 * state is the sampling MPS Phi_j after step j (Sec. "Algorithm").
 * TJM_EBUSY (nothing copied) while the trajectory sits between the halves of
 * a phase-wise step (after tjm_run_advance(-1), before -2): it then holds
 * X = U[dt] Phi_j, which is not a state a run can resume from. */
tjm_status tjm_run_get_state(tjm_ctx* ctx, int64_t run_id, int64_t traj, int* step, int* chi, double* data);

/* tjm_run_set_state -- overwrite trajectory `traj` of a run with an MPS in
 * the layout of tjm_run_get_state and mark it as having completed `step`
 * steps (checkpoint / resume).  The next advance brings the state to
 * right-canonical form, normalises it and rebuilds its environments; random
 * numbers continue from step + 1, so a resumed run reproduces the
 * uninterrupted one. */
tjm_status tjm_run_set_state(tjm_ctx* ctx, int64_t run_id, int64_t traj, int step, const int* chi,
                             const double* data);

/* tjm_run_set_tile_rule -- GEMM tile rule for this run's later launches:
 * 0 (default) 64 x 64 output tiles everywhere; 1 32 x 32 tiles for products
 * with an output dimension <= 32 (small bonds, chain ends).  Both compute the
 * same contractions (results differ only by summation order).  The choice is
 * made by the host autotuner (paper_2501_17913_gb300/autotune.py) from timed
 * launches; it is not from the paper.  Blocks until the setting is on the
 * device; TJM_EINVAL for another rule or an unknown run. */
tjm_status tjm_run_set_tile_rule(tjm_ctx* ctx, int64_t run_id, int rule);

/* tjm_run_status -- per-trajectory status, [n_traj] (TJM_OK or TJM_ENUMERIC;
 * a failed trajectory stops advancing and keeps its last good outputs). */
tjm_status tjm_run_status(tjm_ctx* ctx, int64_t run_id, int* status);

/* tjm_run_free -- release the device memory of a run. */
tjm_status tjm_run_free(tjm_ctx* ctx, int64_t run_id);

/* The CUDA stream (cudaStream_t) all work of this context is issued on. */
void* tjm_stream(tjm_ctx* ctx);

/* Block the host until all work of the context has finished. */
tjm_status tjm_sync(tjm_ctx* ctx);

void tjm_destroy(tjm_ctx* ctx);
const char* tjm_last_error(const tjm_ctx* ctx);

/* Number of kernels launched so far by this context (for launch accounting). */
int64_t tjm_launch_count(const tjm_ctx* ctx);

/* ------------------------------------------------------------------------
 * Kernel-level self tests: one CTA runs one building block of the trajectory
 * kernel on one small problem.  Matrices are row-major complex interleaved;
 * double_precision selects the FP32 (0), FP64 (1) or double-float emulated
 * FP64 (2) instantiation.  They allocate their own device memory and
 * synchronise the device.
 * ---------------------------------------------------------------------- */

/* Householder QR of A (m x n, m, n <= 256): Q (m x k) with orthonormal
 * columns, R (k x n) upper triangular, A = Q R, k = min(m, n).  Moves the
 * MPS orthogonality centre (Methods, Sec. "Matrix product states"). */
tjm_status tjm_selftest_qr(int double_precision, int m, int n, const double* A, double* Q, double* R);

/* One-sided Jacobi SVD of A (m x n): U (m x nn), S (nn, descending),
 * V (n x nn), A = U diag(S) V^H, nn = min(m, n); columns of U belonging to
 * exactly-zero singular values are completed to an orthonormal set.  Used for
 * the truncations of Sec. "1TDVP and 2TDVP as tensor networks". */
tjm_status tjm_selftest_svd(int double_precision, int m, int n, const double* A, double* U, double* S, double* V);

/* C = op(A) op(B) on the tensor cores (tcgen05, TF32 inputs with the 3xTF32
 * split, FP32 accumulation in tensor memory), one CTA: the complex GEMM of
 * the effective-Hamiltonian and environment contractions (Fig. 2 networks).
 * A is M x K and B is K x N, row-major complex doubles rounded to FP32 on the
 * device; conj_a / conj_b conjugate them; a_col_major / b_k_contig store the
 * operands transposed on the device first, so both access patterns of the
 * GEMM are exercised.  C (M x N) is returned as doubles.  M, N, K <= 1024.
 * TJM_ETIMEOUT if the kernel's bounded wait for the tensor cores ran out. */
tjm_status tjm_selftest_tc_cgemm(int M, int N, int K, int conj_a, int conj_b, int a_col_major, int b_k_contig,
                                 const double* A, const double* B, double* C);

/* One effective-Hamiltonian application or environment update of the
 * trajectory kernel (Fig. 2 networks; environment recursion of Sec. "Hybrid
 * strategy"), by the same device functions the sweeps call, on one CTA.
 * Layouts (complex doubles, row-major): Lenv [chl][Dl][chl] (bra, MPO, ket),
 * Renv [Dr][chr][chr] (MPO, ket, bra), W1 [Dl][Dr or Du][2][2] and W2
 * [Du][Dr][2][2] (MPO left, right, out, in).
 *   kind 0  bond:      y[chl][chr]       = sum Lenv[x,w,a] x[a,b] Renv'[w,b,y]  (Renv' is [Dl][chr][chr])
 *   kind 1  one site:  y[chl][2][chr]    = sum Lenv W1 x Renv
 *   kind 2  two sites: y[chl][2][2][chr] = sum Lenv W1 W2 x Renv
 *   kind 3  left env:  y[chr][Dr][chr]   = sum conj(x) Lenv W1 x      (x = A [chl][2][chr])
 *   kind 4  right env: y[Dl][chl][chl]   = sum x W1 Renv conj(x)      (x = B [chl][2][chr])
 * precision TJM_PREC_FP64 or TJM_PREC_FP32 (FP32 contractions; tensor_cores
 * selects tcgen05 or the CUDA cores).  chl, chr <= 64; D <= 8. */
tjm_status tjm_selftest_contract(int kind, int precision, int tensor_cores, int chl, int chr, int Dl, int Du, int Dr,
                                 const double* W1, const double* W2, const double* Lenv, const double* Renv,
                                 const double* x, double* y);

/* exp(i theta T) e_1 for the k x k (k <= 32) real symmetric tridiagonal
 * T = tridiag(beta, alpha, beta): the Lanczos exponential's small factor
 * (Sec. "1TDVP and 2TDVP as tensor networks", Lanczos method).  c: k complex. */
tjm_status tjm_selftest_expm_tridiag(int k, const double* alpha, const double* beta, double theta, double* c);

/* The (u1, u2) pair of the Philox4x32-10 stream for n (trajectory, step,
 * branch) triples under one seed -- the uniforms epsilon of Sec. "Stochastic
 * jump process" exactly as the trajectory kernel draws them. */
tjm_status tjm_selftest_philox(uint64_t seed, const uint64_t* traj, const uint32_t* step, const uint32_t* branch, int n,
                               double* u1, double* u2);

/* ------------------------------------------------------------------------
 * Allocation-free SVD (the paper has no counterpart; this is a library
 * utility).  For callers that cannot let a library allocate device memory:
 * applications whose own pool or arena allocator owns all device memory, and
 * latency-sensitive loops that must not pay for cudaMalloc/cudaFree (cudaFree
 * synchronises the whole device).
 *
 * tjm_svd_noalloc -- the same one-CTA Jacobi SVD as tjm_selftest_svd (same
 * kernel body; double_precision 0 FP32, 1 FP64, 2 double-float), with
 * DEVICE pointers: A (m x n), U (m x nn), S (nn), V (n x nn), nn = min(m, n),
 * row-major complex interleaved doubles (S real), A = U diag(S) V^H, S
 * descending.  The caller owns and provides all four buffers; the call
 * allocates nothing.  Its workspace is one static device array of about
 * 1.1 MB sized for m, n <= TJM_NOALLOC_MAX_DIM, held by every GPU that loads
 * the library until the process exits; larger m or n return TJM_EINVAL.
 * The kernel is queued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting.  The first call on each
 * device looks up the workspace's device address (cudaGetSymbolAddress with
 * that device current); make that first call before any stream capture.
 * Every call on a device shares the one workspace and leaves its contents
 * behind (nothing in it needs clearing): calls whose kernels overlap on the
 * GPU (different streams without ordering) race and corrupt each other.
 * Returns TJM_ECUDA if the launch fails, and also, without launching, if
 * a CUDA error from earlier work is already pending (that error is left in
 * place for the caller to read). */
#define TJM_NOALLOC_MAX_DIM 128
tjm_status tjm_svd_noalloc(int double_precision, int m, int n, const double* A, double* U, double* S, double* V,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TJM_H */

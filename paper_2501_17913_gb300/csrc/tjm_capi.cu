// Host runtime of the batched TJM library: problem preparation, device memory
// for runs, the persistent-kernel launches and the result path behind the C
// ABI declared in include/tjm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "tjm.h"
#include "tjm_kernels.cuh"
#include "tjm_launch.h"
#include "tjm_mpo_layout.h"

using tjm::cx;
typedef std::complex<double> zc;

namespace tjm {
// Ensemble statistics per (sample row, observable): mean and standard error
// over the trajectories of one run, two-pass, fixed summation order.
__global__ void ensemble_kernel(const SlotDev* slots, int n_traj, int n_out, double* mean, double* sem) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_out) return;
  double s = 0.0;
  for (int t = 0; t < n_traj; ++t) s += slots[t].out[e];
  const double mu = s / n_traj;
  double v = 0.0;
  for (int t = 0; t < n_traj; ++t) { const double x = slots[t].out[e] - mu; v += x * x; }
  mean[e] = mu;
  sem[e] = n_traj > 1 ? sqrt(v / (n_traj - 1) / n_traj) : 0.0;
}

}  // namespace tjm

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() { if (p) cudaFree(p); }
};

struct Run {
  int64_t n_traj = 0, first = 0;
  int L = 0, n_obs = 0, n_samples = 0, n_steps = 0, chi_cap = 0;
  std::vector<DevBuf*> bufs;
  tjm::SlotDev* slots = nullptr;     // device [n_traj]
  tjm::SlotDev** order = nullptr;    // device [n_traj] pointers, largest cost first
  tjm::ProbDev* prob = nullptr;      // device
  int* chi = nullptr;                // device [n_traj][L+1]
  double* out = nullptr;             // device [n_traj][n_samples][n_obs]
  double* mean = nullptr;            // device [n_samples][n_obs]
  double* sem = nullptr;
  int* next = nullptr;               // device counter
  cudaEvent_t done = nullptr;
  double cost = 0.0;
  ~Run() {
    for (DevBuf* b : bufs) delete b;
    if (done) cudaEventDestroy(done);
  }
};

}  // namespace

struct tjm_ctx {
  int device = 0;
  tjm_options opt;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t launches = 0;
  // problem
  int L = 0, chi_max = 0, n_jumps = 0, Dmax = 1, shift_ok = 0;
  double dt = 0, trunc_eps = 0;
  std::vector<int> Dbond;
  std::vector<zc> Wm1, WmR, W12, Dhalf, Dfull, jop, jLdL;
  std::vector<long long> Wm1_off, WmR_off, W12_off;
  std::vector<int> jsite;
  std::vector<double> jgamma;
  std::vector<std::vector<zc>> Wsite;   // raw MPO tensors
  // device copies of the problem arrays
  std::vector<DevBuf*> pbufs;
  const int* d_Dbond = nullptr;
  const cx<double>*d_Wm1 = nullptr, *d_WmR = nullptr, *d_W12 = nullptr, *d_Dhalf = nullptr, *d_Dfull = nullptr,
  *d_jop = nullptr, *d_jLdL = nullptr;
  const long long *d_Wm1_off = nullptr, *d_WmR_off = nullptr, *d_W12_off = nullptr;
  const int* d_jsite = nullptr;
  const double* d_jgamma = nullptr;
  // per-CTA scratch
  DevBuf scratch;
  long long scratch_stride = 0;
  int scratch_ctas = 0;
  tjm::ScratchDims sdims = {0, 0, 0, 0, 0};
  std::map<int64_t, std::unique_ptr<Run>> runs;
  int64_t next_run = 1;
  // work list and counter of group launches (tjm_run_group_advance), reused from launch to launch:
  // the stream orders each refill after the previous kernel that reads it
  DevBuf group_order;
  DevBuf group_next;
  ~tjm_ctx() {
    runs.clear();
    for (DevBuf* b : pbufs) delete b;
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

tjm_status fail(tjm_ctx* c, tjm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define TJM_CU(call)                                                                                \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TJM_ENOMEM : TJM_ECUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                      \
  } while (0)

template <class T>
tjm_status upload(tjm_ctx* ctx, std::vector<DevBuf*>& owner, const T* src, size_t count, T** dst) {
  DevBuf* b = new DevBuf;
  owner.push_back(b);
  b->n = std::max<size_t>(count, 1) * sizeof(T);
  TJM_CU(cudaMalloc(&b->p, b->n));
  if (count) TJM_CU(cudaMemcpy(b->p, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *dst = reinterpret_cast<T*>(b->p);
  return TJM_OK;
}

tjm_status alloc(tjm_ctx* ctx, std::vector<DevBuf*>& owner, size_t bytes, void** dst) {
  DevBuf* b = new DevBuf;
  owner.push_back(b);
  b->n = std::max<size_t>(bytes, 16);
  TJM_CU(cudaMalloc(&b->p, b->n));
  *dst = b->p;
  return TJM_OK;
}

zc cplx(const double* p) { return zc(p[0], p[1]); }

// exp(-s A) for a 2x2 Hermitian A = [[a, b], [conj(b), e]]:
// with m = (a + e)/2, r = sqrt(((a - e)/2)^2 + |b|^2) and (A - m)^2 = r^2 I,
// exp(-s A) = e^{-s m} (cosh(s r) I - sinh(s r)/r (A - m I)).
void expm_neg_herm2(const zc A[4], double s, zc out[4]) {
  const double a = A[0].real(), e = A[3].real();
  const zc b = A[1];
  const double m = 0.5 * (a + e);
  const double r = std::sqrt(0.25 * (a - e) * (a - e) + std::norm(b));
  const double em = std::exp(-s * m);
  const double ch = std::cosh(s * r);
  const double sh_r = r > 0 ? std::sinh(s * r) / r : s;
  out[0] = em * (ch - sh_r * (a - m));
  out[1] = em * (-sh_r * b);
  out[2] = em * (-sh_r * std::conj(b));
  out[3] = em * (ch - sh_r * (e - m));
}

size_t szc_of(int prec) { return prec == TJM_PREC_FP64 ? 16 : 8; }
size_t szd_of(int prec) { return prec == TJM_PREC_FP32_DEC32 ? 8 : 16; }   // df64 is 8 bytes like double

// Full bond dimension of bond b in an L-site d=2 chain.
int full_dim(int L, int b) {
  const int e = std::min(b, L - b);
  return e >= 30 ? (1 << 30) : (1 << e);
}

// Product state padded to full bond dimension, right-canonical (exact mode).
// Site l is built from a Householder reflector whose first column is
// phi_l (x) e_0, so the first basis vector of every right block is the product
// state of that block and the other rows complete an orthonormal set.
void pad_product(int L, const std::vector<zc>& phi, std::vector<zc>& data, std::vector<int>& chi) {
  chi.assign(L + 1, 1);
  for (int b = 0; b <= L; ++b) chi[b] = full_dim(L, b);
  std::vector<std::vector<zc>> sites(L);
  for (int l = L - 1; l >= 0; --l) {
    const int cr = chi[l + 1], cl = chi[l], n = 2 * cr;
    std::vector<zc> v(n, 0.0);
    double nv = std::sqrt(std::norm(phi[2 * l]) + std::norm(phi[2 * l + 1]));
    v[0 * cr + 0] = phi[2 * l] / nv;
    v[1 * cr + 0] = phi[2 * l + 1] / nv;
    // H = I - 2 u u^H / |u|^2, u = e_0 - w v with w v_0 real >= 0  =>  H e_0 = w v
    const double av0 = std::abs(v[0]);
    const zc w = av0 > 0 ? std::conj(v[0]) / av0 : zc(1.0, 0.0);
    std::vector<zc> u(n);
    for (int i = 0; i < n; ++i) u[i] = (i == 0 ? 1.0 : 0.0) - w * v[i];
    double uu = 0;
    for (int i = 0; i < n; ++i) uu += std::norm(u[i]);
    std::vector<zc> B((size_t)cl * n);
    for (int a = 0; a < cl; ++a)
      for (int i = 0; i < n; ++i) {
        zc h = (i == a ? 1.0 : 0.0);
        if (uu > 0) h -= 2.0 * u[i] * std::conj(u[a]) / uu;
        B[(size_t)a * n + i] = h;    // row a of B = column a of H
      }
    if (uu > 0)
      for (int i = 0; i < n; ++i) B[i] *= std::conj(w);   // row 0 -> exactly v
    sites[l] = B;
  }
  data.clear();
  for (int l = 0; l < L; ++l) data.insert(data.end(), sites[l].begin(), sites[l].end());
}

int resident(tjm_ctx* ctx) {
  int per_sm = 0, sms = 0;
  const int tc = ctx->opt.tensor_cores;
  switch (ctx->opt.precision) {
    case TJM_PREC_FP64: per_sm = tjm::occupancy_f64(0); break;
    case TJM_PREC_FP32_DEC32: per_sm = tc ? tjm::occupancy_f32d32_tc(1) : tjm::occupancy_f32d32(0); break;
    case TJM_PREC_FP32_DF64: per_sm = tc ? tjm::occupancy_f32df_tc(1) : tjm::occupancy_f32df(0); break;
    default: per_sm = tc ? tjm::occupancy_f32_tc(1) : tjm::occupancy_f32(0); break;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  return std::max(1, per_sm) * std::max(1, sms);
}

tjm_status ensure_scratch(tjm_ctx* ctx, const tjm::ScratchDims& need, int ctas) {
  tjm::ScratchDims d = ctx->sdims;
  d.chi_cap = std::max(d.chi_cap, need.chi_cap);
  d.Dmax = std::max(d.Dmax, need.Dmax);
  d.kmax = std::max(d.kmax, need.kmax);
  d.Lmax = std::max(d.Lmax, need.Lmax);
  d.jmax = std::max(d.jmax, need.jmax);
  const tjm::ScratchMap mp = tjm::scratch_map(d, (int)szc_of(ctx->opt.precision), (int)szd_of(ctx->opt.precision));
  if (ctx->scratch.p && mp.total <= ctx->scratch_stride && ctas <= ctx->scratch_ctas &&
      d.chi_cap == ctx->sdims.chi_cap && d.Dmax == ctx->sdims.Dmax && d.kmax == ctx->sdims.kmax &&
      d.Lmax == ctx->sdims.Lmax && d.jmax == ctx->sdims.jmax)
    return TJM_OK;
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  if (ctx->scratch.p) { cudaFree(ctx->scratch.p); ctx->scratch.p = nullptr; }
  const int nct = std::max(ctas, ctx->scratch_ctas);
  const size_t bytes = (size_t)mp.total * nct;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  if (bytes + (256ull << 20) > fr)
    return fail(ctx, TJM_ENOMEM, "scratch needs %.2f GB, %.2f GB free", bytes / 1e9, fr / 1e9);
  TJM_CU(cudaMalloc(&ctx->scratch.p, bytes));
  ctx->scratch.n = bytes;
  ctx->scratch_stride = mp.total;
  ctx->scratch_ctas = nct;
  ctx->sdims = d;
  return TJM_OK;
}

}  // namespace

extern "C" {

void tjm_default_options(tjm_options* o) {
  if (!o) return;
  o->precision = TJM_PREC_FP32_DF64;
  o->krylov_max = 30;
  o->krylov_tol = 0.0;   // 0: precision default
  o->exact_full_bond = 0;
  o->device = 0;
  o->max_ctas = 0;
  o->energy_shift = 1;
  o->tile_rule = 0;
  o->tensor_cores = 0;
  o->trotter_order = 2;
  o->projection_error = 0;
  o->tc_min_work = 0;
}

const char* tjm_last_error(const tjm_ctx* c) { return c ? c->err.c_str() : "null context"; }
void* tjm_stream(tjm_ctx* c) { return c ? (void*)c->stream : nullptr; }
int64_t tjm_launch_count(const tjm_ctx* c) { return c ? c->launches : 0; }

tjm_status tjm_create(tjm_ctx** out, const tjm_mpo* H, const tjm_jump* jumps, int n_jumps, double dt, int chi_max,
                      double trunc_eps, const tjm_options* opts) {
  if (!out || !H) return TJM_EINVAL;
  *out = nullptr;
  std::unique_ptr<tjm_ctx> hold(new tjm_ctx);
  tjm_ctx* ctx = hold.get();
  tjm_default_options(&ctx->opt);
  if (opts) ctx->opt = *opts;
  tjm_options& o = ctx->opt;
  if (o.precision < 0 || o.precision > 3) return fail(nullptr, TJM_EINVAL, "");
  if (o.tile_rule < 0 || o.tile_rule > 1) return fail(nullptr, TJM_EINVAL, "");
  if (o.tensor_cores < 0 || o.tensor_cores > 1) return fail(nullptr, TJM_EINVAL, "");
  if (o.trotter_order != 1 && o.trotter_order != 2) return fail(nullptr, TJM_EINVAL, "");
  if (o.projection_error < 0 || o.projection_error > 1) return fail(nullptr, TJM_EINVAL, "");
  if (o.tc_min_work < 0) return fail(nullptr, TJM_EINVAL, "");
  if (o.krylov_max <= 0 || o.krylov_max > 30) o.krylov_max = 30;
  if (!(o.krylov_tol > 0)) o.krylov_tol = o.precision == TJM_PREC_FP64 ? 1e-12 : 1e-7;
  const int L = H->L;
  if (L < 2 || H->d != 2 || !H->D || !H->W) return TJM_EINVAL;
  if (!(dt > 0) || chi_max < 1 || chi_max > 64 || !(trunc_eps >= 0) || n_jumps < 0 || (n_jumps && !jumps))
    return TJM_EINVAL;
  if (H->D[0] != 1 || H->D[L] != 1) return TJM_EINVAL;
  ctx->device = o.device;
  {
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return TJM_ECUDA;
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return TJM_ECUDA;
  }
  ctx->L = L;
  ctx->chi_max = chi_max;
  ctx->dt = dt;
  ctx->trunc_eps = trunc_eps;
  ctx->Dbond.assign(H->D, H->D + L + 1);
  ctx->Dmax = 1;
  for (int b = 0; b <= L; ++b) {
    if (ctx->Dbond[b] < 1 || ctx->Dbond[b] > 8) return TJM_EINVAL;
    ctx->Dmax = std::max(ctx->Dmax, ctx->Dbond[b]);
  }
  // raw MPO tensors
  const int d = 2;
  size_t off = 0;
  ctx->Wsite.resize(L);
  for (int l = 0; l < L; ++l) {
    const int Dl = ctx->Dbond[l], Dr = ctx->Dbond[l + 1];
    const size_t n = (size_t)Dl * Dr * d * d;
    ctx->Wsite[l].resize(n);
    for (size_t i = 0; i < n; ++i) ctx->Wsite[l][i] = cplx(H->W + 2 * (off + i));
    off += n;
  }
  auto Wel = [&](int l, int w, int v, int t, int s) -> zc {
    const int Dr = ctx->Dbond[l + 1];
    return ctx->Wsite[l][(((size_t)w * Dr + v) * d + t) * d + s];
  };
  // Finite-state form: channel 0 carries the identity string from the left
  // (column 0 is I in row 0 and zero below it) and the last channel carries it
  // to the right (the last row is I in the last column and zero before it).
  // Then adding -s*I to each site's entry (0, last) adds -s*L*I to H.
  ctx->shift_ok = 1;
  for (int b = 1; b < L; ++b)
    if (ctx->Dbond[b] < 2) ctx->shift_ok = 0;
  auto is_id = [&](int l, int w, int v, double scale) {
    for (int t = 0; t < d; ++t)
      for (int s = 0; s < d; ++s)
        if (Wel(l, w, v, t, s) != zc(t == s ? scale : 0.0)) return false;
    return true;
  };
  for (int l = 0; l < L && ctx->shift_ok; ++l) {
    const int Dl = ctx->Dbond[l], Dr = ctx->Dbond[l + 1];
    if (l + 1 < L)
      for (int w = 0; w < Dl; ++w)
        if (!is_id(l, w, 0, w == 0 ? 1.0 : 0.0)) ctx->shift_ok = 0;
    if (l > 0)
      for (int v = 0; v < Dr; ++v)
        if (!is_id(l, Dl - 1, v, v == Dr - 1 ? 1.0 : 0.0)) ctx->shift_ok = 0;
  }
  if (!ctx->opt.energy_shift) ctx->shift_ok = 0;
  // kernel layouts of the MPO
  {
    tjm_host::MpoLayouts lay;
    tjm_host::mpo_layouts(ctx->Dbond, ctx->Wsite, d, lay);
    ctx->Wm1 = std::move(lay.Wm1);
    ctx->WmR = std::move(lay.WmR);
    ctx->W12 = std::move(lay.W12);
    ctx->Wm1_off = std::move(lay.Wm1_off);
    ctx->WmR_off = std::move(lay.WmR_off);
    ctx->W12_off = std::move(lay.W12_off);
  }
  // jumps, site-major (stable in the caller's order), and the dissipators
  std::vector<int> idx(n_jumps);
  for (int m = 0; m < n_jumps; ++m) {
    idx[m] = m;
    if (jumps[m].site < 0 || jumps[m].site >= L || !(jumps[m].rate >= 0)) return TJM_EINVAL;
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return jumps[a].site < jumps[b].site; });
  std::vector<zc> A((size_t)L * 4, 0.0);
  for (int m : idx) {
    const tjm_jump& J = jumps[m];
    zc op[4], ldl[4];
    for (int q = 0; q < 4; ++q) op[q] = cplx(J.op + 2 * q);
    for (int t = 0; t < 2; ++t)
      for (int s = 0; s < 2; ++s) ldl[t * 2 + s] = std::conj(op[0 * 2 + t]) * op[0 * 2 + s] + std::conj(op[1 * 2 + t]) * op[1 * 2 + s];
    ctx->jsite.push_back(J.site);
    ctx->jgamma.push_back(J.rate);
    for (int q = 0; q < 4; ++q) {
      ctx->jop.push_back(op[q]);
      ctx->jLdL.push_back(ldl[q]);
      A[(size_t)J.site * 4 + q] += J.rate * ldl[q];
    }
  }
  ctx->n_jumps = n_jumps;
  ctx->Dhalf.resize((size_t)L * 4);
  ctx->Dfull.resize((size_t)L * 4);
  for (int l = 0; l < L; ++l) {
    expm_neg_herm2(&A[(size_t)l * 4], 0.25 * dt, &ctx->Dhalf[(size_t)l * 4]);   // exp(-(dt/2)/2 A)
    expm_neg_herm2(&A[(size_t)l * 4], 0.5 * dt, &ctx->Dfull[(size_t)l * 4]);    // exp(-dt/2 A)
  }
  // upload
  tjm_status st;
  auto up_c = [&](const std::vector<zc>& v, const cx<double>** dst) {
    cx<double>* p = nullptr;
    tjm_status s = upload(ctx, ctx->pbufs, reinterpret_cast<const cx<double>*>(v.data()), v.size(), &p);
    *dst = p;
    return s;
  };
  int* dD = nullptr;
  if ((st = upload(ctx, ctx->pbufs, ctx->Dbond.data(), ctx->Dbond.size(), &dD))) return st;
  ctx->d_Dbond = dD;
  if ((st = up_c(ctx->Wm1, &ctx->d_Wm1)) || (st = up_c(ctx->WmR, &ctx->d_WmR)) || (st = up_c(ctx->W12, &ctx->d_W12)) ||
      (st = up_c(ctx->Dhalf, &ctx->d_Dhalf)) || (st = up_c(ctx->Dfull, &ctx->d_Dfull)) ||
      (st = up_c(ctx->jop, &ctx->d_jop)) || (st = up_c(ctx->jLdL, &ctx->d_jLdL)))
    return st;
  long long* po = nullptr;
  if ((st = upload(ctx, ctx->pbufs, ctx->Wm1_off.data(), ctx->Wm1_off.size(), &po))) return st;
  ctx->d_Wm1_off = po;
  if ((st = upload(ctx, ctx->pbufs, ctx->WmR_off.data(), ctx->WmR_off.size(), &po))) return st;
  ctx->d_WmR_off = po;
  if ((st = upload(ctx, ctx->pbufs, ctx->W12_off.data(), ctx->W12_off.size(), &po))) return st;
  ctx->d_W12_off = po;
  int* pj = nullptr;
  if ((st = upload(ctx, ctx->pbufs, ctx->jsite.data(), ctx->jsite.size(), &pj))) return st;
  ctx->d_jsite = pj;
  double* pg = nullptr;
  if ((st = upload(ctx, ctx->pbufs, ctx->jgamma.data(), ctx->jgamma.size(), &pg))) return st;
  ctx->d_jgamma = pg;
  *out = hold.release();
  return TJM_OK;
}

static tjm_status prepare(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                          const tjm_observable* obs, int n_obs1, const tjm_observable2* obs2, int n_obs2,
                          const double* times, int n_times, int64_t* run_id) {
  if (!ctx) return TJM_EINVAL;
  if (!run_id || n_traj < 1 || n_traj > (1LL << 30) || first_traj < 0 || n_obs1 < 0 || (n_obs1 && !obs) ||
      n_obs2 < 0 || (n_obs2 && !obs2) || n_times < 1 || !times)
    return fail(ctx, TJM_EINVAL, "bad run arguments");
  // output columns: one-site observables, two-site ones, then the projection error if requested
  const int n_obs = n_obs1 + n_obs2 + (ctx->opt.projection_error ? 1 : 0);
  TJM_CU(cudaSetDevice(ctx->device));
  const int L = ctx->L;
  const double dt = ctx->dt;
  std::unique_ptr<Run> run(new Run);
  Run& R = *run;
  R.n_traj = n_traj;
  R.first = first_traj;
  R.L = L;
  R.n_obs = n_obs;
  R.n_samples = n_times;
  // output schedule
  std::vector<int> steps(n_times);
  for (int i = 0; i < n_times; ++i) {
    const double q = times[i] / dt;
    const double r = std::round(q);
    if (!(times[i] >= 0) || std::fabs(q - r) > 1e-9 * std::max(1.0, q) || (i && r <= steps[i - 1]))
      return fail(ctx, TJM_EINVAL, "times must be increasing multiples of dt");
    steps[i] = (int)r;
  }
  R.n_steps = steps.back();
  std::vector<int> sample_row(R.n_steps + 1, -1);
  for (int i = 0; i < n_times; ++i) sample_row[steps[i]] = i;
  std::vector<int> osite(n_obs1);
  std::vector<zc> oop((size_t)n_obs1 * 4);
  std::vector<int> osite2(n_obs2), has2(L, 0);
  std::vector<zc> oop2((size_t)n_obs2 * 16);
  for (int o = 0; o < n_obs2; ++o) {
    if (obs2[o].site < 0 || obs2[o].site + 1 >= L) return fail(ctx, TJM_EINVAL, "two-site observable out of range");
    osite2[o] = obs2[o].site;
    has2[obs2[o].site] = 1;
    for (int q = 0; q < 16; ++q) oop2[(size_t)o * 16 + q] = cplx(obs2[o].op + 2 * q);
  }
  for (int o = 0; o < n_obs1; ++o) {
    if (obs[o].site < 0 || obs[o].site >= L) return fail(ctx, TJM_EINVAL, "observable site out of range");
    osite[o] = obs[o].site;
    for (int q = 0; q < 4; ++q) oop[(size_t)o * 4 + q] = cplx(obs[o].op + 2 * q);
  }
  // initial states -> packed MPS blobs
  const int kind = psi0 ? psi0->kind : TJM_STATE_ZERO;
  std::vector<std::vector<zc>> blobs;
  std::vector<std::vector<int>> blob_chi;
  auto product_blob = [&](const double* p) {
    std::vector<zc> phi((size_t)2 * L);
    for (int l = 0; l < L; ++l) {
      if (p) { phi[2 * l] = cplx(p + 4 * l); phi[2 * l + 1] = cplx(p + 4 * l + 2); }
      else { phi[2 * l] = 1.0; phi[2 * l + 1] = 0.0; }
      const double nv = std::sqrt(std::norm(phi[2 * l]) + std::norm(phi[2 * l + 1]));
      if (!(nv > 0)) return false;
      phi[2 * l] /= nv; phi[2 * l + 1] /= nv;
    }
    std::vector<zc> data;
    std::vector<int> chi;
    if (ctx->opt.exact_full_bond) {
      pad_product(L, phi, data, chi);
    } else {
      data = phi;
      chi.assign(L + 1, 1);
    }
    blobs.push_back(data);
    blob_chi.push_back(chi);
    return true;
  };
  if (kind == TJM_STATE_ZERO) {
    product_blob(nullptr);
  } else if (kind == TJM_STATE_PRODUCT) {
    if (!psi0->data || !product_blob(psi0->data)) return fail(ctx, TJM_EINVAL, "bad product state");
  } else if (kind == TJM_STATE_PRODUCT_PER_TRAJ) {
    if (!psi0->data) return fail(ctx, TJM_EINVAL, "bad product states");
    for (int64_t t = 0; t < n_traj; ++t)
      if (!product_blob(psi0->data + (size_t)t * 4 * L)) return fail(ctx, TJM_EINVAL, "bad product state %lld", (long long)t);
  } else if (kind == TJM_STATE_MPS) {
    if (!psi0->data || !psi0->chi || psi0->chi[0] != 1 || psi0->chi[L] != 1 || ctx->opt.exact_full_bond)
      return fail(ctx, TJM_EINVAL, "bad MPS");
    std::vector<int> chi(psi0->chi, psi0->chi + L + 1);
    size_t n = 0;
    for (int l = 0; l < L; ++l) {
      if (chi[l + 1] < 1 || chi[l + 1] > 64) return fail(ctx, TJM_EINVAL, "MPS bond out of range");
      n += (size_t)chi[l] * 2 * chi[l + 1];
    }
    std::vector<zc> data(n);
    for (size_t i = 0; i < n; ++i) data[i] = cplx(psi0->data + 2 * i);
    blobs.push_back(data);
    blob_chi.push_back(chi);
  } else {
    return fail(ctx, TJM_EINVAL, "unknown state kind");
  }
  int chi_cap = ctx->chi_max;
  for (auto& ch : blob_chi)
    for (int x : ch) chi_cap = std::max(chi_cap, x);
  if (chi_cap > 64) return fail(ctx, TJM_EINVAL, "bond dimension above 64 (exact mode needs L <= 12)");
  R.chi_cap = chi_cap;
  const size_t szc = szc_of(ctx->opt.precision);
  const long long cap_site = 2LL * chi_cap * chi_cap;
  const long long cap_env = (long long)ctx->Dmax * chi_cap * chi_cap;
  const size_t bytes_sites = (size_t)n_traj * L * cap_site * szc;
  const size_t bytes_env = (size_t)n_traj * (L + 1) * cap_env * szc;
  {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    if (bytes_sites + 2 * bytes_env + (1ull << 30) > fr)
      return fail(ctx, TJM_ENOMEM, "run needs %.2f GB of trajectory state, %.2f GB free",
                  (bytes_sites + 2 * bytes_env) / 1e9, fr / 1e9);
  }
  tjm_status st;
  void *sites = nullptr, *envL = nullptr, *envR = nullptr, *pchi = nullptr, *pout = nullptr;
  if ((st = alloc(ctx, R.bufs, bytes_sites, &sites)) || (st = alloc(ctx, R.bufs, bytes_env, &envL)) ||
      (st = alloc(ctx, R.bufs, bytes_env, &envR)) ||
      (st = alloc(ctx, R.bufs, (size_t)n_traj * (L + 1) * sizeof(int), &pchi)) ||
      (st = alloc(ctx, R.bufs, (size_t)n_traj * n_times * std::max(n_obs, 1) * sizeof(double), &pout)))
    return st;
  R.chi = (int*)pchi;
  R.out = (double*)pout;
  TJM_CU(cudaMemset(R.out, 0, (size_t)n_traj * n_times * std::max(n_obs, 1) * sizeof(double)));
  std::vector<const cx<double>*> d_blob(blobs.size());
  std::vector<const int*> d_bchi(blobs.size());
  for (size_t b = 0; b < blobs.size(); ++b) {
    cx<double>* p = nullptr;
    if ((st = upload(ctx, R.bufs, reinterpret_cast<const cx<double>*>(blobs[b].data()), blobs[b].size(), &p))) return st;
    d_blob[b] = p;
    int* q = nullptr;
    if ((st = upload(ctx, R.bufs, blob_chi[b].data(), blob_chi[b].size(), &q))) return st;
    d_bchi[b] = q;
  }
  // problem descriptor of this run
  tjm::ProbDev P;
  std::memset(&P, 0, sizeof P);
  P.L = L; P.shift_ok = ctx->shift_ok; P.gemm_rule = ctx->opt.tile_rule; P.chi_max = ctx->chi_max; P.exact = ctx->opt.exact_full_bond; P.krylov_max = ctx->opt.krylov_max;
  P.n_jumps = ctx->n_jumps; P.n_obs = n_obs1; P.n_obs2 = n_obs2; P.n_steps = R.n_steps; P.n_samples = n_times;
  P.trotter_order = ctx->opt.trotter_order;
  P.proj_err = ctx->opt.projection_error ? 1 : 0;
  P.n_cols = n_obs;
  P.dt = dt; P.trunc_eps = ctx->trunc_eps; P.krylov_tol = ctx->opt.krylov_tol;
  P.Dbond = ctx->d_Dbond;
  P.Wm1 = ctx->d_Wm1; P.Wm1_off = ctx->d_Wm1_off;
  P.WmR = ctx->d_WmR; P.WmR_off = ctx->d_WmR_off;
  P.W12 = ctx->d_W12; P.W12_off = ctx->d_W12_off;
  P.Dhalf = ctx->d_Dhalf; P.Dfull = ctx->d_Dfull;
  P.jsite = ctx->d_jsite; P.jop = ctx->d_jop; P.jLdL = ctx->d_jLdL; P.jgamma = ctx->d_jgamma;
  {
    int* p = nullptr;
    if ((st = upload(ctx, R.bufs, osite.data(), osite.size(), &p))) return st;
    P.osite = p;
    cx<double>* q = nullptr;
    if ((st = upload(ctx, R.bufs, reinterpret_cast<const cx<double>*>(oop.data()), oop.size(), &q))) return st;
    P.oop = q;
    int* s = nullptr;
    if ((st = upload(ctx, R.bufs, sample_row.data(), sample_row.size(), &s))) return st;
    P.sample_row = s;
    int* p2 = nullptr;
    if ((st = upload(ctx, R.bufs, osite2.data(), osite2.size(), &p2))) return st;
    P.osite2 = p2;
    cx<double>* q2 = nullptr;
    if ((st = upload(ctx, R.bufs, reinterpret_cast<const cx<double>*>(oop2.data()), oop2.size(), &q2))) return st;
    P.oop2 = q2;
    int* h2 = nullptr;
    if ((st = upload(ctx, R.bufs, has2.data(), has2.size(), &h2))) return st;
    P.site_has2 = h2;
  }
  if ((st = upload(ctx, R.bufs, &P, 1, &R.prob))) return st;
  // slots
  std::vector<tjm::SlotDev> hs((size_t)n_traj);
  for (int64_t t = 0; t < n_traj; ++t) {
    tjm::SlotDev& S = hs[(size_t)t];
    std::memset(&S, 0, sizeof S);
    S.prob = R.prob;
    S.traj_id = (unsigned long long)(first_traj + t);
    S.seed = seed;
    S.step = -1;
    S.status = 0;
    S.chi_cap = chi_cap;
    S.sites = (char*)sites + (size_t)t * L * cap_site * szc;
    S.chi = R.chi + (size_t)t * (L + 1);
    S.envL = (char*)envL + (size_t)t * (L + 1) * cap_env * szc;
    S.envR = (char*)envR + (size_t)t * (L + 1) * cap_env * szc;
    S.cap_site = cap_site;
    S.cap_env = cap_env;
    S.out = R.out + (size_t)t * n_times * n_obs;
    const size_t b = blobs.size() == 1 ? 0 : (size_t)t;
    S.init = d_blob[b];
    S.init_chi = d_bchi[b];
    S.stats.min_margin1 = 1e300;
    S.stats.min_margin2 = 1e300;
  }
  if ((st = upload(ctx, R.bufs, hs.data(), hs.size(), &R.slots))) return st;
  std::vector<tjm::SlotDev*> ord((size_t)n_traj);
  for (int64_t t = 0; t < n_traj; ++t) ord[(size_t)t] = R.slots + t;
  if ((st = upload(ctx, R.bufs, ord.data(), ord.size(), &R.order))) return st;
  void *pm = nullptr, *ps = nullptr, *pn = nullptr;
  if ((st = alloc(ctx, R.bufs, (size_t)n_times * std::max(n_obs, 1) * sizeof(double), &pm)) ||
      (st = alloc(ctx, R.bufs, (size_t)n_times * std::max(n_obs, 1) * sizeof(double), &ps)) ||
      (st = alloc(ctx, R.bufs, sizeof(int) * 4, &pn)))
    return st;
  R.mean = (double*)pm;
  R.sem = (double*)ps;
  R.next = (int*)pn;
  TJM_CU(cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming));
  R.cost = (double)L * chi_cap * chi_cap * chi_cap * (R.n_steps + 1);
  const int64_t id = ctx->next_run++;
  ctx->runs[id] = std::move(run);
  *run_id = id;
  return TJM_OK;
}

int tjm_resident_ctas(const tjm_ctx* ctx) { return ctx ? resident(const_cast<tjm_ctx*>(ctx)) : 0; }

tjm_status tjm_scratch_bytes(const tjm_ctx* ctx, int chi_cap, int L, int64_t* bytes) {
  if (!ctx || !bytes || chi_cap < 1 || chi_cap > 64 || L < 1) return TJM_EINVAL;
  tjm::ScratchDims d = {chi_cap, ctx->Dmax, ctx->opt.krylov_max, L, ctx->n_jumps};
  const tjm::ScratchMap mp = tjm::scratch_map(d, (int)szc_of(ctx->opt.precision), (int)szd_of(ctx->opt.precision));
  *bytes = (int64_t)mp.total * resident(const_cast<tjm_ctx*>(ctx));
  return TJM_OK;
}

tjm_status tjm_run_prepare(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                           const tjm_observable* obs, int n_obs, const double* times, int n_times, int64_t* run_id) {
  return prepare(ctx, psi0, n_traj, first_traj, seed, obs, n_obs, nullptr, 0, times, n_times, run_id);
}

tjm_status tjm_run_prepare2(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                            const tjm_observable* obs, int n_obs, const tjm_observable2* obs2, int n_obs2,
                            const double* times, int n_times, int64_t* run_id) {
  return prepare(ctx, psi0, n_traj, first_traj, seed, obs, n_obs, obs2, n_obs2, times, n_times, run_id);
}

static Run* find_run(tjm_ctx* ctx, int64_t id) {
  auto it = ctx->runs.find(id);
  return it == ctx->runs.end() ? nullptr : it->second.get();
}

static tjm_status launch(tjm_ctx* ctx, tjm::SlotDev* const* order, int n, int* next, int max_steps,
                         const tjm::ScratchDims& need) {
  int ctas = resident(ctx);
  if (ctx->opt.max_ctas > 0) ctas = std::min(ctas, ctx->opt.max_ctas);
  ctas = std::max(1, std::min(ctas, n));
  tjm_status st = ensure_scratch(ctx, need, ctas);
  if (st) return st;
  TJM_CU(cudaMemsetAsync(next, 0, sizeof(int), ctx->stream));
  const bool tc = ctx->opt.tensor_cores && ctx->opt.precision != TJM_PREC_FP64;
  const long long tc_min = tc ? (ctx->opt.tc_min_work > 0 ? ctx->opt.tc_min_work : 16384) : 0;
  using launch_fn = cudaError_t (*)(cudaStream_t, tjm::SlotDev* const*, int, int*, int, int, char*, long long,
                                    tjm::ScratchDims, long long);
  launch_fn fn;
  switch (ctx->opt.precision) {
    case TJM_PREC_FP64: fn = tjm::launch_f64; break;
    case TJM_PREC_FP32_DEC32: fn = tc ? tjm::launch_f32d32_tc : tjm::launch_f32d32; break;
    case TJM_PREC_FP32_DF64: fn = tc ? tjm::launch_f32df_tc : tjm::launch_f32df; break;
    default: fn = tc ? tjm::launch_f32_tc : tjm::launch_f32; break;
  }
  const cudaError_t e = fn(ctx->stream, order, n, next, max_steps, ctas, (char*)ctx->scratch.p, ctx->scratch_stride,
                           ctx->sdims, tc_min);
  if (e != cudaSuccess) return fail(ctx, TJM_ECUDA, "advance kernel launch: %s", cudaGetErrorString(e));
  ctx->launches += 1;
  return TJM_OK;
}

tjm_status tjm_run_advance(tjm_ctx* ctx, int64_t run_id, int max_steps) {
  if (!ctx) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R || max_steps < -2) return fail(ctx, TJM_EINVAL, "unknown run or bad step count");
  TJM_CU(cudaSetDevice(ctx->device));
  tjm::ScratchDims need = {R->chi_cap, ctx->Dmax, ctx->opt.krylov_max, R->L, ctx->n_jumps};
  tjm_status st = launch(ctx, R->order, (int)R->n_traj, R->next, max_steps, need);
  if (st) return st;
  TJM_CU(cudaEventRecord(R->done, ctx->stream));
  return TJM_OK;
}

tjm_status tjm_run_group_advance(tjm_ctx* const* ctxs, const int64_t* run_ids, int n_runs, int max_steps) {
  if (!ctxs || !run_ids || n_runs < 1 || !ctxs[0]) return TJM_EINVAL;
  tjm_ctx* ctx = ctxs[0];
  TJM_CU(cudaSetDevice(ctx->device));
  tjm::ScratchDims need = {0, 1, 1, 0, 0};
  std::vector<std::pair<double, Run*>> rs;
  int64_t total = 0;
  for (int i = 0; i < n_runs; ++i) {
    tjm_ctx* c = ctxs[i];
    if (!c || c->device != ctx->device || c->opt.precision != ctx->opt.precision)
      return fail(ctx, TJM_EINVAL, "group runs must share device and precision");
    Run* R = find_run(c, run_ids[i]);
    if (!R) return fail(ctx, TJM_EINVAL, "unknown run in group");
    need.chi_cap = std::max(need.chi_cap, R->chi_cap);
    need.Dmax = std::max(need.Dmax, c->Dmax);
    need.kmax = std::max(need.kmax, c->opt.krylov_max);
    need.Lmax = std::max(need.Lmax, R->L);
    need.jmax = std::max(need.jmax, c->n_jumps);
    rs.push_back({R->cost, R});
    total += R->n_traj;
    if (c != ctx) {
      // order the other contexts' pending work before this launch
      cudaEvent_t ev;
      TJM_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      TJM_CU(cudaEventRecord(ev, c->stream));
      TJM_CU(cudaStreamWaitEvent(ctx->stream, ev, 0));
      cudaEventDestroy(ev);
    }
  }
  std::stable_sort(rs.begin(), rs.end(), [](const std::pair<double, Run*>& a, const std::pair<double, Run*>& b) {
    return a.first > b.first;
  });
  std::vector<tjm::SlotDev*> ord;
  ord.reserve((size_t)total);
  for (auto& pr : rs)
    for (int64_t t = 0; t < pr.second->n_traj; ++t) ord.push_back(pr.second->slots + t);
  const size_t need_bytes = ord.size() * sizeof(tjm::SlotDev*);
  if (ctx->group_order.n < need_bytes) {
    // grow (rare): the old list may still be read by a kernel in flight
    TJM_CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->group_order.p) { cudaFree(ctx->group_order.p); ctx->group_order.p = nullptr; }
    const size_t bytes = std::max(need_bytes, (size_t)4096);
    TJM_CU(cudaMalloc(&ctx->group_order.p, bytes));
    ctx->group_order.n = bytes;
  }
  if (!ctx->group_next.p) {
    TJM_CU(cudaMalloc(&ctx->group_next.p, 16));
    ctx->group_next.n = 16;
  }
  // stream-ordered refill; pageable host memory is staged before the call returns, so `ord` may go
  TJM_CU(cudaMemcpyAsync(ctx->group_order.p, ord.data(), need_bytes, cudaMemcpyHostToDevice, ctx->stream));
  tjm_status st = launch(ctx, reinterpret_cast<tjm::SlotDev**>(ctx->group_order.p), (int)ord.size(),
                         reinterpret_cast<int*>(ctx->group_next.p), max_steps, need);
  if (!st) {
    for (int i = 0; i < n_runs; ++i) {
      Run* R = find_run(ctxs[i], run_ids[i]);
      cudaEventRecord(R->done, ctx->stream);
      if (ctxs[i] != ctx) cudaStreamWaitEvent(ctxs[i]->stream, R->done, 0);
    }
  }
  return st;
}

tjm_status tjm_run(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                   const tjm_observable* obs, int n_obs, const double* times, int n_times, int64_t* run_id) {
  tjm_status st = prepare(ctx, psi0, n_traj, first_traj, seed, obs, n_obs, nullptr, 0, times, n_times, run_id);
  if (st) return st;
  Run* R = find_run(ctx, *run_id);
  return tjm_run_advance(ctx, *run_id, R->n_steps + 1);
}

tjm_status tjm_run2(tjm_ctx* ctx, const tjm_state* psi0, int64_t n_traj, int64_t first_traj, uint64_t seed,
                    const tjm_observable* obs, int n_obs, const tjm_observable2* obs2, int n_obs2, const double* times,
                    int n_times, int64_t* run_id) {
  tjm_status st = prepare(ctx, psi0, n_traj, first_traj, seed, obs, n_obs, obs2, n_obs2, times, n_times, run_id);
  if (st) return st;
  Run* R = find_run(ctx, *run_id);
  return tjm_run_advance(ctx, *run_id, R->n_steps + 1);
}

tjm_status tjm_poll(tjm_ctx* ctx, int64_t run_id) {
  if (!ctx) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  const cudaError_t e = cudaEventQuery(R->done);
  if (e == cudaErrorNotReady) return TJM_EBUSY;
  if (e != cudaSuccess) return fail(ctx, TJM_ECUDA, "poll: %s", cudaGetErrorString(e));
  return TJM_OK;
}

tjm_status tjm_wait(tjm_ctx* ctx, int64_t run_id, double timeout_s) {
  if (!ctx || !(timeout_s >= 0.0)) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(R->done);
    if (e == cudaSuccess) return TJM_OK;
    if (e != cudaErrorNotReady) return fail(ctx, TJM_ECUDA, "wait: %s", cudaGetErrorString(e));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= timeout_s) return fail(ctx, TJM_ETIMEOUT, "run %lld still executing after %.3f s", (long long)run_id, el);
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

tjm_status tjm_sync(tjm_ctx* ctx) {
  if (!ctx) return TJM_EINVAL;
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  return TJM_OK;
}

static tjm_status fetch_slots(tjm_ctx* ctx, Run* R, std::vector<tjm::SlotDev>& hs) {
  TJM_CU(cudaEventSynchronize(R->done));
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  hs.resize((size_t)R->n_traj);
  TJM_CU(cudaMemcpy(hs.data(), R->slots, hs.size() * sizeof(tjm::SlotDev), cudaMemcpyDeviceToHost));
  return TJM_OK;
}

tjm_status tjm_result(tjm_ctx* ctx, int64_t run_id, double* mean, double* sem, double* per_traj) {
  if (!ctx) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  TJM_CU(cudaSetDevice(ctx->device));
  std::vector<tjm::SlotDev> hs;
  tjm_status st = fetch_slots(ctx, R, hs);
  if (st) return st;
  const int n_out = R->n_samples * R->n_obs;
  if ((mean || sem) && n_out > 0) {
    tjm::ensemble_kernel<<<(n_out + 127) / 128, 128, 0, ctx->stream>>>(R->slots, (int)R->n_traj, n_out, R->mean,
                                                                       R->sem);
    TJM_CU(cudaGetLastError());
    ctx->launches += 1;
    if (mean) TJM_CU(cudaMemcpyAsync(mean, R->mean, n_out * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (sem) TJM_CU(cudaMemcpyAsync(sem, R->sem, n_out * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (per_traj && n_out > 0)
    TJM_CU(cudaMemcpyAsync(per_traj, R->out, (size_t)R->n_traj * n_out * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  int64_t failed = 0;
  for (auto& S : hs) failed += S.status != 0;
  if (failed) return fail(ctx, TJM_ENUMERIC, "%lld trajectories failed numerically", (long long)failed);
  for (auto& S : hs)
    if (S.step < R->n_steps) return fail(ctx, TJM_EBUSY, "run not finished (advance further)");
  return TJM_OK;
}

tjm_status tjm_run_stats(tjm_ctx* ctx, int64_t run_id, tjm_stats* out) {
  if (!ctx || !out) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  std::vector<tjm::SlotDev> hs;
  tjm_status st = fetch_slots(ctx, R, hs);
  if (st) return st;
  std::memset(out, 0, sizeof *out);
  out->n_traj = R->n_traj;
  out->steps_done_min = 1LL << 40;
  out->steps_done_max = -1;
  out->min_margin_jump = 1e300;
  out->min_margin_pick = 1e300;
  for (auto& S : hs) {
    out->steps_done_min = std::min<int64_t>(out->steps_done_min, S.step);
    out->steps_done_max = std::max<int64_t>(out->steps_done_max, S.step);
    out->failed += S.status != 0;
    out->matvec_one_site += S.stats.mv_heff1;
    out->matvec_two_site += S.stats.mv_heff2;
    out->matvec_bond += S.stats.mv_heff0;
    out->env_updates += S.stats.env_updates;
    out->krylov_capped += S.stats.krylov_capped;
    out->jumps += S.stats.jumps;
    out->min_margin_jump = std::min(out->min_margin_jump, S.stats.min_margin1);
    out->min_margin_pick = std::min(out->min_margin_pick, S.stats.min_margin2);
    out->flops_contract += S.stats.flops_contract;
    out->flops_decomp += S.stats.flops_decomp;
    for (int q = 0; q < 12; ++q) out->cycles[q] += S.stats.cyc[q];
  }
  std::vector<int> chi((size_t)R->n_traj * (R->L + 1));
  TJM_CU(cudaMemcpy(chi.data(), R->chi, chi.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < chi.size(); ++i) {
    out->final_bond_sum += chi[i];
    out->final_bond_max = std::max<int64_t>(out->final_bond_max, chi[i]);
  }
  return TJM_OK;
}

tjm_status tjm_run_margins(tjm_ctx* ctx, int64_t run_id, double* m1, double* m2) {
  if (!ctx) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  std::vector<tjm::SlotDev> hs;
  tjm_status st = fetch_slots(ctx, R, hs);
  if (st) return st;
  for (size_t t = 0; t < hs.size(); ++t) {
    if (m1) m1[t] = hs[t].stats.min_margin1;
    if (m2) m2[t] = hs[t].stats.min_margin2;
  }
  return TJM_OK;
}

tjm_status tjm_run_bonds(tjm_ctx* ctx, int64_t run_id, int* chi) {
  if (!ctx || !chi) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  TJM_CU(cudaEventSynchronize(R->done));
  TJM_CU(cudaMemcpy(chi, R->chi, (size_t)R->n_traj * (R->L + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  return TJM_OK;
}

tjm_status tjm_run_get_state(tjm_ctx* ctx, int64_t run_id, int64_t traj, int* step, int* chi, double* data) {
  if (!ctx || !chi || !data) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R || traj < 0 || traj >= R->n_traj) return fail(ctx, TJM_EINVAL, "unknown run or trajectory");
  TJM_CU(cudaEventSynchronize(R->done));
  tjm::SlotDev S;
  TJM_CU(cudaMemcpy(&S, R->slots + traj, sizeof S, cudaMemcpyDeviceToHost));
  // Between the two halves of a phase-wise step (U[dt] applied, D and J not
  // yet) the held MPS is X, not a sampling MPS Phi_j: a checkpoint taken there
  // would be resumed as Phi_j and apply U[dt] twice.
  if (S.flags & 2)
    return fail(ctx, TJM_EBUSY, "trajectory %lld is between U[dt] and D/J of a step (advance -2 first)",
                (long long)traj);
  if (step) *step = S.step;
  const int L = R->L;
  TJM_CU(cudaMemcpy(chi, S.chi, (L + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  const size_t esz = szc_of(ctx->opt.precision);
  std::vector<char> buf((size_t)S.cap_site * esz);
  size_t off = 0;
  for (int l = 0; l < L; ++l) {
    const size_t n = (size_t)chi[l] * 2 * chi[l + 1];
    TJM_CU(cudaMemcpy(buf.data(), (char*)S.sites + (size_t)l * S.cap_site * esz, n * esz, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * n; ++i)
      data[2 * off + i] = esz == 16 ? reinterpret_cast<double*>(buf.data())[i] : reinterpret_cast<float*>(buf.data())[i];
    off += n;
  }
  return TJM_OK;
}

tjm_status tjm_run_set_state(tjm_ctx* ctx, int64_t run_id, int64_t traj, int step, const int* chi,
                             const double* data) {
  if (!ctx || !chi || !data) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R || traj < 0 || traj >= R->n_traj || step < 0 || step > R->n_steps)
    return fail(ctx, TJM_EINVAL, "unknown run or trajectory, or step out of range");
  const int L = R->L;
  if (chi[0] != 1 || chi[L] != 1) return fail(ctx, TJM_EINVAL, "boundary bonds must be 1");
  for (int b = 1; b < L; ++b)
    if (chi[b] < 1 || chi[b] > R->chi_cap) return fail(ctx, TJM_EINVAL, "bond %d out of range", b);
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  tjm::SlotDev S;
  TJM_CU(cudaMemcpy(&S, R->slots + traj, sizeof S, cudaMemcpyDeviceToHost));
  TJM_CU(cudaMemcpy(S.chi, chi, (L + 1) * sizeof(int), cudaMemcpyHostToDevice));
  const size_t esz = szc_of(ctx->opt.precision);
  std::vector<char> buf((size_t)S.cap_site * esz);
  size_t off = 0;
  for (int l = 0; l < L; ++l) {
    const size_t n = (size_t)chi[l] * 2 * chi[l + 1];
    for (size_t i = 0; i < 2 * n; ++i) {
      if (esz == 16) reinterpret_cast<double*>(buf.data())[i] = data[2 * off + i];
      else reinterpret_cast<float*>(buf.data())[i] = (float)data[2 * off + i];
    }
    TJM_CU(cudaMemcpy((char*)S.sites + (size_t)l * S.cap_site * esz, buf.data(), n * esz, cudaMemcpyHostToDevice));
    off += n;
  }
  S.step = step;
  S.flags = 1;
  S.status = 0;
  TJM_CU(cudaMemcpy(R->slots + traj, &S, sizeof S, cudaMemcpyHostToDevice));
  return TJM_OK;
}

tjm_status tjm_run_status(tjm_ctx* ctx, int64_t run_id, int* status) {
  if (!ctx || !status) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  std::vector<tjm::SlotDev> hs;
  tjm_status st = fetch_slots(ctx, R, hs);
  if (st) return st;
  for (size_t t = 0; t < hs.size(); ++t) status[t] = hs[t].status;
  return TJM_OK;
}

tjm_status tjm_run_set_tile_rule(tjm_ctx* ctx, int64_t run_id, int rule) {
  if (!ctx) return TJM_EINVAL;
  Run* R = find_run(ctx, run_id);
  if (!R) return fail(ctx, TJM_EINVAL, "unknown run");
  if (rule < 0 || rule > 1) return fail(ctx, TJM_EINVAL, "tile rule must be 0 or 1");
  cudaSetDevice(ctx->device);
  // stream-ordered: launches issued after this call see the new rule
  TJM_CU(cudaMemcpyAsync(reinterpret_cast<char*>(R->prob) + offsetof(tjm::ProbDev, gemm_rule), &rule, sizeof rule,
                         cudaMemcpyHostToDevice, ctx->stream));
  TJM_CU(cudaStreamSynchronize(ctx->stream));
  return TJM_OK;
}

tjm_status tjm_run_free(tjm_ctx* ctx, int64_t run_id) {
  if (!ctx) return TJM_EINVAL;
  auto it = ctx->runs.find(run_id);
  if (it == ctx->runs.end()) return fail(ctx, TJM_EINVAL, "unknown run");
  cudaStreamSynchronize(ctx->stream);
  ctx->runs.erase(it);
  return TJM_OK;
}

void tjm_destroy(tjm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

}  // extern "C"

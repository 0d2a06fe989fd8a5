// Contraction self test: one CTA applies one effective Hamiltonian or one
// environment update of the trajectory kernel (the networks of the paper's
// Fig. 2 and the environment recursion of Sec. "Hybrid strategy") to given
// tensors, through exactly the device functions the sweeps call, so that
// their output can be compared element by element with a plain contraction.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "tjm.h"
#define TJM_TENSOR_CORES 1    // the tests route contractions either way
#include "tjm_kernels.cuh"
#include "tjm_mpo_layout.h"

namespace tjm {

// kind 0: heff0 on bond 1, 1: heff1 on site 1, 2: heff2 on sites 1-2,
// 3: env_left of site 1 (Lenv[1] -> Lenv[2]), 4: env_right of site 1 (Renv[2] -> Renv[1]).
template <class Tc, class Td>
__global__ void __launch_bounds__(TJM_THREADS, 1)
contract_test_kernel(int kind, SlotDev* S, char* scr, ScratchDims dims, const cx<double>* Lin, int nL, int lb,
                     const cx<double>* Rin, int nR, int rb, const cx<double>* x, int nx, cx<double>* y, int ny,
                     int chl, int chr, int use_tc) {
  extern __shared__ __align__(1024) char smem[];
  tc::cta_setup(&tc_ctl, sizeof(Tc) == 4 && use_tc);
  if (threadIdx.x == 0) gemm_tile_rule = 0;
  __syncthreads();
  Ctx<Tc, Td> c;
  make_ctx(c, S, scr, dims, smem);
  cx<Tc>* Lt = c.Lenv(lb);
  cx<Tc>* Rt = c.Renv(rb);
  for (int i = threadIdx.x; i < nL; i += TJM_THREADS) Lt[i] = cvt<Tc>(Lin[i]);
  for (int i = threadIdx.x; i < nR; i += TJM_THREADS) Rt[i] = cvt<Tc>(Rin[i]);
  cx<Tc>* xin = (kind >= 3) ? c.mps.site(1) : c.theta;
  for (int i = threadIdx.x; i < nx; i += TJM_THREADS) xin[i] = cvt<Tc>(x[i]);
  __syncthreads();
  const cx<Tc>* out = c.w;
  if (kind == 0) heff0(c, 1, chl, chr, xin, c.w);
  else if (kind == 1) heff1(c, 1, xin, c.w);
  else if (kind == 2) heff2(c, 1, chl, chr, xin, c.w);
  else if (kind == 3) { env_left(c, 1); out = c.Lenv(2); }
  else { env_right(c, 1); out = c.Renv(1); }
  __syncthreads();
  for (int i = threadIdx.x; i < ny; i += TJM_THREADS) y[i] = cvt<double>(out[i]);
  tc::cta_teardown(&tc_ctl);
}

}  // namespace tjm

namespace {

struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() { for (void* p : ptrs) cudaFree(p); }
  void* get(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes + 256) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    cudaMemset(p, 0, bytes + 256);
    return p;
  }
};

template <class T>
T* upload(DevMem& d, const void* src, size_t bytes) {
  T* p = reinterpret_cast<T*>(d.get(bytes));
  if (p && bytes) cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
  return p;
}

}  // namespace

extern "C" tjm_status tjm_selftest_contract(int kind, int precision, int tensor_cores, int chl, int chr, int Dl,
                                            int Du, int Dr, const double* W1, const double* W2, const double* Lenv,
                                            const double* Renv, const double* x, double* y) {
  if (kind < 0 || kind > 4 || (precision != TJM_PREC_FP64 && precision != TJM_PREC_FP32) || chl < 1 || chr < 1 ||
      chl > 64 || chr > 64 || Dl < 1 || Dr < 1 || Du < 1 || Dl > 8 || Dr > 8 || Du > 8 || !Lenv || !Renv || !x || !y ||
      (kind != 0 && !W1) || (kind == 2 && !W2))
    return TJM_EINVAL;
  typedef std::complex<double> zc;
  const int d = 2, L = 4;
  // bonds: site 1 spans MPO bonds 1..2 (Dl, Dr); for the two-site block sites 1, 2 span 1..3 (Dl, Du, Dr)
  std::vector<int> Dbond = {1, Dl, kind == 2 ? Du : Dr, kind == 2 ? Dr : 1, 1};
  std::vector<std::vector<zc>> Wsite(L);
  for (int l = 0; l < L; ++l) Wsite[l].assign((size_t)Dbond[l] * Dbond[l + 1] * d * d, zc(0.0));
  const size_t n1 = (size_t)Dl * Dbond[2] * d * d;
  if (kind != 0)
    for (size_t i = 0; i < n1; ++i) Wsite[1][i] = zc(W1[2 * i], W1[2 * i + 1]);
  if (kind == 2)
    for (size_t i = 0; i < (size_t)Du * Dr * d * d; ++i) Wsite[2][i] = zc(W2[2 * i], W2[2 * i + 1]);
  tjm_host::MpoLayouts lay;
  tjm_host::mpo_layouts(Dbond, Wsite, d, lay);
  // input / output sizes and the environments they occupy
  int nL = chl * Dl * chl, nR = 0, lb = 1, rb = 2, nx = 0, ny = 0;
  switch (kind) {
    case 0: nR = Dl * chr * chr; rb = 1; nx = ny = chl * chr; break;
    case 1: nR = Dr * chr * chr; rb = 2; nx = ny = chl * d * chr; break;
    case 2: nR = Dr * chr * chr; rb = 3; nx = ny = chl * d * d * chr; break;
    case 3: nR = 1; rb = 2; nx = chl * d * chr; ny = chr * Dr * chr; break;
    default: nL = 1; nR = Dr * chr * chr; rb = 2; nx = chl * d * chr; ny = Dl * chl * chl; break;
  }
  DevMem m;
  const size_t szc = precision == TJM_PREC_FP64 ? 16 : 8;
  const int cap = 64;
  const long long cap_site = 2LL * d * cap * cap, cap_env = 8LL * cap * cap;   // site slots hold two-site blocks too
  tjm::ScratchDims dims = {cap, 8, 30, L, 0};
  const tjm::ScratchMap mp = tjm::scratch_map(dims, (int)szc, 16);
  int* dD = upload<int>(m, Dbond.data(), Dbond.size() * sizeof(int));
  auto* dWm1 = upload<tjm::cx<double>>(m, lay.Wm1.data(), lay.Wm1.size() * 16);
  auto* dWmR = upload<tjm::cx<double>>(m, lay.WmR.data(), lay.WmR.size() * 16);
  auto* dW12 = upload<tjm::cx<double>>(m, lay.W12.data(), lay.W12.size() * 16);
  auto* o1 = upload<long long>(m, lay.Wm1_off.data(), lay.Wm1_off.size() * 8);
  auto* oR = upload<long long>(m, lay.WmR_off.data(), lay.WmR_off.size() * 8);
  auto* o12 = upload<long long>(m, lay.W12_off.data(), lay.W12_off.size() * 8);
  tjm::ProbDev P;
  std::memset(&P, 0, sizeof P);
  P.L = L; P.chi_max = cap; P.krylov_max = 30; P.shift_ok = 0;
  P.Dbond = dD; P.Wm1 = dWm1; P.Wm1_off = o1; P.WmR = dWmR; P.WmR_off = oR; P.W12 = dW12; P.W12_off = o12;
  auto* dP = upload<tjm::ProbDev>(m, &P, sizeof P);
  std::vector<int> chi = {1, chl, chr, 1, 1};
  int* dchi = upload<int>(m, chi.data(), chi.size() * sizeof(int));
  void* sites = m.get((size_t)L * cap_site * szc);
  void* envL = m.get((size_t)(L + 1) * cap_env * szc);
  void* envR = m.get((size_t)(L + 1) * cap_env * szc);
  char* scr = reinterpret_cast<char*>(m.get((size_t)mp.total));
  tjm::SlotDev S;
  std::memset(&S, 0, sizeof S);
  S.prob = dP; S.chi_cap = cap; S.sites = sites; S.chi = dchi; S.envL = envL; S.envR = envR;
  S.cap_site = cap_site; S.cap_env = cap_env;
  auto* dS = upload<tjm::SlotDev>(m, &S, sizeof S);
  auto* dLin = upload<tjm::cx<double>>(m, Lenv, (size_t)nL * 16);
  auto* dRin = upload<tjm::cx<double>>(m, Renv, (size_t)nR * 16);
  auto* dx = upload<tjm::cx<double>>(m, x, (size_t)nx * 16);
  auto* dy = reinterpret_cast<tjm::cx<double>*>(m.get((size_t)ny * 16));
  if (!dD || !dWm1 || !dWmR || !dW12 || !o1 || !oR || !o12 || !dP || !dchi || !sites || !envL || !envR || !scr ||
      !dS || !dLin || !dRin || !dx || !dy)
    return TJM_ENOMEM;
  cudaError_t e;
  if (precision == TJM_PREC_FP64) {
    const int sm = tjm::smem_bytes<double, double>(false);
    auto k = tjm::contract_test_kernel<double, double>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k<<<1, TJM_THREADS, sm>>>(kind, dS, scr, dims, dLin, nL, lb, dRin, nR, rb, dx, nx, dy, ny, chl, chr, 0);
  } else {
    const int sm = tjm::smem_bytes<float, double>(true);
    auto k = tjm::contract_test_kernel<float, double>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k<<<1, TJM_THREADS, sm>>>(kind, dS, scr, dims, dLin, nL, lb, dRin, nR, rb, dx, nx, dy, ny, chl, chr,
                              tensor_cores);
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return TJM_ECUDA;
  tjm::SlotDev back;
  cudaMemcpy(&back, dS, sizeof back, cudaMemcpyDeviceToHost);
  cudaMemcpy(y, dy, (size_t)ny * 16, cudaMemcpyDeviceToHost);
  return TJM_OK;
}

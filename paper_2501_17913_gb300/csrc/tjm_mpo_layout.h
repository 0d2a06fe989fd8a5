// Host-side kernel layouts of a Hamiltonian MPO (H0 as an MPO, Methods Sec.
// "Matrix product (density) operators"), shared by tjm_create and the
// contraction self test.  For site l with bond dimensions Dl, Dr and d = 2:
//   Wm1[(t v)][(w s)] = W_l[w][v][t][s]   (one-site effective Hamiltonian,
//                                           left environment update)
//   WmR[(w t)][(s v)] = W_l[w][v][t][s]   (right environment update)
// and for the bond (l, l+1) the two-site block
//   W12[(t1 t2 v)][(w s1 s2)] = sum_u W_l[w][u][t1][s1] W_{l+1}[u][v][t2][s2].
#pragma once
#include <complex>
#include <vector>

namespace tjm_host {

typedef std::complex<double> zc;

struct MpoLayouts {
  std::vector<zc> Wm1, WmR, W12;
  std::vector<long long> Wm1_off, WmR_off, W12_off;   // per site / per bond (plus the end of W12)
};

// Wsite[l] is [Dl][Dr][d][d] row-major; Dbond has L + 1 entries.
inline void mpo_layouts(const std::vector<int>& Dbond, const std::vector<std::vector<zc>>& Wsite, int d,
                        MpoLayouts& out) {
  const int L = (int)Wsite.size();
  auto Wel = [&](int l, int w, int v, int t, int s) -> zc {
    const int Dr = Dbond[l + 1];
    return Wsite[l][(((size_t)w * Dr + v) * d + t) * d + s];
  };
  for (int l = 0; l < L; ++l) {
    const int Dl = Dbond[l], Dr = Dbond[l + 1];
    out.Wm1_off.push_back((long long)out.Wm1.size());
    const int O1 = d * Dr, I1 = Dl * d;
    for (int o = 0; o < O1; ++o)
      for (int i = 0; i < I1; ++i) out.Wm1.push_back(Wel(l, i / d, o % Dr, o / Dr, i % d));
    out.WmR_off.push_back((long long)out.WmR.size());
    const int OR = Dl * d, IR = d * Dr;
    for (int o = 0; o < OR; ++o)
      for (int i = 0; i < IR; ++i) out.WmR.push_back(Wel(l, o / d, i % Dr, o % d, i / Dr));
  }
  for (int l = 0; l + 1 < L; ++l) {
    const int Dl = Dbond[l], Du = Dbond[l + 1], Dr = Dbond[l + 2];
    out.W12_off.push_back((long long)out.W12.size());
    const int O = d * d * Dr, I = Dl * d * d;
    for (int o = 0; o < O; ++o)
      for (int i = 0; i < I; ++i) {
        const int t1 = (o / Dr) / d, t2 = (o / Dr) % d, v = o % Dr;
        const int w = i / (d * d), s1 = (i % (d * d)) / d, s2 = i % d;
        zc acc = 0.0;
        for (int u = 0; u < Du; ++u) acc += Wel(l, w, u, t1, s1) * Wel(l + 1, u, v, t2, s2);
        out.W12.push_back(acc);
      }
  }
  out.W12_off.push_back((long long)out.W12.size());
}

}  // namespace tjm_host

// Host driver for the double-float arithmetic of the GPU factorizations
// (csrc/tjm_df64.cuh compiled as plain C++): reads lines "a_hi a_lo b_hi b_lo
// c_hi c_lo" of hexadecimal floats and prints, as hexadecimal floats, the
// (hi, lo) words of a+b, a-b, a*b, a/b, sqrt(|a|), fma(a, b, c), a*b + c*a and
// c + a*b + b*c.
#include <cstdio>

#include "tjm_df64.cuh"

using tjm::df64;

static void out(df64 x) { std::printf(" %a %a", (double)x.hi, (double)x.lo); }

int main() {
  float v[6];
  while (std::scanf("%a %a %a %a %a %a", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
    const df64 a(v[0], v[1]), b(v[2], v[3]), c(v[4], v[5]);
    out(a + b);
    out(a - b);
    out(a * b);
    out(a / b);
    out(sqrt(tjm::fabs(a)));
    out(fma(a, b, c));
    out(tjm::df_dot2(a, b, c, a));
    out(tjm::df_fma2(c, a, b, b, c));
    std::printf("\n");
  }
  return 0;
}

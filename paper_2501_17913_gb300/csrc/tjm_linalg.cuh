// CTA-wide dense factorizations used by the sweeps, in the decomposition
// precision Td (double in the FP64 path, float or double in the FP32 path):
//   * Householder QR with explicit thin Q  (moving the orthogonality centre,
//     Methods Sec. "Matrix product states"; Eq. 1TDVP_ForwardEvolving's QR),
//   * one-sided (Hestenes) Jacobi SVD       (two-site truncation, post-jump
//     compression; Sec. "1TDVP and 2TDVP as tensor networks"),
//   * exp(i theta T) e_1 for the Lanczos tridiagonal T by a scaled Taylor
//     series on one warp (Moler & Van Loan, "Nineteen dubious ways...", the
//     series method with scaling), with a Gershgorin-centred shift.
// Matrices are column-major, in the CTA's shared-memory workspace when the
// factorization precision is FP32 and they fit (64 KB), else in its global
// scratch.  Column (pair) work is dealt to aligned groups of 8 lanes.
#pragma once
#include "tjm_common.cuh"

namespace tjm {

template <class T> struct eps_of;
template <> struct eps_of<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct eps_of<double> { static constexpr double v = 2.220446049250313e-16; };
// double-float: a few units of 2^-48 per operation (tjm_df64.cuh); 2^-46 bounds them
template <> struct eps_of<df64> { static constexpr double v = 1.4210854715202004e-14; };

// |z| without squaring z: max(|x|, |y|) sqrt(1 + (min / max)^2).
template <class T>
__device__ __forceinline__ T cabs_scaled(cx<T> z) {
  const T ax = fabs(z.x), ay = fabs(z.y);
  const T m = ax > ay ? ax : ay;
  if (!(m > T(0))) return T(0);
  const T rx = ax / m, ry = ay / m;
  return m * sqrt(rx * rx + ry * ry);
}

// ------------------------------------------------------------------ QR
// x[:, c] <- (I - tau v v^H) x[:, c] for columns c0 <= c < c1 of x (column-major,
// leading dimension m), acting on rows j..m-1 where v lives.  One aligned
// group of 8 lanes per column, so a warp works on four columns at once and
// each dot product needs only a 3-step shuffle reduction; the groups of a
// warp start their walk down the column 8 rows apart, so their shared-memory
// reads fall in different banks.
// If nrm is given, the group that owns column c0 also stores there the
// squared norm of that column's rows j+1..m-1 after the update.
template <class T>
__device__ __forceinline__ void grp_reflect(int m, int j, const cx<T>* v, T tj, cx<T>* x, int c0, int c1,
                                            T* nrm = nullptr) {
  const int gl = threadIdx.x & 7, grp = threadIdx.x >> 3;
  const unsigned gmask = 0xffu << ((threadIdx.x & 31) & 24);
  const int len = m - j;
  if (len <= 0) return;
  const int i0 = j + (gl + 8 * (grp & 3)) % len;
  for (int c = c0 + grp; c < c1; c += TJM_THREADS / 8) {
    cx<T>* xc = x + (long long)c * m;
    cx<T> s = czero<T>();
    for (int t = gl, i = i0; t < len; t += 8) {
      cfma_cj(s, v[i], xc[i]);
      i += 8; if (i >= m) i -= len;
    }
    s.x = grp8_sum(s.x, gmask);
    s.y = grp8_sum(s.y, gmask);
    const cx<T> f = mk(-tj * s.x, -tj * s.y);
    T q2 = T(0);
    for (int t = gl, i = i0; t < len; t += 8) {
      cx<T> y = xc[i];
      cfma(y, f, v[i]);
      xc[i] = y;
      if (i > j) q2 += norm2(y);
      i += 8; if (i >= m) i -= len;
    }
    if (nrm && c == c0) {
      q2 = grp8_sum(q2, gmask);
      if (gl == 0) *nrm = q2;
    }
  }
}

// a: m x n column-major (lda = m), factorised in place.  k = min(m, n).
// On exit q (m x k, column-major) holds the thin Q, r (k x n, column-major,
// ldr = k) holds R.  tau / rdiag: k entries of scratch each.  With q == a the
// thin Q is formed in place in the first k columns of a (the workspace can
// then live in shared memory).
template <class T>
__device__ __noinline__ void blk_qr(int m, int n, cx<T>* a, cx<T>* q, cx<T>* r, cx<T>* rdiag, T* tau, double* red) {
  const int k = m < n ? m : n;
  // A remaining column below eps * ||A||_F is rounding noise: no reflector is
  // built from it (its 1/(v^H v) would overflow in FP32) and it is left as is,
  // a backward error of at most eps * ||A||_F.
  double fro2 = 0.0;
  for (long long e = threadIdx.x; e < (long long)m * n; e += TJM_THREADS) fro2 += (double)norm2(a[e]);
  fro2 = blk_sum(fro2, red);
  const T negl = (T)(eps_of<T>::v * eps_of<T>::v * fro2);
  // cn[j & 1]: squared norm of rows j..m-1 of the pivot column j.  It is
  // produced by the group that applies reflector j-1 to column j, so no
  // block-wide reduction stands between two reflectors.
  T* cn = reinterpret_cast<T*>(red + 256);
  const int gl = threadIdx.x & 7, grp = threadIdx.x >> 3;
  const unsigned gmask = 0xffu << ((threadIdx.x & 31) & 24);
  if (threadIdx.x < 8) {
    T s2 = T(0);
    for (int i = threadIdx.x; i < m; i += 8) s2 += norm2(a[i]);
    s2 = grp8_sum(s2, 0xffu);
    if (threadIdx.x == 0) cn[0] = s2;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    cx<T>* col = a + (long long)j * m;
    if (threadIdx.x == 0) {
      const cx<T> al = col[j];
      const T s2 = cn[j & 1];
      if (s2 <= negl) {
        tau[j] = (T)0; rdiag[j] = al;
      } else {
        const T sig = sqrt(s2);
        const T aa = sqrt(norm2(al));
        const T px = aa > (T)0 ? al.x / aa : (T)1, py = aa > (T)0 ? al.y / aa : (T)0;
        const cx<T> be = mk(-px * sig, -py * sig);
        col[j] = al - be;
        tau[j] = (T)1 / (s2 + aa * sig);          // 2 / (v^H v)
        rdiag[j] = be;
      }
    }
    __syncthreads();
    const T tj = tau[j];
    T* nx = j + 1 < k ? &cn[(j + 1) & 1] : nullptr;
    if (tj != (T)0) {
      grp_reflect<T>(m, j, col, tj, a, j + 1, n, nx);
    } else if (nx && grp == 0) {
      const cx<T>* xc = a + (long long)(j + 1) * m;
      T s2 = T(0);
      for (int i = j + 1 + gl; i < m; i += 8) s2 += norm2(xc[i]);
      s2 = grp8_sum(s2, gmask);
      if (gl == 0) *nx = s2;
    }
    __syncthreads();
  }
  __syncthreads();
  // R (k x n)
  for (int e = threadIdx.x; e < k * n; e += TJM_THREADS) {
    const int i = e % k, c = e / k;
    cx<T> v = czero<T>();
    if (c > i) v = a[(long long)c * m + i];
    else if (c == i) v = rdiag[i];
    r[(long long)c * k + i] = v;
  }
  __syncthreads();
  if (q == a) {
    // Q = H_0 ... H_{k-1} [I_k; 0] formed in place in the first k columns of a:
    // for j from k-1 down to 0, apply H_j to columns j+1..k-1 (rows j..m-1;
    // their rows <= j are zero), then replace column j, which holds v_j, by
    // H_j e_j = e_j - tau_j v_j conj(v_j[j]).
    for (int e = threadIdx.x; e < k * k; e += TJM_THREADS) {
      const int i = e % k, c = e / k;
      if (i < c) a[(long long)c * m + i] = czero<T>();
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
      const T tj = tau[j];
      cx<T>* v = a + (long long)j * m;
      const cx<T> vj = v[j];              // column j is rewritten below, after the barrier
      if (tj != (T)0) grp_reflect<T>(m, j, v, tj, a, j + 1, k);
      const cx<T> f = mk(-tj * vj.x, tj * vj.y);            // -tau conj(v_j)
      __syncthreads();
      for (int i = j + threadIdx.x; i < m; i += TJM_THREADS) {
        const cx<T> x = v[i];
        cx<T> y = czero<T>();
        if (tj != (T)0) y = f * x;
        if (i == j) y = y + mk((T)1, (T)0);
        v[i] = y;
      }
      __syncthreads();
    }
    return;
  }
  // Q = H_0 ... H_{k-1} [I_k; 0] into the separate buffer q
  for (int e = threadIdx.x; e < m * k; e += TJM_THREADS) {
    const int i = e % m, c = e / m;
    q[e] = (i == c) ? mk((T)1, (T)0) : czero<T>();
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj != (T)0) grp_reflect<T>(m, j, a + (long long)j * m, tj, q, j, k);
    __syncthreads();
  }
}

// One pass of classical Gram-Schmidt over the columns q[:, perm[0..n-1]]
// (column-major, len rows), in that order, each normalised first: columns
// that are already orthonormal to about 1e-6 come out orthonormal to working
// precision.  Projections use compensated warp sums.  red: shared memory,
// 2 * n + 64 doubles.
template <class T>
__device__ __noinline__ void blk_cgs_perm(int len, int n, cx<T>* q, const int* perm, double* red) {
  const int gl = threadIdx.x & 7, grp = threadIdx.x >> 3;
  const unsigned gmask = 0xffu << ((threadIdx.x & 31) & 24);
  T* h = reinterpret_cast<T*>(red + 64);
  for (int c = 0; c < n; ++c) {
    cx<T>* qc = q + (long long)perm[c] * len;
    if (c > 0) {
      // one aligned group of 8 lanes per projection
      for (int o = grp; o < c; o += TJM_THREADS / 8) {
        const cx<T>* qo = q + (long long)perm[o] * len;
        T hx = T(0), hy = T(0);
        for (int i = gl; i < len; i += 8) {
          const cx<T> x = qo[i], y = qc[i];
          hx = fma(x.x, y.x, fma(x.y, y.y, hx));
          hy = fma(x.x, y.y, fma(-x.y, y.x, hy));
        }
        grp8_sum_acc2(hx, hy, gmask);
        if (gl == 0) { h[2 * o] = hx; h[2 * o + 1] = hy; }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < len; i += TJM_THREADS) {
        cx<T> a = qc[i];
        for (int o = 0; o < c; ++o) {
          const cx<T> x = q[(long long)perm[o] * len + i];
          a.x -= h[2 * o] * x.x - h[2 * o + 1] * x.y;
          a.y -= h[2 * o] * x.y + h[2 * o + 1] * x.x;
        }
        qc[i] = a;
      }
    }
    T nr = T(0);
    for (int i = threadIdx.x; i < len; i += TJM_THREADS) nr += norm2(qc[i]);
    nr = blk_sum_pos(nr, red);
    const T f = nr > (T)0 ? (T)1 / sqrt(nr) : (T)0;
    for (int i = threadIdx.x; i < len; i += TJM_THREADS) qc[i] = mk(qc[i].x * f, qc[i].y * f);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Jacobi SVD
// a: mm x nn column-major with mm >= nn (the caller transposes when needed).
// On exit: u (mm x nn) orthonormal columns sorted by decreasing singular
// value, s[nn], v (nn x nn) with a = u diag(s) v^H.  Columns of u that belong
// to exactly-zero singular values are completed to an orthonormal set.
// vw: nn x nn rotation accumulator; sv: nn scratch values; iw: 2 nn ints.
// Returns the sweep count.
template <class T>
__device__ __noinline__ int blk_svd_jacobi(int mm, int nn, cx<T>* a, cx<T>* u, T* s, cx<T>* v, cx<T>* vw, T* sv,
                                           int* iw, double* red, bool complete) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int rot_count;
  for (int e = threadIdx.x; e < nn * nn; e += TJM_THREADS) vw[e] = (e % nn == e / nn) ? mk((T)1, (T)0) : czero<T>();
  // rotate while |a_p^H a_q| > tol sqrt(|a_p|^2 |a_q|^2); the products are
  // reduced with compensation (FP32) or in FP64, so the test resolves below tol
  const T tol = (T)(sizeof(T) == 4 ? 8.0 * eps_of<T>::v : eps_of<T>::v * (double)mm);
  // Columns whose norm falls below eps * ||A||_F carry only rounding noise.
  // They are set to exactly zero and take no further part in rotations:
  // otherwise every sweep re-orthogonalises them, shrinks them by another
  // factor eps and eventually drives them into the denormal range, where the
  // rotation phases stop being unitary.
  double fro2 = 0.0;
  for (long long e = threadIdx.x; e < (long long)mm * nn; e += TJM_THREADS) fro2 += (double)norm2(a[e]);
  fro2 = blk_sum(fro2, red);
  const T negl = (T)(eps_of<T>::v * eps_of<T>::v * fro2);
  const int ne = nn + (nn & 1);
  // Each pair of columns is handled by an aligned group of 8 lanes (4 pairs
  // per warp): the per-pair cross-lane reduction is then 3 shuffle steps
  // instead of 5, over a quarter of the lanes.  Groups of one warp start
  // their column walk 8 elements apart, so their shared-memory reads fall in
  // different banks.
  const int gl = threadIdx.x & 7, grp = threadIdx.x >> 3;
  const unsigned gmask = 0xffu << (lane & 24);
  const int off = 8 * (grp & 3);
  const int ia0 = (gl + off) % mm, iv0 = (gl + off) % nn;
  int sweep = 0;
  for (; sweep < 40 && nn > 1; ++sweep) {
    if (threadIdx.x == 0) rot_count = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int pr = grp; pr < ne / 2; pr += TJM_THREADS / 8) {
        // circle-method pairing: position 0 fixed, the others rotate
        const int pa = pr, pb = ne - 1 - pr;
        const int p = pa == 0 ? 0 : ((pa - 1 + rnd) % (ne - 1)) + 1;
        const int qq = ((pb - 1 + rnd) % (ne - 1)) + 1;
        if (p >= nn || qq >= nn) continue;
        cx<T>* ap = a + (long long)p * mm;
        cx<T>* aq = a + (long long)qq * mm;
        T al0 = T(0), be0 = T(0);
        cx<T> ga0 = czero<T>();
        for (int r = gl, i = ia0; r < mm; r += 8) {
          const cx<T> x = ap[i], y = aq[i];
          al0 += norm2(x); be0 += norm2(y); cfma_cj(ga0, x, y);
          i += 8; if (i >= mm) i -= mm;
        }
        // column norms add positive terms (no cancellation); the product is
        // reduced with compensation in FP32
        const T al = grp8_sum(al0, gmask), be = grp8_sum(be0, gmask);
        grp8_sum_acc2(ga0.x, ga0.y, gmask);
        const cx<T> ga = ga0;
        if (al <= negl || be <= negl) {
          if (al <= negl && al != (T)0) for (int i = gl; i < mm; i += 8) ap[i] = czero<T>();
          if (be <= negl && be != (T)0) for (int i = gl; i < mm; i += 8) aq[i] = czero<T>();
          continue;
        }
        // |ga| and the test scaled so that no product of two squared norms is formed: in double-float
        // (FP32 exponent range) |ga|^2 and al * be of noise-level columns underflow, and a phase
        // ga / |ga| computed from underflowed values is not unitary
        const T ag = cabs_scaled(ga);
        if (!(ag > tol * sqrt(al) * sqrt(be))) continue;
        const T zeta = (be - al) / ((T)2 * ag);
        // tan of the rotation angle, sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); beyond |zeta| = 1e8 it is
        // sign(zeta) / (2 |zeta|) to within 1e-16 relative, which also keeps zeta^2 from overflowing the
        // FP32 exponent range of double-float
        const T az = fabs(zeta);
        const T t = (zeta >= (T)0 ? (T)1 : (T)-1) / (az > T(1e8f) ? (T)2 * az : az + sqrt((T)1 + zeta * zeta));
        const T c = (T)1 / sqrt((T)1 + t * t), sn = c * t;
        const cx<T> ph = mk(ga.x / ag, -ga.y / ag);           // e^{-i phi}
        // [a_p, a_q] <- [a_p, a_q] [[c, sn], [-sn e^{-i phi}, c e^{-i phi}]]
        const T msn = -sn;
        for (int r = gl, i = ia0; r < mm; r += 8) {
          const cx<T> x = ap[i], y = ph * aq[i];
          ap[i] = rot_comb(c, x, msn, y);
          aq[i] = rot_comb(sn, x, c, y);
          i += 8; if (i >= mm) i -= mm;
        }
        cx<T>* vp = vw + (long long)p * nn;
        cx<T>* vq = vw + (long long)qq * nn;
        for (int r = gl, i = iv0; r < nn; r += 8) {
          const cx<T> x = vp[i], y = ph * vq[i];
          vp[i] = rot_comb(c, x, msn, y);
          vq[i] = rot_comb(sn, x, c, y);
          i += 8; if (i >= nn) i -= nn;
        }
        if (gl == 0) atomicAdd(&rot_count, 1);
      }
      __syncthreads();
    }
    const int rc = rot_count;
    __syncthreads();
    if (rc == 0) break;
  }
  // singular values (unsorted in sv), descending order (ties by index)
  for (int c = warp; c < nn; c += TJM_WARPS) {
    const cx<T>* ac = a + (long long)c * mm;
    double acc = 0.0;
    for (int i = lane; i < mm; i += 32) acc += (double)norm2(ac[i]);
    acc = warp_sum(acc);
    if (lane == 0) sv[c] = (T)sqrt(acc);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nn; c += TJM_THREADS) {
    int rank = 0;
    const T x = sv[c];
    for (int i = 0; i < nn; ++i) rank += (sv[i] > x) || (sv[i] == x && i < c);
    iw[rank] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += TJM_THREADS) s[e] = sv[iw[e]];
  const bool f32 = sizeof(T) == 4;
  if constexpr (sizeof(T) == 4) {
    // In FP32 the converged columns are orthogonal only to tol (about 5e-7)
    // and the accumulated rotations drift by a similar amount; sites cut from
    // U or V must be isometries to working precision, because every
    // environment and transfer contraction along the chain assumes it.
    int nz = 0;
    for (int c = 0; c < nn; ++c) nz += sv[c] > (T)0;
    blk_cgs_perm<T>(mm, nz, a, iw, red);
    blk_cgs_perm<T>(nn, nn, vw, iw, red);
  }
  for (long long e = threadIdx.x; e < (long long)mm * nn; e += TJM_THREADS) {
    const int i = (int)(e % mm), c = (int)(e / mm);
    const T sc = sv[iw[c]];
    const cx<T> x = a[(long long)iw[c] * mm + i];
    u[e] = sc > (T)0 ? (f32 ? x : mk(x.x / sc, x.y / sc)) : czero<T>();
  }
  for (long long e = threadIdx.x; e < (long long)nn * nn; e += TJM_THREADS) {
    const int i = (int)(e % nn), c = (int)(e / nn);
    v[e] = vw[(long long)iw[c] * nn + i];
  }
  __syncthreads();
  // complete columns of exactly-zero singular values (Gram-Schmidt on unit
  // vectors e_cand, scanned cyclically; the residuals of all mm candidates sum
  // to the dimension still free, so one of them exceeds 1/mm and the
  // threshold 0.5/mm is always met)
  if (!complete) return sweep;
  int cand = 0;
  const double accept = 0.5 / mm;
  for (int c = 0; c < nn; ++c) {
    if (s[c] > (T)0) continue;
    cx<T>* uc = u + (long long)c * mm;
    for (int tries = 0; tries < mm; ++tries, cand = (cand + 1) % mm) {
      for (int i = threadIdx.x; i < mm; i += TJM_THREADS) uc[i] = (i == cand) ? mk((T)1, (T)0) : czero<T>();
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int o = 0; o < nn; ++o) {
          if (o == c || (s[o] == (T)0 && o > c)) continue;
          const cx<T>* uo = u + (long long)o * mm;
          double hx = 0.0, hy = 0.0;
          for (int i = threadIdx.x; i < mm; i += TJM_THREADS) {
            const cx<T> x = uo[i], y = uc[i];
            hx += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
            hy += (double)x.x * (double)y.y - (double)x.y * (double)y.x;
          }
          hx = blk_sum(hx, red);
          hy = blk_sum(hy, red);
          for (int i = threadIdx.x; i < mm; i += TJM_THREADS) {
            const cx<T> x = uo[i];
            const double xr = (double)x.x, xi = (double)x.y;
            uc[i] = uc[i] - mk((T)(hx * xr - hy * xi), (T)(hx * xi + hy * xr));
          }
          __syncthreads();
        }
      }
      double n2 = 0.0;
      for (int i = threadIdx.x; i < mm; i += TJM_THREADS) n2 += (double)norm2(uc[i]);
      n2 = blk_sum(n2, red);
      if (n2 > accept) {
        const T f = (T)(1.0 / sqrt(n2));
        for (int i = threadIdx.x; i < mm; i += TJM_THREADS) uc[i] = f * uc[i];
        __syncthreads();
        cand = (cand + 1) % mm;
        break;
      }
    }
  }
  __syncthreads();
  return sweep;
}

// ------------------------------------------------------------------ exp of the Lanczos tridiagonal
// Called by ONE full warp.  c[0..k-1] = exp(i theta T) e_1 with
// T = tridiag(beta; alpha; beta), k <= 32.  Lane j holds component j.
__device__ inline void warp_expm_tridiag(int k, const double* alpha, const double* beta, double theta,
                                         cx<double>* c) {
  const int j = threadIdx.x & 31;
  const bool on = j < k;
  double aj = on ? alpha[j] : 0.0;
  double amax = on ? aj : -1e300, amin = on ? aj : 1e300;
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
  }
  const double sh = 0.5 * (amax + amin);
  const double bj = (on && j + 1 < k) ? beta[j] : 0.0;          // coupling j <-> j+1
  const double bm = __shfl_up_sync(0xffffffffu, bj, 1);
  const double bjm = (j > 0 && on) ? bm : 0.0;                  // coupling j-1 <-> j
  const double ad = on ? aj - sh : 0.0;
  const double rho = warp_max(on ? fabs(ad) + fabs(bj) + fabs(bjm) : 0.0);
  int nsc = (int)ceil(fabs(theta) * rho / 0.5);
  if (nsc < 1) nsc = 1;
  const double h = theta / nsc;
  double xr = (j == 0) ? 1.0 : 0.0, xi = 0.0;
  for (int st = 0; st < nsc; ++st) {
    double sr = xr, si = xi, tr = xr, ti = xi;
    for (int n = 1; n <= 16; ++n) {
      // t <- (i h / n) (T - sh) t
      const double ur = __shfl_down_sync(0xffffffffu, tr, 1), ui = __shfl_down_sync(0xffffffffu, ti, 1);
      const double lr = __shfl_up_sync(0xffffffffu, tr, 1), li = __shfl_up_sync(0xffffffffu, ti, 1);
      double yr = ad * tr + bj * ur + bjm * lr;
      double yi = ad * ti + bj * ui + bjm * li;
      if (!on) { yr = 0.0; yi = 0.0; }
      const double f = h / n;
      tr = -f * yi;
      ti = f * yr;
      sr += tr; si += ti;
    }
    xr = sr; xi = si;
  }
  // multiply by exp(i theta sh)
  double cs, sn;
  sincos(theta * sh, &sn, &cs);
  if (on) c[j] = mk(cs * xr - sn * xi, cs * xi + sn * xr);
}

}  // namespace tjm

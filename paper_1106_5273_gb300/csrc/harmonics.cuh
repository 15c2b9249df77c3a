// Solid harmonics and translation-operator entries (host and device).
//
// Basis (Sec. 3.1: spherical-harmonic Laplace expansions).  With P_n^m the
// associated Legendre function without the Condon-Shortley phase,
//   R_n^m(x) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!       (regular)
//   I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m phi} / r^{n+1}    (irregular)
//   X_n^{-m} = (-1)^m conj(X_n^m)
// satisfy 1/|x-y| = sum conj(R_n^m(y)) I_n^m(x) (|y|<|x|),
// R_n^m(a+b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b) and
// I_j^k(t-y) = sum_{n,m} conj(R_n^m(y)) I_{j+n}^{k+m}(t).
// Stored coefficients are scaled by nu_n^m = sqrt((n+m)!(n-m)!) and by the
// cell side a (the normalisation of Sec. 4.2 that keeps single precision
// usable):  M~ = M nu / a^n,  L~ = L a^{n+1} / nu,  R~ = nu R (|R~| <= r^n).
// The resulting operators (a_t target side, a_s source side):
//   P2M  M~_n^m = sum_j q_j conj(R~_n^m(y_j / a))
//   M2M  M~_n^m = r^n sum_{k,l} nu_n^m/(nu_k^l nu_{n-k}^{m-l}) conj(R~_k^l(beta)) M~'_{n-k}^{m-l}
//        (r = a_child/a_parent, beta = (c_child - c_parent)/a_child)
//   M2L  L~_n^m = (-1)^n sum_{j,k} (a_s/a_t)^j/(nu_n^m nu_j^k) conj(M~_j^k I_{j+n}^{k+m}(tau))
//        (tau = (c_t - c_s)/a_t)
//   L2L  L~'_n^m = sum_{k,l} r^{n+k+1} nu_{n+k}^{m+l}/(nu_n^m nu_k^l) L~_{n+k}^{m+l} R~_k^l(beta)
//   L2P  Phi(x) = (1/a) sum L~_n^m R~_n^m((x-c)/a)
#pragma once

#include <math.h>

#include "common.cuh"

namespace fmm {

struct cd {
  double re, im;
};
__host__ __device__ inline cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline cd cconj(cd a) { return {a.re, -a.im}; }
__host__ __device__ inline cd cscale(cd a, double s) { return {a.re * s, a.im * s}; }

// Complex index for m >= 0: n(n+1)/2 + m.
__host__ __device__ inline int cidx(int n, int m) { return n * (n + 1) / 2 + m; }

__host__ __device__ inline double factorial_d(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

__host__ __device__ inline double nu_d(int n, int m) {
  if (m < 0) m = -m;
  return sqrt(factorial_d(n + m) * factorial_d(n - m));
}

// Unnormalized irregular harmonics I_n^m(x), n < D, m >= 0, into I[cidx].
__host__ __device__ inline void irregular_table_d(double x, double y, double z, int D, cd* I) {
  double r2 = x * x + y * y + z * z;
  double inv_r2 = 1.0 / r2;
  I[0] = {1.0 / sqrt(r2), 0.0};
  for (int m = 1; m < D; ++m) {
    cd prev = I[cidx(m - 1, m - 1)];
    cd xy = {x, y};
    I[cidx(m, m)] = cscale(cmul(prev, xy), (2.0 * m - 1.0) * inv_r2);
  }
  for (int m = 0; m < D; ++m) {
    for (int n = m + 1; n < D; ++n) {
      cd a = cscale(I[cidx(n - 1, m)], (2.0 * n - 1.0) * z);
      if (n - 2 >= m) {
        cd b = cscale(I[cidx(n - 2, m)], (double)((n - 1) * (n - 1) - m * m));
        a.re -= b.re;
        a.im -= b.im;
      }
      I[cidx(n, m)] = cscale(a, inv_r2);
    }
  }
}

// Normalized regular harmonics R~_n^m(x), n < p, m >= 0 (FP64).
__host__ __device__ inline void regular_table_d(double x, double y, double z, int p, cd* R) {
  double r2 = x * x + y * y + z * z;
  R[0] = {1.0, 0.0};
  for (int m = 1; m < p; ++m) {
    cd prev = R[cidx(m - 1, m - 1)];
    cd xy = {x, y};
    R[cidx(m, m)] = cscale(cmul(prev, xy), sqrt((2.0 * m - 1.0) / (2.0 * m)));
  }
  for (int m = 0; m < p; ++m) {
    for (int n = m + 1; n < p; ++n) {
      cd a = cscale(R[cidx(n - 1, m)], (2.0 * n - 1.0) * z);
      if (n - 2 >= m) {
        cd b = cscale(R[cidx(n - 2, m)], r2 * sqrt((double)(n + m - 1) * (double)(n - m - 1)));
        a.re -= b.re;
        a.im -= b.im;
      }
      R[cidx(n, m)] = cscale(a, 1.0 / sqrt((double)(n + m) * (double)(n - m)));
    }
  }
}

// X_n^m for any m from a table of m >= 0 (X^{-m} = (-1)^m conj(X^m)).
__host__ __device__ inline cd harm_get(const cd* T, int n, int m) {
  if (m >= 0) return T[cidx(n, m)];
  cd v = cconj(T[cidx(n, -m)]);
  return (m & 1) ? cd{-v.re, -v.im} : v;
}

// Real-matrix entry of the normalized M2L operator (row: output (n,m,po),
// column: input (j,k,pi)), given the irregular table I (degrees < 2p-1) at
// tau and the scale ratio a_s/a_t.  See the header comment for the formula.
__host__ __device__ inline double m2l_entry(const cd* I, int n, int m, int po, int j, int k, int pi,
                                            double ratio_pow_j) {
  double s = ((n & 1) ? -1.0 : 1.0) * ratio_pow_j / (nu_d(n, m) * nu_d(j, k));
  cd A = cconj(harm_get(I, j + n, k + m));
  cd B = {0.0, 0.0};
  if (k > 0) {
    B = cconj(harm_get(I, j + n, m - k));
    if (k & 1) B = {-B.re, -B.im};
  }
  // Y = s [ a (A + B) + i b (B - A) ]  with input a + i b
  if (pi == 0) return po == 0 ? s * (A.re + B.re) : s * (A.im + B.im);
  return po == 0 ? -s * (B.im - A.im) : s * (B.re - A.re);
}

}  // namespace fmm

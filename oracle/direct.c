/*
 * Oracle (test infrastructure only; never linked into the product path).
 *
 * Plain FP64 direct sum of the regularized Biot-Savart velocity (Eq. 1 with the
 * Gaussian cutoff of Eq. 2) and of the classical vortex-stretching term (Eq. 3,
 * read as (gamma_i . grad) u), over all source particles and an explicit list of
 * periodic image shifts.
 *
 * With d = x_i - x_j + shift, r = |d|, rho = r / sigma_j, c = sqrt(2/pi):
 *   g(rho) = erf(rho/sqrt 2) - c rho exp(-rho^2/2)                    (Eq. 2)
 *   S      = g / r^3
 *   T      = (c exp(-rho^2/2) / sigma_j^3 - 3 S) / r^2   ( = S'(r)/r )
 *   u_i   += S (gamma_j x d) / (4 pi)                                (Eq. 1)
 *   s_i   += [S (gamma_j x gamma_i) + T (gamma_i . d)(gamma_j x d)] / (4 pi)  (Eq. 3)
 * or, with transpose != 0, the transpose scheme s = (grad u)^T gamma_i:
 *   s_i   += [S (gamma_i x gamma_j) + T (gamma_i . (gamma_j x d)) d] / (4 pi)
 * For rho^2 < 1/4 the closed forms lose digits to cancellation, so S and T come
 * from the Taylor series of g(rho)/rho^3 in rho^2 (term-by-term integral of
 * g'(rho) = c rho^2 exp(-rho^2/2)).
 *
 * The pair with the same index and a zero shift is skipped when skip_self != 0:
 * its exact contribution is zero (d = 0 and gamma_i x gamma_i = 0).
 */
#include <math.h>
#include <stdint.h>

#define ORACLE_C_SQRT_2_OVER_PI 0.79788456080286535588
#define ORACLE_INV_4PI 0.07957747154594766788

/* S*sigma^3 and T*sigma^5 as functions of u = rho^2, by the series. */
static void series_ST(double u, double* Sh, double* Th) {
  /* a_k = c (-1)^k / (2^k k! (2k+3)) */
  double a = ORACLE_C_SQRT_2_OVER_PI / 3.0; /* k = 0 */
  double sS = 0.0, sT = 0.0, uk = 1.0, ukm1 = 0.0;
  for (int k = 0; k < 20; ++k) {
    if (k > 0) {
      a = ORACLE_C_SQRT_2_OVER_PI * ((k & 1) ? -1.0 : 1.0);
      double den = (2.0 * k + 3.0);
      for (int q = 1; q <= k; ++q) den *= 2.0 * q;
      a /= den;
    }
    sS += a * uk;
    if (k >= 1) sT += 2.0 * k * a * ukm1;
    ukm1 = uk;
    uk *= u;
  }
  *Sh = sS;
  *Th = sT;
}

/* S and T for one pair (r2 = |d|^2). */
static void pair_ST(double r2, double sigma, double* S, double* T) {
  double s2 = sigma * sigma;
  double u = r2 / s2;
  if (u < 0.25) {
    double Sh, Th;
    series_ST(u, &Sh, &Th);
    *S = Sh / (s2 * sigma);
    *T = Th / (s2 * s2 * sigma);
    return;
  }
  double r = sqrt(r2);
  double rho = r / sigma;
  double e = exp(-0.5 * u);
  double g = erf(rho / sqrt(2.0)) - ORACLE_C_SQRT_2_OVER_PI * rho * e;
  double s = g / (r2 * r);
  *S = s;
  *T = (ORACLE_C_SQRT_2_OVER_PI * e / (s2 * sigma) - 3.0 * s) / r2;
}

/* Exported for the pins: S and T of one pair. */
void oracle_pair_ST(double r2, double sigma, double* S, double* T) { pair_ST(r2, sigma, S, T); }

/*
 * u[nt,3], s[nt,3] (overwritten) at targets xt[nt,3] with target strengths
 * gt[nt,3] (needed for s only) from sources xs[ns,3], gs[ns,3], sig[ns].
 * img[nimg,3] are shifts added to d (nimg >= 1; pass one zero shift for free
 * space).  If skip_self, target i and source i are the same particle.
 * transpose selects the stretching scheme (0 classical, 1 transpose).
 */
void oracle_direct(int64_t nt, const double* xt, const double* gt, int64_t ns,
                   const double* xs, const double* gs, const double* sig,
                   int64_t nimg, const double* img, int skip_self, int transpose,
                   double* u, double* s) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    double ux = 0, uy = 0, uz = 0, sx = 0, sy = 0, sz = 0;
    const double gix = gt[3 * i], giy = gt[3 * i + 1], giz = gt[3 * i + 2];
    for (int64_t m = 0; m < nimg; ++m) {
      const double ox = img[3 * m], oy = img[3 * m + 1], oz = img[3 * m + 2];
      const int zero_shift = (ox == 0.0 && oy == 0.0 && oz == 0.0);
      for (int64_t j = 0; j < ns; ++j) {
        if (skip_self && zero_shift && j == i) continue;
        double dx = (xt[3 * i] - xs[3 * j]) + ox;
        double dy = (xt[3 * i + 1] - xs[3 * j + 1]) + oy;
        double dz = (xt[3 * i + 2] - xs[3 * j + 2]) + oz;
        double r2 = dx * dx + dy * dy + dz * dz;
        double S, T;
        pair_ST(r2, sig[j], &S, &T);
        double gx = gs[3 * j], gy = gs[3 * j + 1], gz = gs[3 * j + 2];
        /* gamma_j x d */
        double cx = gy * dz - gz * dy, cy = gz * dx - gx * dz, cz = gx * dy - gy * dx;
        ux += S * cx; uy += S * cy; uz += S * cz;
        /* gamma_j x gamma_i */
        double kx = gy * giz - gz * giy, ky = gz * gix - gx * giz, kz = gx * giy - gy * gix;
        if (transpose) {
          /* gamma_i x gamma_j = -(gamma_j x gamma_i); gamma_i . (gamma_j x d) */
          double tw = T * (gix * cx + giy * cy + giz * cz);
          sx += tw * dx - S * kx; sy += tw * dy - S * ky; sz += tw * dz - S * kz;
        } else {
          double td = T * (gix * dx + giy * dy + giz * dz);
          sx += S * kx + td * cx; sy += S * ky + td * cy; sz += S * kz + td * cz;
        }
      }
    }
    u[3 * i] = ux * ORACLE_INV_4PI; u[3 * i + 1] = uy * ORACLE_INV_4PI; u[3 * i + 2] = uz * ORACLE_INV_4PI;
    s[3 * i] = sx * ORACLE_INV_4PI; s[3 * i + 1] = sy * ORACLE_INV_4PI; s[3 * i + 2] = sz * ORACLE_INV_4PI;
  }
}

/* Number of OpenMP threads the direct sum uses (reported with CPU timings). */
int oracle_num_threads(void) {
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    {
#ifdef _OPENMP
      extern int omp_get_num_threads(void);
      n = omp_get_num_threads();
#endif
    }
  }
  return n;
}

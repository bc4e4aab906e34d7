// Gauss rule of a symmetric tridiagonal matrix (Eq. quadratic: nodes are the
// eigenvalues of T, weights the squared first components of its normalized
// eigenvectors; Golub and Welsch 1969).
//
// Symmetric QR iteration with implicit Wilkinson shifts (Golub & Van Loan,
// "Matrix Computations", Sec. 8.3): each step chases the bulge of one Givens
// rotation down the unreduced block; the first row of the accumulated
// rotation product is carried along, which is all the Gauss rule needs.
// Compiled for both host and device so the solver can be tested on a CPU.
#pragma once

#include <math.h>

namespace slaq {

#ifdef __CUDACC__
#define SLAQ_HD __host__ __device__
#else
#define SLAQ_HD
#endif

// 1/sqrt(x) for x > 0 (the device's reciprocal square root; FP64 division
// and hypot are slow on GB300's small FP64 units)
SLAQ_HD inline double rnorm(double x2) {
#ifdef __CUDA_ARCH__
  return rsqrt(x2);
#else
  return 1.0 / sqrt(x2);
#endif
}

// d[0..m): diagonal (overwritten by the nodes), e[0..m-1): off-diagonal
// (e[i] couples i and i+1; destroyed), w[0..m): squared first components.
// Nodes come out in ascending order.  Returns 0, or 1 without convergence.
SLAQ_HD inline int tridiag_gauss(double *d, double *e, double *w, int m) {
  const double eps = 2.220446049250313e-16;
  const double tiny = 2.2250738585072014e-308;
  for (int i = 0; i < m; ++i) w[i] = (i == 0) ? 1.0 : 0.0;  // first row of the rotations
  int hi = m - 1;
  int steps = 0;
  while (hi > 0) {
    if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi])) + tiny) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo])) + tiny) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++steps > 40 * m) return 1;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
    const double a = d[hi - 1], b = e[hi - 1], c = d[hi];
    const double delta = 0.5 * (a - c);
    const double den = delta + copysign(hypot(delta, b), delta);
    const double mu = c - (b / den) * b;
    double x = d[lo] - mu, y = e[lo];
    for (int k = lo; k < hi; ++k) {
      // rotation G in plane (k, k+1) with G^T (x, y) = (r, 0)
      const double r2 = x * x + y * y;
      double r = 0.0, cs = 1.0, sn = 0.0;
      if (r2 > 1e-290) {
        const double ir = rnorm(r2);
        r = r2 * ir;
        cs = x * ir;
        sn = -y * ir;
      } else if (r2 > 0.0) {  // tiny entries: scaled form
        r = hypot(x, y);
        cs = x / r;
        sn = -y / r;
      }
      if (k > lo) e[k - 1] = r;  // bulge annihilated
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      const double cc = cs * cs, ss = sn * sn, csn = cs * sn;
      d[k] = cc * dk - 2.0 * csn * ek + ss * dk1;
      d[k + 1] = ss * dk + 2.0 * csn * ek + cc * dk1;
      e[k] = csn * (dk - dk1) + (cc - ss) * ek;
      if (k + 1 < hi) {
        const double bulge = -sn * e[k + 1];
        e[k + 1] = cs * e[k + 1];
        x = e[k];
        y = bulge;
      }
      const double wp = w[k], wq = w[k + 1];
      w[k] = cs * wp - sn * wq;
      w[k + 1] = sn * wp + cs * wq;
    }
  }
  for (int i = 0; i < m; ++i) w[i] = w[i] * w[i];
  // insertion sort of the nodes, weights alongside
  for (int i = 1; i < m; ++i) {
    const double di = d[i], wi = w[i];
    int j = i - 1;
    while (j >= 0 && d[j] > di) {
      d[j + 1] = d[j];
      w[j + 1] = w[j];
      --j;
    }
    d[j + 1] = di;
    w[j + 1] = wi;
  }
  return 0;
}

}  // namespace slaq

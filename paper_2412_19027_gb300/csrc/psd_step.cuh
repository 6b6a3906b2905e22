// Step length of one side of a PSD cone, the arithmetic of one thread of the
// PSD step-length kernel.  Host and device code: the CUDA path includes it from
// cones.cu, and a CPU test compiles it with a host compiler to check it against
// the oracle without a GPU.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define CLR_HD __host__ __device__
#else
#define CLR_HD
#endif

namespace clr {

#ifndef __CUDACC__
using std::fabs;
using std::fmin;
using std::isfinite;
using std::sqrt;
#endif

constexpr double kPsdSqrt2 = 1.4142135623730951;

// Step length of one side of a PSD cone of order k <= KM (one thread): the largest
// alpha with S + alpha dS PSD, alpha = -1 / lambda_min(L^{-1} dS L^{-T}), S = L L'
// (Sec. 2.2: the symmetric-cone step is the cone's own ratio test).  lambda_min by
// Householder tridiagonalisation of X = L^{-1} dS L^{-T} (Golub and Van Loan,
// Matrix Computations, Sec. 8.3.1) and bisection on Sturm counts of the
// tridiagonal matrix (the number of negative pivots of T - x I in its LDL'
// recurrence is the number of eigenvalues below x), from the Gershgorin bound
// to a relative width of 1e-14.  Infinity when lambda_min >= 0; zero when S is
// not positive definite in floating point or X is not finite (no step).
template <int KM>
CLR_HD double psd_step_side(const double* __restrict__ v, const double* __restrict__ dv, int k) {
  double L[KM * KM], W[KM * KM];  // row-major; L lower, W full then X in its lower part
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= j; ++i) {
      double x = v[j * (j + 1) / 2 + i], y = dv[j * (j + 1) / 2 + i];
      if (i != j) {
        x /= kPsdSqrt2;
        y /= kPsdSqrt2;
      }
      L[j * KM + i] = x;
      W[i * KM + j] = y;
      W[j * KM + i] = y;
    }
  // Cholesky S = L L' (by columns, left-looking)
  for (int j = 0; j < k; ++j) {
    double d = L[j * KM + j];
    for (int l = 0; l < j; ++l) d -= L[j * KM + l] * L[j * KM + l];
    if (!(d > 0)) return 0.0;
    const double ljj = sqrt(d), r = 1.0 / ljj;
    L[j * KM + j] = ljj;
    for (int i = j + 1; i < k; ++i) {
      double a = L[i * KM + j];
      for (int l = 0; l < j; ++l) a -= L[i * KM + l] * L[j * KM + l];
      L[i * KM + j] = a * r;
    }
  }
  // W = L^{-1} dS, then X = W L^{-T} (lower part, over W's lower part)
  for (int i = 0; i < k; ++i) {
    const double r = 1.0 / L[i * KM + i];
    for (int c = 0; c < k; ++c) {
      double a = W[i * KM + c];
      for (int l = 0; l < i; ++l) a -= L[i * KM + l] * W[l * KM + c];
      W[i * KM + c] = a * r;
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= i; ++j) {
      double a = W[i * KM + j];
      for (int l = 0; l < j; ++l) a -= W[i * KM + l] * L[j * KM + l];
      W[i * KM + j] = a / L[j * KM + j];
    }
  // Householder tridiagonalisation of X (lower part): diagonal a, subdiagonal b
  double a[KM], b[KM];
  double* u = L;  // (L no longer needed) the Householder vector, then p
  double* pv = L + KM;
  for (int j = 0; j + 2 < k; ++j) {
    const double x0 = W[(j + 1) * KM + j];
    double al2 = 0.0;
    for (int i = j + 1; i < k; ++i) al2 += W[i * KM + j] * W[i * KM + j];
    if (al2 - x0 * x0 <= 0.0) {  // the column is already tridiagonal
      b[j] = x0;
      continue;
    }
    const double nrm = sqrt(al2);
    const double be = x0 >= 0.0 ? -nrm : nrm;  // the new subdiagonal entry
    const double tau = (be - x0) / be;         // H = I - tau u u', u_{j+1} = 1
    const double sc = 1.0 / (x0 - be);
    u[j + 1] = 1.0;
    for (int i = j + 2; i < k; ++i) u[i] = W[i * KM + j] * sc;
    double pu = 0.0;
    for (int i = j + 1; i < k; ++i) {  // p = tau X22 u
      double acc = 0.0;
      for (int l = j + 1; l < k; ++l) acc += (i >= l ? W[i * KM + l] : W[l * KM + i]) * u[l];
      pv[i] = tau * acc;
      pu += pv[i] * u[i];
    }
    const double h = 0.5 * tau * pu;
    for (int i = j + 1; i < k; ++i) pv[i] -= h * u[i];  // w = p - (tau/2)(p'u) u
    for (int i = j + 1; i < k; ++i)                     // X22 -= u w' + w u'
      for (int l = j + 1; l <= i; ++l) W[i * KM + l] -= u[i] * pv[l] + pv[i] * u[l];
    b[j] = be;
  }
  bool fin = true;
  for (int i = 0; i < k; ++i) {
    a[i] = W[i * KM + i];
    fin = fin && isfinite(a[i]);
  }
  if (k >= 2) b[k - 2] = W[(k - 1) * KM + (k - 2)];
  for (int i = 0; i + 1 < k; ++i) fin = fin && isfinite(b[i]);
  if (!fin) return 0.0;
  // number of eigenvalues below x: negative pivots of T - x I
  auto below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      double t = a[i] - x;
      if (i > 0) t -= (b[i - 1] * b[i - 1]) / d;
      if (t == 0.0) t = -1e-300;
      cnt += t < 0.0;
      d = t;
    }
    return cnt;
  };
  if (below(0.0) == 0) return INFINITY;
  double lo = INFINITY;
  for (int i = 0; i < k; ++i)
    lo = fmin(lo, a[i] - (i > 0 ? fabs(b[i - 1]) : 0.0) - (i + 1 < k ? fabs(b[i]) : 0.0));
  double hi = 0.0;
  for (int it = 0; it < 80 && hi - lo > 1e-14 * fabs(lo); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (below(mid) > 0) hi = mid;
    else lo = mid;
  }
  return -1.0 / (0.5 * (lo + hi));
}

}  // namespace clr

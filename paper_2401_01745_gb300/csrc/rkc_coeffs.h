// Algorithm 1 (get_stages, get_coeffs) in one definition for the host
// runtime and for the device-resident step kernel, so that both derive the
// same stage counts and coefficients from the same spectral radii.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define EMRKC_HD __host__ __device__
#else
#define EMRKC_HD
#endif

namespace emrkc {

// get_stages without division or square root (one device thread's FP64
// divisions and square roots are slow): the smallest s >= 1 with
// beta s^2 >= x = dt rho, from an FP32 estimate corrected by FP64
// comparisons of beta s^2 with x.  x not finite or beyond 1e15 gives 1 << 24
// (no step has that many stages).
EMRKC_HD inline int rkc_stages_mul(double x, double beta) {
  if (!(x > beta)) return 1;  // also x NaN
  if (!(x < 1e15)) return 1 << 24;
  int s = (int)ceilf(sqrtf((float)x / (float)beta));
  if (s < 1) s = 1;
  while (s > 1 && beta * (double)(s - 1) * (double)(s - 1) >= x) --s;
  while (beta * (double)s * (double)s < x) ++s;
  return s;
}

// get_stages: smallest s >= 1 with beta s^2 >= dt rho, beta = 2 - 4 eps / 3;
// l_s = beta s^2 (the length of the stability interval).  Every path takes
// its stage counts from this definition (the device-resident step calls
// rkc_stages_mul with beta computed once).
EMRKC_HD inline int rkc_stages(double dt, double rho, double eps, double* l_s) {
  const double beta = 2.0 - 4.0 * eps / 3.0;
  const int s = rkc_stages_mul(dt * rho, beta);
  if (l_s) *l_s = beta * (double)s * (double)s;
  return s;
}

// Coefficient tables for s = 1 .. smax in one array: four blocks (mu, nu,
// kappa, c) of rkc_table_len(smax) entries, row s (s + 1 entries) at
// rkc_table_row(s) of each block, then 1 / (beta s^2) and 1 / mu_1 for
// s = 0 .. smax.
EMRKC_HD inline int rkc_table_row(int s) { return (s - 1) * (s + 2) / 2; }
EMRKC_HD inline int rkc_table_len(int smax) { return rkc_table_row(smax + 1); }
EMRKC_HD inline int rkc_table_doubles(int smax) { return 4 * rkc_table_len(smax) + 2 * (smax + 1); }

// get_coeffs into mu, nu, kappa, c [0 .. s]: Chebyshev T_j(w0) by the
// three-term recurrence and T_s'(w0) = s U_{s-1}(w0), U by its own
// recurrence (a first pass for T_s and U_{s-1}, a second for the stages).
EMRKC_HD inline void rkc_coeffs(int s, double eps, double* mu, double* nu, double* kappa, double* c) {
  const double w0 = 1.0 + eps / ((double)s * (double)s);
  double Ta = 1.0, Tb = w0;        // T_{j-1}, T_j at j = 1
  double Ua = 1.0, Ub = 2.0 * w0;  // U_{j-1}, U_j at j = 1
  for (int j = 1; j < s; ++j) {
    const double Tn = 2.0 * w0 * Tb - Ta;
    const double Un = 2.0 * w0 * Ub - Ua;
    Ta = Tb;
    Tb = Tn;
    Ua = Ub;
    Ub = Un;
  }
  // Tb = T_s(w0), Ua = U_{s-1}(w0)
  const double w1 = Tb / ((double)s * Ua);
  mu[0] = nu[0] = kappa[0] = c[0] = 0.0;
  mu[1] = w1 / w0;
  nu[1] = kappa[1] = 0.0;
  c[1] = mu[1];
  double Tm2 = 1.0, Tm1 = w0;  // T_{j-2}, T_{j-1} at j = 2
  for (int j = 2; j <= s; ++j) {
    const double Tj = 2.0 * w0 * Tm1 - Tm2;
    // b_j = 1 / T_j(w0)
    mu[j] = 2.0 * w1 * Tm1 / Tj;
    nu[j] = 2.0 * w0 * Tm1 / Tj;
    kappa[j] = -Tm2 / Tj;
    c[j] = nu[j] * c[j - 1] + kappa[j] * c[j - 2] + mu[j];
    Tm2 = Tm1;
    Tm1 = Tj;
  }
}

}  // namespace emrkc

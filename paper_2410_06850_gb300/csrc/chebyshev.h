// Coefficients of the fine Chebyshev smoother (host; plain C++, also compiled by
// the host-logic tests).  The sweep e_{k+1} = e_k + a_k (e_k - e_{k-1}) +
// b_k D^-1 (r - A e_k), a_0 = 0, applied `degree` times, damps the spectrum of
// D^-1 A on [lo, hi] = [lmax / ratio, 1.1 lmax] by the scaled Chebyshev
// polynomial T_m((hi + lo - 2 lam) / (hi - lo)) / T_m((hi + lo) / (hi - lo)),
// m = degree (three-term recurrence of the Chebyshev semi-iteration).
#pragma once

namespace thermo {

inline void chebyshev_coefficients(double lmax, double ratio, int degree, double* a, double* b) {
  const double lo = lmax / ratio, hi = 1.1 * lmax;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  a[0] = 0.0;
  b[0] = 1.0 / theta;
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    a[k] = rn * rho;
    b[k] = 2.0 * rn / delta;
    rho = rn;
  }
}

}  // namespace thermo

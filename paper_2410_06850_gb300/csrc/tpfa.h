// The paper's cell-centred two-point flux approximation (Sec. 2.2 Eqs. (4)-(5))
// per cell, on the host and the device: one temperature per element, the flux
// of an internal face -kappa_F (t_b - t_a) / h with the harmonic face mean
// kappa_F = 2 / (1/kappa_a + 1/kappa_b), integrated over the face (area |F|:
// transmissibility tau_F = kappa_F |F| / h); a face on Gamma_D carries the flux
// to T_D over half a cell (tau = 2 kappa_c |F| / h); Gamma_N faces carry none.
// Also the design-dependent source f0 (1 - x^p) (Sec. 2.1 Eq. (1)) and the
// adjoint sensitivity of the mean temperature (Sec. 2.3, Eqs. (6)-(7)).
//
// Layout: natural cell order c = i + Nx (j + Ny k), FP64.  Dirichlet faces: one
// byte per cell, bit 0/1 the -x/+x face, 2/3 -y/+y, 4/5 -z/+z (meaningful on the
// box boundary only).  The kernels in tpfa.cu are grid-stride wrappers; the host
// test (tests/test_host_tpfa.py) compiles these functions with the host C++
// compiler and compares them with the oracle.
#pragma once
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define TPFA_HD __host__ __device__ __forceinline__
#else
#define TPFA_HD inline
#endif

namespace thermo {

struct TpfaGrid {
  int nx, ny, nz;       // cells per axis
  double hx, hy, hz;    // cell edges
};

TPFA_HD double tpfa_harm(double a, double b) { return 2.0 / (1.0 / a + 1.0 / b); }

// |F| / h per axis
TPFA_HD void tpfa_ah(const TpfaGrid& g, double& ax, double& ay, double& az) {
  ax = g.hy * g.hz / g.hx;
  ay = g.hx * g.hz / g.hy;
  az = g.hx * g.hy / g.hz;
}

// sum of the Dirichlet transmissibilities of cell c (coefficient of T_D)
TPFA_HD double tpfa_tau_d(const TpfaGrid& g, double kc, uint8_t m) {
  if (!m) return 0.0;
  double ax, ay, az;
  tpfa_ah(g, ax, ay, az);
  double s = 0.0;
  if (m & 1u) s += ax;
  if (m & 2u) s += ax;
  if (m & 4u) s += ay;
  if (m & 8u) s += ay;
  if (m & 16u) s += az;
  if (m & 32u) s += az;
  return 2.0 * kc * s;
}

// (A t)_c = sum_F tau_F (t_c - t_nb) + tau_D t_c
TPFA_HD double tpfa_row(const TpfaGrid& g, const double* kappa, const uint8_t* dface, const double* t, long long c) {
  const int i = (int)(c % g.nx);
  const long long r = c / g.nx;
  const int j = (int)(r % g.ny), k = (int)(r / g.ny);
  const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
  double ax, ay, az;
  tpfa_ah(g, ax, ay, az);
  const double kc = kappa[c], tc = t[c];
  double s = 0.0;
  if (i > 0) s += ax * tpfa_harm(kc, kappa[c - sx]) * (tc - t[c - sx]);
  if (i + 1 < g.nx) s += ax * tpfa_harm(kc, kappa[c + sx]) * (tc - t[c + sx]);
  if (j > 0) s += ay * tpfa_harm(kc, kappa[c - sy]) * (tc - t[c - sy]);
  if (j + 1 < g.ny) s += ay * tpfa_harm(kc, kappa[c + sy]) * (tc - t[c + sy]);
  if (k > 0) s += az * tpfa_harm(kc, kappa[c - sz]) * (tc - t[c - sz]);
  if (k + 1 < g.nz) s += az * tpfa_harm(kc, kappa[c + sz]) * (tc - t[c + sz]);
  return s + tpfa_tau_d(g, kc, dface[c]) * tc;
}

// b_c = f0 (1 - x_c^p) |K| + tau_D T_D
TPFA_HD double tpfa_rhs(const TpfaGrid& g, double xc, double p, double f0, double kc, uint8_t m, double TD) {
  const double vol = g.hx * g.hy * g.hz;
  return f0 * (1.0 - pow(xc, p)) * vol + tpfa_tau_d(g, kc, m) * TD;
}

// dc/dx_e = u^T (df/dx_e - dA/dx_e t + db_D/dx_e) for the mean temperature c,
// u the adjoint (A u = 1/M): dkappa_e/dx_e = p x_e^(p-1) (kmax - kmin); a face
// (e, nb) contributes -dtau/dkappa_e (u_e - u_nb)(t_e - t_nb) with
// dtau/dkappa_e = tau^2 / (2 (|F|/h) kappa_e^2); a Dirichlet face
// -2 (|F|/h) u_e (t_e - T_D); the source -f0 p x_e^(p-1) |K| u_e.
TPFA_HD double tpfa_sens(const TpfaGrid& g, const double* kappa, const uint8_t* dface, const double* x, double p,
                         double kmin, double kmax, double f0, double TD, const double* t, const double* u,
                         long long e) {
  const int i = (int)(e % g.nx);
  const long long r = e / g.nx;
  const int j = (int)(r % g.ny), k = (int)(r / g.ny);
  const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
  double ax, ay, az;
  tpfa_ah(g, ax, ay, az);
  const double ke = kappa[e], te = t[e], ue = u[e];
  double s = 0.0;
  auto face = [&](double ah, long long nb) {
    const double tau = ah * tpfa_harm(ke, kappa[nb]);
    s -= tau * tau / (2.0 * ah * ke * ke) * (ue - u[nb]) * (te - t[nb]);
  };
  if (i > 0) face(ax, e - sx);
  if (i + 1 < g.nx) face(ax, e + sx);
  if (j > 0) face(ay, e - sy);
  if (j + 1 < g.ny) face(ay, e + sy);
  if (k > 0) face(az, e - sz);
  if (k + 1 < g.nz) face(az, e + sz);
  const uint8_t m = dface[e];
  if (m) s -= tpfa_tau_d(g, 1.0, m) * ue * (te - TD);  // tau_D / kappa_e = 2 sum |F|/h
  const double xp1 = (p == 1.0) ? 1.0 : pow(x[e], p - 1.0);
  const double vol = g.hx * g.hy * g.hz;
  return p * xp1 * (kmax - kmin) * s - f0 * p * xp1 * vol * ue;
}

}  // namespace thermo

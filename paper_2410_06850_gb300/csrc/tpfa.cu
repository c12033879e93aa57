// The paper's cell-centred TPFA operator (Sec. 2.2 Eqs. (4)-(5)), its
// design-dependent right-hand side (Sec. 2.1 Eq. (1)) and the mean-temperature
// adjoint sensitivity (Sec. 2.3 Eqs. (6)-(7)) as grid-stride kernels over the
// per-cell functions of tpfa.h, behind context-free C entry points.
#include <math.h>

#include <cmath>

#include "../../include/thermo.h"
#include "common.cuh"
#include "kernels.h"
#include "tpfa.h"

namespace thermo {

static int tpfa_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

__global__ void k_tpfa_kappa(long long M, const double* __restrict__ x, double p, double kmin, double kmax,
                             double* __restrict__ kappa) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x)
    kappa[c] = kmin + pow(x[c], p) * (kmax - kmin);
}
__global__ void k_tpfa_apply(TpfaGrid g, const double* __restrict__ kappa, const uint8_t* __restrict__ dface,
                             const double* __restrict__ t, double* __restrict__ y) {
  const long long M = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x)
    y[c] = tpfa_row(g, kappa, dface, t, c);
}
__global__ void k_tpfa_rhs(TpfaGrid g, const double* __restrict__ x, double p, double f0,
                           const double* __restrict__ kappa, const uint8_t* __restrict__ dface, double TD,
                           double* __restrict__ b) {
  const long long M = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x)
    b[c] = tpfa_rhs(g, x[c], p, f0, kappa[c], dface[c], TD);
}
__global__ void k_tpfa_sens(TpfaGrid g, const double* __restrict__ kappa, const uint8_t* __restrict__ dface,
                            const double* __restrict__ x, double p, double kmin, double kmax, double f0, double TD,
                            const double* __restrict__ t, const double* __restrict__ u, double* __restrict__ dc) {
  const long long M = (long long)g.nx * g.ny * g.nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x)
    dc[e] = tpfa_sens(g, kappa, dface, x, p, kmin, kmax, f0, TD, t, u, e);
}

}  // namespace thermo

using namespace thermo;

static bool tpfa_grid(const int grid[3], const double h[3], TpfaGrid& g) {
  if (!grid || !h) return false;
  for (int k = 0; k < 3; ++k)
    if (grid[k] < 1 || !(h[k] > 0.0) || !std::isfinite(h[k])) return false;
  g.nx = grid[0];
  g.ny = grid[1];
  g.nz = grid[2];
  g.hx = h[0];
  g.hy = h[1];
  g.hz = h[2];
  return true;
}
static thermo_status tpfa_status(cudaError_t e) { return e == cudaSuccess ? THERMO_OK : THERMO_ECUDA; }

extern "C" thermo_status thermo_tpfa_conductivity(long long M, const double* x, double p, double kmin, double kmax,
                                                  double* kappa, void* stream) {
  if (M < 1 || !x || !kappa || !(p >= 1.0) || !(kmin > 0.0) || !(kmax >= kmin)) return THERMO_EINVAL;
  note_launch(), k_tpfa_kappa<<<tpfa_blocks(M), 256, 0, (cudaStream_t)stream>>>(M, x, p, kmin, kmax, kappa);
  return tpfa_status(cudaGetLastError());
}

extern "C" thermo_status thermo_tpfa_apply(const int grid[3], const double h[3], const double* kappa,
                                           const uint8_t* dirichlet_faces, const double* t, double* y, void* stream) {
  TpfaGrid g;
  if (!tpfa_grid(grid, h, g) || !kappa || !dirichlet_faces || !t || !y || t == y) return THERMO_EINVAL;
  const long long M = (long long)g.nx * g.ny * g.nz;
  note_launch(), k_tpfa_apply<<<tpfa_blocks(M), 256, 0, (cudaStream_t)stream>>>(g, kappa, dirichlet_faces, t, y);
  return tpfa_status(cudaGetLastError());
}

extern "C" thermo_status thermo_tpfa_rhs(const int grid[3], const double h[3], const double* x, double p, double f0,
                                         const double* kappa, const uint8_t* dirichlet_faces, double TD, double* b,
                                         void* stream) {
  TpfaGrid g;
  if (!tpfa_grid(grid, h, g) || !x || !kappa || !dirichlet_faces || !b || !(p >= 1.0)) return THERMO_EINVAL;
  const long long M = (long long)g.nx * g.ny * g.nz;
  note_launch(),
      k_tpfa_rhs<<<tpfa_blocks(M), 256, 0, (cudaStream_t)stream>>>(g, x, p, f0, kappa, dirichlet_faces, TD, b);
  return tpfa_status(cudaGetLastError());
}

extern "C" thermo_status thermo_tpfa_sensitivity(const int grid[3], const double h[3], const double* x, double p,
                                                 double kmin, double kmax, double f0, const double* kappa,
                                                 const uint8_t* dirichlet_faces, double TD, const double* t,
                                                 const double* u, double* dc, void* stream) {
  TpfaGrid g;
  if (!tpfa_grid(grid, h, g) || !x || !kappa || !dirichlet_faces || !t || !u || !dc || !(p >= 1.0))
    return THERMO_EINVAL;
  const long long M = (long long)g.nx * g.ny * g.nz;
  note_launch(), k_tpfa_sens<<<tpfa_blocks(M), 256, 0, (cudaStream_t)stream>>>(g, kappa, dirichlet_faces, x, p, kmin,
                                                                               kmax, f0, TD, t, u, dc);
  return tpfa_status(cudaGetLastError());
}

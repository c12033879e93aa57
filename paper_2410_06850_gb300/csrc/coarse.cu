// Coarse levels of the multigrid cycle (Sec. 3, Algorithm 1, grids >= 1).
//
// Level l >= 1 lives on an mx x my x mz grid of cells with L unknowns per
// cell (the local spectral basis of Eq. (8)/(9)).  Its Galerkin operator has
// the 27-neighbour block structure of the cell grid: tiles[c][n][i][j] with
// neighbour n = (dx+1) + 3(dy+1) + 9(dz+1), row i of cell c and column j of
// the neighbour; tiles to cells outside the grid are zero and skipped.
// Vectors are x[c*L + i].  Templates on T = double (FP64 form) or float
// (mixed form); accumulation is in T.
#include "common.cuh"
#include "kernels.h"
#include "coarse_dev.cuh"

namespace thermo {

__device__ __forceinline__ long long nbr_cell(const CLevel& lv, long long c, int n, bool& ok) {
  const int cx = (int)(c % lv.mx);
  const long long t = c / lv.mx;
  const int cy = (int)(t % lv.my), cz = (int)(t / lv.my);
  const int nx = cx + (n % 3) - 1, ny = cy + (n / 3) % 3 - 1, nz = cz + n / 9 - 1;
  ok = nx >= 0 && ny >= 0 && nz >= 0 && nx < lv.mx && ny < lv.my && nz < lv.mz;
  return nx + (long long)lv.mx * (ny + (long long)lv.my * nz);
}

// row . x of one tile row; with a compile-time L that fills whole 16-byte
// vectors (rows and cell vectors then start on 16-byte boundaries) the loads
// are 16 bytes wide
template <class T, int LT>
__device__ __forceinline__ T row_dot(const T* __restrict__ row, const T* __restrict__ xv, int L) {
  T s = T(0);
  if constexpr (LT > 0 && sizeof(T) == 4 && LT % 4 == 0) {
#pragma unroll
    for (int j = 0; j < LT; j += 4) {
      const float4 a = *reinterpret_cast<const float4*>(row + j);
      const float4 b = *reinterpret_cast<const float4*>(xv + j);
      s = fma(a.x, b.x, s);
      s = fma(a.y, b.y, s);
      s = fma(a.z, b.z, s);
      s = fma(a.w, b.w, s);
    }
  } else if constexpr (LT > 0 && sizeof(T) == 8 && LT % 2 == 0) {
#pragma unroll
    for (int j = 0; j < LT; j += 2) {
      const double2 a = *reinterpret_cast<const double2*>(row + j);
      const double2 b = *reinterpret_cast<const double2*>(xv + j);
      s = fma(a.x, b.x, s);
      s = fma(a.y, b.y, s);
    }
  } else {
    for (int j = 0; j < L; ++j) s += row[j] * xv[j];
  }
  return s;
}

// (A x)_row for row (c, i); LT > 0: compile-time L, LT == 0: runtime lv.L
template <class T, int LT>
__device__ __forceinline__ T tile_row(const CLevel& lv, const T* __restrict__ tiles, const T* __restrict__ x,
                                      long long c, int i) {
  const int L = LT > 0 ? LT : lv.L;
  T s = T(0);
  for (int n = 0; n < 27; ++n) {
    bool ok;
    const long long nc = nbr_cell(lv, c, n, ok);
    if (!ok) continue;
    s += row_dot<T, LT>(tiles + (((c * 27 + n) * L) + i) * (long long)L, x + nc * L, L);
  }
  return s;
}

template <class T, int LT>
__global__ void k_capply(CLevel lv, const T* __restrict__ tiles, const T* __restrict__ x, T* __restrict__ y) {
  const long long nrow = lv.ncell * lv.L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / lv.L;
    const int i = (int)(t - c * lv.L);
    y[t] = tile_row<T, LT>(lv, tiles, x, c, i);
  }
}

template <class T, int LT>
__global__ void k_cresidual(CLevel lv, const T* __restrict__ tiles, const T* __restrict__ r, const T* __restrict__ e,
                            T* __restrict__ res) {
  const long long nrow = lv.ncell * lv.L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / lv.L;
    const int i = (int)(t - c * lv.L);
    res[t] = r[t] - tile_row<T, LT>(lv, tiles, e, c, i);
  }
}

// e = Dinv r  (first l1-block-Jacobi sweep from zero)
template <class T>
__global__ void k_csmooth0(CLevel lv, const T* __restrict__ Dinv, const T* __restrict__ r, T* __restrict__ e) {
  const long long nrow = lv.ncell * lv.L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x)
    csmooth0_item<T>(lv, Dinv, r, e, t);
}

// out = e + Dinv (r - A e): cells_per_cta cells, L threads each
template <class T, int LT>
__global__ void k_csmooth(CLevel lv, const T* __restrict__ tiles, const T* __restrict__ Dinv, const T* __restrict__ r,
                          const T* __restrict__ e, T* __restrict__ out, int cpc) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* res = reinterpret_cast<T*>(sm_raw);
  const int L = LT > 0 ? LT : lv.L;
  const int lc = threadIdx.x / L, i = threadIdx.x - lc * L;
  const long long c = (long long)blockIdx.x * cpc + lc;
  const bool act = lc < cpc && c < lv.ncell;
  if (act) res[lc * L + i] = r[c * L + i] - tile_row<T, LT>(lv, tiles, e, c, i);
  __syncthreads();
  if (act) {
    const T* D = Dinv + (c * L + i) * (long long)L;
    T s = T(0);
    for (int j = 0; j < L; ++j) s += D[j] * res[lc * L + j];
    out[c * L + i] = e[c * L + i] + s;
  }
}

// Levels with many vectors per cell (L >= 12): one CTA per cell (ccell_cell in
// coarse_dev.cuh: the cell's 27 tiles staged into shared memory with 16-byte
// copies, the 27 neighbour vectors gathered beside them, partial row sums
// combined over the neighbours in fixed order).
//   MODE 0: out = A x;  MODE 1: out = r - A x;  MODE 2: out = x + Dinv (r - A x)
template <class T, int MODE>
__global__ void k_ccell(CLevel lv, const T* __restrict__ tiles, const T* __restrict__ Dinv, const T* __restrict__ r,
                        const T* __restrict__ x, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  ccell_cell<T, MODE>(lv, tiles, Dinv, r, x, out, blockIdx.x, sm_raw);
}
template <class T, int MODE>
static void launch_ccell(const CLevel& lv, const T* tiles, const T* Dinv, const T* r, const T* x, T* out,
                         cudaStream_t st) {
  const int nt = ((27 * lv.L + 31) / 32) * 32;
  const size_t sm = ccell_smem_bytes<T>(lv.L);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_ccell<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launch(), k_ccell<T, MODE><<<(unsigned)lv.ncell, nt > 1024 ? 1024 : nt, sm, st>>>(lv, tiles, Dinv, r, x, out);
}
constexpr int CCELL_MIN_L = 12;

// rc[G][k] = sum_{c in G} sum_i Psi[G][lc*Lf + i][k] res[c][i]
template <class T>
__global__ void k_crestrict(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ res,
                            T* __restrict__ rc) {
  const long long nout = cs.ncell * cs.L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nout; t += (long long)gridDim.x * blockDim.x)
    crestrict_item<T>(f, cs, Psi, res, rc, t);
}

// The same restriction with Q = g^3 <= 32 threads per output (one per cell of
// the group, lanes of one warp), their partial sums over the cell's Lf basis
// rows combined by a fixed shuffle tree: Q times the parallelism for the small
// deep levels, where one thread per output left most of the GPU idle.
template <class T, int Q>
__global__ void k_crestrict_q(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ res,
                              T* __restrict__ rc) {
  crestrict_q_item<T, Q>(f, cs, Psi, res, rc, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// e[c][i] += sum_k Psi[G(c)][lc*Lf + i][k] ec[G][k]
template <class T>
__global__ void k_cprolong(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ ec,
                           T* __restrict__ e) {
  const long long nrow = f.ncell * f.L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x)
    cprolong_item<T>(f, cs, Psi, ec, e, t);
}

// y = Ainv x (coarsest solve by the precomputed FP64 inverse), one warp per row
template <class T>
__global__ void k_gemv(int n, const double* __restrict__ A, const T* __restrict__ x, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double* xs = reinterpret_cast<double*>(sm_raw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (double)x[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= n) return;
  gemv_row<T>(n, A, xs, y, row, lane);
}

static int cgrid(long long n, int nt = 256) {
  long long b = (n + nt - 1) / nt;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

#define LT_DISPATCH(L, CALL)                 \
  switch (L) {                               \
    case 4: { constexpr int LT = 4; CALL; } break;  \
    case 8: { constexpr int LT = 8; CALL; } break;  \
    case 16: { constexpr int LT = 16; CALL; } break; \
    case 17: { constexpr int LT = 17; CALL; } break; \
    default: { constexpr int LT = 0; CALL; } break;  \
  }

template <class T>
cudaError_t coarse_apply(const CLevel& lv, const T* tiles, const T* x, T* y, cudaStream_t st) {
  if (lv.L >= CCELL_MIN_L) {
    launch_ccell<T, 0>(lv, tiles, nullptr, nullptr, x, y, st);
    return cudaGetLastError();
  }
  note_launch();
  LT_DISPATCH(lv.L, (k_capply<T, LT><<<cgrid(lv.ncell * lv.L), 256, 0, st>>>(lv, tiles, x, y)));
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_residual(const CLevel& lv, const T* tiles, const T* r, const T* e, T* res, cudaStream_t st) {
  if (lv.L >= CCELL_MIN_L) {
    launch_ccell<T, 1>(lv, tiles, nullptr, r, e, res, st);
    return cudaGetLastError();
  }
  note_launch();
  LT_DISPATCH(lv.L, (k_cresidual<T, LT><<<cgrid(lv.ncell * lv.L), 256, 0, st>>>(lv, tiles, r, e, res)));
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_smooth0(const CLevel& lv, const T* Dinv, const T* r, T* e, cudaStream_t st) {
  note_launch(), k_csmooth0<T><<<cgrid(lv.ncell * lv.L), 256, 0, st>>>(lv, Dinv, r, e);
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_smooth(const CLevel& lv, const T* tiles, const T* Dinv, const T* r, const T* e, T* out,
                          cudaStream_t st) {
  if (lv.L >= CCELL_MIN_L) {
    launch_ccell<T, 2>(lv, tiles, Dinv, r, e, out, st);
    return cudaGetLastError();
  }
  const int cpc = lv.L >= 128 ? 1 : 128 / lv.L;
  const long long nb = (lv.ncell + cpc - 1) / cpc;
  const int nt = ((cpc * lv.L + 31) / 32) * 32;
  const size_t sm = (size_t)cpc * lv.L * sizeof(T);
  note_launch();
  LT_DISPATCH(lv.L, (k_csmooth<T, LT><<<(unsigned)nb, nt, sm, st>>>(lv, tiles, Dinv, r, e, out, cpc)));
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_restrict(const CLevel& f, const CLevel& cs, const T* Psi, const T* res, T* rc, cudaStream_t st) {
  const long long nout = cs.ncell * cs.L;
  const int q = cs.g * cs.g * cs.g;
  if (q == 8) {
    const long long nb = (nout * 8 + 255) / 256;
    note_launch(), k_crestrict_q<T, 8><<<(unsigned)nb, 256, 0, st>>>(f, cs, Psi, res, rc);
  } else {
    note_launch(), k_crestrict<T><<<cgrid(nout, 128), 128, 0, st>>>(f, cs, Psi, res, rc);
  }
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_prolong(const CLevel& f, const CLevel& cs, const T* Psi, const T* ec, T* e, cudaStream_t st) {
  note_launch(), k_cprolong<T><<<cgrid(f.ncell * f.L), 256, 0, st>>>(f, cs, Psi, ec, e);
  return cudaGetLastError();
}
template <class T>
cudaError_t dense_gemv(int n, const double* Ainv, const T* x, T* y, cudaStream_t st) {
  const int rows_per = 8;
  const size_t sm = (size_t)n * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_gemv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launch(), k_gemv<T><<<(n + rows_per - 1) / rows_per, rows_per * 32, sm, st>>>(n, Ainv, x, y);
  return cudaGetLastError();
}

#define INST_C(T)                                                                                          \
  template cudaError_t coarse_apply<T>(const CLevel&, const T*, const T*, T*, cudaStream_t);               \
  template cudaError_t coarse_residual<T>(const CLevel&, const T*, const T*, const T*, T*, cudaStream_t);  \
  template cudaError_t coarse_smooth0<T>(const CLevel&, const T*, const T*, T*, cudaStream_t);             \
  template cudaError_t coarse_smooth<T>(const CLevel&, const T*, const T*, const T*, const T*, T*,         \
                                        cudaStream_t);                                                     \
  template cudaError_t coarse_restrict<T>(const CLevel&, const CLevel&, const T*, const T*, T*,            \
                                          cudaStream_t);                                                   \
  template cudaError_t coarse_prolong<T>(const CLevel&, const CLevel&, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t dense_gemv<T>(int, const double*, const T*, T*, cudaStream_t);
INST_C(double)
INST_C(float)

}  // namespace thermo

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
  const int L = lv.L;
  const long long nrow = lv.ncell * L;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / L;
    const int i = (int)(t - c * L);
    const T* D = Dinv + (c * L + i) * (long long)L;
    const T* rv = r + c * L;
    T s = T(0);
    for (int j = 0; j < L; ++j) s += D[j] * rv[j];
    e[t] = s;
  }
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

// Levels with many vectors per cell (L >= 12): one CTA per cell.  The cell's
// 27 tiles (contiguous, 27 L^2 values) are staged into shared memory with
// coalesced loads by all threads, the 27 neighbour vectors gathered beside
// them; thread (n, i) forms the partial row sum of tile n, then the rows are
// summed over the 27 neighbours in fixed order (deterministic).
//   MODE 0: out = A x;  MODE 1: out = r - A x;  MODE 2: out = x + Dinv (r - A x)
template <class T, int MODE>
__global__ void k_ccell(CLevel lv, const T* __restrict__ tiles, const T* __restrict__ Dinv, const T* __restrict__ r,
                        const T* __restrict__ x, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int L = lv.L;
  const int LL = L * L;
  constexpr int V = 16 / sizeof(T);      // elements per 16-byte chunk
  const long long c = blockIdx.x;
  // the cell's 27 tiles start at element c * 27 L^2, generally not on a 16-byte
  // boundary: copy the aligned 16-byte chunks that cover them (the allocation
  // has slack past its end) and index the tiles from the head offset
  const long long e0 = c * 27 * (long long)LL;
  const long long a0 = e0 & ~(long long)(V - 1);
  const int head = (int)(e0 - a0);
  const int nchunk = (int)((e0 + 27 * LL - a0 + V - 1) / V);
  T* buf = reinterpret_cast<T*>(sm_raw);  // nchunk * V elements
  T* ts = buf + head;                     // [27][L][L]
  T* xs = buf + ((nchunk * V + V - 1) / V) * V;  // [27][L] (zero outside the grid)
  T* part = xs + 27 * L;                 // [27][L]
  T* res = part + 27 * L;                // [L]
  const int cx = (int)(c % lv.mx);
  const long long tt = c / lv.mx;
  const int cy = (int)(tt % lv.my), cz = (int)(tt / lv.my);
  // asynchronous 16-byte copies (all in flight at once), completed before the barrier
  for (int k = threadIdx.x; k < nchunk; k += blockDim.x) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(buf + (long long)k * V);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(tiles + a0 + (long long)k * V)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int k = threadIdx.x; k < 27 * L; k += blockDim.x) {
    const int n = k / L, j = k - n * L;
    const int nx = cx + n % 3 - 1, ny = cy + (n / 3) % 3 - 1, nz = cz + n / 9 - 1;
    T v = T(0);
    if (nx >= 0 && ny >= 0 && nz >= 0 && nx < lv.mx && ny < lv.my && nz < lv.mz)
      v = x[(nx + (long long)lv.mx * (ny + (long long)lv.my * nz)) * L + j];
    xs[k] = v;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  for (int idx = threadIdx.x; idx < 27 * L; idx += blockDim.x) {
    const int n = idx / L;
    const T* row = ts + (long long)idx * L;  // tile n, row i
    const T* xv = xs + n * L;
    T s = T(0), s2 = T(0);
    int j = 0;
    for (; j + 1 < L; j += 2) {
      s = fma(row[j], xv[j], s);
      s2 = fma(row[j + 1], xv[j + 1], s2);
    }
    if (j < L) s = fma(row[j], xv[j], s);
    part[idx] = s + s2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    T s = T(0);
    for (int n = 0; n < 27; ++n) s += part[n * L + i];
    if (MODE == 0)
      out[c * L + i] = s;
    else if (MODE == 1)
      out[c * L + i] = r[c * L + i] - s;
    else
      res[i] = r[c * L + i] - s;
  }
  if (MODE == 2) {
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      const T* D = Dinv + (c * L + i) * (long long)L;
      T s = T(0);
      for (int j = 0; j < L; ++j) s = fma(D[j], res[j], s);
      out[c * L + i] = x[c * L + i] + s;
    }
  }
}
template <class T, int MODE>
static void launch_ccell(const CLevel& lv, const T* tiles, const T* Dinv, const T* r, const T* x, T* out,
                         cudaStream_t st) {
  const int nt = ((27 * lv.L + 31) / 32) * 32;
  const size_t V = 16 / sizeof(T);
  const size_t sm = ((size_t)27 * lv.L * lv.L + 2 * V + (size_t)55 * lv.L) * sizeof(T);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_ccell<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_launch(), k_ccell<T, MODE><<<(unsigned)lv.ncell, nt > 1024 ? 1024 : nt, sm, st>>>(lv, tiles, Dinv, r, x, out);
}
constexpr int CCELL_MIN_L = 12;

// rc[G][k] = sum_{c in G} sum_i Psi[G][lc*Lf + i][k] res[c][i]
template <class T>
__global__ void k_crestrict(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ res,
                            T* __restrict__ rc) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
  const long long nout = cs.ncell * Lc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nout; t += (long long)gridDim.x * blockDim.x) {
    const long long G = t / Lc;
    const int k = (int)(t - G * Lc);
    const int gx = (int)(G % cs.mx);
    const long long tt = G / cs.mx;
    const int gy = (int)(tt % cs.my), gz = (int)(tt / cs.my);
    const T* ps = Psi + G * (long long)nloc * Lc;
    T s = T(0);
    for (int lz = 0; lz < g; ++lz)
      for (int ly = 0; ly < g; ++ly)
        for (int lx = 0; lx < g; ++lx) {
          const long long c = (gx * g + lx) + (long long)f.mx * ((gy * g + ly) + (long long)f.my * (gz * g + lz));
          const int lc = lx + g * (ly + g * lz);
          for (int i = 0; i < Lf; ++i) s += ps[(long long)(lc * Lf + i) * Lc + k] * res[c * Lf + i];
        }
    rc[t] = s;
  }
}

// The same restriction with Q = g^3 <= 32 threads per output (one per cell of
// the group, lanes of one warp), their partial sums over the cell's Lf basis
// rows combined by a fixed shuffle tree: Q times the parallelism for the small
// deep levels, where one thread per output left most of the GPU idle.
template <class T, int Q>
__global__ void k_crestrict_q(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ res,
                              T* __restrict__ rc) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
  const long long nout = cs.ncell * Lc;
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lc = (int)(gt % Q);
  const long long t = gt / Q;
  T s = T(0);
  if (t < nout) {
    const long long G = t / Lc;
    const int k = (int)(t - G * Lc);
    const int gx = (int)(G % cs.mx);
    const long long tt = G / cs.mx;
    const int gy = (int)(tt % cs.my), gz = (int)(tt / cs.my);
    const int lx = lc % g, ly = (lc / g) % g, lz = lc / (g * g);
    const long long c = (gx * g + lx) + (long long)f.mx * ((gy * g + ly) + (long long)f.my * (gz * g + lz));
    const T* ps = Psi + G * (long long)nloc * Lc + (long long)lc * Lf * Lc + k;
    const T* rv = res + c * Lf;
    for (int i = 0; i < Lf; ++i) s = fma(ps[(long long)i * Lc], rv[i], s);
  }
#pragma unroll
  for (int o = Q / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (t < nout && lc == 0) rc[t] = s;
}

// e[c][i] += sum_k Psi[G(c)][lc*Lf + i][k] ec[G][k]
template <class T>
__global__ void k_cprolong(CLevel f, CLevel cs, const T* __restrict__ Psi, const T* __restrict__ ec,
                           T* __restrict__ e) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
  const long long nrow = f.ncell * Lf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrow; t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / Lf;
    const int i = (int)(t - c * Lf);
    const int cx = (int)(c % f.mx);
    const long long tt = c / f.mx;
    const int cy = (int)(tt % f.my), cz = (int)(tt / f.my);
    const long long G = (cx / g) + (long long)cs.mx * ((cy / g) + (long long)cs.my * (cz / g));
    const int lc = (cx % g) + g * ((cy % g) + g * (cz % g));
    const T* ps = Psi + G * (long long)nloc * Lc + (long long)(lc * Lf + i) * Lc;
    const T* ev = ec + G * Lc;
    T s = T(0);
    for (int k = 0; k < Lc; ++k) s += ps[k] * ev[k];
    e[t] += s;
  }
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
  const double* a = A + (long long)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += a[j] * xs[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = (T)s;
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

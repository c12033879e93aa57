// Dense FP64 Cholesky factorisation and explicit inverse of the coarsest
// Galerkin operator (the direct coarse solve of Sec. 3 Algorithm 1; the paper
// uses a sparse LU in Sec. 4, and A_L is SPD, so a Cholesky factor serves).
//
// Blocked in 64 x 64 tiles, right-looking:
//   for each block column k:  L_kk = chol(A_kk)                (one CTA)
//                             L_ik = A_ik L_kk^-T, i > k       (one CTA per tile row)
//                             A_ij -= L_ik L_jk^T, i >= j > k  (one CTA per tile)
// then W = L^-1 block row by block row,
//   W_ii = L_ii^-1,  W_ic = -L_ii^-1 sum_{k=c}^{i-1} L_ik W_kc  (c < i),
// and A^-1 = W^T W (lower tiles, mirrored).  About 4 n/64 launches in all
// (the unblocked form took two per column).  A matrix order that is not a
// multiple of 64 is padded with identity rows and columns inside the tiles;
// nothing outside n x n is read or written.  A non-positive or non-finite
// pivot records its (1-based) index in *status (the first one only) and is
// replaced by 1 so that the remaining kernels finish on finite data.
#include "common.cuh"
#include "kernels.h"

namespace thermo {

namespace {

constexpr int DB = 64;        // tile edge
constexpr int DLD = DB + 1;   // shared-memory leading dimension (odd: conflict-free columns)
constexpr int DNT = 256;      // threads per CTA (16 x 16, 4 x 4 outputs each)
constexpr size_t TILE_SMEM = 2 * (size_t)DB * DLD * sizeof(double);

// s[r][c] (r, c < 64) = element (r0 + r, c0 + c) of the n x n row-major M, or of
// its transpose when T; outside the matrix: the identity's entry.
template <bool T>
__device__ void load_tile(double* s, const double* M, int n, int r0, int c0) {
  for (int i = threadIdx.x; i < DB * DB; i += blockDim.x) {
    const int a = i / DB, b = i % DB;  // b runs fastest: coalesced along the stored rows
    if (T) {  // s[b][a] = M[c0 + a][r0 + b]
      const int gr = c0 + a, gc = r0 + b;
      s[b * DLD + a] = (gr < n && gc < n) ? M[(long long)gr * n + gc] : (r0 + b == c0 + a ? 1.0 : 0.0);
    } else {  // s[a][b] = M[r0 + a][c0 + b]
      const int gr = r0 + a, gc = c0 + b;
      s[a * DLD + b] = (gr < n && gc < n) ? M[(long long)gr * n + gc] : (gr == gc ? 1.0 : 0.0);
    }
  }
}

// acc[r][c] += sum_k sA[4ty + r][k] sB[k][4tx + c]
__device__ __forceinline__ void tile_mma(double (&acc)[4][4], const double* sA, const double* sB) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 4
  for (int k = 0; k < DB; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = sA[(4 * ty + r) * DLD + k];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = sB[k * DLD + 4 * tx + c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
  }
}

// Cholesky of the diagonal tile k (lower part of A in place); first bad pivot -> *status
__global__ void __launch_bounds__(DNT) k_potrf_tile(int n, double* A, int k, int* status) {
  __shared__ double s[DB][DLD];
  const int k0 = k * DB, tid = threadIdx.x;
  for (int i = tid; i < DB * DB; i += DNT) {
    const int r = i / DB, c = i % DB;
    const bool in = k0 + r < n && k0 + c < n;
    s[r][c] = c > r ? 0.0 : (in ? A[(long long)(k0 + r) * n + k0 + c] : (r == c ? 1.0 : 0.0));
  }
  __syncthreads();
  for (int j = 0; j < DB; ++j) {
    if (tid == 0) {
      const double d = s[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (k0 + j < n) atomicCAS(status, 0, k0 + j + 1);
        s[j][j] = 1.0;
      } else {
        s[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double djj = s[j][j];
    for (int r = j + 1 + tid; r < DB; r += DNT) s[r][j] /= djj;
    __syncthreads();
    const int m = DB - 1 - j;
    for (int i = tid; i < m * m; i += DNT) {
      const int r = j + 1 + i / m, c = j + 1 + i % m;
      if (c <= r) s[r][c] -= s[r][j] * s[c][j];
    }
    __syncthreads();
  }
  for (int i = tid; i < DB * DB; i += DNT) {
    const int r = i / DB, c = i % DB;
    if (c <= r && k0 + r < n && k0 + c < n) A[(long long)(k0 + r) * n + k0 + c] = s[r][c];
  }
}

// L_ik = A_ik L_kk^-T for tile rows i = k + 1 + blockIdx.x (one row of the tile per thread)
__global__ void __launch_bounds__(DB) k_trsm_tile(int n, double* A, int k) {
  extern __shared__ double sm_d[];
  double(*sL)[DLD] = reinterpret_cast<double(*)[DLD]>(sm_d);
  double(*sP)[DLD] = reinterpret_cast<double(*)[DLD]>(sm_d + DB * DLD);
  const int k0 = k * DB, i0 = (k + 1 + blockIdx.x) * DB, r = threadIdx.x;
  load_tile<false>(&sL[0][0], A, n, k0, k0);
  load_tile<false>(&sP[0][0], A, n, i0, k0);
  __syncthreads();
  // row r of X with X L^T = P: x_j = p_j / L_jj, then p_c -= x_j L_cj for c > j
  for (int j = 0; j < DB; ++j) {
    const double xj = sP[r][j] / sL[j][j];
    sP[r][j] = xj;
    for (int c = j + 1; c < DB; ++c) sP[r][c] -= xj * sL[c][j];
  }
  if (i0 + r < n)
    for (int c = 0; c < DB && k0 + c < n; ++c) A[(long long)(i0 + r) * n + k0 + c] = sP[r][c];
}

// tile pair index p -> (i, j), j <= i, of a lower triangle of tiles
__device__ __forceinline__ void tri_pair(int p, int& i, int& j) {
  i = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  j = p - i * (i + 1) / 2;
}

// trailing update A_ij -= L_ik L_jk^T for tiles k < j <= i
__global__ void __launch_bounds__(DNT) k_syrk_tile(int n, double* A, int k) {
  extern __shared__ double sm_d[];
  double* sA = sm_d;
  double* sB = sm_d + DB * DLD;
  int i, j;
  tri_pair(blockIdx.x, i, j);
  i += k + 1;
  j += k + 1;
  load_tile<false>(sA, A, n, i * DB, k * DB);  // L_ik
  load_tile<true>(sB, A, n, k * DB, j * DB);   // (L_jk)^T: sB[kk][c] = L[j*DB + c][k*DB + kk]
  __syncthreads();
  double acc[4][4] = {};
  tile_mma(acc, sA, sB);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int gr = i * DB + 4 * ty + rr, gc = j * DB + 4 * tx + cc;
      if (gr < n && gc < n) A[(long long)gr * n + gc] -= acc[rr][cc];
    }
}

// inverse of the lower triangular diagonal tile i of L -> Dinv[i] (DB x DB, row-major)
__global__ void __launch_bounds__(DB) k_trtri_tile(int n, const double* L, double* Dinv) {
  extern __shared__ double sm_d[];
  double(*sL)[DLD] = reinterpret_cast<double(*)[DLD]>(sm_d);
  double(*sX)[DLD] = reinterpret_cast<double(*)[DLD]>(sm_d + DB * DLD);
  const int i = blockIdx.x, c = threadIdx.x;
  load_tile<false>(&sL[0][0], L, n, i * DB, i * DB);
  for (int r = 0; r < DB; ++r) sX[r][c] = (r == c) ? 1.0 : 0.0;
  __syncthreads();
  // column c of X with L X = I (forward substitution, column per thread)
  for (int j = 0; j < DB; ++j) {
    const double xj = sX[j][c] / sL[j][j];
    sX[j][c] = xj;
    for (int r = j + 1; r < DB; ++r) sX[r][c] -= sL[r][j] * xj;
  }
  double* out = Dinv + (long long)i * DB * DB;
  for (int r = 0; r < DB; ++r) out[r * DB + c] = (r >= c) ? sX[r][c] : 0.0;
}

// block row i of W = L^-1: W_ic = -Dinv_i sum_{k=c}^{i-1} L_ik W_kc (c = blockIdx.x < i), W_ii = Dinv_i
__global__ void __launch_bounds__(DNT) k_winv_row(int n, const double* L, const double* Dinv, double* W, int i) {
  extern __shared__ double sm_d[];
  double* sA = sm_d;
  double* sB = sm_d + DB * DLD;
  const int c = blockIdx.x, tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double* Di = Dinv + (long long)i * DB * DB;
  if (c == i) {
    for (int e = threadIdx.x; e < DB * DB; e += DNT) {
      const int r = e / DB, cc = e % DB;
      if (i * DB + r < n && i * DB + cc < n) W[(long long)(i * DB + r) * n + i * DB + cc] = Di[e];
    }
    return;
  }
  double acc[4][4] = {};
  for (int k = c; k < i; ++k) {
    load_tile<false>(sA, L, n, i * DB, k * DB);
    load_tile<false>(sB, W, n, k * DB, c * DB);
    __syncthreads();
    tile_mma(acc, sA, sB);
    __syncthreads();
  }
  // T = acc -> sB; Dinv_i -> sA; W_ic = -Dinv_i T
  for (int e = threadIdx.x; e < DB * DB; e += DNT) sA[(e / DB) * DLD + e % DB] = Di[e];
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) sB[(4 * ty + rr) * DLD + 4 * tx + cc] = acc[rr][cc];
  __syncthreads();
  double w[4][4] = {};
  tile_mma(w, sA, sB);
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int gr = i * DB + 4 * ty + rr, gc = c * DB + 4 * tx + cc;
      if (gr < n && gc < n) W[(long long)gr * n + gc] = -w[rr][cc];
    }
}

// X_ab = sum_{k >= a} W_ka^T W_kb for tiles b <= a; X_ba = X_ab^T
__global__ void __launch_bounds__(DNT) k_wtw_tile(int n, int nt, const double* W, double* X) {
  extern __shared__ double sm_d[];
  double* sA = sm_d;
  double* sB = sm_d + DB * DLD;
  int a, b;
  tri_pair(blockIdx.x, a, b);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k = a; k < nt; ++k) {
    load_tile<true>(sA, W, n, a * DB, k * DB);   // sA[r][kk] = W[k*DB + kk][a*DB + r]
    load_tile<false>(sB, W, n, k * DB, b * DB);  // sB[kk][c] = W[k*DB + kk][b*DB + c]
    __syncthreads();
    tile_mma(acc, sA, sB);
    __syncthreads();
  }
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int gr = a * DB + 4 * ty + rr, gc = b * DB + 4 * tx + cc;
      if (gr < n && gc < n) {
        X[(long long)gr * n + gc] = acc[rr][cc];
        X[(long long)gc * n + gr] = acc[rr][cc];
      }
    }
}

__global__ void k_symm(int n, double* A) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n * n;
       w += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(w / n), j = (int)(w % n);
    if (i > j) {
      const double v = 0.5 * (A[(long long)i * n + j] + A[(long long)j * n + i]);
      A[(long long)i * n + j] = v;
      A[(long long)j * n + i] = v;
    }
  }
}

}  // namespace

long long cholesky_work_size(int n) {
  const long long nt = (n + DB - 1) / DB;
  return (long long)n * n + nt * DB * DB;
}

// A (n x n, symmetrised here) is overwritten by its Cholesky factor (lower
// part); Ainv receives A^-1; work holds cholesky_work_size(n) doubles.
cudaError_t cholesky_inverse(int n, double* A, double* Ainv, double* work, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nt = (n + DB - 1) / DB;
  double* W = work;
  double* Dinv = work + (long long)n * n;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_syrk_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_trsm_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_trtri_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_winv_row, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_wtw_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) !=
      cudaSuccess)
    return e;
  long long nb = ((long long)n * n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  note_launch(), k_symm<<<(unsigned)nb, 256, 0, st>>>(n, A);
  for (int k = 0; k < nt; ++k) {
    note_launch(), k_potrf_tile<<<1, DNT, 0, st>>>(n, A, k, status);
    const int rest = nt - 1 - k;
    if (rest > 0) {
      note_launch(), k_trsm_tile<<<rest, DB, TILE_SMEM, st>>>(n, A, k);
      note_launch(), k_syrk_tile<<<rest * (rest + 1) / 2, DNT, TILE_SMEM, st>>>(n, A, k);
    }
  }
  note_launch(), k_trtri_tile<<<nt, DB, TILE_SMEM, st>>>(n, A, Dinv);
  for (int i = 0; i < nt; ++i) note_launch(), k_winv_row<<<i + 1, DNT, TILE_SMEM, st>>>(n, A, Dinv, W, i);
  note_launch(), k_wtw_tile<<<nt * (nt + 1) / 2, DNT, TILE_SMEM, st>>>(n, nt, W, Ainv);
  return cudaGetLastError();
}

}  // namespace thermo

// CTA-wide FP32 solver for the K smallest eigenpairs of a small dense
// symmetric matrix held in shared memory, used by the local spectral problems
// of Sec. 3 (Eq. (8) per block, Eq. (9) per group) before their FP64
// Rayleigh-Ritz refinement.
//
//   1. Householder reduction to tridiagonal form T = Q^T A Q (Q = H_0 ... H_{n-3},
//      H_k = I - tau_k v_k v_k^T), reflectors kept in the columns of A below the
//      subdiagonal;
//   2. the K smallest eigenvalues of T by bisection on Sturm counts;
//   3. eigenvectors of T by inverse iteration (tridiagonal elimination with
//      partial pivoting, three steps from a fixed start), Gram-Schmidt against the
//      earlier members of a cluster of close eigenvalues (gap < 1e-3 ||T||), so
//      that a degenerate cluster yields an orthonormal basis of its space;
//   4. back-transformation y <- Q y.
// About (4/3) n^3 flops for step 1, O(K n) for the rest, against a full
// diagonalisation by Jacobi sweeps.  The FP64 refinement that follows works on
// the span of these K >= L vectors, so FP32 accuracy here only has to place
// the L wanted vectors inside that span.
#pragma once
#include "common.cuh"

namespace thermo {

__device__ double cta_sum(double v, double* sh);  // setup.cu

// 1. in place: A (n x n, leading dimension lda, full symmetric storage) ->
// d[0..n-1], e[0..n-2]; reflector k in A[k+1..n-1][k] (v[k+1] = x0 - alpha), tau[k].
// p: n floats of scratch.  blockDim.x must be 256 (the update's 16 x 16 grid).
__device__ void eig_tridiag(float* A, int lda, int n, float* d, float* e, float* tau, float* p, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k + 2 < n; ++k) {
    double s = 0.0;
    for (int i = k + 2 + tid; i < n; i += nt) {
      const float v = A[i * lda + k];
      s += (double)v * v;
    }
    s = cta_sum(s, sh);
    if (tid == 0) {
      const float x0 = A[(k + 1) * lda + k];
      d[k] = A[k * lda + k];
      if (s == 0.0) {
        tau[k] = 0.f;
        e[k] = x0;
      } else {
        const double mu = sqrt((double)x0 * x0 + s);
        const float alpha = (float)(x0 > 0.f ? -mu : mu);
        const float v0 = x0 - alpha;  // no cancellation: alpha has the opposite sign of x0
        tau[k] = (float)(2.0 / ((double)v0 * v0 + s));
        e[k] = alpha;
        A[(k + 1) * lda + k] = v0;
      }
    }
    __syncthreads();
    const float t = tau[k];
    if (t == 0.f) continue;  // uniform: every thread reads the same shared value
    // p = t A22 v: four threads per row (a fixed shuffle tree combines them)
    for (int i0 = k + 1; i0 < n; i0 += nt / 4) {
      const int i = i0 + (tid >> 2);
      float acc = 0.f;
      if (i < n) {
        const float* row = A + i * lda;
        for (int j = k + 1 + (tid & 3); j < n; j += 4) acc = fmaf(row[j], A[j * lda + k], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (i < n && (tid & 3) == 0) p[i] = t * acc;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = k + 1 + tid; i < n; i += nt) pv += (double)p[i] * A[i * lda + k];
    pv = cta_sum(pv, sh);
    const float kc = (float)(0.5 * t * pv);
    for (int i = k + 1 + tid; i < n; i += nt) p[i] -= kc * A[i * lda + k];  // w = p - K v
    __syncthreads();
    // rank-2 update on a 16 x 16 thread grid (no index division)
    for (int i = k + 1 + (tid >> 4); i < n; i += nt / 16) {
      const float vi = A[i * lda + k], wi = p[i];
      float* row = A + i * lda;
      for (int j = k + 1 + (tid & 15); j < n; j += 16) row[j] -= vi * p[j] + wi * A[j * lda + k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(n - 2) * lda + n - 2];
      e[n - 2] = A[(n - 1) * lda + n - 2];
    }
    d[n - 1] = A[(n - 1) * lda + n - 1];
  }
  __syncthreads();
}

// number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots; e2 =
// the squared off-diagonal; a fast division: only the signs of the pivots count)
__device__ __forceinline__ int eig_sturm(const float* d, const float* e2, int n, float x, float pivmin) {
  float q = d[0] - x;
  int c = q < 0.f ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = d[i] - x - __fdividef(e2[i - 1], q);
    c += q < 0.f ? 1 : 0;
  }
  return c;
}

// 2. (threads j < K) lam[j] = the j-th smallest eigenvalue; tn[0] = Gershgorin bound of ||T||;
// e2: n floats of scratch (the squared off-diagonal)
__device__ void eig_bisect(const float* d, const float* e, int n, int K, float* lam, float* tn, float* e2) {
  for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) e2[i] = e[i] * e[i];
  __syncthreads();
  const int j = threadIdx.x;
  if (j < K) {
    float lo = 3.0e38f, hi = -3.0e38f;
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i < n - 1 ? fabsf(e[i]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
    }
    const float norm = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), 1e-30f);
    const float pivmin = 1e-30f * norm, tol = 2e-7f * norm;
    float a = lo, b = hi;
    for (int it = 0; it < 80 && b - a > tol; ++it) {
      const float mid = 0.5f * (a + b);
      if (mid <= a || mid >= b) break;
      if (eig_sturm(d, e2, n, mid, pivmin) > j)
        b = mid;
      else
        a = mid;
    }
    lam[j] = 0.5f * (a + b);
    if (j == 0) tn[0] = norm;
  }
  __syncthreads();
}

// 3. (one thread per cluster of close eigenvalues) eigenvectors of T: row j of
// Y (leading dimension ldy) for lam[j].  Each inverse-iteration step factors
// T - lam I with partial pivoting row by row while it eliminates the
// right-hand side (U kept: 3 n floats of lu per eigenvalue), then back-substitutes.
__device__ void eig_tri_vectors(const float* d, const float* e, int n, int K, const float* lam, float tnorm, float* Y,
                                int ldy, float* lu) {
  const int jh = threadIdx.x;
  const float ctol = 1e-3f * tnorm, eps = 1.2e-7f * tnorm;
  const bool head = jh < K && (jh == 0 || lam[jh] - lam[jh - 1] >= ctol);
  if (head) {
    float* ud = lu + (size_t)jh * 3 * n;
    float* us = ud + n;
    float* us2 = us + n;
    for (int j = jh; j < K && (j == jh || lam[j] - lam[j - 1] < ctol); ++j) {
      const float l = lam[j];
      float* y = Y + (size_t)j * ldy;
      for (int i = 0; i < n; ++i) y[i] = 1.f + 0.125f * (float)(((i * 7 + j * 13) % 11) - 5);
      for (int it = 0; it < 3; ++it) {
        float cd = d[0] - l, cs = n > 1 ? e[0] : 0.f, yc = y[0];
        for (int i = 0; i + 1 < n; ++i) {
          const float sub = e[i], nd = d[i + 1] - l, ns = (i + 1 < n - 1) ? e[i + 1] : 0.f, yn = y[i + 1];
          if (fabsf(cd) >= fabsf(sub)) {  // row i pivots
            if (cd == 0.f) cd = eps;
            const float m = __fdividef(sub, cd);
            ud[i] = cd, us[i] = cs, us2[i] = 0.f, y[i] = yc;
            cd = nd - m * cs;
            cs = ns;
            yc = yn - m * yc;
          } else {  // rows i and i+1 exchanged
            const float m = __fdividef(cd, sub);
            ud[i] = sub, us[i] = nd, us2[i] = ns, y[i] = yn;
            cd = cs - m * nd;
            cs = -m * ns;
            yc = yc - m * yn;
          }
        }
        ud[n - 1] = cd != 0.f ? cd : eps;
        y[n - 1] = yc;
        for (int i = n - 1; i >= 0; --i) {
          float s = y[i];
          if (i + 1 < n) s -= us[i] * y[i + 1];
          if (i + 2 < n) s -= us2[i] * y[i + 2];
          y[i] = __fdividef(s, ud[i]);
        }
        for (int q = jh; q < j; ++q) {  // orthogonalise against the cluster's earlier vectors
          const float* yq = Y + (size_t)q * ldy;
          float dt = 0.f;
          for (int i = 0; i < n; ++i) dt = fmaf(yq[i], y[i], dt);
          for (int i = 0; i < n; ++i) y[i] = fmaf(-dt, yq[i], y[i]);
        }
        float nn = 0.f, mx = 0.f;
        for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(y[i]));
        const float sc = mx > 0.f ? 1.f / mx : 1.f;  // scale first: no overflow in the norm
        for (int i = 0; i < n; ++i) {
          y[i] *= sc;
          nn = fmaf(y[i], y[i], nn);
        }
        const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
        for (int i = 0; i < n; ++i) y[i] *= inv;
      }
    }
  }
  __syncthreads();
}

// 4. rows of Y (K vectors) <- Q y, applying H_{n-3} ... H_0 (one warp per vector)
__device__ void eig_back(const float* A, int lda, int n, const float* tau, float* Y, int ldy, int K) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = w; j < K; j += nw) {
    float* y = Y + (size_t)j * ldy;
    for (int k = n - 3; k >= 0; --k) {
      const float t = tau[k];
      if (t == 0.f) continue;
      float s = 0.f;
      for (int i = k + 1 + lane; i < n; i += 32) s = fmaf(A[i * lda + k], y[i], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float f = t * s;
      for (int i = k + 1 + lane; i < n; i += 32) y[i] = fmaf(-f, A[i * lda + k], y[i]);
      __syncwarp();
    }
  }
  __syncthreads();
}

// Shared-memory floats of eig_lowest's scratch (d, e, tau, p, ||T||) and of
// its per-eigenvalue factor storage lu (which may alias memory that is free
// until eig_lowest returns)
__host__ __device__ inline size_t eig_scratch_floats(int n) { return 4 * (size_t)n + 4; }
__host__ __device__ inline size_t eig_lu_floats(int n, int K) { return 3 * (size_t)n * K; }

// The K smallest eigenpairs of the symmetric A (destroyed): lam[0..K-1]
// ascending, eigenvectors in the rows of Y (K x n, leading dimension ldy).
__device__ void eig_lowest(float* A, int lda, int n, int K, float* lam, float* Y, int ldy, float* scr, float* lu,
                           double* sh) {
  float* d = scr;
  float* e = d + n;
  float* tau = e + n;
  float* p = tau + n;
  float* tn = p + n;
  eig_tridiag(A, lda, n, d, e, tau, p, sh);
  eig_bisect(d, e, n, K, lam, tn, p);
  eig_tri_vectors(d, e, n, K, lam, tn[0], Y, ldy, lu);
  eig_back(A, lda, n, tau, Y, ldy, K);
}

}  // namespace thermo

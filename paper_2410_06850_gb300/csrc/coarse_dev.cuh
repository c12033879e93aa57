// Per-cell and per-item device bodies of the coarse-level operations (the
// kernels of coarse.cu are thin grid-stride or one-cell wrappers around them).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace thermo {

// One cell of a level with many vectors per cell, by the whole CTA: the cell's
// 27 tiles (contiguous, 27 L^2 values) are staged into shared memory with
// coalesced 16-byte copies, the 27 neighbour vectors gathered beside them;
// thread (n, i) forms the partial row sum of tile n, then the rows are summed
// over the 27 neighbours in fixed order (deterministic).
//   MODE 0: out = A x;  MODE 1: out = r - A x;  MODE 2: out = x + Dinv (r - A x)
// Shared memory: ccell_smem_bytes(L).  Every thread of the CTA must call it; a
// CTA that loops over cells needs a barrier between two calls.
template <class T>
__host__ __device__ inline size_t ccell_smem_bytes(int L) {
  const size_t V = 16 / sizeof(T);
  return ((size_t)27 * L * L + 2 * V + (size_t)55 * L) * sizeof(T);
}
template <class T, int MODE>
__device__ __forceinline__ void ccell_cell(const CLevel& lv, const T* __restrict__ tiles, const T* __restrict__ Dinv,
                                           const T* __restrict__ r, const T* __restrict__ x, T* __restrict__ out,
                                           long long c, unsigned char* sm_raw) {
  const int L = lv.L;
  const int LL = L * L;
  constexpr int V = 16 / sizeof(T);      // elements per 16-byte chunk
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

// e[t] = (Dinv r)[t] for dof t = (c, i): the first l1-block-Jacobi sweep from zero
template <class T>
__device__ __forceinline__ void csmooth0_item(const CLevel& lv, const T* __restrict__ Dinv, const T* __restrict__ r,
                                              T* __restrict__ e, long long t) {
  const int L = lv.L;
  const long long c = t / L;
  const int i = (int)(t - c * L);
  const T* D = Dinv + (c * L + i) * (long long)L;
  const T* rv = r + c * L;
  T s = T(0);
  for (int j = 0; j < L; ++j) s += D[j] * rv[j];
  e[t] = s;
}

// restriction with Q = g^3 <= 32 lanes per output (one per cell of the group),
// combined by a fixed shuffle tree; gt = global thread index, every lane of the
// warp must call it (t >= nout: contributes nothing)
template <class T, int Q>
__device__ __forceinline__ void crestrict_q_item(const CLevel& f, const CLevel& cs, const T* __restrict__ Psi,
                                                 const T* __restrict__ res, T* __restrict__ rc, long long gt) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
  const long long nout = cs.ncell * Lc;
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

// restriction, one thread per output (any group size)
template <class T>
__device__ __forceinline__ void crestrict_item(const CLevel& f, const CLevel& cs, const T* __restrict__ Psi,
                                               const T* __restrict__ res, T* __restrict__ rc, long long t) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
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

// e[c][i] += sum_k Psi[G(c)][lc*Lf + i][k] ec[G][k] for row t = (c, i)
template <class T>
__device__ __forceinline__ void cprolong_item(const CLevel& f, const CLevel& cs, const T* __restrict__ Psi,
                                              const T* __restrict__ ec, T* __restrict__ e, long long t) {
  const int g = cs.g, Lf = f.L, Lc = cs.L;
  const int nloc = g * g * g * Lf;
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

// row of y = Ainv x by one warp (x already in shared memory as doubles)
template <class T>
__device__ __forceinline__ void gemv_row(int n, const double* __restrict__ A, const double* xs, T* __restrict__ y,
                                         int row, int lane) {
  const double* a = A + (long long)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += a[j] * xs[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = (T)s;
}

}  // namespace thermo

// Internal definitions shared by the libthermo CUDA sources.
//
// Device layout ("padded"): every nodal array has one ghost node on each
// side of every axis and a row pitch P that is a multiple of 32 elements, so
// that row starts are 128/256-byte aligned and stencil kernels need no
// boundary branches.  Node (x, y, z), x in [-1, Nx+1], is stored at
//     base + ((z+1)*RYn + (y+1))*P + x,     RYn = Ny + 3,  base = 32,
// i.e. the left ghost of a row is the last pad word of the previous row and
// the right ghost is the first pad word of the row itself (P >= Nx + 3).
// Element arrays use the same pitch with RYe = Ny + 2 and a ghost ring of
// zero conductivity, which yields the natural (adiabatic) boundary for free.
// Every pad / ghost word is zero at all times: kernels write interior
// entries only.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "zchunks.h"

namespace thermo {

typedef __nv_bfloat16 bf16;

struct Geom {
  int Nx, Ny, Nz;           // elements per axis
  int nx, ny, nz;           // nodes per axis (N + 1)
  long long P;              // row pitch in elements (multiple of 32)
  long long RYn, RYe;       // rows per plane: nodes (Ny + 3), elements (Ny + 2)
  long long base;           // offset of row 0 (32)
  long long nsize;          // padded nodal array length
  long long esize;          // padded element array length
  long long mwr;            // Dirichlet bitmask words per row (P / 32)
  long long msize;          // bitmask words
  double c[8];              // K0[a][b] = c[a ^ b] (unit conductivity)
  int cube;                 // c[1] = c[2] = c[4] = 0 (hx = hy = hz)
  double vol;               // hx * hy * hz
  // level-1 block partition
  int b;                    // block edge (elements)
  int nbx, nby, nbz;        // blocks per axis
  // fine tile decomposition (nodes); tiles are block-aligned
  int TX, TY, ZC;           // tile width / height, z planes per CTA chunk
  int NZ2, NZD;             // z chunks (ragged) of the two-nodes-per-lane and float-float engines
  int NZ3;                  // z chunks of the separable FP32 engine (0: engine not used)
  // bounded waits of the TMA-staged fine kernels (one word per context, on its device)
  int* err;                 // set to 1 by a kernel whose stage wait gave up
  long long wait;           // stage wait limit in clock64 cycles after a first non-blocking test
};

__host__ __device__ __forceinline__ long long nidx(const Geom& g, int x, int y, int z) {
  return g.base + ((long long)(z + 1) * g.RYn + (y + 1)) * g.P + x;
}
__host__ __device__ __forceinline__ long long eidx(const Geom& g, int ex, int ey, int ez) {
  return g.base + ((long long)(ez + 1) * g.RYe + (ey + 1)) * g.P + ex;
}
__host__ __device__ __forceinline__ long long mword(const Geom& g, int x, int y, int z) {
  return ((long long)(z + 1) * g.RYn + (y + 1)) * g.mwr + (x >> 5);
}
__device__ __forceinline__ bool is_dir(const Geom& g, const uint32_t* m, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.nx || y >= g.ny || z >= g.nz) return false;
  return (__ldg(m + mword(g, x, y, z)) >> (x & 31)) & 1u;
}
// level-1 block coordinate of node coordinate i along an axis with nb blocks
__host__ __device__ __forceinline__ int blk_of(int i, int b, int nb) {
  int q = i / b;
  return q < nb ? q : nb - 1;
}

// storage <-> compute conversions
template <class S> struct Cv;
template <> struct Cv<double> {
  typedef double C;
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct Cv<float> {
  typedef float C;
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <> struct Cv<bf16> {
  typedef float C;
  static __device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Deterministic block reduction of one double per thread (fixed tree order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) s += sh[i];
  }
  return s;  // valid in thread 0
}

// number of kernel launches issued by this library (process-wide, host side)
void note_launch();
long long launch_count();

}  // namespace thermo

// Layout conversion, SIMP conductivity, load vector, the FP64 Krylov vector
// updates with deterministic reductions, the adjoint sensitivity, and the
// SIMP harness kernels (density filter, OC update).
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "splitmix.h"
#include "fconv.h"

namespace thermo {

constexpr int VNT = 256;
constexpr int VEC_BLOCKS_MAX = 152 * 8;

// ---------------------------------------------------------------------------
// deterministic multi-CTA reduction of K doubles (fixed order everywhere)
template <int K>
__device__ __forceinline__ bool reduce_k(double (&v)[K], const Reducer& red, double (&res)[K]) {
  __shared__ double sh[32];
  __shared__ bool last;
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = block_sum<VNT>(v[k], sh);
  const unsigned nblk = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red.partial[K * blockIdx.x + k] = s[k];
    __threadfence();
    last = (atomicAdd(red.counter, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += VNT) a += __ldcg(red.partial + K * i + k);
    res[k] = block_sum<VNT>(a, sh);
  }
  if (threadIdx.x == 0) *red.counter = 0u;
  return true;
}

// interior nodes are visited as (row, pair) items: rows (y,z) in [0,ny)x[0,nz),
// pairs of x in [0, nx] (the odd tail pairs with the zero right ghost)
struct Rows {
  long long nrows, ppr, items;
};
static Rows rows_of(const Geom& g) {
  Rows r;
  r.nrows = (long long)g.ny * g.nz;
  r.ppr = (g.nx + 1) / 2;
  r.items = r.nrows * r.ppr;
  return r;
}
__device__ __forceinline__ long long item_index(const Geom& g, long long it, long long ppr) {
  if (it < (1LL << 32)) {  // 32-bit divisions (every grid this library accepts in practice)
    const unsigned u = (unsigned)it, q = (unsigned)ppr;
    const unsigned row = u / q, pr = u - row * q;
    const unsigned z = row / (unsigned)g.ny, y = row - z * (unsigned)g.ny;
    return g.base + ((long long)(z + 1) * g.RYn + (y + 1)) * g.P + 2 * (long long)pr;
  }
  const long long row = it / ppr, pr = it - row * ppr;
  const long long z = row / g.ny, y = row - z * g.ny;
  return g.base + ((z + 1) * g.RYn + (y + 1)) * g.P + 2 * pr;
}

static int vec_blocks(long long items) {
  long long b = (items + VNT - 1) / VNT;
  if (b > VEC_BLOCKS_MAX) b = VEC_BLOCKS_MAX;
  if (b < 1) b = 1;
  return (int)b;
}

template <class T>
__device__ __forceinline__ double2 ld2(const T* p);
template <>
__device__ __forceinline__ double2 ld2<double>(const double* p) {
  return *reinterpret_cast<const double2*>(p);
}
template <>
__device__ __forceinline__ double2 ld2<float>(const float* p) {
  float2 f = *reinterpret_cast<const float2*>(p);
  return make_double2(f2d_int(f.x), f2d_int(f.y));
}
template <>
__device__ __forceinline__ double2 ld2<bf16>(const bf16* p) {
  __nv_bfloat162 f = *reinterpret_cast<const __nv_bfloat162*>(p);
  return make_double2(__bfloat162float(f.x), __bfloat162float(f.y));
}
template <class T>
__device__ __forceinline__ void st2(T* p, double2 v);
template <>
__device__ __forceinline__ void st2<double>(double* p, double2 v) {
  *reinterpret_cast<double2*>(p) = v;
}
template <>
__device__ __forceinline__ void st2<float>(float* p, double2 v) {
  *reinterpret_cast<float2*>(p) = make_float2(d2f_int(v.x), d2f_int(v.y));
}
template <>
__device__ __forceinline__ void st2<bf16>(bf16* p, double2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

// ---------------------------------------------------------------------------
// layout conversion (natural <-> padded), masks, conductivity, load

__global__ void k_pack_nodes(Geom g, const double* __restrict__ nat, double* __restrict__ pad) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    pad[nidx(g, x, y, z)] = nat[i];
  }
}
__global__ void k_unpack_nodes(Geom g, const double* __restrict__ pad, double* __restrict__ nat) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    nat[i] = pad[nidx(g, x, y, z)];
  }
}
static int grid1(long long n, int nt = 256) {
  long long b = (n + nt - 1) / nt;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}
cudaError_t pack_nodes(const Geom& g, const double* nat, double* pad, cudaStream_t st) {
  note_launch(), k_pack_nodes<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, nat, pad);
  return cudaGetLastError();
}
cudaError_t unpack_nodes(const Geom& g, const double* pad, double* nat, cudaStream_t st) {
  note_launch(), k_unpack_nodes<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, pad, nat);
  return cudaGetLastError();
}

__global__ void k_mask_bits(Geom g, const uint8_t* __restrict__ nat, uint32_t* __restrict__ bits) {
  const long long nw = (long long)g.ny * g.nz * g.mwr;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x) {
    const long long row = w / g.mwr;
    const int wx = (int)(w - row * g.mwr);
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    uint32_t m = 0;
    for (int bit = 0; bit < 32; ++bit) {
      const int x = wx * 32 + bit;
      if (x < g.nx && nat[x + (long long)g.nx * (y + (long long)g.ny * z)]) m |= 1u << bit;
    }
    bits[mword(g, wx * 32, y, z)] = m;
  }
}
cudaError_t mask_to_bits(const Geom& g, const uint8_t* nat, uint32_t* bits, cudaStream_t st) {
  note_launch(), k_mask_bits<<<grid1((long long)g.ny * g.nz * g.mwr), 256, 0, st>>>(g, nat, bits);
  return cudaGetLastError();
}
__global__ void k_count(const uint8_t* __restrict__ m, long long n, int* out) {
  int c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += m[i] ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}
cudaError_t count_mask(const Geom& g, const uint8_t* nat, long long n, int* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(int), st);
  note_launch(), k_count<<<grid1(n), 256, 0, st>>>(nat, n, out);
  return cudaGetLastError();
}

// Sec. 2.1 Eq. (1): kappa_e = kmin + x_e^p (kmax - kmin), kept in FP64, FP32 and
// (optional, k16) BF16; klo (optional) is the float remainder kappa - (double)k32, so that k32 + klo is a
// float-float copy of the FP64 value (used by the float-float fine apply)
template <class X>  // the stored design: double, or float when it is given in FP32
__global__ void k_simp(Geom g, const X* __restrict__ x, double p, double kmin, double kmax,
                       double* __restrict__ k64, float* __restrict__ k32, bf16* __restrict__ k16,
                       float* __restrict__ klo) {
  const long long M = (long long)g.Nx * g.Ny * g.Nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.Nx);
    const long long t = e / g.Nx;
    const int ey = (int)(t % g.Ny), ez = (int)(t / g.Ny);
    const double k = kmin + pow((double)x[e], p) * (kmax - kmin);
    const long long i = eidx(g, ex, ey, ez);
    const float kh = (float)k;
    k64[i] = k;
    k32[i] = kh;
    if (k16) k16[i] = __float2bfloat16_rn(kh);
    if (klo) klo[i] = (float)(k - (double)kh);
  }
}
template <class X>
cudaError_t simp_kappa(const Geom& g, const X* x, double p, double kmin, double kmax, double* k64, float* k32,
                       bf16* k16, float* klo, cudaStream_t st) {
  note_launch(), k_simp<X><<<grid1((long long)g.Nx * g.Ny * g.Nz), 256, 0, st>>>(g, x, p, kmin, kmax, k64, k32, k16, klo);
  return cudaGetLastError();
}
template cudaError_t simp_kappa<double>(const Geom&, const double*, double, double, double, double*, float*, bf16*,
                                        float*, cudaStream_t);
template cudaError_t simp_kappa<float>(const Geom&, const float*, double, double, double, double*, float*, bf16*,
                                       float*, cudaStream_t);

__global__ void k_widen(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
cudaError_t widen_f32(const float* a, double* b, long long n, cudaStream_t st) {
  note_launch(), k_widen<<<grid1(n), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

// f_i = sum_{e contains i} q_e |e| / 8
__global__ void k_load(Geom g, const double* __restrict__ q, double* __restrict__ f) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    double s = 0.0;
    for (int dz = -1; dz <= 0; ++dz)
      for (int dy = -1; dy <= 0; ++dy)
        for (int dx = -1; dx <= 0; ++dx) {
          const int ex = x + dx, ey = y + dy, ez = z + dz;
          if (ex < 0 || ey < 0 || ez < 0 || ex >= g.Nx || ey >= g.Ny || ez >= g.Nz) continue;
          s += q[ex + (long long)g.Nx * (ey + (long long)g.Ny * ez)];
        }
    f[nidx(g, x, y, z)] = s * g.vol * 0.125;
  }
}
cudaError_t load_vector(const Geom& g, const double* q, double* f, cudaStream_t st) {
  note_launch(), k_load<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, q, f);
  return cudaGetLastError();
}

// b_F = f_F - (A_N T_D)_F, b_D = T_D  (Dirichlet lifting; A_N unmasked)
__global__ void k_dir_rhs(Geom g, const uint32_t* __restrict__ bits, const double* __restrict__ k64,
                          const double* __restrict__ f, const double* __restrict__ TD, double* __restrict__ b) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const long long ni = nidx(g, x, y, z);
    if (is_dir(g, bits, x, y, z)) {
      b[ni] = TD ? TD[ni] : 0.0;
      continue;
    }
    if (!TD) {  // T_D = 0: nothing to lift
      b[ni] = f[ni];
      continue;
    }
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ex = x - 1 + dx, ey = y - 1 + dy, ez = z - 1 + dz;
          const double k = k64[eidx(g, ex, ey, ez)];
          if (k == 0.0) continue;
          const int a = (1 - dx) | ((1 - dy) << 1) | ((1 - dz) << 2);
          for (int bb = 0; bb < 8; ++bb) {
            const int xx = ex + (bb & 1), yy = ey + ((bb >> 1) & 1), zz = ez + (bb >> 2);
            if (!is_dir(g, bits, xx, yy, zz)) continue;
            s += k * g.c[a ^ bb] * TD[nidx(g, xx, yy, zz)];
          }
        }
    b[ni] = f[ni] - s;
  }
}
cudaError_t dirichlet_rhs(const Geom& g, const uint32_t* bits, const double* k64, const double* f,
                          const double* TDpad, double* b, cudaStream_t st) {
  note_launch(), k_dir_rhs<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, bits, k64, f, TDpad, b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Krylov vector kernels (FP64 accumulation, deterministic)

// r = b - Ax, rr = r.r
__global__ void __launch_bounds__(VNT) k_residual(Geom g, Rows R, const double* __restrict__ b,
                                                  const double* __restrict__ Ax, double* __restrict__ r,
                                                  Reducer red, double* rr) {
  double v[1] = {0.0}, res[1];
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 bb = ld2<double>(b + i), aa = ld2<double>(Ax + i);
    double2 rv = make_double2(bb.x - aa.x, bb.y - aa.y);
    st2<double>(r + i, rv);
    v[0] += rv.x * rv.x + rv.y * rv.y;
  }
  if (reduce_k<1>(v, red, res) && threadIdx.x == 0) *rr = res[0];
}
cudaError_t vec_residual(const Geom& g, const double* b, const double* Ax, double* r, const Reducer& red, double* rr,
                         cudaStream_t st) {
  Rows R = rows_of(g);
  note_launch(), k_residual<<<vec_blocks(R.items), VNT, 0, st>>>(g, R, b, Ax, r, red, rr);
  return cudaGetLastError();
}

template <class Tb>
__global__ void __launch_bounds__(VNT) k_dot(Geom g, Rows R, const double* __restrict__ a, const Tb* __restrict__ b,
                                             Reducer red, double* out) {
  double v[1] = {0.0}, res[1];
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 x = ld2<double>(a + i), y = ld2<Tb>(b + i);
    v[0] += x.x * y.x + x.y * y.y;
  }
  if (reduce_k<1>(v, red, res) && threadIdx.x == 0) *out = res[0];
}
cudaError_t vec_dot(const Geom& g, const double* a, const void* b, int b_kind, const Reducer& red, double* out,
                    cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (b_kind == 0)
    note_launch(), k_dot<double><<<nb, VNT, 0, st>>>(g, R, a, (const double*)b, red, out);
  else if (b_kind == 1)
    note_launch(), k_dot<float><<<nb, VNT, 0, st>>>(g, R, a, (const float*)b, red, out);
  else
    note_launch(), k_dot<bf16><<<nb, VNT, 0, st>>>(g, R, a, (const bf16*)b, red, out);
  return cudaGetLastError();
}

template <class Td>
__global__ void __launch_bounds__(VNT) k_cvt(Geom g, Rows R, const double* __restrict__ s, Td* __restrict__ d) {
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    st2<Td>(d + i, ld2<double>(s + i));
  }
}
cudaError_t vec_copy_cvt(const Geom& g, const double* src, void* dst, int kind, cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (kind == 0)
    note_launch(), k_cvt<double><<<nb, VNT, 0, st>>>(g, R, src, (double*)dst);
  else if (kind == 1)
    note_launch(), k_cvt<float><<<nb, VNT, 0, st>>>(g, R, src, (float*)dst);
  else
    note_launch(), k_cvt<bf16><<<nb, VNT, 0, st>>>(g, R, src, (bf16*)dst);
  return cudaGetLastError();
}

// a.b over free (non-Dirichlet) interior nodes only
__global__ void __launch_bounds__(VNT) k_dot_free(Geom g, Rows R, const uint32_t* __restrict__ bits,
                                                  const double* __restrict__ a, const double* __restrict__ b,
                                                  Reducer red, double* out) {
  double v[1] = {0.0}, res[1];
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long row = it / R.ppr, pr = it - row * R.ppr;
    const int z = (int)(row / g.ny), y = (int)(row - (row / g.ny) * g.ny);
    const long long i = item_index(g, it, R.ppr);
    double2 x = ld2<double>(a + i), w = ld2<double>(b + i);
    const int x0 = (int)(2 * pr);
    if (!is_dir(g, bits, x0, y, z)) v[0] += x.x * w.x;
    if (!is_dir(g, bits, x0 + 1, y, z)) v[0] += x.y * w.y;
  }
  if (reduce_k<1>(v, red, res) && threadIdx.x == 0) *out = res[0];
}
cudaError_t vec_dot_free(const Geom& g, const uint32_t* bits, const double* a, const double* b, const Reducer& red,
                         double* out, cudaStream_t st) {
  Rows R = rows_of(g);
  note_launch(), k_dot_free<<<vec_blocks(R.items), VNT, 0, st>>>(g, R, bits, a, b, red, out);
  return cudaGetLastError();
}

// alpha = rz / pq;  u += alpha p;  r -= alpha q;  rr = r.r;  rzo = r.z_old;  r_lp = (low) r
template <class Tz, class Tr>
__global__ void __launch_bounds__(VNT) k_cg_update(Geom g, Rows R, double* __restrict__ u, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ q,
                                                   const Tz* __restrict__ z, Tr* __restrict__ rlp, CgScalars* sc,
                                                   Reducer red) {
  const double pq = sc->pq, rz = sc->rz;
  const bool ok = (pq > 0.0) && isfinite(pq) && isfinite(rz);
  const double alpha = ok ? rz / pq : 0.0;
  double v[2] = {0.0, 0.0}, res[2];
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 uu = ld2<double>(u + i), rr = ld2<double>(r + i), pp = ld2<double>(p + i), qq = ld2<double>(q + i);
    uu.x += alpha * pp.x;
    uu.y += alpha * pp.y;
    rr.x -= alpha * qq.x;
    rr.y -= alpha * qq.y;
    st2<double>(u + i, uu);
    st2<double>(r + i, rr);
    v[0] = fma(rr.x, rr.x, v[0]);
    v[0] = fma(rr.y, rr.y, v[0]);
    if (z) {
      double2 zz = ld2<Tz>(z + i);
      v[1] = fma(rr.x, zz.x, v[1]);
      v[1] = fma(rr.y, zz.y, v[1]);
    }
    if (rlp) st2<Tr>(rlp + i, rr);
  }
  if (reduce_k<2>(v, red, res) && threadIdx.x == 0) {
    sc->rr = res[0];
    sc->rzo = res[1];
    sc->alpha = alpha;
    if (!ok) sc->flag = 1;
  }
}

template <class Tz>
static cudaError_t cg_update_t(const Geom& g, double* u, double* r, const double* p, const double* q, const Tz* z,
                               void* rlp, int rk, CgScalars* sc, const Reducer& red, cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (rk == 1)
    note_launch(), k_cg_update<Tz, float><<<nb, VNT, 0, st>>>(g, R, u, r, p, q, z, (float*)rlp, sc, red);
  else if (rk == 2)
    note_launch(), k_cg_update<Tz, bf16><<<nb, VNT, 0, st>>>(g, R, u, r, p, q, z, (bf16*)rlp, sc, red);
  else
    note_launch(), k_cg_update<Tz, double><<<nb, VNT, 0, st>>>(g, R, u, r, p, q, z, (double*)rlp, sc, red);
  return cudaGetLastError();
}
cudaError_t cg_update(const Geom& g, double* u, double* r, const double* p, const double* q, const void* z_old,
                      int zk, void* r_lp, int rk, CgScalars* sc, const Reducer& red, cudaStream_t st) {
  if (zk == 1) return cg_update_t<float>(g, u, r, p, q, (const float*)z_old, r_lp, rk, sc, red, st);
  if (zk == 2) return cg_update_t<bf16>(g, u, r, p, q, (const bf16*)z_old, r_lp, rk, sc, red, st);
  return cg_update_t<double>(g, u, r, p, q, (const double*)z_old, r_lp, rk, sc, red, st);
}

// rzn = r.z; beta for p' = z + beta p:
//   flexible 0: rzn / rz (standard PCG)
//   flexible 1: -(z.q) / (p.q), q = A p of the previous direction (flexible CG with explicit
//               A-orthogonalisation against the last direction, Notay's truncated form)
//   flexible 2: (rzn - r.z_old) / rz (Polak-Ribiere)
//   rz = rzn
template <class Tz>
__global__ void __launch_bounds__(VNT) k_beta(Geom g, Rows R, const double* __restrict__ r, const Tz* __restrict__ z,
                                              const double* __restrict__ q, int flexible, CgScalars* sc, Reducer red) {
  double v[2] = {0.0, 0.0}, res[2];
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 rr = ld2<double>(r + i), zz = ld2<Tz>(z + i);
    v[0] = fma(rr.x, zz.x, v[0]);
    v[0] = fma(rr.y, zz.y, v[0]);
    if (flexible == 1) {
      const double2 qq = ld2<double>(q + i);
      v[1] = fma(zz.x, qq.x, v[1]);
      v[1] = fma(zz.y, qq.y, v[1]);
    }
  }
  if (reduce_k<2>(v, red, res) && threadIdx.x == 0) {
    const double rzn = res[0];
    const double rz = sc->rz;
    double beta;
    if (flexible == 1)
      beta = -res[1] / sc->pq;
    else if (flexible == 2)
      beta = (rzn - sc->rzo) / rz;
    else
      beta = rzn / rz;
    if (!isfinite(beta)) {
      beta = 0.0;
      sc->flag = 1;
    }
    sc->rzn = rzn;
    sc->beta = beta;
    sc->rz = rzn;
  }
}
cudaError_t cg_beta_dot(const Geom& g, const double* r, const void* z, int zk, const double* q, int flexible,
                        CgScalars* sc, const Reducer& red, cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (zk == 1)
    note_launch(), k_beta<float><<<nb, VNT, 0, st>>>(g, R, r, (const float*)z, q, flexible, sc, red);
  else if (zk == 2)
    note_launch(), k_beta<bf16><<<nb, VNT, 0, st>>>(g, R, r, (const bf16*)z, q, flexible, sc, red);
  else
    note_launch(), k_beta<double><<<nb, VNT, 0, st>>>(g, R, r, (const double*)z, q, flexible, sc, red);
  return cudaGetLastError();
}

// p = z + beta p   (first: p = z)
template <class Tz>
__global__ void __launch_bounds__(VNT) k_pupd(Geom g, Rows R, const Tz* __restrict__ z, double* __restrict__ p,
                                              const CgScalars* sc, int first) {
  const double beta = first ? 0.0 : sc->beta;
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 zz = ld2<Tz>(z + i);
    if (!first) {
      double2 pp = ld2<double>(p + i);
      zz.x += beta * pp.x;
      zz.y += beta * pp.y;
    }
    st2<double>(p + i, zz);
  }
}
cudaError_t cg_pupdate(const Geom& g, const void* z, int zk, double* p, const CgScalars* sc, int first,
                       cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (zk == 1)
    note_launch(), k_pupd<float><<<nb, VNT, 0, st>>>(g, R, (const float*)z, p, sc, first);
  else if (zk == 2)
    note_launch(), k_pupd<bf16><<<nb, VNT, 0, st>>>(g, R, (const bf16*)z, p, sc, first);
  else
    note_launch(), k_pupd<double><<<nb, VNT, 0, st>>>(g, R, (const double*)z, p, sc, first);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(VNT) k_axpy(Geom g, Rows R, double a, const double* __restrict__ x,
                                              double* __restrict__ y) {
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 xx = ld2<double>(x + i), yy = ld2<double>(y + i);
    yy.x += a * xx.x;
    yy.y += a * xx.y;
    st2<double>(y + i, yy);
  }
}
cudaError_t vec_axpy_pad(const Geom& g, double a, const double* x, double* y, cudaStream_t st) {
  Rows R = rows_of(g);
  note_launch(), k_axpy<<<vec_blocks(R.items), VNT, 0, st>>>(g, R, a, x, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sec. 2.3: dc_e = -p x_e^(p-1) (kmax - kmin) u_e^T K0 u_e, with
// u_e^T K0 u_e = sum_{a<b} (-K0[a][b]) (u_a - u_b)^2 (rows of K0 sum to zero).
template <class X>
__global__ void k_sens(Geom g, const double* __restrict__ u, const X* __restrict__ x, double p, double kmin,
                       double kmax, double* __restrict__ dc) {
  const long long M = (long long)g.Nx * g.Ny * g.Nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.Nx);
    const long long t = e / g.Nx;
    const int ey = (int)(t % g.Ny), ez = (int)(t / g.Ny);
    double ue[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) ue[a] = u[nidx(g, ex + (a & 1), ey + ((a >> 1) & 1), ez + (a >> 2))];
    double E = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = a + 1; b < 8; ++b) {
        const double d = ue[a] - ue[b];
        E -= g.c[a ^ b] * d * d;
      }
    const double xe = (double)x[e];
    const double dk = p * ((p == 1.0) ? 1.0 : pow(xe, p - 1.0)) * (kmax - kmin);
    dc[e] = -dk * E;
  }
}
template <class X>
cudaError_t sensitivity(const Geom& g, const double* upad, const X* x, double p, double kmin, double kmax,
                        double* dc, cudaStream_t st) {
  note_launch(), k_sens<X><<<grid1((long long)g.Nx * g.Ny * g.Nz), 256, 0, st>>>(g, upad, x, p, kmin, kmax, dc);
  return cudaGetLastError();
}
template cudaError_t sensitivity<double>(const Geom&, const double*, const double*, double, double, double, double*,
                                         cudaStream_t);
template cudaError_t sensitivity<float>(const Geom&, const double*, const float*, double, double, double, double*,
                                        cudaStream_t);

// ---------------------------------------------------------------------------
// SIMP harness: hat-weight density filter and OC candidate (not in the paper)
__global__ void k_filter(int Nx, int Ny, int Nz, const double* __restrict__ in, double* __restrict__ out,
                         double rmin, int transpose) {
  const long long M = (long long)Nx * Ny * Nz;
  const int R = (int)ceil(rmin) - 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % Nx);
    const long long t = e / Nx;
    const int ey = (int)(t % Ny), ez = (int)(t / Ny);
    double s = 0.0, ws = 0.0;
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          const double w = rmin - sqrt((double)(dx * dx + dy * dy + dz * dz));
          if (w <= 0.0) continue;
          const int jx = ex + dx, jy = ey + dy, jz = ez + dz;
          if (jx < 0 || jy < 0 || jz < 0 || jx >= Nx || jy >= Ny || jz >= Nz) continue;
          const long long j = jx + (long long)Nx * (jy + (long long)Ny * jz);
          if (!transpose) {
            s += w * in[j];
            ws += w;
          } else {
            // weight of e in row j, normalised by row j's sum
            double wj = 0.0;
            for (int cz = -R; cz <= R; ++cz)
              for (int cy = -R; cy <= R; ++cy)
                for (int cx = -R; cx <= R; ++cx) {
                  const double w2 = rmin - sqrt((double)(cx * cx + cy * cy + cz * cz));
                  if (w2 <= 0.0) continue;
                  const int kx = jx + cx, ky = jy + cy, kz = jz + cz;
                  if (kx < 0 || ky < 0 || kz < 0 || kx >= Nx || ky >= Ny || kz >= Nz) continue;
                  wj += w2;
                }
            s += w / wj * in[j];
          }
        }
    out[e] = transpose ? s : s / ws;
  }
}
// ---------------------------------------------------------------------------
// Resolution change of a field (Sec. 3 interpolation technique: a design, or a
// solution, carried from an N^3 run to an (rN)^3 one).  kind 0: element field,
// piecewise constant; 1: element field, trilinear between cell centres (fine
// centre at (i + 1/2)/r - 1/2 in coarse-centre units), constant beyond the
// outermost centres; 2: nodal field, the coarse trilinear function at the fine
// nodes.  Products and sums are rounded one by one (no fused multiply-add) in
// the order x, y, z, so that the result does not depend on contraction.
struct RsAxis {
  int i0, i1;
  double t;
};
__device__ __forceinline__ RsAxis rs_axis(int i, int N, int r, int kind) {
  RsAxis a;
  if (kind == 1) {
    const double s = __dsub_rn(__ddiv_rn((double)i + 0.5, (double)r), 0.5);
    int k = (int)floor(s);
    double t = __dsub_rn(s, (double)k);
    if (k < 0) {
      k = 0;
      t = 0.0;
    } else if (k >= N - 1) {
      k = N - 1;
      t = 0.0;
    }
    a.i0 = k;
    a.i1 = k + 1 < N ? k + 1 : N - 1;
    a.t = t;
  } else {  // nodal
    int k = i / r;
    if (k > N - 1) k = N - 1;
    a.i0 = k;
    a.i1 = k + 1;
    a.t = __dsub_rn(__ddiv_rn((double)i, (double)r), (double)k);
  }
  return a;
}
__device__ __forceinline__ double rs_lerp(double a, double b, double t) {
  return __dadd_rn(__dmul_rn(a, __dsub_rn(1.0, t)), __dmul_rn(b, t));
}
__global__ void k_resample(int3 nc, int3 nf, int3 r, int kind, const double* __restrict__ in, double* __restrict__ out) {
  // nc / nf: extents of the coarse / fine arrays (elements, or nodes for kind 2)
  const long long n = (long long)nf.x * nf.y * nf.z;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(o % nf.x);
    const long long t = o / nf.x;
    const int iy = (int)(t % nf.y), iz = (int)(t / nf.y);
    if (kind == 0) {
      out[o] = in[(ix / r.x) + (long long)nc.x * ((iy / r.y) + (long long)nc.y * (iz / r.z))];
      continue;
    }
    const int Nx = kind == 2 ? nc.x - 1 : nc.x, Ny = kind == 2 ? nc.y - 1 : nc.y, Nz = kind == 2 ? nc.z - 1 : nc.z;
    const RsAxis ax = rs_axis(ix, Nx, r.x, kind), ay = rs_axis(iy, Ny, r.y, kind), az = rs_axis(iz, Nz, r.z, kind);
    auto at = [&](int z, int y, int x) { return in[x + (long long)nc.x * (y + (long long)nc.y * z)]; };
    const double c00 = rs_lerp(at(az.i0, ay.i0, ax.i0), at(az.i0, ay.i0, ax.i1), ax.t);
    const double c10 = rs_lerp(at(az.i0, ay.i1, ax.i0), at(az.i0, ay.i1, ax.i1), ax.t);
    const double c01 = rs_lerp(at(az.i1, ay.i0, ax.i0), at(az.i1, ay.i0, ax.i1), ax.t);
    const double c11 = rs_lerp(at(az.i1, ay.i1, ax.i0), at(az.i1, ay.i1, ax.i1), ax.t);
    out[o] = rs_lerp(rs_lerp(c00, c10, ay.t), rs_lerp(c01, c11, ay.t), az.t);
  }
}
cudaError_t resample_field(const int gc[3], const double* in, const int gf[3], double* out, int kind, cudaStream_t st) {
  const int e = kind == 2 ? 1 : 0;
  const int3 nc = make_int3(gc[0] + e, gc[1] + e, gc[2] + e), nf = make_int3(gf[0] + e, gf[1] + e, gf[2] + e);
  const int3 r = make_int3(gf[0] / gc[0], gf[1] / gc[1], gf[2] / gc[2]);
  const long long n = (long long)nf.x * nf.y * nf.z;
  note_launch(), k_resample<<<grid1(n), 256, 0, st>>>(nc, nf, r, kind, in, out);
  return cudaGetLastError();
}

cudaError_t density_filter(int Nx, int Ny, int Nz, const double* in, double* out, double rmin, int transpose,
                           cudaStream_t st) {
  note_launch(), k_filter<<<grid1((long long)Nx * Ny * Nz), 256, 0, st>>>(Nx, Ny, Nz, in, out, rmin, transpose);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(VNT) k_oc(long long M, const double* __restrict__ x, const double* __restrict__ dc,
                                            const double* __restrict__ dv, const double* __restrict__ cs, double lmid,
                                            double move, double* __restrict__ xn, Reducer red, double* vol) {
  double v[1] = {0.0}, res[1];
  for (long long e = blockIdx.x * (long long)VNT + threadIdx.x; e < M; e += (long long)gridDim.x * VNT) {
    const double xe = x[e];
    const double ratio = fmax(-dc[e], 0.0) / (dv[e] * lmid);
    double c = xe * sqrt(ratio);
    c = fmin(fmin(c, xe + move), 1.0);
    c = fmax(fmax(c, xe - move), 0.0);
    xn[e] = c;
    v[0] += cs[e] * c;
  }
  if (reduce_k<1>(v, red, res) && threadIdx.x == 0) *vol = res[0] / (double)M;
}
cudaError_t oc_candidate(long long M, const double* x, const double* dc, const double* dv, const double* colsum,
                         double lmid, double move, double* xnew, const Reducer& red, double* vol, cudaStream_t st) {
  note_launch(), k_oc<<<vec_blocks(M), VNT, 0, st>>>(M, x, dc, dv, colsum, lmid, move, xnew, red, vol);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(VNT) k_maxdiff(long long M, const double* __restrict__ a,
                                                 const double* __restrict__ b, Reducer red, double* out) {
  // max via the deterministic reducer: accumulate max in a sum-free way
  __shared__ double sh[VNT];
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)VNT + threadIdx.x; e < M; e += (long long)gridDim.x * VNT)
    m = fmax(m, fabs(a[e] - b[e]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = VNT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    red.partial[blockIdx.x] = sh[0];
    __threadfence();
    last = (atomicAdd(red.counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double r = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) r = fmax(r, __ldcg(red.partial + i));
    *out = r;
    *red.counter = 0u;
  }
}
cudaError_t max_abs_diff(long long M, const double* a, const double* b, const Reducer& red, double* out,
                         cudaStream_t st) {
  note_launch(), k_maxdiff<<<vec_blocks(M), VNT, 0, st>>>(M, a, b, red, out);
  return cudaGetLastError();
}


// d = (double) s on padded arrays (s: 0 f64, 1 f32, 2 bf16)
template <class Ts>
__global__ void __launch_bounds__(VNT) k_to64(Geom g, Rows R, const Ts* __restrict__ s, double* __restrict__ d) {
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    st2<double>(d + i, ld2<Ts>(s + i));
  }
}
cudaError_t vec_to_f64(const Geom& g, const void* src, int kind, double* dst, cudaStream_t st) {
  Rows R = rows_of(g);
  const int nb = vec_blocks(R.items);
  if (kind == 0)
    note_launch(), k_to64<double><<<nb, VNT, 0, st>>>(g, R, (const double*)src, dst);
  else if (kind == 1)
    note_launch(), k_to64<float><<<nb, VNT, 0, st>>>(g, R, (const float*)src, dst);
  else
    note_launch(), k_to64<bf16><<<nb, VNT, 0, st>>>(g, R, (const bf16*)src, dst);
  return cudaGetLastError();
}

// u_i += sum_j Phi_ij ec[B(i)][j]  (prolongation from level 1 into an FP64 vector;
// Phi and ec stored as C, FP64 sums)
template <class C>
__global__ void k_prolong_add(Geom g, const C* __restrict__ phi, int L, const C* __restrict__ ec,
                              double* __restrict__ u) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const long long nd = nidx(g, x, y, z);
    const long long cell = blk_of(x, g.b, g.nbx) + (long long)g.nbx * (blk_of(y, g.b, g.nby) + (long long)g.nby * blk_of(z, g.b, g.nbz));
    double s = 0.0;
    for (int a = 0; a < L; ++a) s += (double)phi[nd * L + a] * (double)ec[cell * L + a];
    u[nd] += s;
  }
}
template <class C>
cudaError_t fine_prolong_add(const Geom& g, const C* phi, int L1, const C* ec, double* u, cudaStream_t st) {
  note_launch(), k_prolong_add<C><<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, phi, L1, ec, u);
  return cudaGetLastError();
}
template cudaError_t fine_prolong_add<double>(const Geom&, const double*, int, const double*, double*, cudaStream_t);
template cudaError_t fine_prolong_add<float>(const Geom&, const float*, int, const float*, double*, cudaStream_t);

// v = 0 on Dirichlet nodes (padded FP64)
__global__ void k_mask_dir(Geom g, const uint32_t* __restrict__ bits, double* __restrict__ v) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    if (is_dir(g, bits, x, y, z)) v[nidx(g, x, y, z)] = 0.0;
  }
}
cudaError_t vec_mask_dir(const Geom& g, const uint32_t* bits, double* v, cudaStream_t st) {
  note_launch(), k_mask_dir<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, bits, v);
  return cudaGetLastError();
}

// dst = src on the Dirichlet nodes (padded layout); other nodes untouched
__global__ void k_copy_dir(Geom g, const uint32_t* __restrict__ bits, const double* __restrict__ src,
                           double* __restrict__ dst) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    if (is_dir(g, bits, x, y, z)) dst[nidx(g, x, y, z)] = src[nidx(g, x, y, z)];
  }
}
cudaError_t vec_copy_dir(const Geom& g, const uint32_t* bits, const double* src, double* dst, cudaStream_t st) {
  note_launch(), k_copy_dir<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, bits, src, dst);
  return cudaGetLastError();
}

// seeded start vector of the power iteration: u_i - 1/2 at the natural node index i,
// u_i the SplitMix64 uniform of stream POWER_SEED (splitmix.h; 53 bits), zero on
// Dirichlet nodes.  A random start has weight on the top of the spectrum of D^-1 A,
// which a smooth or periodic start lacks on uniform media.
constexpr unsigned long long POWER_SEED = 101ull;
__global__ void k_power_start(Geom g, const uint32_t* __restrict__ bits, double* __restrict__ v) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    v[nidx(g, x, y, z)] = is_dir(g, bits, x, y, z) ? 0.0 : splitmix_u01(POWER_SEED, (unsigned long long)i) - 0.5;
  }
}
cudaError_t power_start(const Geom& g, const uint32_t* bits, double* v, cudaStream_t st) {
  note_launch(), k_power_start<<<grid1((long long)g.nx * g.ny * g.nz), 256, 0, st>>>(g, bits, v);
  return cudaGetLastError();
}
__global__ void __launch_bounds__(VNT) k_scale(Geom g, Rows R, double a, double* __restrict__ v) {
  for (long long it = blockIdx.x * (long long)VNT + threadIdx.x; it < R.items; it += (long long)gridDim.x * VNT) {
    const long long i = item_index(g, it, R.ppr);
    double2 x = ld2<double>(v + i);
    x.x *= a;
    x.y *= a;
    st2<double>(v + i, x);
  }
}
cudaError_t vec_scale(const Geom& g, double a, double* v, cudaStream_t st) {
  Rows R = rows_of(g);
  note_launch(), k_scale<<<vec_blocks(R.items), VNT, 0, st>>>(g, R, a, v);
  return cudaGetLastError();
}

__global__ void k_fill(double* __restrict__ a, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = v;
}
cudaError_t fill_const(double* a, long long n, double v, cudaStream_t st) {
  note_launch(), k_fill<<<grid1(n), 256, 0, st>>>(a, n, v);
  return cudaGetLastError();
}

}  // namespace thermo

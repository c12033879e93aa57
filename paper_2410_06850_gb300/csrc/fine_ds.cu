// FP64-accurate fine operator apply on the FP32 pipes (float-float arithmetic).
//
// q = A p with the Q1 operator of Sec. 2.2 Eq. (5) (cubic elements), plus the
// fused CG reduction p.q, for the outer FP64 CG.  GB300 issues FP64 at about
// 1/60 of its FP32 rate, so the plain FP64 kernel is bound by its ~41 FP64
// instructions per node.  This kernel keeps every value as an unevaluated
// sum of two floats (hi + lo, 47-48 significant bits) and uses error-free
// transformations: TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2) for sums and
// differences, and the FMA form of TwoProduct (Dekker 1971, with the exact
// product error recovered by one fused multiply-add) for products.  Each lane
// evaluates two neighbouring nodes at once with packed f32x2 instructions.
//
// Cancellation: the rows have zero sum on the Neumann part, so the stencil is
// evaluated in difference form,
//   (A p)_i = c3 sum_j w_ij (p_j - p_i),   c3 = -h/12,
// over the 12 face-diagonal neighbours (w = sum of the two elements sharing
// the edge) and the 8 body-diagonal ones (w = kappa of the one element); the
// axis neighbours couple with weight 0 on cubes.  Dirichlet neighbours carry
// p_j = 0 (CG directions vanish there), Dirichlet rows return 0, ghost
// elements have kappa = 0.  The result is as accurate as the FP64 sum form.
//
// Engine: a CTA owns 64 x TY nodes (two per lane, one row per warp) and marches
// over one of NZD ragged z chunks; one elected thread stages each plane of p (FP64), of kappa
// (hi and lo floats) and of the Dirichlet bits with TMA tensor copies into an
// mbarrier ring; all threads split the landed FP64 plane into hi/lo float
// planes (integer arithmetic, no FP64 pipe) before the plane is used.  The
// closing column (x = Nx) and row (y = Ny), 0.8% of the nodes at 256^3, are
// evaluated first by a small grid-stride kernel (ds_edge) whose block partials
// of p.q open the reduction buffer.  FP64 work per node: one add to assemble
// q and one fused multiply-add for p.q.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace thermo {

namespace {

constexpr int DTY = 8;               // rows per tile (max), one warp each
constexpr int DNT = 32 * DTY;        // the closing column / row go to ds_edge
constexpr int DTX = 64;              // nodes per tile row (two per lane)
constexpr int DSX = 4;               // staged rows start at x0 - DSX (16-byte aligned)
constexpr int DW = 72;               // staged row width (x0 - 4 .. x0 + 67)
constexpr int DMW = 8;               // staged mask words per row
constexpr int DNS = 6;               // TMA ring stages (3 resident + 3 in flight)

constexpr size_t up128(size_t x) { return (x + 127) / 128 * 128; }
constexpr size_t BV = up128((size_t)(DTY + 3) * DW * 8);   // p plane (FP64) with halo
constexpr size_t BK = up128((size_t)(DTY + 2) * DW * 4);   // kappa hi (or lo) plane
constexpr size_t BM = up128((size_t)(DTY + 1) * DMW * 4);  // Dirichlet words
constexpr size_t STB = BV + 2 * BK + BM;
constexpr size_t BPAIR = up128((size_t)(DTY + 3) * DW * 4);  // one hi (or lo) plane of p
constexpr size_t SMEM = 256 + DNS * STB + 3 * 2 * BPAIR;

struct DsArgs {
  Geom g;
  const double* v;  // p (padded)
  double* out;      // q = A p (padded)
  const uint32_t* mask;
  float c3h, c3l;   // -h/12 as a float-float pair
  double* partial;  // dot partials: [0, nedge) from ds_edge, then one per CTA
  unsigned* counter;
  double* dot;
  int nedge;        // partials written by ds_edge before this kernel
};
struct alignas(64) DsMaps {
  CUtensorMap v, kh, kl, m;
};

// ---- packed float-float arithmetic (two nodes per lane)
__device__ __forceinline__ float2 F2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, F2(-1.f, -1.f), a); }  // exact negation, one rounding

struct DD {  // two float-float values: node 0 in .x, node 1 in .y
  float2 h, l;
};

// a + b, TwoSum on the high parts, low parts added (result unnormalised)
__device__ __forceinline__ DD dd_add(const DD& a, const DD& b) {
  const float2 s = add2(a.h, b.h);
  const float2 bb = sub2(s, a.h);
  const float2 e = add2(sub2(a.h, sub2(s, bb)), sub2(b.h, bb));
  return DD{s, add2(e, add2(a.l, b.l))};
}
// a - b, TwoSum on the high parts
__device__ __forceinline__ DD dd_sub(const DD& a, const DD& b) {
  const float2 s = sub2(a.h, b.h);
  const float2 bb = sub2(s, a.h);                              // ~ -b.h
  const float2 e = sub2(sub2(a.h, sub2(s, bb)), add2(b.h, bb));  // exact error of s
  return DD{s, add2(e, sub2(a.l, b.l))};
}
// acc += w * d: exact high product (FMA TwoProduct), cross terms into the low
// part, TwoSum of the high parts (w.l * d.l is below the format's precision)
__device__ __forceinline__ void dd_fma_acc(DD& acc, const DD& w, const DD& d) {
  const float2 ph = mul2(w.h, d.h);
  const float2 pe = fma2(w.h, d.h, F2(-ph.x, -ph.y));
  const float2 cr = fma2(w.h, d.l, mul2(w.l, d.h));
  const float2 s = add2(acc.h, ph);
  const float2 bb = sub2(s, acc.h);
  const float2 e = add2(sub2(acc.h, sub2(s, bb)), sub2(ph, bb));
  acc.h = s;
  acc.l = add2(acc.l, add2(e, add2(pe, cr)));
}

// FP64 -> (hi, lo) floats without the FP64 pipe: hi keeps the leading 24
// significant bits (truncated), lo the next 23 (exact).  Values whose
// remainder would leave the normal float range (|x| < 2^-80 or > 2^127) take
// the conversion instructions; zero is handled exactly.
__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int E = (int)((h32 >> 20) & 0x7ffu);
  if (E >= 943 && E <= 1150) {
    const unsigned sign = h32 & 0x80000000u;
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    hi = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | m23);
    const unsigned r23 = (l32 & 0x1fffffffu) >> 6;                       // next 23 bits
    const float rf = __fsub_rn(__uint_as_float(0x4b000000u | r23), 8388608.0f);  // exact integer r23
    const float sc = __uint_as_float((unsigned)(E - 1069 + 127) << 23);  // 2^(E - 1075 + 6)
    lo = __uint_as_float(__float_as_uint(__fmul_rn(rf, sc)) | sign);
  } else if ((b << 1) == 0ull) {
    hi = 0.f;
    lo = 0.f;
  } else {
    hi = __double2float_rz(x);
    lo = __double2float_rn(x - (double)hi);
  }
}
// float -> double by exponent re-bias (normal floats; zero and subnormals give 0)
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 0xffu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// ---- scalar float-float helpers (edge kernel)
struct D1 {
  float h, l;
};
__device__ __forceinline__ D1 d1_split(double x) {
  D1 r;
  split_d(x, r.h, r.l);
  return r;
}
__device__ __forceinline__ D1 d1_sub(const D1& a, const D1& b) {
  const float s = __fsub_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fsub_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fadd_rn(b.h, bb));
  return D1{s, __fadd_rn(e, __fsub_rn(a.l, b.l))};
}
__device__ __forceinline__ void d1_fma_acc(D1& acc, const D1& w, const D1& d) {
  const float ph = __fmul_rn(w.h, d.h);
  const float pe = __fmaf_rn(w.h, d.h, -ph);
  const float cr = __fmaf_rn(w.h, d.l, __fmul_rn(w.l, d.h));
  const float s = __fadd_rn(acc.h, ph);
  const float bb = __fsub_rn(s, acc.h);
  const float e = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, __fadd_rn(pe, cr)));
}

// closing column x = Nx (all y, z) and closing row y = Ny (x < Nx, all z):
// per node, the sum over its 8 elements of kappa_e times the differences to
// the element's three face-diagonal nodes and its body-diagonal node (the
// same operator as the tile kernel, grouped by element); the zero padding of
// the node and element arrays supplies every off-domain neighbour.
template <bool DOT>
__global__ void __launch_bounds__(256) ds_edge(const Geom g, const double* __restrict__ v, const float* __restrict__ khi,
                                               const float* __restrict__ klo, const uint32_t* __restrict__ mask,
                                               double* __restrict__ out, float c3h, float c3l,
                                               double* __restrict__ partial) {
  __shared__ double sh[256];
  const long long ncol = (long long)(g.Ny + 1) * (g.Nz + 1);  // x = Nx
  const long long nrow = (long long)g.Nx * (g.Nz + 1);        // y = Ny, x < Nx
  double dacc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncol + nrow;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (i < ncol) {
      x = g.Nx;
      y = (int)(i % (g.Ny + 1));
      z = (int)(i / (g.Ny + 1));
    } else {
      const long long j = i - ncol;
      x = (int)(j % g.Nx);
      y = g.Ny;
      z = (int)(j / g.Nx);
    }
    const double pd = v[nidx(g, x, y, z)];
    const D1 pc = d1_split(pd);
    D1 acc{0.f, 0.f};
#pragma unroll
    for (int sz = -1; sz <= 1; sz += 2)
#pragma unroll
      for (int sy = -1; sy <= 1; sy += 2)
#pragma unroll
        for (int sx = -1; sx <= 1; sx += 2) {
          const long long e = eidx(g, sx < 0 ? x - 1 : x, sy < 0 ? y - 1 : y, sz < 0 ? z - 1 : z);
          const D1 k{khi[e], klo[e]};
          d1_fma_acc(acc, k, d1_sub(d1_split(v[nidx(g, x + sx, y + sy, z)]), pc));
          d1_fma_acc(acc, k, d1_sub(d1_split(v[nidx(g, x + sx, y, z + sz)]), pc));
          d1_fma_acc(acc, k, d1_sub(d1_split(v[nidx(g, x, y + sy, z + sz)]), pc));
          d1_fma_acc(acc, k, d1_sub(d1_split(v[nidx(g, x + sx, y + sy, z + sz)]), pc));
        }
    const float yh = __fmul_rn(acc.h, c3h);
    const float ye = __fmaf_rn(acc.h, c3h, -yh);
    const float yl = __fadd_rn(ye, __fmaf_rn(acc.h, c3l, __fmul_rn(acc.l, c3h)));
    const double q = is_dir(g, mask, x, y, z) ? 0.0 : f2d(yh) + f2d(yl);
    out[nidx(g, x, y, z)] = q;
    if (DOT) dacc = fma(pd, q, dacc);
  }
  if (DOT) {
    sh[threadIdx.x] = dacc;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
      if ((int)threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
  }
}

template <bool DOT>
__global__ void __launch_bounds__(DNT, 2) ds_apply(const __grid_constant__ DsArgs a, const __grid_constant__ DsMaps tm) {
  const Geom& g = a.g;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned char* stages = smem_raw + 128;
  unsigned char* pairs = stages + DNS * STB;  // 3 slots x (hi plane, lo plane)
  __shared__ int stage_bad;
  __shared__ double dsh[DTY];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int TY = g.TY;
  const int x0 = blockIdx.x * DTX, y0 = blockIdx.y * TY;
  int zs, ze;
  zchunk(g.Nz, g.NZD, blockIdx.z, zs, ze);
  const int mx = (x0 >> 5) & ~3;
  const unsigned bytesV = (unsigned)((TY + 3) * DW * 8), bytesK = (unsigned)((TY + 2) * DW * 4);
  const unsigned bytesM = (unsigned)((TY + 1) * DMW * 4);
  auto stage_of = [&](int q) { return (q - zs + 1) % DNS; };
  auto base_of = [&](int q) { return stages + (size_t)stage_of(q) * STB; };
  auto sV = [&](int q) { return reinterpret_cast<const double*>(base_of(q)); };
  auto sKh = [&](int q) { return reinterpret_cast<const float*>(base_of(q) + BV); };
  auto sKl = [&](int q) { return reinterpret_cast<const float*>(base_of(q) + BV + BK); };
  auto sM = [&](int q) { return reinterpret_cast<const uint32_t*>(base_of(q) + BV + 2 * BK); };
  auto pslot = [&](int q) { return ((q - zs + 3) % 3); };
  auto pH = [&](int q) { return reinterpret_cast<float*>(pairs + (size_t)pslot(q) * 2 * BPAIR); };
  auto pL = [&](int q) { return reinterpret_cast<float*>(pairs + (size_t)pslot(q) * 2 * BPAIR + BPAIR); };

  // group q: node plane q of p, element plane q-1 of kappa, Dirichlet bits of node plane q-1
  auto issue = [&](int q) {
    const bool hv = q <= ze + 1;
    const int qk = q - 1;
    const bool hk = qk >= zs - 1 && qk <= ze;
    const bool hc = qk >= zs && qk <= ze;
    const unsigned bytes = (hv ? bytesV : 0u) + (hk ? 2u * bytesK : 0u) + (hc ? bytesM : 0u);
    const int s = stage_of(q);
    uint64_t* bar = bars + s;
    unsigned char* b = stages + (size_t)s * STB;
    mbar_expect_tx(bar, bytes);
    if (hv) tma_load3(b, &tm.v, x0 - DSX, y0, q + 1, bar);
    if (hk) {
      tma_load3(b + BV, &tm.kh, x0 - DSX, y0, qk + 1, bar);
      tma_load3(b + BV + BK, &tm.kl, x0 - DSX, y0, qk + 1, bar);
    }
    if (hc) tma_load3(b + BV + 2 * BK, &tm.m, mx, y0 + 1, qk + 1, bar);
  };
  auto wait_group = [&](int q) {
    if (stage_bad) return;
    const unsigned parity = (unsigned)(((q - zs + 1) / DNS) & 1);
    if (!mbar_wait_limited(bars + stage_of(q), parity, g.wait)) {  // bounded: give up, flag, never hang
      stage_bad = 1;
      atomicExch(g.err, 1);
    }
  };

  if (tid == 0) {
    stage_bad = 0;
    for (int s = 0; s < DNS; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int qhi = zs - 2;  // last group issued (thread 0)
  if (tid == 0)
    for (int q = zs - 1; q < zs - 1 + (DNS - 3); ++q) issue(q), qhi = q;

  const float2 c3h = F2(a.c3h, a.c3h), c3l = F2(a.c3l, a.c3l);
  double dacc = 0.0;

  // node pair (x0 + c, x0 + c + 1) on tile row r of node plane t
  auto pair = [&](int t, int r, int c) {
    const int sc = c + DSX;  // staged column of node x0 + c
    // conductivity pairs k[a][b][s]: element plane t-1+a, element row y-1+b (staged row r+b),
    // side s = 0: elements (c-1, c), s = 1: elements (c, c+1)
    DD k[2][2][2];
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      const float* kh = sKh(t + aa);
      const float* kl = sKl(t + aa);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int o = (r + bb) * DW + sc;
        const float hm = kh[o - 1], lm = kl[o - 1];
        const float2 h01 = *reinterpret_cast<const float2*>(kh + o);
        const float2 l01 = *reinterpret_cast<const float2*>(kl + o);
        k[aa][bb][0] = DD{F2(hm, h01.x), F2(lm, l01.x)};
        k[aa][bb][1] = DD{h01, l01};
      }
    }
    // centre values
    const float* c0h = pH(t);
    const float* c0l = pL(t);
    const int oc = (r + 1) * DW + sc;
    const DD pc{*reinterpret_cast<const float2*>(c0h + oc), *reinterpret_cast<const float2*>(c0l + oc)};
    DD acc{F2(0.f, 0.f), F2(0.f, 0.f)};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const float* ph = pH(t + dz);
      const float* pl = pL(t + dz);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        if (dz == 0 && dy == 0) continue;
        const int o = (r + 1 + dy) * DW + sc;
        const float2 h01 = *reinterpret_cast<const float2*>(ph + o);
        const float2 l01 = *reinterpret_cast<const float2*>(pl + o);
        const DD vm{F2(ph[o - 1], h01.x), F2(pl[o - 1], l01.x)};  // x - 1
        const DD vp{F2(h01.y, ph[o + 2]), F2(l01.y, pl[o + 2])};  // x + 1
        const int ia = dz < 0 ? 0 : 1, ib = dy < 0 ? 0 : 1;
        if (dz == 0) {
          // xy face diagonals: weight = the two elements of the column (x-side, y-side) stacked in z
          dd_fma_acc(acc, dd_add(k[0][ib][0], k[1][ib][0]), dd_sub(vm, pc));
          dd_fma_acc(acc, dd_add(k[0][ib][1], k[1][ib][1]), dd_sub(vp, pc));
        } else if (dy == 0) {
          // xz face diagonals: the two elements stacked in y
          dd_fma_acc(acc, dd_add(k[ia][0][0], k[ia][1][0]), dd_sub(vm, pc));
          dd_fma_acc(acc, dd_add(k[ia][0][1], k[ia][1][1]), dd_sub(vp, pc));
        } else {
          // yz face diagonal (same x): the two elements side by side in x; body diagonals: one element
          const DD v0{h01, l01};
          dd_fma_acc(acc, dd_add(k[ia][ib][0], k[ia][ib][1]), dd_sub(v0, pc));
          dd_fma_acc(acc, k[ia][ib][0], dd_sub(vm, pc));
          dd_fma_acc(acc, k[ia][ib][1], dd_sub(vp, pc));
        }
      }
    }
    // q = c3 * acc, then to FP64
    const float2 yh = mul2(acc.h, c3h);
    const float2 ye = fma2(acc.h, c3h, F2(-yh.x, -yh.y));
    const float2 yl = add2(ye, fma2(acc.h, c3l, mul2(acc.l, c3h)));
    const int xx = x0 + c, yy = y0 + r;
    const uint32_t mw = sM(t + 1)[r * DMW + ((xx >> 5) - mx)];
    double q0 = ((mw >> (xx & 31)) & 1u) ? 0.0 : f2d(yh.x) + f2d(yl.x);
    double q1 = ((mw >> ((xx + 1) & 31)) & 1u) ? 0.0 : f2d(yh.y) + f2d(yl.y);
    const long long n = nidx(g, xx, yy, t);
    const double* pv = sV(t) + (r + 1) * DW + sc;  // FP64 p of the pair (for the dot)
    *reinterpret_cast<double2*>(a.out + n) = make_double2(q0, q1);
    if (DOT) dacc = fma(pv[1], q1, fma(pv[0], q0, dacc));
  };

  const int nsplit = (TY + 3) * DW;
  for (int t = zs - 2; t <= ze; ++t) {
    wait_group(t + 1);
    __syncthreads();
    if (tid == 0 && !stage_bad) {  // after a wait gave up no stage is refilled
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(t + DNS - 2);
      qhi = t + DNS - 2;
    }
    if (t + 1 <= ze + 1) {  // split the landed p plane into hi / lo floats
      const double* src = sV(t + 1);
      float* dh = pH(t + 1);
      float* dl = pL(t + 1);
      for (int i = tid; i < nsplit; i += DNT) {
        float hi, lo;
        split_d(src[i], hi, lo);
        dh[i] = hi;
        dl[i] = lo;
      }
    }
    __syncthreads();
    if (t < zs) continue;
    if (w < TY) pair(t, w, 2 * lane);
  }
  if (tid == 0) mbar_drain(bars, DNS, zs - 1, qhi);

  if (DOT) {
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_down_sync(0xffffffffu, dacc, o);
    __syncthreads();
    if (lane == 0) dsh[w] = dacc;
    __shared__ bool last;
    __syncthreads();
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < DTY; ++i) s += dsh[i];
      a.partial[a.nedge + bid] = s;
      __threadfence();
      last = (atomicAdd(a.counter, 1u) == nblk - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const unsigned ntot = nblk + (unsigned)a.nedge;  // the edge kernel's partials come first
      double v = 0.0;
      for (unsigned i = tid; i < ntot; i += DNT) v += __ldcg(a.partial + i);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) dsh[w] = v;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < DTY; ++i) s += dsh[i];
        *a.dot = s;
        *a.counter = 0u;
      }
    }
  }
}

}  // namespace

bool fine_ds_supported(const Geom& g) { return g.cube && g.Nx % DTX == 0 && g.TY <= DTY; }

unsigned fine_ds_num_ctas(const Geom& g) { return (unsigned)(g.Nx / DTX) * (g.Ny / g.TY) * g.NZD; }

int fine_ds_tiles_xy(const Geom& g) { return (g.Nx / DTX) * (g.Ny / g.TY); }

int fine_ds_ctas_per_sm() {
  int n = 0;
  cudaFuncSetAttribute(ds_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ds_apply<true>, DNT, SMEM) != cudaSuccess) n = 0;
  return n;
}

cudaError_t fine_apply_ds(const Geom& g, const uint32_t* mask, const float* khi, const float* klo, const double* u,
                          double* y, double* partial, unsigned* counter, double* dot, cudaStream_t st) {
  if (!fine_ds_supported(g)) return cudaErrorInvalidValue;
  DsArgs a;
  memset(&a, 0, sizeof a);
  a.g = g;
  a.v = u;
  a.out = y;
  a.mask = mask;
  const double c3 = g.c[3];
  const float h = (float)c3;
  a.c3h = h;
  a.c3l = (float)(c3 - (double)h);
  a.partial = partial;
  a.counter = counter;
  a.dot = dot;
  DsMaps tm;
  cudaError_t e;
  if ((e = get_map(&tm.v, u + g.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, g.P, g.RYn, g.nz + 2, DW, g.TY + 3)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.kh, khi + g.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.P, g.RYe, g.Nz + 2, DW, g.TY + 2)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.kl, klo + g.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.P, g.RYe, g.Nz + 2, DW, g.TY + 2)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.m, mask, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, g.mwr, g.RYn, g.nz + 2, DMW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  const dim3 grid(g.Nx / DTX, g.Ny / g.TY, g.NZD);
  const long long nedge_nodes = (long long)(g.Ny + 1) * (g.Nz + 1) + (long long)g.Nx * (g.Nz + 1);
  const int eb = (int)std::min<long long>((nedge_nodes + 255) / 256, 512);
  a.nedge = dot ? eb : 0;
  if (dot) {
    note_launch(), ds_edge<true><<<eb, 256, 0, st>>>(g, u, khi, klo, mask, y, a.c3h, a.c3l, partial);
    cudaFuncSetAttribute(ds_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    note_launch(), ds_apply<true><<<grid, DNT, SMEM, st>>>(a, tm);
  } else {
    note_launch(), ds_edge<false><<<eb, 256, 0, st>>>(g, u, khi, klo, mask, y, a.c3h, a.c3l, nullptr);
    cudaFuncSetAttribute(ds_apply<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    note_launch(), ds_apply<false><<<grid, DNT, SMEM, st>>>(a, tm);
  }
  return cudaGetLastError();
}

}  // namespace thermo

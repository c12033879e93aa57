// FP32-compute fine sweeps and applies, two nodes per lane (packed f32x2).
//
// The fine smoother of the V-cycle (Sec. 3, Algorithm 1: the three-term
// Chebyshev / damped-Jacobi sweep e' = e + a (e - e_prev) + b D^-1 (r - A e))
// and the low-precision operator apply, for FP32 or BF16 storage with FP32
// arithmetic on cubic elements.  A CTA owns 64 x TY nodes: one row per warp,
// two neighbouring nodes per lane evaluated with packed f32x2 instructions,
// marching over one of NZ2 ragged z chunks (chosen so that the CTAs fill
// whole waves of the GPU).  One elected thread stages each plane of the
// iterate (with halo), of kappa, of the Dirichlet bits and of the centre
// arrays r and e_prev with TMA tensor copies into an mbarrier ring (waits
// bounded, failures flagged).  A ninth warp evaluates, from the same stages,
// the closing column (x = Nx, lanes = rows) of the last tile in x and the
// closing row (y = Ny) of the last tile in y.  Grids
// whose Nx is not a multiple of 64, or non-cubic elements, use the one-node-
// per-lane engine of fine.cu.
//
// Operator (cubic Q1, node-centred gather, Sec. 2.2 Eq. (5)):
//   (A v)_i = c0 K8 v_i + c3 (sum_xy zp v + sum_xz yp v + sum_yz xp v + sum_diag kappa v)
// K8 = the 8 conductivities around the node, zp / yp / xp = the two elements
// sharing a face-diagonal edge (stacked in z / y / x), the diagonal terms one
// element each.  The Jacobi diagonal is c0 K8.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace thermo {

namespace {

constexpr int QTY = 8;               // rows per tile (max), one warp each
constexpr int QNT = 32 * (QTY + 1);  // + one warp for the closing column / row
constexpr int QTX = 64;        // nodes per tile row (two per lane)
constexpr int QMW = 8;         // staged mask words per row
constexpr int QNS = 6;         // TMA ring stages (4 resident + 2 in flight)
constexpr int QRW = 72;        // staged centre row width: x0 .. x0 + 71 (closing column included)

template <class S>
struct QHalo {  // staged row: x0 - SX .. x0 - SX + W - 1 (16-byte aligned start and width)
  static constexpr int SX = sizeof(S) == 2 ? 8 : 4;
  static constexpr int W = sizeof(S) == 2 ? 80 : 72;
};
constexpr size_t qup(size_t x) { return (x + 127) / 128 * 128; }
template <class S, bool HR, bool HW>
struct QLay {
  static constexpr size_t BV = qup((size_t)(QTY + 3) * QHalo<S>::W * sizeof(S));
  static constexpr size_t BK = qup((size_t)(QTY + 2) * QHalo<S>::W * sizeof(S));
  static constexpr size_t BM = qup((size_t)(QTY + 1) * QMW * 4);
  static constexpr size_t BR = HR ? qup((size_t)(QTY + 1) * QRW * sizeof(S)) : 0;
  static constexpr size_t BW = HW ? qup((size_t)(QTY + 1) * QRW * sizeof(S)) : 0;
  static constexpr size_t STB = BV + BK + BM + BR + BW;
  static constexpr size_t SMEM = 256 + QNS * STB;
};

template <class S, class To>
struct QArgs {
  Geom g;
  const S* v;    // iterate / input (null: zero)
  const S* r;    // sweep right-hand side
  const S* w;    // previous iterate (null: zero)
  To* out;
  const S* kap;
  const uint32_t* mask;
  float cA, cB;  // e' = e + cA (e - w) + cB D^-1 (r - A e)
  float c0, c3;  // K0 coefficients
};
struct alignas(64) QMaps {
  CUtensorMap v, k, m, r, w;
};

__device__ __forceinline__ float2 Q2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 qadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 qmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 qfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class S>
__device__ __forceinline__ float ldf(const S* p) { return Cv<S>::ld(p); }
template <class S>
__device__ __forceinline__ float2 ld2(const S* p);  // two consecutive values, p 2-element aligned
template <>
__device__ __forceinline__ float2 ld2<float>(const float* p) { return *reinterpret_cast<const float2*>(p); }
template <>
__device__ __forceinline__ float2 ld2<bf16>(const bf16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
template <class T>
__device__ __forceinline__ void st2(T* p, float2 v);
template <>
__device__ __forceinline__ void st2<float>(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
template <>
__device__ __forceinline__ void st2<bf16>(bf16* p, float2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
}

// VAR: bit 0 iterate present, bit 1 a(e - w) term, bit 2 previous iterate staged
template <class S, class To, int OP, int VAR>
__global__ void __launch_bounds__(QNT, 3) q_tile(const __grid_constant__ QArgs<S, To> a, const __grid_constant__ QMaps tm) {
  constexpr bool SM = OP == 1;                 // smoother sweep (else apply)
  constexpr bool HV = !SM || (VAR & 1);
  constexpr bool HCA = SM && (VAR & 2);
  constexpr bool HW = SM && (VAR & 4);
  constexpr int SX = QHalo<S>::SX, W = QHalo<S>::W;
  typedef QLay<S, SM, HW> LY;
  constexpr size_t BV = LY::BV, BK = LY::BK, BM = LY::BM, BR = LY::BR, STB = LY::STB;
  const Geom& g = a.g;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned char* stages = smem_raw + 128;
  __shared__ int stage_bad;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int TY = g.TY;
  const int x0 = blockIdx.x * QTX, y0 = blockIdx.y * TY;
  int zs, ze;
  zchunk(g.Nz, g.NZ2, blockIdx.z, zs, ze);
  const int mx = (x0 >> 5) & ~3;
  const unsigned bytesV = (unsigned)((TY + 3) * W * sizeof(S)), bytesK = (unsigned)((TY + 2) * W * sizeof(S));
  const unsigned bytesM = (unsigned)((TY + 1) * QMW * 4), bytesR = (unsigned)((TY + 1) * QRW * sizeof(S));
  auto stage_of = [&](int q) { return (q - zs + 1) % QNS; };
  auto base_of = [&](int q) { return stages + (size_t)stage_of(q) * STB; };
  auto sV = [&](int q) { return reinterpret_cast<const S*>(base_of(q)); };
  auto sK = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV); };
  auto sM = [&](int q) { return reinterpret_cast<const uint32_t*>(base_of(q) + BV + BK); };
  auto sR = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV + BK + BM); };
  auto sW = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV + BK + BM + BR); };

  // group q: node plane q of v, element plane q-1 of kappa, mask / r / w of node plane q-1
  auto issue = [&](int q) {
    const bool hv = HV && q <= ze + 1;
    const int qk = q - 1;
    const bool hk = qk >= zs - 1 && qk <= ze;
    const bool hc = qk >= zs && qk <= ze;
    const unsigned bytes = (hv ? bytesV : 0u) + (hk ? bytesK : 0u) + (hc ? bytesM : 0u) + (hc && SM ? bytesR : 0u) +
                           (hc && HW ? bytesR : 0u);
    const int s = stage_of(q);
    uint64_t* bar = bars + s;
    unsigned char* b = stages + (size_t)s * STB;
    mbar_expect_tx(bar, bytes);
    if (hv) tma_load3(b, &tm.v, x0 - SX, y0, q + 1, bar);
    if (hk) tma_load3(b + BV, &tm.k, x0 - SX, y0, qk + 1, bar);
    if (hc) {
      tma_load3(b + BV + BK, &tm.m, mx, y0 + 1, qk + 1, bar);
      if (SM) tma_load3(b + BV + BK + BM, &tm.r, x0, y0 + 1, qk + 1, bar);
      if (HW) tma_load3(b + BV + BK + BM + BR, &tm.w, x0, y0 + 1, qk + 1, bar);
    }
  };
  auto wait_group = [&](int q) {
    if (stage_bad) return;
    const unsigned parity = (unsigned)(((q - zs + 1) / QNS) & 1);
    if (!mbar_wait_limited(bars + stage_of(q), parity, g.wait)) {  // bounded: give up, flag, never hang
      stage_bad = 1;
      atomicExch(g.err, 1);
    }
  };

  if (tid == 0) {
    stage_bad = 0;
    for (int s = 0; s < QNS; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  static_assert(QNS == 6, "the two-plane step keeps four groups resident and two in flight");
  int qhi = zs + 2;  // last group issued (thread 0)
  if (tid == 0)
    for (int q = zs - 1; q <= zs + 2; ++q) issue(q);

  const float2 c0 = Q2(a.c0, a.c0), c3 = Q2(a.c3, a.c3);
  const bool lastx = x0 + QTX == g.Nx, lasty = y0 + TY == g.Ny;

  // Values carried in registers from node plane t-1 to t (a warp marches in z
  // over the same row): the element plane t-1 conductivities (kappa at x-1,
  // x, x+1 of element rows y-1, y) and the iterate on node plane t (x-1 .. x+2
  // of rows y-1, y, y+1), so that each step reads one new plane of each from
  // shared memory instead of two of kappa and three of the iterate.
  float ck[2][3], cv[3][4];
  bool carried = false;

  // update of the two nodes (x0 + c, x0 + c + 1) of tile row r (0..TY) in node plane t
  auto pair_row = [&](int t, int r, int c) {
    const int sc = c + SX;
    // conductivities kf[a][b][.]: element plane t-1+a, element row y-1+b, x-1 / x / x+1
    float kf[2][2][3];
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      if (aa == 0 && carried) {
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
          for (int q = 0; q < 3; ++q) kf[0][bb][q] = ck[bb][q];
        continue;
      }
      const S* kp = sK(t + aa);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int o = (r + bb) * W + sc;
        const float2 k01 = ld2<S>(kp + o);
        kf[aa][bb][0] = ldf<S>(kp + o - 1);
        kf[aa][bb][1] = k01.x;
        kf[aa][bb][2] = k01.y;
      }
    }
    // k[a][b][s]: side s (0: elements (x-1, x) of the two nodes, 1: elements (x, x+1))
    float2 k[2][2][2];
#pragma unroll
    for (int aa = 0; aa < 2; ++aa)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        k[aa][bb][0] = Q2(kf[aa][bb][0], kf[aa][bb][1]);
        k[aa][bb][1] = Q2(kf[aa][bb][1], kf[aa][bb][2]);
      }
    float2 zp[2][2], yp[2][2], xp[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        zp[i][j] = qadd(k[0][i][j], k[1][i][j]);
        yp[i][j] = qadd(k[i][0][j], k[i][1][j]);
        xp[i][j] = qadd(k[i][j][0], k[i][j][1]);
      }
    const float2 K8 = qadd(qadd(zp[0][0], zp[0][1]), qadd(zp[1][0], zp[1][1]));
    float2 Av = Q2(0.f, 0.f), ctr = Q2(0.f, 0.f);
    if (HV) {
      // vf[dz][dy][.]: iterate at x-1, x, x+1, x+2 of node plane t+dz, row y+dy
      float vf[3][3][4];
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        if (dz == 0 && carried) {
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int q = 0; q < 4; ++q) vf[1][dy][q] = cv[dy][q];
          continue;
        }
        const S* vp = sV(t + dz);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int o = (r + 1 + dy) * W + sc;
          const float2 v01 = ld2<S>(vp + o);
          vf[dz + 1][dy + 1][0] = ldf<S>(vp + o - 1);
          vf[dz + 1][dy + 1][1] = v01.x;
          vf[dz + 1][dy + 1][2] = v01.y;
          vf[dz + 1][dy + 1][3] = ldf<S>(vp + o + 2);
        }
      }
      float2 s = Q2(0.f, 0.f);
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const float* vv = vf[dz + 1][dy + 1];
          const float2 v01 = Q2(vv[1], vv[2]);
          if (dz == 0 && dy == 0) {
            ctr = v01;
            continue;
          }
          const float2 vl = Q2(vv[0], vv[1]);  // x - 1
          const float2 vr = Q2(vv[2], vv[3]);  // x + 1
          const int ia = dz < 0 ? 0 : 1, ib = dy < 0 ? 0 : 1;
          if (dz == 0) {  // xy face diagonals
            s = qfma(zp[ib][0], vl, s);
            s = qfma(zp[ib][1], vr, s);
          } else if (dy == 0) {  // xz face diagonals
            s = qfma(yp[ia][0], vl, s);
            s = qfma(yp[ia][1], vr, s);
          } else {  // yz face diagonal and the two body diagonals
            s = qfma(xp[ia][ib], v01, s);
            s = qfma(k[ia][ib][0], vl, s);
            s = qfma(k[ia][ib][1], vr, s);
          }
        }
      }
      Av = qfma(qmul(c0, K8), ctr, qmul(c3, s));
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int q = 0; q < 4; ++q) cv[dy][q] = vf[2][dy][q];
    }
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int q = 0; q < 3; ++q) ck[bb][q] = kf[1][bb][q];
    carried = true;
    float2 e;
    if (!SM) {
      e = Av;
    } else {
      const float2 rr = ld2<S>(sR(t + 1) + r * QRW + c);
      const float2 d = qmul(c0, K8);
      const float2 inv = Q2(__frcp_rn(d.x), __frcp_rn(d.y));
      e = qmul(qmul(Q2(a.cB, a.cB), qadd(rr, Q2(-Av.x, -Av.y))), inv);
      if (HV) e = qadd(e, ctr);
      if (HCA) {
        const float2 wv = HW ? ld2<S>(sW(t + 1) + r * QRW + c) : Q2(0.f, 0.f);
        e = qfma(Q2(a.cA, a.cA), qadd(ctr, Q2(-wv.x, -wv.y)), e);
      }
    }
    const int xx = x0 + c, yy = y0 + r;
    const uint32_t mw = sM(t + 1)[r * QMW + ((xx >> 5) - mx)];
    if ((mw >> (xx & 31)) & 1u) e.x = 0.f;
    if ((mw >> ((xx + 1) & 31)) & 1u) e.y = 0.f;
    st2<To>(a.out + nidx(g, xx, yy, t), e);
  };

  // the closing-column node (x0 + 64, y0 + r) of node plane t, one per lane of the
  // extra warp (lanes = rows): per element, kappa times its three face-diagonal
  // nodes and its body-diagonal node (the same operator grouped by element)
  auto col_node = [&](int t, int r) {
    const int sc = QTX + SX;
    float K8 = 0.f, s = 0.f;
#pragma unroll
    for (int ia = 0; ia < 2; ++ia)
#pragma unroll
      for (int ib = 0; ib < 2; ++ib)
#pragma unroll
        for (int is = 0; is < 2; ++is) {
          const float ke = ldf<S>(sK(t + ia) + (r + ib) * W + sc - 1 + is);
          K8 += ke;
          if (HV) {
            const int dx = is ? 1 : -1, dy = ib ? 1 : -1, dz = ia ? 1 : -1;
            const S* v0 = sV(t);
            const S* vz = sV(t + dz);
            const float f = ldf<S>(v0 + (r + 1 + dy) * W + sc + dx) + ldf<S>(vz + (r + 1) * W + sc + dx) +
                            ldf<S>(vz + (r + 1 + dy) * W + sc) + ldf<S>(vz + (r + 1 + dy) * W + sc + dx);
            s = fmaf(ke, f, s);
          }
        }
    const float ctr = HV ? ldf<S>(sV(t) + (r + 1) * W + sc) : 0.f;
    const float Av = HV ? a.c0 * K8 * ctr + a.c3 * s : 0.f;
    float e;
    if (!SM) {
      e = Av;
    } else {
      const float rr = ldf<S>(sR(t + 1) + r * QRW + QTX);
      e = a.cB * (rr - Av) * __frcp_rn(a.c0 * K8);
      if (HV) e += ctr;
      if (HCA) e += a.cA * (ctr - (HW ? ldf<S>(sW(t + 1) + r * QRW + QTX) : 0.f));
    }
    const int xx = x0 + QTX, yy = y0 + r;
    const uint32_t mw = sM(t + 1)[r * QMW + ((xx >> 5) - mx)];
    if ((mw >> (xx & 31)) & 1u) e = 0.f;
    Cv<To>::st(a.out + nidx(g, xx, yy, t), e);
  };

  auto plane = [&](int t) {
    if (w < TY) {
      pair_row(t, w, 2 * lane);
    } else if (w == QTY) {  // extra warp: closing column (lanes = rows) and closing row
      if (lastx && (lane < TY || (lasty && lane == TY))) col_node(t, lane);
      if (lasty) pair_row(t, TY, 2 * lane);
    }
  };
  // Two node planes per CTA barrier: a step reads groups t-1 .. t+2 and, once
  // every warp has left the previous step (which read t-3 .. t), refills the
  // two stages that step released with groups t+3 and t+4.
  for (int t = zs; t <= ze; t += 2) {
    if (t == zs) {
      wait_group(zs - 1);
      wait_group(zs);
    }
    wait_group(t + 1);
    __syncthreads();
    if (tid == 0 && !stage_bad) {  // after a wait gave up no stage is refilled
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(t + 3);
      issue(t + 4);
      qhi = t + 4;
    }
    plane(t);
    if (t + 1 <= ze) {
      wait_group(t + 2);
      plane(t + 1);
    }
  }
  if (tid == 0) mbar_drain(bars, QNS, zs - 1, qhi);
}

template <class T>
struct QDT;
template <>
struct QDT<float> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <>
struct QDT<bf16> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

template <class S, class To, int OP, int VAR>
cudaError_t q_launch(const QArgs<S, To>& a, cudaStream_t st) {
  constexpr bool SM = OP == 1;
  constexpr bool HW = SM && (VAR & 4);
  constexpr bool HV = !SM || (VAR & 1);
  typedef QLay<S, SM, HW> LY;
  const Geom& g = a.g;
  QMaps tm;
  cudaError_t e;
  const int es = (int)sizeof(S);
  if ((e = get_map(&tm.v, HV ? a.v + g.base : nullptr, QDT<S>::v, es, g.P, g.RYn, g.nz + 2, QHalo<S>::W, g.TY + 3)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.k, a.kap + g.base, QDT<S>::v, es, g.P, g.RYe, g.Nz + 2, QHalo<S>::W, g.TY + 2)) != cudaSuccess)
    return e;
  if ((e = get_map(&tm.m, a.mask, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, g.mwr, g.RYn, g.nz + 2, QMW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.r, SM ? a.r + g.base : nullptr, QDT<S>::v, es, g.P, g.RYn, g.nz + 2, QRW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  if ((e = get_map(&tm.w, HW ? a.w + g.base : nullptr, QDT<S>::v, es, g.P, g.RYn, g.nz + 2, QRW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  auto k = q_tile<S, To, OP, VAR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
  const dim3 grid(g.Nx / QTX, g.Ny / g.TY, g.NZ2);
  note_launch(), k<<<grid, QNT, LY::SMEM, st>>>(a, tm);
  return cudaGetLastError();
}

template <class S, class To>
QArgs<S, To> qargs(const Geom& g, const uint32_t* mask, const S* kap) {
  QArgs<S, To> a;
  memset(&a, 0, sizeof a);
  a.g = g;
  a.mask = mask;
  a.kap = kap;
  a.c0 = (float)g.c[0];
  a.c3 = (float)g.c[3];
  return a;
}

}  // namespace

bool fine2_supported(const Geom& g) { return g.cube && g.Nx % QTX == 0 && g.TY <= QTY; }

int fine2_tiles_xy(const Geom& g) { return (g.Nx / QTX) * (g.Ny / g.TY); }

int fine2_ctas_per_sm() {
  typedef QLay<float, true, true> LY;
  auto k = q_tile<float, float, 1, 7>;
  int n = 0;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, QNT, LY::SMEM) != cudaSuccess) n = 0;
  return n;
}

template <class S, class To>
cudaError_t fine2_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e, const S* w, To* out,
                         float cA, float cB, cudaStream_t st) {
  auto a = qargs<S, To>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.w = (e != nullptr) ? w : nullptr;
  a.out = out;
  a.cA = cA;
  a.cB = cB;
  if (e == nullptr) return q_launch<S, To, 1, 0>(a, st);
  if (cA == 0.f) return q_launch<S, To, 1, 1>(a, st);
  if (w == nullptr) return q_launch<S, To, 1, 3>(a, st);
  return q_launch<S, To, 1, 7>(a, st);
}

template <class S>
cudaError_t fine2_apply(const Geom& g, const uint32_t* mask, const S* kap, const S* u, S* y, cudaStream_t st) {
  auto a = qargs<S, S>(g, mask, kap);
  a.v = u;
  a.out = y;
  return q_launch<S, S, 0, 1>(a, st);
}

template cudaError_t fine2_smooth<float, float>(const Geom&, const uint32_t*, const float*, const float*, const float*,
                                                const float*, float*, float, float, cudaStream_t);
template cudaError_t fine2_smooth<bf16, bf16>(const Geom&, const uint32_t*, const bf16*, const bf16*, const bf16*,
                                              const bf16*, bf16*, float, float, cudaStream_t);
template cudaError_t fine2_smooth<bf16, float>(const Geom&, const uint32_t*, const bf16*, const bf16*, const bf16*,
                                               const bf16*, float*, float, float, cudaStream_t);
template cudaError_t fine2_apply<float>(const Geom&, const uint32_t*, const float*, const float*, float*, cudaStream_t);
template cudaError_t fine2_apply<bf16>(const Geom&, const uint32_t*, const bf16*, const bf16*, bf16*, cudaStream_t);

}  // namespace thermo

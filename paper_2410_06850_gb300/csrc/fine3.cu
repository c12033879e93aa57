// FP32 fine-grid sweeps and applies on cubic elements from a separable form of
// the Q1 operator (Sec. 2.2 Eq. (5)): the fine smoother of the cycle (Sec. 3,
// Algorithm 1: e' = e + a (e - e_prev) + b D^-1 (r - A e)) and the FP32 apply.
//
// Operator.  For a cube of edge h, K0 = (h/12) (4 on the diagonal, 0 between
// nodes one edge apart, -1 between nodes two or three coordinates apart).
// With S_e the sum of the eight nodal values of element e this gives, for a
// node i with the conductivities kappa_e of its eight elements,
//   (A v)_i = (h/12) [ 5 K8 v_i + sum_{j axis neighbour} W_ij v_j - sum_{e ∋ i} kappa_e S_e ],
// K8 the sum of the eight kappa_e and W_ij the sum of kappa over the four
// elements that contain the edge ij.  Every term is a sum of box sums, which
// the kernel builds incrementally:
//   B(ex, ey) on a node plane  = v over the 4 nodes of the face (ex..ex+1, ey..ey+1),
//   S = B(plane z) + B(plane z+1),  T = kappa S for the element layer between,
//   C(x, y) = T over the 4 elements (x-1..x, y-1..y) of a layer,
// and the same pair and quadruple sums of kappa give the edge weights and K8.
//
// Layout.  A warp owns one x column of 32 lanes (lane l: node x0 - 1 + l; the
// outputs are lanes 1..30) and R node rows in y; a CTA stacks NW warps in y
// and marches over a ragged chunk of node planes in z.  x neighbours come by
// warp shuffles, y neighbours from the thread's own registers, z neighbours
// from the values carried from the previous plane: each node plane of v and
// each element plane of kappa is read once from shared memory.  One elected
// thread stages, per node plane, the iterate (rows y0-1 .. y0+NW R), kappa,
// r, e_prev and the Dirichlet bits with TMA tensor copies into an mbarrier
// ring (bounded waits, as in the other fine kernels); ghost planes, rows and
// columns of the padded layout hold zeros, so boundary nodes need no special
// code.  About 50 instructions per node and no CTA barrier besides the ring's
// one per plane.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace thermo {

namespace {

constexpr int R3 = 4;            // node rows per warp
constexpr int NW3 = 8;           // warps per CTA (stacked in y)
constexpr int TY3 = R3 * NW3;    // node rows per CTA
constexpr int TX3 = 30;          // output nodes per CTA row (lanes 1..30)
constexpr int WB3 = 36;          // staged row width (floats): x0 - 4 .. x0 + 31 at most
constexpr int MW3 = 8;           // staged mask words per row
constexpr int NS3 = 4;           // TMA ring stages
constexpr int NT3 = 32 * NW3;

constexpr size_t up128(size_t x) { return (x + 127) / 128 * 128; }
struct Lay3 {
  static constexpr size_t BV = up128((size_t)(TY3 + 2) * WB3 * 4);
  static constexpr size_t BK = up128((size_t)(TY3 + 1) * WB3 * 4);
  static constexpr size_t BM = up128((size_t)TY3 * MW3 * 4);
  static constexpr size_t BR = up128((size_t)TY3 * WB3 * 4);
  static constexpr size_t STB = BV + BK + BM + 2 * BR;  // v, kappa, mask, r, e_prev
  static constexpr size_t SMEM = 256 + NS3 * STB;
};

template <class To>
struct Args3 {
  Geom g;
  const float* v;  // iterate / input (null: zero)
  const float* r;  // sweep right-hand side (null for the apply)
  const float* w;  // previous iterate (null: zero)
  To* out;
  const float* kap;
  const uint32_t* mask;
  float cA, cB;    // e' = e + cA (e - w) + cB D^-1 (r - A e)
  float cc;        // h / 12
};
struct Maps3 {
  CUtensorMap v, k, m, r, w;
};

// OP 0: out = A v; OP 1: sweep; OP 2: residual out = r - A v.  VAR bit 0:
// iterate present, bit 1: cA (e - w) term, bit 2: w staged (else zero).
template <class To, int OP, int VAR>
__global__ void __launch_bounds__(NT3, 2) f3_tile(const __grid_constant__ Args3<To> a,
                                                  const __grid_constant__ Maps3 tm) {
  constexpr bool SM = OP == 1;
  constexpr bool HRS = OP >= 1;  // r staged
  constexpr bool HV = !SM || (VAR & 1);
  constexpr bool HCA = SM && (VAR & 2);
  constexpr bool HW = SM && (VAR & 4);
  constexpr int R = R3;
  typedef Lay3 LY;
  const Geom& g = a.g;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned char* stages = smem_raw + 128;
  __shared__ int stage_bad;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
  int zs, ze;
  zchunk(g.Nz, g.NZ3, blockIdx.z, zs, ze);
  const int xs = ((x0 - 1) >> 2) << 2;  // staged column 0 (16-byte aligned, may be negative)
  const int mx = (x0 >> 5) & ~3;        // first staged mask word
  const int x = x0 - 1 + lane;          // this lane's node column
  const int cx = x - xs;                // its staged column
  const int ya = y0 + w * R;            // first node row of this warp
  const unsigned bytesV = (unsigned)((TY3 + 2) * WB3 * 4), bytesK = (unsigned)((TY3 + 1) * WB3 * 4);
  const unsigned bytesM = (unsigned)(TY3 * MW3 * 4), bytesR = (unsigned)(TY3 * WB3 * 4);
  auto stage_of = [&](int q) { return (q - zs + 1) % NS3; };
  auto base_of = [&](int q) { return stages + (size_t)stage_of(q) * LY::STB; };
  // group q: node plane q of v (rows y0-1 ..), element plane q-1 of kappa (rows y0-1 ..),
  // mask / r / w of node plane q-1 (rows y0 ..)
  auto issue = [&](int q) {
    const bool hv = HV && q <= ze + 1;
    const int qk = q - 1;
    const bool hk = qk >= zs - 1 && qk <= ze;
    const bool hc = qk >= zs && qk <= ze;
    const unsigned bytes = (hv ? bytesV : 0u) + (hk ? bytesK : 0u) + (hc ? bytesM : 0u) + (hc && HRS ? bytesR : 0u) +
                           (hc && HW ? bytesR : 0u);
    const int s = stage_of(q);
    uint64_t* bar = bars + s;
    unsigned char* b = stages + (size_t)s * LY::STB;
    mbar_expect_tx(bar, bytes);
    if (hv) tma_load3(b, &tm.v, xs, y0, q + 1, bar);
    if (hk) tma_load3(b + LY::BV, &tm.k, xs, y0, qk + 1, bar);
    if (hc) {
      tma_load3(b + LY::BV + LY::BK, &tm.m, mx, y0 + 1, qk + 1, bar);
      if (HRS) tma_load3(b + LY::BV + LY::BK + LY::BM, &tm.r, xs, y0 + 1, qk + 1, bar);
      if (HW) tma_load3(b + LY::BV + LY::BK + LY::BM + LY::BR, &tm.w, xs, y0 + 1, qk + 1, bar);
    }
  };
  auto wait_group = [&](int q) {
    if (stage_bad) return;
    const unsigned parity = (unsigned)(((q - zs + 1) / NS3) & 1);
    if (!mbar_wait_limited(bars + stage_of(q), parity, g.wait)) {  // bounded: give up, flag, never hang
      stage_bad = 1;
      atomicExch(g.err, 1);
    }
  };
  if (tid == 0) {
    stage_bad = 0;
    for (int s = 0; s < NS3; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int qhi = zs - 2;  // last group issued (thread 0)
  if (tid == 0)
    for (int q = zs - 1; q < zs - 1 + NS3; ++q) issue(q), qhi = q;

  // per-thread constants of the z march (no address arithmetic inside the loop):
  // staged offsets of this thread's first row, its Dirichlet word and bit, its
  // output rows' validity, and the output pointer of its first row, advanced
  // by one plane per step
  const float cA = a.cA, cB = a.cB, cc = a.cc, cc4 = 4.f * a.cc;
  const int Nx = g.Nx, Ny = g.Ny;
  const int offV = w * R * WB3 + cx;                      // v, kappa, r, w rows start at w R
  const int xm = x < 0 ? 0 : x;                           // (lane 0 of the first tile: never stored)
  const int offM = w * R * MW3 + ((xm >> 5) - mx);
  const unsigned bitM = 1u << (xm & 31);
  const long long pstride = g.RYn * g.P;
  unsigned rowok = 0;
#pragma unroll
  for (int i = 0; i < R; ++i)
    if (lane >= 1 && lane <= TX3 && x <= Nx && ya + i <= Ny) rowok |= 1u << i;
  To* op = a.out + nidx(g, xm, ya, zs);
  const long long P = g.P;

  // values of the layer below / the plane below, carried from one node plane to
  // the next in two register sets used alternately (no copies)
  struct Carry {
    float vm[R], vc[R + 2], B[R + 1], C[R], Ky[R], Kym[R], Kx[R + 1], Kxy[R];
  };
  Carry c0, c1;
  // kappa sums of an element layer from its staged rows ya-1 .. ya+R-1
  auto layer_kappa = [&](const float* kp, Carry& o, float (&kn)[R + 1]) {
#pragma unroll
    for (int j = 0; j <= R; ++j) kn[j] = kp[j * WB3];
#pragma unroll
    for (int j = 0; j <= R; ++j) o.Kx[j] = __shfl_up_sync(0xffffffffu, kn[j], 1) + kn[j];  // elements x-1, x
#pragma unroll
    for (int i = 0; i < R; ++i) {
      o.Ky[i] = kn[i] + kn[i + 1];  // element column x, rows y-1, y
      o.Kym[i] = __shfl_up_sync(0xffffffffu, o.Ky[i], 1);
      o.Kxy[i] = o.Kx[i] + o.Kx[i + 1];
    }
  };
  // face sums B of a node plane from its staged rows ya-1 .. ya+R
  auto plane_B = [&](const float* vp, float (&vv)[R + 2], float (&B)[R + 1]) {
#pragma unroll
    for (int j = 0; j < R + 2; ++j) vv[j] = vp[j * WB3];
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      const float p = vv[j] + vv[j + 1];
      B[j] = p + __shfl_down_sync(0xffffffffu, p, 1);
    }
  };
  // layer box sums C from the face sums below (Bb) and above (Ba)
  auto layer_C = [&](const float (&kn)[R + 1], const float (&Bb)[R + 1], const float (&Ba)[R + 1], float (&C)[R]) {
    float T[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) T[j] = kn[j] * (Bb[j] + Ba[j]);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float ty = T[i] + T[i + 1];
      C[i] = ty + __shfl_up_sync(0xffffffffu, ty, 1);
    }
  };
  auto stage_ptr = [&](int q) { return stages + (size_t)((unsigned)(q - zs + 1) % NS3) * LY::STB; };

  // prologue: node plane zs-1 (group zs-1), then layer zs-1/2 (group zs)
  {
    float vpre[R + 2], Bpre[R + 1], kn[R + 1];
    wait_group(zs - 1);
    if (HV) plane_B(reinterpret_cast<const float*>(stage_ptr(zs - 1)) + offV, vpre, Bpre);
    wait_group(zs);
    const unsigned char* sb = stage_ptr(zs);
    if (HV) {
      plane_B(reinterpret_cast<const float*>(sb) + offV, c0.vc, c0.B);
#pragma unroll
      for (int i = 0; i < R; ++i) c0.vm[i] = vpre[i + 1];
    }
    layer_kappa(reinterpret_cast<const float*>(sb + LY::BV) + offV, c0, kn);
    if (HV) layer_C(kn, Bpre, c0.B, c0.C);
  }
  __syncthreads();
  if (tid == 0 && !stage_bad) {  // after a wait gave up no stage is refilled
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    issue(zs - 1 + NS3);
    issue(zs + NS3);
    qhi = zs + NS3;
  }

  // node plane t from the layer below (cu) and group t+1; the layer above goes to nx
  auto step = [&](int t, Carry& cu, Carry& nx) {
    wait_group(t + 1);
    const unsigned char* sb = stage_ptr(t + 1);
    const float* sv = reinterpret_cast<const float*>(sb) + offV;
    const float* sk = reinterpret_cast<const float*>(sb + LY::BV) + offV;
    const uint32_t* smk = reinterpret_cast<const uint32_t*>(sb + LY::BV + LY::BK) + offM;
    const float* sr = reinterpret_cast<const float*>(sb + LY::BV + LY::BK + LY::BM) + offV;
    const float* sw = reinterpret_cast<const float*>(sb + LY::BV + LY::BK + LY::BM + LY::BR) + offV;
    float kn[R + 1];
    if (HV) plane_B(sv, nx.vc, nx.B);
    layer_kappa(sk, nx, kn);
    if (HV) layer_C(kn, cu.B, nx.B, nx.C);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float K8 = cu.Kxy[i] + nx.Kxy[i];
      float Av = 0.f, ctr = 0.f;
      if (HV) {
        ctr = cu.vc[i + 1];
        const float vxp = __shfl_down_sync(0xffffffffu, ctr, 1), vxm = __shfl_up_sync(0xffffffffu, ctr, 1);
        float E = (cu.Ky[i] + nx.Ky[i]) * vxp;
        E = fmaf(cu.Kym[i] + nx.Kym[i], vxm, E);
        E = fmaf(cu.Kx[i + 1] + nx.Kx[i + 1], cu.vc[i + 2], E);
        E = fmaf(cu.Kx[i] + nx.Kx[i], cu.vc[i], E);
        E = fmaf(nx.Kxy[i], nx.vc[i + 1], E);
        E = fmaf(cu.Kxy[i], cu.vm[i], E);
        Av = cc * (fmaf(5.f * K8, ctr, E) - (cu.C[i] + nx.C[i]));
        nx.vm[i] = ctr;
      }
      float e;
      if (OP == 0) {
        e = Av;
      } else if (OP == 2) {
        e = sr[i * WB3] - Av;
      } else {
        // D = (h/3) K8; every lane evaluates (its staged columns exist), only valid ones store
        e = __fdividef(cB * (sr[i * WB3] - Av), cc4 * K8);
        if (HV) e += ctr;
        if (HCA) e = fmaf(cA, ctr - (HW ? sw[i * WB3] : 0.f), e);
      }
      if (smk[i * MW3] & bitM) e = 0.f;
      if (rowok & (1u << i)) Cv<To>::st(op + i * P, e);
    }
    op += pstride;
    __syncthreads();
    if (tid == 0 && !stage_bad) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(t + 1 + NS3);
      qhi = t + 1 + NS3;
    }
  };
  for (int t = zs; t <= ze; t += 2) {
    step(t, c0, c1);
    if (t + 1 <= ze) step(t + 1, c1, c0);
  }
  if (tid == 0) mbar_drain(bars, NS3, zs - 1, qhi);
}

template <class To, int OP, int VAR>
cudaError_t f3_launch(const Args3<To>& a, cudaStream_t st) {
  constexpr bool SM = OP == 1;
  constexpr bool HRS = OP >= 1;
  constexpr bool HW = SM && (VAR & 4);
  constexpr bool HV = !SM || (VAR & 1);
  const Geom& g = a.g;
  Maps3 tm;
  cudaError_t e;
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if ((e = get_map(&tm.v, HV ? a.v + g.base : nullptr, F32, 4, g.P, g.RYn, g.nz + 2, WB3, TY3 + 2)) != cudaSuccess)
    return e;
  if ((e = get_map(&tm.k, a.kap + g.base, F32, 4, g.P, g.RYe, g.Nz + 2, WB3, TY3 + 1)) != cudaSuccess) return e;
  if ((e = get_map(&tm.m, a.mask, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, g.mwr, g.RYn, g.nz + 2, MW3, TY3)) != cudaSuccess)
    return e;
  if ((e = get_map(&tm.r, HRS ? a.r + g.base : nullptr, F32, 4, g.P, g.RYn, g.nz + 2, WB3, TY3)) != cudaSuccess)
    return e;
  if ((e = get_map(&tm.w, HW ? a.w + g.base : nullptr, F32, 4, g.P, g.RYn, g.nz + 2, WB3, TY3)) != cudaSuccess)
    return e;
  auto k = f3_tile<To, OP, VAR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay3::SMEM);
  const dim3 grid(fine3_tiles_x(g), fine3_tiles_y(g), g.NZ3);
  note_launch(), k<<<grid, NT3, Lay3::SMEM, st>>>(a, tm);
  return cudaGetLastError();
}

// rc[B][j] = sum over the nodes i of level-1 block B of Phi[i][j] res[i] (Phi
// node-major, L values per node).  One CTA per strip of blocks sharing (by, bz):
// thread x walks the strip's node rows (4 per axis, 5 for the last block of an
// axis, which also owns the closing node plane / row), each row read with
// coalesced loads; the last thread of a row also takes the closing node x = Nx.
// The four threads of a block then combine by a fixed shuffle tree.
template <int L>
__global__ void k_blk_restrict(Geom g, const float* __restrict__ res, const float* __restrict__ phi,
                               float* __restrict__ rc) {
  const int by = blockIdx.x, bz = blockIdx.y, x = threadIdx.x;
  const int b = g.b;
  const int ylo = by * b, yhi = (by == g.nby - 1) ? g.Ny : ylo + b - 1;
  const int zlo = bz * b, zhi = (bz == g.nbz - 1) ? g.Nz : zlo + b - 1;
  float acc[L];
#pragma unroll
  for (int j = 0; j < L; ++j) acc[j] = 0.f;
  const bool closing = x == g.Nx - 1;  // also owns node x = Nx
  for (int z = zlo; z <= zhi; ++z)
    for (int y = ylo; y <= yhi; ++y) {
      const long long n = nidx(g, x, y, z);
      const float rv = res[n];
      const float* ph = phi + n * L;
      if constexpr (L == 4) {  // node-major Phi: 16-byte aligned rows of four
        const float4 p4 = *reinterpret_cast<const float4*>(ph);
        acc[0] = fmaf(p4.x, rv, acc[0]);
        acc[1] = fmaf(p4.y, rv, acc[1]);
        acc[2] = fmaf(p4.z, rv, acc[2]);
        acc[3] = fmaf(p4.w, rv, acc[3]);
      } else {
#pragma unroll
        for (int j = 0; j < L; ++j) acc[j] = fmaf(ph[j], rv, acc[j]);
      }
      if (closing) {
        const float r2 = res[n + 1];
#pragma unroll
        for (int j = 0; j < L; ++j) acc[j] = fmaf(ph[L + j], r2, acc[j]);
      }
    }
  // blocks of 4 threads along x (b = 4): fixed-order shuffle tree
#pragma unroll
  for (int j = 0; j < L; ++j) {
    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 1);
    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 2);
  }
  if ((x & 3) == 0) {
    const long long B = (x >> 2) + (long long)g.nbx * (by + (long long)g.nby * bz);
#pragma unroll
    for (int j = 0; j < L; ++j) rc[B * L + j] = acc[j];
  }
}

template <class To>
Args3<To> args3(const Geom& g, const uint32_t* mask, const float* kap) {
  Args3<To> a;
  memset(&a, 0, sizeof a);
  a.g = g;
  a.mask = mask;
  a.kap = kap;
  a.cc = (float)(-g.c[3]);  // h / 12 for cubic elements
  return a;
}

}  // namespace

bool fine3_supported(const Geom& g) { return g.cube && g.NZ3 > 0; }
int fine3_tiles_x(const Geom& g) { return (g.nx + TX3 - 1) / TX3; }
int fine3_tiles_y(const Geom& g) { return (g.ny + TY3 - 1) / TY3; }

int fine3_ctas_per_sm() {
  auto k = f3_tile<float, 1, 7>;
  int n = 0;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay3::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT3, Lay3::SMEM) != cudaSuccess) n = 0;
  return n;
}

template <class To>
cudaError_t fine3_smooth(const Geom& g, const uint32_t* mask, const float* kap, const float* r, const float* e,
                         const float* w, To* out, float cA, float cB, cudaStream_t st) {
  auto a = args3<To>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.w = (e != nullptr) ? w : nullptr;
  a.out = out;
  a.cA = cA;
  a.cB = cB;
  if (e == nullptr) return f3_launch<To, 1, 0>(a, st);
  if (cA == 0.f) return f3_launch<To, 1, 1>(a, st);
  if (w == nullptr) return f3_launch<To, 1, 3>(a, st);
  return f3_launch<To, 1, 7>(a, st);
}

cudaError_t fine3_apply(const Geom& g, const uint32_t* mask, const float* kap, const float* u, float* y,
                        cudaStream_t st) {
  auto a = args3<float>(g, mask, kap);
  a.v = u;
  a.out = y;
  return f3_launch<float, 0, 1>(a, st);
}

bool fine3_restrict_supported(const Geom& g, int L1) {
  return fine3_supported(g) && g.b == 4 && g.Nx <= 1024 && g.Nx % 32 == 0 && L1 == 4;
}

// level-1 restriction of the cycle (Algorithm 1): res = r - A e (FP32, zero on
// Gamma_D) by the separable engine into `res`, then rc = Phi^T res block by block
cudaError_t fine3_restrict(const Geom& g, const uint32_t* mask, const float* kap, const float* r, const float* e,
                           const float* phi, float* res, float* rc, int L1, cudaStream_t st) {
  if (!fine3_restrict_supported(g, L1)) return cudaErrorInvalidValue;
  auto a = args3<float>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.out = res;
  cudaError_t err = f3_launch<float, 2, 1>(a, st);
  if (err != cudaSuccess) return err;
  note_launch(), k_blk_restrict<4><<<dim3(g.nby, g.nbz), g.Nx, 0, st>>>(g, res, phi, rc);
  return cudaGetLastError();
}

template cudaError_t fine3_smooth<float>(const Geom&, const uint32_t*, const float*, const float*, const float*,
                                         const float*, float*, float, float, cudaStream_t);

}  // namespace thermo

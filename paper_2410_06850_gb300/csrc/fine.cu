// Fine-grid kernels: matrix-free Q1 operator and the fine part of the
// multigrid cycle (Sec. 3, Algorithm 1).
//
// One z-marching engine serves every fine-grid pass.  A CTA owns a TX x TY
// tile of nodes (TX <= 32 columns = lanes, TY <= 8 rows = one warp each) and
// marches over ZC node planes.  Each plane of the input field (one-node
// halo), of the element conductivity, of the Dirichlet bitmask and of the
// centre-only arrays of the epilogue (r, w, or Phi) is staged into shared
// memory by one elected thread with TMA tensor copies
// (cp.async.bulk.tensor) into a ring of stages, each guarded by an
// mbarrier with a byte-count transaction; three planes stay resident for
// the stencil and the rest are in flight.  Every lane keeps the 3x3 windows
// of its node for the two previous planes in registers (z unrolled by three
// so the windows rotate without moves) and reads only the new plane.  The
// tile on the high face of an axis also owns the closing node plane: an
// extra warp computes the closing column (lanes = rows) and the closing row
// (lanes = columns) from the resident stages.
//
// Operator (node-centred gather of A = sum_e kappa_e K0_e, K0[a][b] =
// c[a ^ b]): with the 8 elements around node i indexed (dx,dy,dz),
//   (A v)_i = c0 K8 v_i + c3 sum_xy zp v + c5 sum_xz yp v + c6 sum_yz xp v
//           + c7 sum_diag kappa v  [+ c1/c2/c4 axis terms, non-cubic boxes]
// where K8 is the sum of the 8 conductivities and zp/yp/xp are sums of the
// two elements sharing an edge (Sec. 2.2 Eq. (5) realised for Q1).
// Dirichlet rows are identities.  Inputs of the hot kernels vanish on
// Gamma_D by construction (Krylov directions, cycle iterates); the MASKIN
// variants zero them on load for arbitrary inputs.
#include <cuda.h>

#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace thermo {

enum FineOp { F_APPLY = 0, F_SMOOTH = 1, F_RESTRICT = 3 };

constexpr int TYM = 8;            // rows per tile (max), one warp each
constexpr int FNT = 32 * (TYM + 1);  // + one warp for the closing column / row
constexpr int MBW = 8;            // staged mask words per row
constexpr int CWD = 40;           // staged centre row width (elements)
constexpr int PNODE = 33;         // Phi nodes per staged centre row

template <class S>
struct Halo {
  static constexpr int SX = sizeof(S) == 2 ? 8 : 4;   // halo rows start at x0 - SX (16-byte aligned)
  static constexpr int W = sizeof(S) == 2 ? 48 : 40;  // halo row width (elements)
};
template <class C, int LP>
struct PhiBox {  // staged Phi row width in elements of C (16-byte multiple)
  static constexpr int PW = ((PNODE * LP * (int)sizeof(C) + 15) / 16) * 16 / (int)sizeof(C);
};

// Stage layout (bytes; 128-aligned parts): halo field, conductivity, mask,
// centre r, centre w, centre Phi.
template <class S, int OP, int LP, bool HWW>
struct FLay {
  typedef typename Cv<S>::C C;
  static constexpr size_t A = 128;
  static constexpr size_t up(size_t x) { return (x + A - 1) / A * A; }
  static constexpr bool HR = OP == F_SMOOTH || OP == F_RESTRICT;
  static constexpr bool HP = OP == F_RESTRICT;
  static constexpr int PW = PhiBox<C, LP>::PW;
  static constexpr size_t BV = up((size_t)(TYM + 3) * Halo<S>::W * sizeof(S));
  static constexpr size_t BK = up((size_t)(TYM + 2) * Halo<S>::W * sizeof(S));
  static constexpr size_t BM = up((size_t)(TYM + 1) * MBW * 4);
  static constexpr size_t BR = HR ? up((size_t)(TYM + 1) * CWD * sizeof(S)) : 0;
  static constexpr size_t BW = HWW ? BR : 0;
  static constexpr size_t BP = HP ? up((size_t)(TYM + 1) * PW * sizeof(C)) : 0;
  static constexpr size_t STB = BV + BK + BM + BR + BW + BP;
  static constexpr int NS = sizeof(S) == 8 ? 4 : 6;  // ring stages: 3 resident + NS-3 in flight
  static constexpr size_t SMEM = 256 + (size_t)NS * STB;  // + barriers + alignment slack
};

struct alignas(64) TMaps {
  CUtensorMap v, k, m, r, w, p;
};

template <class S, class To>
struct FineArgs {
  typedef typename Cv<S>::C C;
  Geom g;
  const S* v;       // APPLY: u; SMOOTH/RESTRICT: e (null: e = 0)
  const S* r;       // smoother right-hand side / residual source
  const S* w;       // SMOOTH: previous iterate of the three-term recurrence (null: zero)
  To* out;
  const S* kap;     // element conductivity (padded)
  const uint32_t* mask;
  const C* phi;     // level-1 basis [nsize][L1]
  C* rc;            // level-1 restricted residual [cells][L1]
  C cA;             // coefficient of (v - w)
  C omega;          // coefficient of D^-1 (r - A v)
  C cc[8];          // K0 coefficients c[a ^ b] in the compute type (converted on the host)
  double* partial;  // dot partials, one per CTA
  unsigned* counter;
  double* dot;
};

template <class C, bool CUBE>
__device__ __forceinline__ C stencil(const C (&vm)[3][3], const C (&v0)[3][3], const C (&vp)[3][3],
                                     const C (&km)[2][2], const C (&kp)[2][2], const C* cc, C& K8) {
  C zp[2][2], yp[2][2], xp[2][2];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) zp[dy][dx] = km[dy][dx] + kp[dy][dx];
#pragma unroll
  for (int dx = 0; dx < 2; ++dx) {
    yp[0][dx] = km[0][dx] + km[1][dx];
    yp[1][dx] = kp[0][dx] + kp[1][dx];
  }
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
    xp[0][dy] = km[dy][0] + km[dy][1];
    xp[1][dy] = kp[dy][0] + kp[dy][1];
  }
  K8 = zp[0][0] + zp[0][1] + zp[1][0] + zp[1][1];
  C sxy = zp[0][0] * v0[0][0] + zp[0][1] * v0[0][2] + zp[1][0] * v0[2][0] + zp[1][1] * v0[2][2];
  C sxz = yp[0][0] * vm[1][0] + yp[0][1] * vm[1][2] + yp[1][0] * vp[1][0] + yp[1][1] * vp[1][2];
  C syz = xp[0][0] * vm[0][1] + xp[0][1] * vm[2][1] + xp[1][0] * vp[0][1] + xp[1][1] * vp[2][1];
  C sbd = km[0][0] * vm[0][0] + km[0][1] * vm[0][2] + km[1][0] * vm[2][0] + km[1][1] * vm[2][2] +
          kp[0][0] * vp[0][0] + kp[0][1] * vp[0][2] + kp[1][0] * vp[2][0] + kp[1][1] * vp[2][2];
  C y;
  if (CUBE) {
    // c3 = c5 = c6 = c7 for cubes
    y = cc[0] * K8 * v0[1][1] + cc[3] * (sxy + sxz + syz + sbd);
  } else {
    C sx = (zp[0][0] + zp[1][0]) * v0[1][0] + (zp[0][1] + zp[1][1]) * v0[1][2];
    C sy = (zp[0][0] + zp[0][1]) * v0[0][1] + (zp[1][0] + zp[1][1]) * v0[2][1];
    C sz = (xp[0][0] + xp[0][1]) * vm[1][1] + (xp[1][0] + xp[1][1]) * vp[1][1];
    y = cc[0] * K8 * v0[1][1] + cc[3] * sxy + cc[5] * sxz + cc[6] * syz + cc[7] * sbd +
        cc[1] * sx + cc[2] * sy + cc[4] * sz;
  }
  return y;
}


// VAR (sweeps): bit 0 input iterate present, bit 1 three-term (cA) term, bit 2 w present
template <class S, class To, int OP, bool CUBE, int L1, bool DOT, bool MASKIN, int VAR>
__global__ void __launch_bounds__(FNT, sizeof(S) == 8 ? 1 : (OP == F_RESTRICT ? 2 : 3)) fine_tile(const __grid_constant__ FineArgs<S, To> a,
                                                 const __grid_constant__ TMaps tm) {
  typedef typename Cv<S>::C C;
  constexpr int LP = L1 > 0 ? L1 : 1;
  constexpr int SX = Halo<S>::SX, W = Halo<S>::W, PW = PhiBox<C, LP>::PW;
  constexpr bool HV = OP != F_SMOOTH || (VAR & 1);
  constexpr bool HCA = OP == F_SMOOTH && (VAR & 2);
  constexpr bool HWW = OP == F_SMOOTH && (VAR & 4);
  constexpr bool HR = OP == F_SMOOTH || OP == F_RESTRICT;
  constexpr bool HP = OP == F_RESTRICT && L1 > 0;
  constexpr int NS = FLay<S, OP, LP, HWW>::NS;
  typedef FLay<S, OP, LP, HWW> LY;
  constexpr size_t BV = LY::BV, BK = LY::BK, BM = LY::BM, BR = LY::BR, BW = LY::BW, STB = LY::STB;
  const Geom& g = a.g;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // TMA destinations must be 128-byte aligned: align the dynamic base by hand
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);  // NS barriers in the first 128 bytes
  unsigned char* stages = smem_raw + 128;
  __shared__ int stage_bad;  // a stage wait gave up: skip the remaining waits (results invalid, flagged)
  __shared__ C red[TYM + 2][8][LP];  // restriction scratch: rows, block columns, vectors
  __shared__ C redc[TYM + 1][LP];
  __shared__ double dsh[TYM + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int TX = g.TX, TY = g.TY;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool lastx = (x0 + TX == g.Nx), lasty = (y0 + TY == g.Ny);
  const int zs = blockIdx.z * g.ZC;
  const int ze = (zs + g.ZC == g.Nz) ? g.Nz : zs + g.ZC - 1;
  const bool rowwarp = w < TY;        // warps beyond TY (and the extra warp) hold no row
  const bool extra = w == TYM;        // closing column / row warp
  const bool xact = lane < TX;
  const int x = x0 + lane, y = y0 + w;
  const int mx = (x0 >> 5) & ~3;      // first staged mask word
  // compute-type coefficients straight from the parameter bank (no FP64 conversions per node)
  const C* ccv = a.cc;
  const C c0 = a.cc[0];

  // stage bytes of one group
  const unsigned bytesV = (unsigned)((TY + 3) * W * sizeof(S)), bytesK = (unsigned)((TY + 2) * W * sizeof(S));
  const unsigned bytesM = (unsigned)((TY + 1) * MBW * 4), bytesR = (unsigned)((TY + 1) * CWD * sizeof(S));
  const unsigned bytesP = (unsigned)((TY + 1) * PW * sizeof(C));
  auto stage_of = [&](int q) { return (q - zs + 1) % NS; };
  auto base_of = [&](int q) { return stages + (size_t)stage_of(q) * STB; };
  auto sV = [&](int q) { return reinterpret_cast<const S*>(base_of(q)); };
  auto sK = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV); };
  auto sM = [&](int q) { return reinterpret_cast<const uint32_t*>(base_of(q) + BV + BK); };
  auto sR = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV + BK + BM); };
  auto sW = [&](int q) { return reinterpret_cast<const S*>(base_of(q) + BV + BK + BM + BR); };
  auto sP = [&](int q) { return reinterpret_cast<const C*>(base_of(q) + BV + BK + BM + BR + BW); };

  // group q: node plane q, element plane q-1, mask + centre arrays of plane q-1
  auto issue = [&](int q) {
    const bool hv = HV && q <= ze + 1;
    const int qk = q - 1;
    const bool hk = qk >= zs - 1 && qk <= ze;
    const bool hc = qk >= zs && qk <= ze;
    const unsigned bytes = (hv ? bytesV : 0u) + (hk ? bytesK : 0u) + (hc ? bytesM : 0u) +
                           (hc && HR ? bytesR : 0u) + (hc && HWW ? bytesR : 0u) + (hc && HP ? bytesP : 0u);
    const int s = stage_of(q);
    uint64_t* bar = bars + s;
    unsigned char* b = stages + (size_t)s * STB;
    mbar_expect_tx(bar, bytes);  // always arrive, so every stage's phases stay in step
    if (hv) tma_load3(b, &tm.v, x0 - SX, y0, q + 1, bar);
    if (hk) tma_load3(b + BV, &tm.k, x0 - SX, y0, qk + 1, bar);
    if (hc) {
      tma_load3(b + BV + BK, &tm.m, mx, y0 + 1, qk + 1, bar);
      if (HR) tma_load3(b + BV + BK + BM, &tm.r, x0, y0 + 1, qk + 1, bar);
      if (HWW) tma_load3(b + BV + BK + BM + BR, &tm.w, x0, y0 + 1, qk + 1, bar);
      if (HP) tma_load3(b + BV + BK + BM + BR + BW, &tm.p, x0 * LP, y0 + 1, qk + 1, bar);
    }
  };
  auto wait_group = [&](int q) {
    if (stage_bad) return;
    const unsigned parity = (unsigned)(((q - zs + 1) / NS) & 1);
    if (!mbar_wait_limited(bars + stage_of(q), parity, g.wait)) {  // bounded: give up, flag, never hang
      stage_bad = 1;
      atomicExch(g.err, 1);
    }
  };

  if (tid == 0) {
    stage_bad = 0;
    for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int qhi = zs - 2;  // last group issued (thread 0)
  if (tid == 0)
    for (int q = zs - 1; q < zs - 1 + (NS - 3); ++q) issue(q), qhi = q;

  C VA[3][3], VB[3][3], VC[3][3], KA[2][2], KB[2][2], KC[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) VA[i][j] = VB[i][j] = VC[i][j] = C(0);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) KA[i][j] = KB[i][j] = KC[i][j] = C(0);
  C acc[LP], accR[LP];
#pragma unroll
  for (int j = 0; j < LP; ++j) acc[j] = accR[j] = C(0);
  double dacc = 0.0;

  // epilogue of one node; ci: staged centre column, crow: staged centre row
  auto node = [&](int xx, int yy, int t, int crow, int ccol, const C (&vm)[3][3], const C (&v0)[3][3],
                  const C (&vp)[3][3], const C (&km)[2][2], const C (&kp)[2][2], C (&ac)[LP]) {
    C K8;
    const C Av0 = stencil<C, CUBE>(vm, v0, vp, km, kp, ccv, K8);
    const C Av = HV ? Av0 : C(0);
    const long long n = nidx(g, xx, yy, t);
    const uint32_t mw = sM(t + 1)[crow * MBW + ((xx >> 5) - mx)];
    const bool dir = (mw >> (xx & 31)) & 1u;
    if (OP == F_APPLY) {
      C yv = Av;
      if (dir) yv = MASKIN ? Cv<S>::ld(a.v + n) : C(0);
      Cv<To>::st(a.out + n, yv);
      if (DOT) dacc += (double)v0[1][1] * (double)yv;
    } else if (OP == F_SMOOTH) {
      const C rr = Cv<S>::ld(sR(t + 1) + crow * CWD + ccol);
      const C d = c0 * K8;
      C inv;
      if (sizeof(C) == 4) {
        inv = (C)__frcp_rn((float)d);
      } else {
        const double i0 = (double)__frcp_rn((float)d);  // FP32 seed, one FP64 Newton step
        inv = (C)(i0 * (2.0 - (double)d * i0));
      }
      C e = a.omega * (rr - Av) * inv;
      if (HV) e += v0[1][1];
      if (HCA) e += a.cA * (v0[1][1] - (HWW ? Cv<S>::ld(sW(t + 1) + crow * CWD + ccol) : C(0)));
      if (dir) e = C(0);
      Cv<To>::st(a.out + n, e);
    } else if (OP == F_RESTRICT) {
      const C rr = Cv<S>::ld(sR(t + 1) + crow * CWD + ccol);
      const C sres = dir ? C(0) : rr - Av;
      const C* ph = sP(t + 1) + crow * PW + ccol * LP;
#pragma unroll
      for (int j = 0; j < LP; ++j) ac[j] += sres * ph[j];
    }
  };

  // windows of any staged node (row sr = y - (y0-1) - 1, column sc = x - (x0 - SX) - 1)
  auto win = [&](int t, int sr, int sc, C (&vm)[3][3], C (&v0)[3][3], C (&vp)[3][3], C (&km)[2][2],
                 C (&kp)[2][2]) {
    const S* a0 = sV(t - 1);
    const S* a1 = sV(t);
    const S* a2 = sV(t + 1);
    const S* k0 = sK(t);
    const S* k1 = sK(t + 1);
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        const int o = (sr + oy) * W + sc + ox;
        vm[oy][ox] = HV ? Cv<S>::ld(a0 + o) : C(0);
        v0[oy][ox] = HV ? Cv<S>::ld(a1 + o) : C(0);
        vp[oy][ox] = HV ? Cv<S>::ld(a2 + o) : C(0);
      }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int o = (sr + dy) * W + sc + dx;
        km[dy][dx] = Cv<S>::ld(k0 + o);
        kp[dy][dx] = Cv<S>::ld(k1 + o);
      }
  };

  auto restrict_flush = [&](int t) {
    if (OP != F_RESTRICT) return;
    const int bz = blk_of(t, 4, g.nbz);
    const int zend = (bz == g.nbz - 1) ? g.Nz : bz * 4 + 3;
    if (t != zend) return;  // uniform across the CTA
    const int nbl = TX / 4;
    if (rowwarp) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        C v = xact ? acc[j] : C(0);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (xact && (lane & 3) == 0) red[w][lane >> 2][j] = v;
        acc[j] = C(0);
      }
    }
    if (extra) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        if (lane <= TY) redc[lane][j] = lastx ? acc[j] : C(0);  // closing column, row y0 + lane
        C v = (lasty && xact) ? accR[j] : C(0);                 // closing row
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (xact && (lane & 3) == 0) red[TYM + 1][lane >> 2][j] = v;
        acc[j] = accR[j] = C(0);
      }
    }
    __syncthreads();
    for (int o = tid; o < nbl * (TY / 4) * LP; o += FNT) {
      const int j = o % LP, lb = o / LP, bxl = lb % nbl, byl = lb / nbl;
      C s = C(0);
      for (int rr = 0; rr < 4; ++rr) s += red[byl * 4 + rr][bxl][j];
      if (lastx && bxl == nbl - 1) {
        for (int rr = 0; rr < 4; ++rr) s += redc[byl * 4 + rr][j];
        if (lasty && byl == TY / 4 - 1) s += redc[TY][j];
      }
      if (lasty && byl == TY / 4 - 1) s += red[TYM + 1][bxl][j];
      const long long cell = (x0 / 4 + bxl) + (long long)g.nbx * ((y0 / 4 + byl) + (long long)g.nby * bz);
      a.rc[cell * LP + j] = s;
    }
  };

  auto step = [&](int t, C (&Vm)[3][3], C (&V0)[3][3], C (&Vp)[3][3], C (&Km)[2][2], C (&Kp)[2][2]) {
    wait_group(t + 1);
    __syncthreads();
    if (MASKIN && HV) {
      // zero the landed node plane t+1 on Gamma_D (inputs may be arbitrary there)
      S* d = const_cast<S*>(sV(t + 1));
      for (int i = tid; i < (TY + 3) * W; i += FNT) {
        const int ly = i / W, lx = i - ly * W;
        if (is_dir(g, a.mask, x0 - SX + lx, y0 - 1 + ly, t + 1)) Cv<S>::st(d + i, C(0));
      }
      __syncthreads();
    }
    if (tid == 0 && !stage_bad) {  // after a wait gave up no stage is refilled
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier generic accesses before TMA writes
      issue(t + NS - 2);
      qhi = t + NS - 2;
    }
    if (rowwarp) {
      const S* s1 = sV(t + 1);
      const S* k1 = sK(t + 1);
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) Vp[oy][ox] = HV ? Cv<S>::ld(s1 + (w + oy) * W + lane + SX - 1 + ox) : C(0);
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) Kp[dy][dx] = Cv<S>::ld(k1 + (w + dy) * W + lane + SX - 1 + dx);
      if (t >= zs && xact) node(x, y, t, w, lane, Vm, V0, Vp, Km, Kp, acc);
    } else if (extra && t >= zs) {
      C vm[3][3], v0[3][3], vp[3][3], km[2][2], kp[2][2];
      // closing column x0 + TX, row y0 + lane; row y0 + TY only in the last tile row (else the
      // next tile owns that node and a second evaluation would count twice in the dot)
      if (lastx && (lane < TY || (lasty && lane == TY))) {
        win(t, lane, TX + SX - 1, vm, v0, vp, km, kp);
        node(x0 + TX, y0 + lane, t, lane, TX, vm, v0, vp, km, kp, acc);
      }
      if (lasty && xact) {  // closing row y0 + TY, column x0 + lane
        win(t, TY, lane + SX - 1, vm, v0, vp, km, kp);
        node(x, y0 + TY, t, TY, lane, vm, v0, vp, km, kp, accR);
      }
    }
    if (t >= zs) restrict_flush(t);
  };

  for (int t = zs - 2; t <= ze; t += 3) {
    step(t, VA, VB, VC, KA, KB);
    if (t + 1 > ze) break;
    step(t + 1, VB, VC, VA, KB, KC);
    if (t + 2 > ze) break;
    step(t + 2, VC, VA, VB, KC, KA);
  }
  if (tid == 0) mbar_drain(bars, NS, zs - 1, qhi);

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
      for (int i = 0; i < TYM + 1; ++i) s += dsh[i];
      a.partial[bid] = s;
      __threadfence();
      last = (atomicAdd(a.counter, 1u) == nblk - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double v = 0.0;
      for (unsigned i = tid; i < nblk; i += FNT) v += __ldcg(a.partial + i);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) dsh[w] = v;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < TYM + 1; ++i) s += dsh[i];
        *a.dot = s;
        *a.counter = 0u;
      }
    }
  }
}

// e[n] += sum_j Phi[n][j] ec[cell(n)][j]  (level-1 prolongation, in place)
template <class S, int L1>
__global__ void k_prolong(Geom g, const typename Cv<S>::C* __restrict__ phi, const typename Cv<S>::C* __restrict__ ec,
                          S* __restrict__ e) {
  typedef typename Cv<S>::C C;
  const long long rows = (long long)g.ny * g.nz;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < rows * g.nx;
       it += (long long)gridDim.x * blockDim.x) {
    const long long row = it / g.nx;
    const int x = (int)(it - row * g.nx);
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long n = nidx(g, x, y, z);
    const long long cell =
        blk_of(x, 4, g.nbx) + (long long)g.nbx * (blk_of(y, 4, g.nby) + (long long)g.nby * blk_of(z, 4, g.nbz));
    C s = C(0);
    if (L1 == 4 && sizeof(C) == 4) {
      const float4 p = *reinterpret_cast<const float4*>(phi + n * 4);
      const float4 c = *reinterpret_cast<const float4*>(ec + cell * 4);
      s = (C)(p.x * c.x + p.y * c.y + p.z * c.z + p.w * c.w);
    } else {
#pragma unroll
      for (int j = 0; j < L1; ++j) s += phi[n * L1 + j] * ec[cell * L1 + j];
    }
    Cv<S>::st(e + n, Cv<S>::ld(e + n) + s);
  }
}

// ---------------------------------------------------------------------------
// host side: tensor maps (cached per buffer and box) and launchers

template <class T>
struct DT;
template <>
struct DT<double> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
};
template <>
struct DT<float> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <>
struct DT<bf16> {
  static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

static dim3 fine_grid(const Geom& g) { return dim3(g.Nx / g.TX, g.Ny / g.TY, g.Nz / g.ZC); }

template <class S, class To, int OP, int L1, bool DOT, bool MASKIN = false, int VAR = 1>
static cudaError_t launch_fine(const FineArgs<S, To>& a, cudaStream_t st) {
  typedef typename Cv<S>::C C;
  constexpr int LP = L1 > 0 ? L1 : 1;
  constexpr bool HWW = OP == F_SMOOTH && (VAR & 4);
  typedef FLay<S, OP, LP, HWW> LY;
  const Geom& g = a.g;
  TMaps tm;
  cudaError_t e;
  const int es = (int)sizeof(S);
  const S* vb = a.v ? a.v + g.base : nullptr;
  if ((e = get_map(&tm.v, vb, DT<S>::v, es, g.P, g.RYn, g.nz + 2, Halo<S>::W, g.TY + 3)) != cudaSuccess) return e;
  if ((e = get_map(&tm.k, a.kap + g.base, DT<S>::v, es, g.P, g.RYe, g.Nz + 2, Halo<S>::W, g.TY + 2)) != cudaSuccess)
    return e;
  if ((e = get_map(&tm.m, a.mask, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, g.mwr, g.RYn, g.nz + 2, MBW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  const S* rb = (OP != F_APPLY && a.r) ? a.r + g.base : nullptr;
  if ((e = get_map(&tm.r, rb, DT<S>::v, es, g.P, g.RYn, g.nz + 2, CWD, g.TY + 1)) != cudaSuccess) return e;
  const S* wb = (HWW && a.w) ? a.w + g.base : nullptr;
  if ((e = get_map(&tm.w, wb, DT<S>::v, es, g.P, g.RYn, g.nz + 2, CWD, g.TY + 1)) != cudaSuccess) return e;
  const C* pb = (OP == F_RESTRICT && a.phi) ? a.phi + g.base * LP : nullptr;
  if ((e = get_map(&tm.p, pb, DT<C>::v, (int)sizeof(C), g.P * LP, g.RYn, g.nz + 2, PhiBox<C, LP>::PW, g.TY + 1)) !=
      cudaSuccess)
    return e;
  auto k = a.g.cube ? fine_tile<S, To, OP, true, L1, DOT, MASKIN, VAR> : fine_tile<S, To, OP, false, L1, DOT, MASKIN, VAR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
  note_launch(), k<<<fine_grid(a.g), FNT, LY::SMEM, st>>>(a, tm);
  return cudaGetLastError();
}

unsigned fine_num_ctas(const Geom& g) {
  dim3 d = fine_grid(g);
  return d.x * d.y * d.z;
}

template <class S, class To>
static FineArgs<S, To> fargs(const Geom& g, const uint32_t* mask, const S* kap) {
  FineArgs<S, To> a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.mask = mask;
  a.kap = kap;
  for (int i = 0; i < 8; ++i) a.cc[i] = (typename Cv<S>::C)g.c[i];
  return a;
}

// y = A u (FP64), optionally dot = u . y (deterministic).  mask_input: treat
// the input as arbitrary on Gamma_D (zero it on load); otherwise the caller
// guarantees u = 0 there (Krylov directions).
cudaError_t fine_apply_f64(const Geom& g, const uint32_t* mask, const double* kap, const double* u, double* y,
                           double* partial, unsigned* counter, double* dot, cudaStream_t st, bool mask_input) {
  auto a = fargs<double, double>(g, mask, kap);
  a.v = u;
  a.out = y;
  if (mask_input) return launch_fine<double, double, F_APPLY, 0, false, true>(a, st);
  if (dot) {
    a.partial = partial;
    a.counter = counter;
    a.dot = dot;
    return launch_fine<double, double, F_APPLY, 0, true>(a, st);
  }
  return launch_fine<double, double, F_APPLY, 0, false>(a, st);
}

template <class S>
cudaError_t fine_apply_lp(const Geom& g, const uint32_t* mask, const S* kap, const S* u, S* y, cudaStream_t st,
                          bool mask_input) {
  if constexpr (sizeof(S) == 4) {
    if (!mask_input && fine3_supported(g)) return fine3_apply(g, mask, kap, u, y, st);
  }
  if (!mask_input && fine2_supported(g)) return fine2_apply<S>(g, mask, kap, u, y, st);
  auto a = fargs<S, S>(g, mask, kap);
  a.v = u;
  a.out = y;
  if (mask_input) return launch_fine<S, S, F_APPLY, 0, false, true>(a, st);
  return launch_fine<S, S, F_APPLY, 0, false>(a, st);
}
template cudaError_t fine_apply_lp<float>(const Geom&, const uint32_t*, const float*, const float*, float*, cudaStream_t,
                                          bool);
template cudaError_t fine_apply_lp<bf16>(const Geom&, const uint32_t*, const bf16*, const bf16*, bf16*, cudaStream_t,
                                         bool);

#define L1_DISPATCH(L1rt, CALL)                                  \
  switch (L1rt) {                                                \
    case 1: { constexpr int LL = 1; CALL; } break;               \
    case 2: { constexpr int LL = 2; CALL; } break;               \
    case 3: { constexpr int LL = 3; CALL; } break;               \
    case 4: { constexpr int LL = 4; CALL; } break;               \
    case 5: { constexpr int LL = 5; CALL; } break;               \
    case 6: { constexpr int LL = 6; CALL; } break;               \
    case 8: { constexpr int LL = 8; CALL; } break;               \
    default: return cudaErrorInvalidValue;                       \
  }

// FP32/BF16 sweeps on grids the two-nodes-per-lane engine covers (fine2.cu)
template <class S, class To>
static cudaError_t fine2_smooth_dispatch(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e,
                                         const S* w, To* out, float cA, float cB, cudaStream_t st) {
  if constexpr (sizeof(S) == 8) {
    return cudaErrorInvalidValue;
  } else {
    if constexpr (sizeof(S) == 4 && sizeof(To) == 4) {
      if (fine3_supported(g)) return fine3_smooth<To>(g, mask, kap, r, e, w, out, cA, cB, st);
    }
    return fine2_smooth<S, To>(g, mask, kap, r, e, w, out, cA, cB, st);
  }
}

// One sweep e' = e + cA (e - w) + cB D^-1 (r - A e); e == nullptr: e' = cB D^-1 r.
template <class S, class To>
cudaError_t fine_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e, const S* w,
                        To* out, typename Cv<S>::C cA, typename Cv<S>::C cB, cudaStream_t st) {
  if (sizeof(S) < 8 && (fine2_supported(g) || (sizeof(S) == 4 && fine3_supported(g))))
    return fine2_smooth_dispatch(g, mask, kap, r, e, w, out, (float)cA, (float)cB, st);
  auto a = fargs<S, To>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.w = (e != nullptr) ? w : nullptr;
  a.out = out;
  a.cA = cA;
  a.omega = cB;
  if (e == nullptr) return launch_fine<S, To, F_SMOOTH, 0, false, false, 0>(a, st);
  if (cA == typename Cv<S>::C(0)) return launch_fine<S, To, F_SMOOTH, 0, false, false, 1>(a, st);
  if (w == nullptr) return launch_fine<S, To, F_SMOOTH, 0, false, false, 3>(a, st);
  return launch_fine<S, To, F_SMOOTH, 0, false, false, 7>(a, st);
}

template <class S>
cudaError_t fine_restrict(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e,
                          const typename Cv<S>::C* phi, typename Cv<S>::C* rc, int L1, cudaStream_t st) {
  auto a = fargs<S, S>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.phi = phi;
  a.rc = rc;
  L1_DISPATCH(L1, return (launch_fine<S, S, F_RESTRICT, LL, false>(a, st)));
  return cudaSuccess;
}

// e += Phi ec (level-1 prolongation, in place)
template <class S>
cudaError_t fine_prolong(const Geom& g, const typename Cv<S>::C* phi, const typename Cv<S>::C* ec, S* e, int L1,
                         cudaStream_t st) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  L1_DISPATCH(L1, (note_launch(), k_prolong<S, LL><<<(unsigned)nb, 256, 0, st>>>(g, phi, ec, e)));
  return cudaGetLastError();
}

#define INST_FINE(S, To)                                                                                        \
  template cudaError_t fine_smooth<S, To>(const Geom&, const uint32_t*, const S*, const S*, const S*, const S*, \
                                          To*, Cv<S>::C, Cv<S>::C, cudaStream_t);
INST_FINE(double, double)
INST_FINE(float, float)
INST_FINE(bf16, bf16)
INST_FINE(bf16, float)
template cudaError_t fine_restrict<double>(const Geom&, const uint32_t*, const double*, const double*,
                                           const double*, const double*, double*, int, cudaStream_t);
template cudaError_t fine_restrict<float>(const Geom&, const uint32_t*, const float*, const float*, const float*,
                                          const float*, float*, int, cudaStream_t);
template cudaError_t fine_restrict<bf16>(const Geom&, const uint32_t*, const bf16*, const bf16*, const bf16*,
                                         const float*, float*, int, cudaStream_t);
template cudaError_t fine_prolong<double>(const Geom&, const double*, const double*, double*, int, cudaStream_t);
template cudaError_t fine_prolong<float>(const Geom&, const float*, const float*, float*, int, cudaStream_t);
template cudaError_t fine_prolong<bf16>(const Geom&, const float*, const float*, bf16*, int, cudaStream_t);

}  // namespace thermo

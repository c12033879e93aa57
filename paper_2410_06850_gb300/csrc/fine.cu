// Fine-grid kernels: matrix-free Q1 operator and the fine part of the
// multigrid cycle (Sec. 3, Algorithm 1).
//
// One z-marching tile engine serves every fine-grid pass.  A CTA owns a
// TX x TY tile of nodes (block-aligned; the tile on the high face of an axis
// also owns the closing node plane) and marches over ZC node planes.  Per
// plane it stages the next node plane of the input field (with a one-node
// halo) and the next element plane of conductivity in shared memory (double
// buffered, one barrier per plane); each thread keeps its 3x3 column of the
// two previous node planes and 2x2 conductivities of the previous element
// plane in registers, so a node costs 9 + 4 shared loads.
//
// Operator (node-centred gather of A = sum_e kappa_e K0_e, K0[a][b] =
// c[a ^ b]): with the 8 elements around node i indexed (dx,dy,dz),
//   (A v)_i = c0 K8 v_i + c3 sum_xy zp v + c5 sum_xz yp v + c6 sum_yz xp v
//           + c7 sum_diag kappa v  [+ c1/c2/c4 axis terms, non-cubic boxes]
// where K8 is the sum of the 8 conductivities and zp/yp/xp are sums of the
// two elements sharing an edge (Sec. 2.2 Eq. (5) realised for Q1).
// Dirichlet nodes: inputs are masked to zero on load (no coupling to
// Gamma_D columns) and the row is the identity.
#include "common.cuh"
#include "kernels.h"

namespace thermo {

enum FineOp { F_APPLY = 0, F_SMOOTH = 1, F_DIAG = 2, F_RESTRICT = 3, F_PSMOOTH = 4 };

constexpr int FINE_NT = 320;  // >= (TX+1)(TY+1) = 297 for 32 x 8 tiles

template <class S, class To>
struct FineArgs {
  typedef typename Cv<S>::C C;
  Geom g;
  const S* kap;
  const S* v;       // APPLY: u; SMOOTH/RESTRICT: e; PSMOOTH: e before prolongation
  const S* r;       // smoother right-hand side / residual source
  To* out;
  const uint32_t* mask;
  const C* phi;     // level-1 basis [nsize][L1]
  const C* ec;      // level-1 correction [cells][L1]
  C* rc;            // level-1 restricted residual [cells][L1]
  C omega;
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

template <class S, class To, int OP, bool CUBE, int L1, bool DOT>
__global__ void __launch_bounds__(FINE_NT) fine_tile(FineArgs<S, To> a) {
  typedef typename Cv<S>::C C;
  const Geom& g = a.g;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = g.TX, TY = g.TY;
  const int VW = TX + 3, VH = TY + 3, KW = TX + 2, KH = TY + 2;
  C* vbuf = reinterpret_cast<C*>(smem_raw);
  C* kbuf = vbuf + 2 * VW * VH;
  C* red = kbuf + 2 * KW * KH;  // RESTRICT scratch [(TX+1)(TY+1)][L1]
  __shared__ double dsh[32];
  __shared__ C cc[8];
  const int tid = threadIdx.x;
  if (tid < 8) cc[tid] = (C)g.c[tid];
  const int tx = tid % (TX + 1), ty = tid / (TX + 1);
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool lastx = (x0 + TX == g.Nx), lasty = (y0 + TY == g.Ny);
  const int zs = blockIdx.z * g.ZC;
  const int ze = (zs + g.ZC == g.Nz) ? g.Nz : zs + g.ZC - 1;
  const int x = x0 + tx, y = y0 + ty;
  const bool mapped = ty <= TY;
  const bool active = mapped && (tx < TX || lastx) && (ty < TY || lasty);
  const int rtx = mapped ? tx : 0, rty = mapped ? ty : 0;  // safe smem read coords

  C vm[3][3], v0[3][3], vp[3][3], km[2][2], kp[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) vm[i][j] = v0[i][j] = vp[i][j] = C(0);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) km[i][j] = kp[i][j] = C(0);

  C acc[L1 > 0 ? L1 : 1];
#pragma unroll
  for (int j = 0; j < (L1 > 0 ? L1 : 1); ++j) acc[j] = C(0);
  double dacc = 0.0;

  for (int t = zs - 2; t <= ze; ++t) {
    const int buf = t & 1;
    C* vb = vbuf + buf * VW * VH;
    C* kb = kbuf + buf * KW * KH;
    if (OP != F_DIAG) {
      const int zz = t + 1;
      for (int i = tid; i < VW * VH; i += FINE_NT) {
        const int lx = i % VW, ly = i / VW;
        const int xx = x0 - 1 + lx, yy = y0 - 1 + ly;
        const long long n = nidx(g, xx, yy, zz);
        C val = Cv<S>::ld(a.v + n);
        if (OP == F_PSMOOTH && L1 > 0) {
          if (xx >= 0 && yy >= 0 && zz >= 0 && xx <= g.Nx && yy <= g.Ny && zz <= g.Nz) {
            const long long cell =
                blk_of(xx, g.b, g.nbx) + (long long)g.nbx * (blk_of(yy, g.b, g.nby) + (long long)g.nby * blk_of(zz, g.b, g.nbz));
#pragma unroll
            for (int j = 0; j < (L1 > 0 ? L1 : 1); ++j) val += a.phi[n * L1 + j] * a.ec[cell * L1 + j];
          }
        }
        if (is_dir(g, a.mask, xx, yy, zz)) val = C(0);
        vb[i] = val;
      }
    }
    if (t >= zs - 1) {
      for (int i = tid; i < KW * KH; i += FINE_NT) {
        const int lx = i % KW, ly = i / KW;
        kb[i] = Cv<S>::ld(a.kap + eidx(g, x0 - 1 + lx, y0 - 1 + ly, t));
      }
    }
    __syncthreads();
    if (OP != F_DIAG) {
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) vp[oy][ox] = vb[(rty + oy) * VW + rtx + ox];
    }
    if (t >= zs - 1) {
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) kp[dy][dx] = kb[(rty + dy) * KW + rtx + dx];
    }
    if (t >= zs && active) {
      C K8;
      const C Av = stencil<C, CUBE>(vm, v0, vp, km, kp, cc, K8);
      const long long n = nidx(g, x, y, t);
      const bool dir = is_dir(g, a.mask, x, y, t);
      if (OP == F_APPLY) {
        C yv = Av;
        if (dir) yv = Cv<S>::ld(a.v + n);
        Cv<To>::st(a.out + n, yv);
        if (DOT) dacc += (double)v0[1][1] * (double)yv;
      } else if (OP == F_SMOOTH || OP == F_PSMOOTH) {
        const C rr = Cv<S>::ld(a.r + n);
        C e = v0[1][1] + a.omega * (rr - Av) / (cc[0] * K8);
        if (dir) e = C(0);
        Cv<To>::st(a.out + n, e);
      } else if (OP == F_DIAG) {
        const C rr = Cv<S>::ld(a.r + n);
        C e = a.omega * rr / (cc[0] * K8);
        if (dir) e = C(0);
        Cv<To>::st(a.out + n, e);
      } else if (OP == F_RESTRICT) {
        const C rr = Cv<S>::ld(a.r + n);
        const C s = dir ? C(0) : rr - Av;
#pragma unroll
        for (int j = 0; j < (L1 > 0 ? L1 : 1); ++j) acc[j] += s * a.phi[n * L1 + j];
      }
    }
    if (OP == F_RESTRICT && L1 > 0 && t >= zs) {
      const int bz = blk_of(t, g.b, g.nbz);
      const int zend = (bz == g.nbz - 1) ? g.Nz : bz * g.b + g.b - 1;
      if (t == zend) {  // uniform across the CTA
        if (mapped) {
#pragma unroll
          for (int j = 0; j < L1; ++j) red[(ty * (TX + 1) + tx) * L1 + j] = active ? acc[j] : C(0);
        }
        __syncthreads();
        const int nlx = TX / g.b, nly = TY / g.b;
        for (int o = tid; o < nlx * nly * L1; o += FINE_NT) {
          const int j = o % L1, lb = o / L1, lbx = lb % nlx, lby = lb / nlx;
          const int xa = lbx * g.b, xb = (lbx == nlx - 1 && lastx) ? TX + 1 : xa + g.b;
          const int ya = lby * g.b, yb = (lby == nly - 1 && lasty) ? TY + 1 : ya + g.b;
          C s = C(0);
          for (int yy = ya; yy < yb; ++yy)
            for (int xx = xa; xx < xb; ++xx) s += red[(yy * (TX + 1) + xx) * L1 + j];
          const long long cell = (x0 / g.b + lbx) + (long long)g.nbx * ((y0 / g.b + lby) + (long long)g.nby * bz);
          a.rc[cell * L1 + j] = s;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < L1; ++j) acc[j] = C(0);
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        vm[i][j] = v0[i][j];
        v0[i][j] = vp[i][j];
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) km[i][j] = kp[i][j];
  }

  if (DOT) {
    const double s = block_sum<FINE_NT>(dacc, dsh);
    __shared__ bool last;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
      a.partial[bid] = s;
      __threadfence();
      const unsigned prev = atomicAdd(a.counter, 1u);
      last = (prev == nblk - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double v = 0.0;
      for (unsigned i = tid; i < nblk; i += FINE_NT) v += __ldcg(a.partial + i);
      v = block_sum<FINE_NT>(v, dsh);
      if (tid == 0) {
        *a.dot = v;
        *a.counter = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host launchers

static dim3 fine_grid(const Geom& g) { return dim3(g.Nx / g.TX, g.Ny / g.TY, g.Nz / g.ZC); }

template <class S>
static size_t fine_smem(const Geom& g, int L1) {
  typedef typename Cv<S>::C C;
  size_t n = 2 * (size_t)(g.TX + 3) * (g.TY + 3) + 2 * (size_t)(g.TX + 2) * (g.TY + 2) +
             (size_t)(g.TX + 1) * (g.TY + 1) * (L1 > 0 ? L1 : 0);
  return n * sizeof(C);
}

template <class S, class To, int OP, int L1, bool DOT>
static cudaError_t launch_fine(const FineArgs<S, To>& a, int L1rt, cudaStream_t st) {
  const size_t sm = fine_smem<S>(a.g, OP == F_RESTRICT ? L1rt : 0);
  if (a.g.cube) {
    auto k = fine_tile<S, To, OP, true, L1, DOT>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launch(), k<<<fine_grid(a.g), FINE_NT, sm, st>>>(a);
  } else {
    auto k = fine_tile<S, To, OP, false, L1, DOT>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launch(), k<<<fine_grid(a.g), FINE_NT, sm, st>>>(a);
  }
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
  return a;
}

// y = A u (FP64), optionally dot = u . y (deterministic)
cudaError_t fine_apply_f64(const Geom& g, const uint32_t* mask, const double* kap, const double* u, double* y,
                           double* partial, unsigned* counter, double* dot, cudaStream_t st) {
  auto a = fargs<double, double>(g, mask, kap);
  a.v = u;
  a.out = y;
  if (dot) {
    a.partial = partial;
    a.counter = counter;
    a.dot = dot;
    return launch_fine<double, double, F_APPLY, 0, true>(a, 0, st);
  }
  return launch_fine<double, double, F_APPLY, 0, false>(a, 0, st);
}

template <class S>
cudaError_t fine_apply_lp(const Geom& g, const uint32_t* mask, const S* kap, const S* u, S* y, cudaStream_t st) {
  auto a = fargs<S, S>(g, mask, kap);
  a.v = u;
  a.out = y;
  return launch_fine<S, S, F_APPLY, 0, false>(a, 0, st);
}
template cudaError_t fine_apply_lp<float>(const Geom&, const uint32_t*, const float*, const float*, float*, cudaStream_t);
template cudaError_t fine_apply_lp<bf16>(const Geom&, const uint32_t*, const bf16*, const bf16*, bf16*, cudaStream_t);

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

// Fine part of the cycle, storage S (double / float / bf16), compute C.
template <class S, class To>
cudaError_t fine_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e, To* out,
                        typename Cv<S>::C omega, cudaStream_t st) {
  auto a = fargs<S, To>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.out = out;
  a.omega = omega;
  if (e == nullptr) return launch_fine<S, To, F_DIAG, 0, false>(a, 0, st);
  return launch_fine<S, To, F_SMOOTH, 0, false>(a, 0, st);
}

template <class S>
cudaError_t fine_restrict(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e,
                          const typename Cv<S>::C* phi, typename Cv<S>::C* rc, int L1, cudaStream_t st) {
  auto a = fargs<S, S>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.phi = phi;
  a.rc = rc;
  L1_DISPATCH(L1, return (launch_fine<S, S, F_RESTRICT, LL, false>(a, LL, st)));
  return cudaSuccess;
}

template <class S, class To>
cudaError_t fine_prolong_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e,
                                const typename Cv<S>::C* phi, const typename Cv<S>::C* ec, To* out,
                                typename Cv<S>::C omega, int L1, cudaStream_t st) {
  auto a = fargs<S, To>(g, mask, kap);
  a.r = r;
  a.v = e;
  a.phi = phi;
  a.ec = ec;
  a.out = out;
  a.omega = omega;
  L1_DISPATCH(L1, return (launch_fine<S, To, F_PSMOOTH, LL, false>(a, LL, st)));
  return cudaSuccess;
}

#define INST_FINE(S, To)                                                                                       \
  template cudaError_t fine_smooth<S, To>(const Geom&, const uint32_t*, const S*, const S*, const S*, To*,   \
                                          Cv<S>::C, cudaStream_t);                                           \
  template cudaError_t fine_prolong_smooth<S, To>(const Geom&, const uint32_t*, const S*, const S*, const S*, \
                                                  const Cv<S>::C*, const Cv<S>::C*, To*, Cv<S>::C, int,      \
                                                  cudaStream_t);
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

}  // namespace thermo

// Host orchestration and the C ABI of libthermo (see include/thermo.h).
//
// The context owns every device buffer in the padded layout of common.cuh.
// Solve = FP64 (flexible) preconditioned CG (Sec. 4) around the multigrid
// cycle of Algorithm 1 (Sec. 3), generalised to the context's number of
// levels; all per-iteration work runs in this library's kernels, with one
// host readback of the device scalars per convergence check.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/thermo.h"
#include "common.cuh"
#include "kernels.h"
#include "chebyshev.h"
#include "tma.cuh"

using namespace thermo;

namespace thermo {
static long long g_launches = 0;
void note_launch() { ++g_launches; }
long long launch_count() { return g_launches; }
}  // namespace thermo

namespace {

struct Lev {
  CLevel cl;
  double* T64 = nullptr;   // Galerkin tiles [ncell][27][L][L]
  float* T32 = nullptr;
  double* Di64 = nullptr;  // l1 block inverses [ncell][L][L]
  float* Di32 = nullptr;
  double* Psi64 = nullptr; // (l >= 2) [ncell][g^3 Lprev][L]
  float* Psi32 = nullptr;
  uint8_t* act = nullptr;
  double* eig = nullptr;
  double* Dc = nullptr;    // row-sum corrections for later levels [nt][ncell][L][L]
  int ntc = 0;
  // cycle vectors (FP64 form and FP32 form)
  double *r64 = nullptr, *e64 = nullptr, *t64 = nullptr, *s64 = nullptr;
  float *r32 = nullptr, *e32 = nullptr, *t32 = nullptr, *s32 = nullptr;
};

}  // namespace

// event-pair timer of one kernel class (see thermo_kernel_timers)
struct KTimer {
  static const int CAP = 4096;
  std::vector<cudaEvent_t> ev;  // 2 * CAP events, created on enable
  int used = 0;                 // pairs recorded in the current solve
  double ms = 0.0, bytes = 0.0, flops = 0.0, pend_bytes = 0.0, pend_flops = 0.0;
  long long launches = 0;
};

struct thermo_ctx {
  std::string err;
  std::vector<double> hist;  // relative recursive residual at each check of the last solve
  bool kt_on = false;
  KTimer kt[THERMO_KT_COUNT];
  double coarse_bytes = 0.0;  // algorithmic bytes of the coarse launches of the current cycle (timers on)
  cudaStream_t st = nullptr;
  thermo_options opt;
  Geom g;
  int L1 = 4;
  double h[3] = {1.0, 1.0, 1.0};  // element edges
  long long nnode = 0, nelem = 0;
  std::vector<void*> allocs;
  bool dry = false;          // allocation plan only: count bytes, allocate nothing
  long long plan_bytes = 0;
  bool lean = false;         // FP32-only hierarchy (opt.lean)
  double* slab64 = nullptr;  // u, r, p, q (lean: also the FP64 set-up intermediates)
  float* slab32 = nullptr;   // r32, z32, ea32, eb32, ec32, tmp32 (lean: also the row-sum corrections)
  long long slab64_n = 0, slab32_n = 0;  // elements
  // fine data
  uint32_t* bits = nullptr;
  double* k64 = nullptr;
  float* k32 = nullptr;
  bf16* k16 = nullptr;
  float* klo = nullptr;  // kappa - (double)k32: with k32 a float-float copy of k64
  double* xd = nullptr;     // design copy (natural; FP64 input)
  float* xf = nullptr;      // design copy (natural; FP32 input, opt.density_fp32)
  double *f = nullptr, *blift = nullptr, *TD = nullptr, *zero64 = nullptr;
  double *u = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *bv = nullptr, *tmp = nullptr, *z64 = nullptr;
  double *ea64 = nullptr, *eb64 = nullptr, *ec64 = nullptr;
  float *r32 = nullptr, *z32 = nullptr, *ea32 = nullptr, *eb32 = nullptr, *ec32 = nullptr, *tmp32 = nullptr;
  bf16 *r16 = nullptr, *ea16 = nullptr, *eb16 = nullptr, *ec16 = nullptr;
  // fine smoother coefficients: e' = e + sa[k] (e - e_prev) + sb[k] D^-1 (r - A e), k < nsweep
  int nsweep = 2;
  double sa[64], sb[64];
  double lmax = 0.0;
  double* phi64 = nullptr;
  float* phi32 = nullptr;
  // levels 1..nlev (index 0 unused)
  int nlev = 0;
  Lev lev[THERMO_MAX_LEVELS + 1];
  double* Ainv = nullptr;
  double* cholA = nullptr;
  double* cholW = nullptr;     // scratch of the blocked factorisation / inverse
  int ncoarse = 0;
  int* gcum_dev = nullptr;
  // scalars and reductions
  CgScalars* sc = nullptr;
  CgScalars* sc_h = nullptr;  // pinned
  Reducer red;
  int* status_dev = nullptr;
  int* status_h = nullptr;     // pinned
  double* dscal = nullptr;     // device scratch scalars [16]
  double* dscal_h = nullptr;   // pinned
  bool have_density = false, have_precond = false;
  double sp = 3, skmin = 1e-3, skmax = 1;
  double t_setup_ms = 0.0;
  int ndir = 0;
  double* colsum = nullptr;    // filter column sums (OC)
  double* xnew = nullptr;
  double rmin_cs = -1.0;
};

static thermo_status fail(thermo_ctx* c, thermo_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}
#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, THERMO_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                        \
  } while (0)

template <class T>
static cudaError_t dalloc(thermo_ctx* ctx, T** p, size_t n) {
  if (ctx->dry) {
    ctx->plan_bytes += (long long)((n * sizeof(T) + 64 + 511) & ~(size_t)511);
    *p = nullptr;
    return cudaSuccess;
  }
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, n * sizeof(T) + 64);
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(v);
  e = cudaMemsetAsync(v, 0, n * sizeof(T) + 64, ctx->st);
  *p = (T*)v;
  return e;
}

// The context's stage time-out word is nonzero when one of its TMA-staged fine
// kernels gave up waiting for a plane since the last check: that launch's
// results are invalid.  Reads and resets the word (synchronises the stream).
static thermo_status stage_check(thermo_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->status_h + 4, ctx->g.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->status_h[4] == 0) return THERMO_OK;
  CK(cudaMemsetAsync(ctx->g.err, 0, sizeof(int), ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return fail(ctx, THERMO_ECUDA, "a fine-grid kernel gave up waiting for a TMA stage (its results are invalid)");
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
extern "C" thermo_status thermo_default_options(const int grid[3], thermo_options* opt) {
  if (!grid || !opt) return THERMO_EINVAL;
  memset(opt, 0, sizeof(*opt));
  for (int k = 0; k < 3; ++k)
    if (grid[k] <= 0 || grid[k] % 4) return THERMO_EINVAL;
  int m = grid[0] / 4;
  for (int k = 1; k < 3; ++k) m = grid[k] / 4 < m ? grid[k] / 4 : m;
  int lv = 1;
  std::vector<int> groups;
  // coarsest level: 4^3 cells (1,088 unknowns) up to 32^3 level-1 cells; above
  // that 8^3 cells (8,704 unknowns), the exact coarse-coarse solve that keeps the
  // iteration count flat in the contrast
  const int stop = m > 32 ? 8 : 4;
  while (m > stop && m % 2 == 0 && lv < THERMO_MAX_LEVELS) {
    m /= 2;
    ++lv;
  }
  opt->levels = lv;
  opt->block = 4;
  opt->nvec[0] = 4;
  for (int l = 1; l < lv; ++l) {
    opt->group[l] = 2;
    opt->nvec[l] = (l == 1 && lv > 2) ? 8 : 17;
  }
  opt->nu_fine = 2;
  opt->nu_coarse = 1;
  opt->omega = 2.0 / 3.0;
  opt->prec = THERMO_MIXED;
  opt->pc = THERMO_PC_MMG;
  opt->guess = THERMO_GUESS_COARSE;
  opt->max_iter = 10000;
  opt->flexible = -1;
  opt->check_every = 1;
  opt->smoother = 1;
  opt->cheb_degree = 5;
  opt->cheb_ratio = 30.0;
  opt->power_iters = 15;
  opt->outer_apply = 0;
  opt->nu_growth = 2;
  opt->w_from = 3;
  opt->restart_decades = 0;
  return THERMO_OK;
}

static int pick_tile(int N, int b, int maxt) {
  for (int t = maxt - maxt % b; t >= b; t -= b)
    if (N % t == 0) return t;
  return 0;
}

// Validation, geometry, hierarchy shape and every device buffer of a context
// whose options are set.  With ctx->dry, buffers are only counted
// (ctx->plan_bytes) and nothing touches a GPU.
static thermo_status build_context(thermo_ctx* ctx, const int grid[3], const double h[3], bool has_dval) {
  const thermo_options& opt = ctx->opt;
  for (int k = 0; k < 3; ++k) {
    if (grid[k] <= 0 || !(h[k] > 0.0)) return fail(ctx, THERMO_EINVAL, "grid and h must be positive");
  }
  const int b = opt.block;
  if (b != 4) return fail(ctx, THERMO_EINVAL, "block must be 4 (fine kernels assign one block row per warp)");
  if (opt.levels < 1 || opt.levels > THERMO_MAX_LEVELS) return fail(ctx, THERMO_EINVAL, "levels out of range");
  if (grid[0] % b || grid[1] % b || grid[2] % b) return fail(ctx, THERMO_EINVAL, "grid must be a multiple of block");
  if (opt.nu_fine < 1 || opt.nu_coarse < 1 || opt.nu_fine > 64) return fail(ctx, THERMO_EINVAL, "smoothing sweeps must be in [1, 64]");
  if (opt.smoother != 0 && opt.smoother != 1) return fail(ctx, THERMO_EINVAL, "smoother must be 0 (Jacobi) or 1 (Chebyshev)");
  if (opt.flexible < -1 || opt.flexible > 2) return fail(ctx, THERMO_EINVAL, "flexible must be -1, 0, 1 or 2");
  if (opt.nu_growth < 1 || opt.nu_growth > 8) return fail(ctx, THERMO_EINVAL, "nu_growth must be in 1..8");
  if (opt.w_from < 0) return fail(ctx, THERMO_EINVAL, "w_from must be >= 0");
  if (!(opt.restart_decades >= 0.0)) return fail(ctx, THERMO_EINVAL, "restart_decades must be >= 0");
  if (opt.outer_apply < 0 || opt.outer_apply > 2) return fail(ctx, THERMO_EINVAL, "outer_apply must be 0, 1 or 2");
  if (opt.smoother == 1 && (opt.cheb_degree < 1 || opt.cheb_degree > 64 || !(opt.cheb_ratio > 1.0) || opt.power_iters < 1))
    return fail(ctx, THERMO_EINVAL, "Chebyshev needs 1 <= degree <= 64, ratio > 1, power_iters >= 1");
  if (opt.nvec[0] < 1 || opt.nvec[0] > 6) return fail(ctx, THERMO_EINVAL, "nvec[0] must be in 1..6");
  if (opt.density_fp32 != 0 && opt.density_fp32 != 1) return fail(ctx, THERMO_EINVAL, "density_fp32 must be 0 or 1");
  if (opt.fine_engine != 0 && opt.fine_engine != 1) return fail(ctx, THERMO_EINVAL, "fine_engine must be 0 or 1");
  if (!(opt.eig_threshold >= 0.0) || !std::isfinite(opt.eig_threshold))
    return fail(ctx, THERMO_EINVAL, "eig_threshold must be finite and >= 0");
  for (int k = 0; k < 3; ++k) ctx->h[k] = h[k];
  Geom& g = ctx->g;
  memset(&g, 0, sizeof(g));
  g.Nx = grid[0];
  g.Ny = grid[1];
  g.Nz = grid[2];
  g.nx = g.Nx + 1;
  g.ny = g.Ny + 1;
  g.nz = g.Nz + 1;
  g.P = ((g.Nx + 3 + 31) / 32) * 32;
  g.RYn = g.Ny + 3;
  g.RYe = g.Ny + 2;
  g.base = 32;
  g.nsize = g.base + (long long)(g.nz + 2) * g.RYn * g.P + 64;
  g.esize = g.base + (long long)(g.Nz + 2) * g.RYe * g.P + 64;
  g.mwr = ((g.P / 32 + 3) / 4) * 4;  // mask rows padded to 16 bytes (TMA row stride)
  g.msize = (long long)(g.nz + 2) * g.RYn * g.mwr + 8;
  {
    // K0[a][b] = c[a ^ b] from the Kronecker form (k (x) m (x) m etc.)
    const double hx = h[0], hy = h[1], hz = h[2];
    const double ax = hy * hz / hx, ay = hx * hz / hy, az = hx * hy / hz;
    for (int pat = 0; pat < 8; ++pat) {
      const int px = pat & 1, py = (pat >> 1) & 1, pz = (pat >> 2) & 1;
      auto k1 = [](int d) { return d ? -1.0 : 1.0; };
      auto m1 = [](int d) { return d ? 1.0 / 6.0 : 1.0 / 3.0; };
      g.c[pat] = ax * k1(px) * m1(py) * m1(pz) + ay * m1(px) * k1(py) * m1(pz) + az * m1(px) * m1(py) * k1(pz);
    }
    g.cube = (fabs(g.c[1]) <= 1e-14 * fabs(g.c[0]) && fabs(g.c[2]) <= 1e-14 * fabs(g.c[0]) &&
              fabs(g.c[4]) <= 1e-14 * fabs(g.c[0]) && fabs(g.c[3] - g.c[7]) <= 1e-14 * fabs(g.c[0]) &&
              fabs(g.c[5] - g.c[7]) <= 1e-14 * fabs(g.c[0]) && fabs(g.c[6] - g.c[7]) <= 1e-14 * fabs(g.c[0]))
                 ? 1
                 : 0;
    if (g.cube) {
      g.c[1] = g.c[2] = g.c[4] = 0.0;
      g.c[3] = g.c[5] = g.c[6] = g.c[7];
    }
    g.vol = hx * hy * hz;
  }
  g.b = b;
  g.nbx = g.Nx / b;
  g.nby = g.Ny / b;
  g.nbz = g.Nz / b;
  g.TX = (g.Nx % 32 == 0) ? 32 : (g.Nx % 16 == 0 ? 16 : (g.Nx % 8 == 0 ? 8 : 0));
  g.TY = pick_tile(g.Ny, b, 8);
  g.ZC = 0;
  if (g.TX && g.TY) {
    // planes per CTA: the largest chunk that still gives >= 8 CTAs per SM
    const long long cols = (long long)(g.Nx / g.TX) * (g.Ny / g.TY);
    for (int zc : {32, 16, 8, 4}) {
      if (g.Nz % zc) continue;
      if (!g.ZC) g.ZC = zc;
      if (cols * (g.Nz / zc) >= 152LL * 8) {
        g.ZC = zc;
        break;
      }
      g.ZC = zc;
    }
  }
  if (!g.TX || !g.TY || !g.ZC) return fail(ctx, THERMO_EINVAL, "unsupported grid / block combination");
  g.NZ2 = g.NZD = g.Nz / g.ZC;
  if (!ctx->dry) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
    if (sms > 0 && fine2_supported(g)) g.NZ2 = balanced_zchunks(fine2_tiles_xy(g), (long long)sms * fine2_ctas_per_sm(), g.Nz);
    g.NZ3 = 0;
    if (sms > 0 && g.cube && opt.fine_engine == 0) {
      const int per = fine3_ctas_per_sm();
      if (per > 0)
        g.NZ3 = balanced_zchunks((long long)fine3_tiles_x(g) * fine3_tiles_y(g), (long long)sms * per, g.Nz);
    }
    if (sms > 0 && fine_ds_supported(g))
      g.NZD = balanced_zchunks(fine_ds_tiles_xy(g), (long long)sms * fine_ds_ctas_per_sm(), g.Nz);
  }
  ctx->L1 = opt.nvec[0];
  ctx->nnode = (long long)g.nx * g.ny * g.nz;
  ctx->nelem = (long long)g.Nx * g.Ny * g.Nz;
  // hierarchy shape
  ctx->nlev = opt.levels;
  {
    int mx = g.nbx, my = g.nby, mz = g.nbz;
    for (int l = 1; l <= ctx->nlev; ++l) {
      CLevel& cl = ctx->lev[l].cl;
      if (l >= 2) {
        const int gg = opt.group[l - 1];
        if (gg < 1 || mx % gg || my % gg || mz % gg)
          return fail(ctx, THERMO_EINVAL, "level %d: cells not divisible by group %d", l, gg);
        mx /= gg;
        my /= gg;
        mz /= gg;
        cl.g = gg;
      } else {
        cl.g = 1;
      }
      cl.mx = mx;
      cl.my = my;
      cl.mz = mz;
      cl.L = opt.nvec[l - 1];
      cl.ncell = (long long)mx * my * mz;
      if (cl.L < 1 || cl.L > 32) return fail(ctx, THERMO_EINVAL, "nvec out of range at level %d", l);
      if (l >= 2) {
        const int n = cl.g * cl.g * cl.g * ctx->lev[l - 1].cl.L;
        if (n > 180) return fail(ctx, THERMO_EINVAL, "level %d local eigenproblem too large (%d > 180)", l, n);
      }
    }
    const CLevel& top = ctx->lev[ctx->nlev].cl;
    ctx->ncoarse = (int)(top.ncell * top.L);
    if (ctx->ncoarse > 20000) return fail(ctx, THERMO_EINVAL, "coarsest level too large (%d)", ctx->ncoarse);
  }
  // allocations
  const long long ns = g.nsize, es = g.esize;
  const long long nsa = (ns + 127) & ~63LL;  // slab stride: 64-element multiple, >= 64 elements of slack
  const bool fp64 = opt.prec == THERMO_FP64;
  if (opt.lean != 0 && opt.lean != 1) return fail(ctx, THERMO_EINVAL, "lean must be 0 or 1");
  if (opt.lean && (fp64 || opt.pc != THERMO_PC_MMG))
    return fail(ctx, THERMO_EINVAL, "lean needs a mixed-precision MMG context");
  ctx->lean = opt.lean != 0;
  const bool lean = ctx->lean;
  CK(dalloc(ctx, &ctx->g.err, 1));  // stage time-out word of this context's fine kernels
  ctx->g.wait = kStageWait;
  CK(dalloc(ctx, &ctx->bits, g.msize));
  CK(dalloc(ctx, &ctx->k64, es));
  CK(dalloc(ctx, &ctx->k32, es));
  if (opt.prec == THERMO_MIXED_BF16S) CK(dalloc(ctx, &ctx->k16, es));
  CK(dalloc(ctx, &ctx->klo, es));
  if (opt.density_fp32)
    CK(dalloc(ctx, &ctx->xf, ctx->nelem));
  else
    CK(dalloc(ctx, &ctx->xd, ctx->nelem));
  for (double** pp : {&ctx->f, &ctx->blift, &ctx->tmp}) CK(dalloc(ctx, pp, ns));
  // a solve's own right-hand side: the lean form shares tmp (no entry point that
  // uses tmp runs inside a solve)
  if (opt.lean)
    ctx->bv = ctx->tmp;
  else
    CK(dalloc(ctx, &ctx->bv, ns));
  if (has_dval) CK(dalloc(ctx, &ctx->TD, ns));
  if (!lean) CK(dalloc(ctx, &ctx->zero64, ns));
  if (fp64 || opt.pc != THERMO_PC_MMG) CK(dalloc(ctx, &ctx->z64, ns));
  if (fp64) {
    CK(dalloc(ctx, &ctx->ea64, ns));
    CK(dalloc(ctx, &ctx->eb64, ns));
    CK(dalloc(ctx, &ctx->ec64, ns));
  }
  // set-up intermediates that the lean form keeps in the slabs: FP64 Phi, each
  // level's FP64 Psi (one at a time), the row-sum corrections of all levels
  long long psi_max = 0, dc_total = 0;
  for (int l = 1; l <= ctx->nlev; ++l) {
    const CLevel& cl = ctx->lev[l].cl;
    if (l >= 2) {
      const long long np = cl.ncell * (long long)cl.g * cl.g * cl.g * ctx->lev[l - 1].cl.L * cl.L;
      psi_max = np > psi_max ? np : psi_max;
    }
    dc_total += (long long)(ctx->nlev - l) * cl.ncell * cl.L * cl.L;
  }
  {
    // u, r, p, q: one slab (lean: also FP64 Phi, then each level's FP64 Psi)
    long long n64 = 4 * nsa;
    if (lean) {
      n64 = std::max(n64, ns * ctx->L1);
      n64 = std::max(n64, psi_max);
    }
    CK(dalloc(ctx, &ctx->slab64, n64));
    ctx->slab64_n = n64;
    // r32, z32, ea32, eb32, ec32, tmp32: one slab (lean: also the row-sum corrections)
    long long n32 = 6 * nsa;
    const bool dc_in_slab = lean && 2 * dc_total <= n32;
    CK(dalloc(ctx, &ctx->slab32, n32));
    ctx->slab32_n = n32;
    if (!ctx->dry) {
      double* s64 = ctx->slab64;
      ctx->u = s64;
      ctx->r = s64 + nsa;
      ctx->p = s64 + 2 * nsa;
      ctx->q = s64 + 3 * nsa;
      float* s32 = ctx->slab32;
      float** v32[6] = {&ctx->r32, &ctx->z32, &ctx->ea32, &ctx->eb32, &ctx->ec32, &ctx->tmp32};
      for (int k = 0; k < 6; ++k) *v32[k] = s32 + k * nsa;
      if (lean) ctx->phi64 = s64;
      if (dc_in_slab) {
        double* d = reinterpret_cast<double*>(s32);
        for (int l = 1; l <= ctx->nlev; ++l) {
          Lev& lv = ctx->lev[l];
          lv.ntc = ctx->nlev - l;
          if (lv.ntc > 0) {
            lv.Dc = d;
            d += (long long)lv.ntc * lv.cl.ncell * lv.cl.L * lv.cl.L;
          }
          if (l >= 2) lv.Psi64 = s64;
        }
      } else if (lean) {
        for (int l = 2; l <= ctx->nlev; ++l) ctx->lev[l].Psi64 = s64;
      }
    }
    if (lean && !dc_in_slab)
      for (int l = 1; l < ctx->nlev; ++l) {
        Lev& lv = ctx->lev[l];
        lv.ntc = ctx->nlev - l;
        CK(dalloc(ctx, &lv.Dc, (long long)lv.ntc * lv.cl.ncell * lv.cl.L * lv.cl.L));
      }
  }
  if (opt.prec == THERMO_MIXED_BF16S) {
    for (bf16** pp : {&ctx->r16, &ctx->ea16, &ctx->eb16, &ctx->ec16}) CK(dalloc(ctx, pp, ns));
  }
  if (!lean) CK(dalloc(ctx, &ctx->phi64, ns * ctx->L1));
  CK(dalloc(ctx, &ctx->phi32, ns * ctx->L1));
  for (int l = 1; l <= ctx->nlev; ++l) {
    Lev& lv = ctx->lev[l];
    const CLevel& cl = lv.cl;
    const long long nd = cl.ncell * cl.L;
    const long long nt = cl.ncell * 27 * cl.L * cl.L;
    if (!lean || l == ctx->nlev) CK(dalloc(ctx, &lv.T64, nt));
    if (l < ctx->nlev) CK(dalloc(ctx, &lv.T32, nt));
    if (!lean) CK(dalloc(ctx, &lv.Di64, cl.ncell * cl.L * cl.L));
    CK(dalloc(ctx, &lv.Di32, cl.ncell * cl.L * cl.L));
    if (l >= 2) {
      const long long np = cl.ncell * (long long)cl.g * cl.g * cl.g * ctx->lev[l - 1].cl.L * cl.L;
      if (!lean) CK(dalloc(ctx, &lv.Psi64, np));
      CK(dalloc(ctx, &lv.Psi32, np));
    }
    CK(dalloc(ctx, &lv.act, nd));
    CK(dalloc(ctx, &lv.eig, nd));
    lv.ntc = ctx->nlev - l;
    if (!lean && lv.ntc > 0) CK(dalloc(ctx, &lv.Dc, (long long)lv.ntc * cl.ncell * cl.L * cl.L));
    if (!lean) {
      CK(dalloc(ctx, &lv.r64, nd));
      CK(dalloc(ctx, &lv.e64, nd));
    }
    if (fp64) {
      CK(dalloc(ctx, &lv.t64, nd));
      CK(dalloc(ctx, &lv.s64, nd));
    }
    for (float** pp : {&lv.r32, &lv.e32, &lv.t32, &lv.s32}) CK(dalloc(ctx, pp, nd));
  }
  CK(dalloc(ctx, &ctx->Ainv, (long long)ctx->ncoarse * ctx->ncoarse));
  CK(dalloc(ctx, &ctx->cholA, (long long)ctx->ncoarse * ctx->ncoarse));
  CK(dalloc(ctx, &ctx->cholW, cholesky_work_size(ctx->ncoarse)));
  {
    std::vector<int> gc(THERMO_MAX_LEVELS, 1);
    int acc = 1;
    for (int l = 2; l <= ctx->nlev; ++l) {
      acc *= ctx->lev[l].cl.g;
      gc[l - 2] = acc;
    }
    CK(dalloc(ctx, &ctx->gcum_dev, THERMO_MAX_LEVELS));
    if (!ctx->dry)
      CK(cudaMemcpyAsync(ctx->gcum_dev, gc.data(), THERMO_MAX_LEVELS * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  }
  CK(dalloc(ctx, &ctx->sc, 1));
  CK(dalloc(ctx, &ctx->dscal, 16));
  CK(dalloc(ctx, &ctx->status_dev, 4));
  {
    unsigned nf = fine_num_ctas(g);
    if (fine_ds_supported(g) && fine_ds_num_ctas(g) + 512 > nf) nf = fine_ds_num_ctas(g) + 512;
    const long long np = (long long)(nf > 8192 ? nf : 8192) * 2;
    CK(dalloc(ctx, &ctx->red.partial, np));
    CK(dalloc(ctx, &ctx->red.counter, 4));
    ctx->red.nblocks = (int)np;
  }
  if (ctx->dry) return THERMO_OK;
  CK(cudaMallocHost((void**)&ctx->sc_h, sizeof(CgScalars)));
  CK(cudaMallocHost((void**)&ctx->status_h, 8 * sizeof(int)));
  CK(cudaMallocHost((void**)&ctx->dscal_h, 16 * sizeof(double)));
  return THERMO_OK;
}

extern "C" thermo_status thermo_create(const int grid[3], const double h[3], const uint8_t* mask, const double* dval,
                                       const double* source, void* stream, const thermo_options* opt_in,
                                       thermo_ctx** out) {
  if (!out) return THERMO_EINVAL;
  *out = nullptr;
  if (!grid || !h || !mask || !source) return THERMO_EINVAL;
  thermo_options opt;
  if (opt_in)
    opt = *opt_in;
  else if (thermo_default_options(grid, &opt) != THERMO_OK)
    return THERMO_EINVAL;
  thermo_ctx* ctx = new (std::nothrow) thermo_ctx();
  if (!ctx) return THERMO_ENOMEM;
  *out = ctx;
  ctx->st = (cudaStream_t)stream;
  ctx->opt = opt;
  {
    const thermo_status s = build_context(ctx, grid, h, dval != nullptr);
    if (s != THERMO_OK) return s;
  }
  const Geom& g = ctx->g;
  // boundary data and load
  CK(mask_to_bits(g, mask, ctx->bits, ctx->st));
  CK(count_mask(g, mask, ctx->nnode, ctx->status_dev + 3, ctx->st));
  CK(cudaMemcpyAsync(ctx->status_h, ctx->status_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->ndir = ctx->status_h[3];
  if (ctx->ndir == 0) return fail(ctx, THERMO_EINVAL, "empty Dirichlet set: the operator is singular");
  if (dval) CK(pack_nodes(g, dval, ctx->TD, ctx->st));
  CK(load_vector(g, source, ctx->f, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_plan_bytes(const int grid[3], const thermo_options* opt_in, int has_dval,
                                           long long* bytes) {
  if (!grid || !bytes) return THERMO_EINVAL;
  thermo_options opt;
  if (opt_in)
    opt = *opt_in;
  else if (thermo_default_options(grid, &opt) != THERMO_OK)
    return THERMO_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (grid[k] <= 0) return THERMO_EINVAL;
  thermo_ctx* ctx = new (std::nothrow) thermo_ctx();
  if (!ctx) return THERMO_ENOMEM;
  ctx->opt = opt;
  ctx->dry = true;
  const double h[3] = {1.0 / grid[0], 1.0 / grid[1], 1.0 / grid[2]};
  const thermo_status s = build_context(ctx, grid, h, has_dval != 0);
  if (s == THERMO_OK) *bytes = ctx->plan_bytes;
  delete ctx;
  return s;
}

extern "C" void thermo_destroy(thermo_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  for (KTimer& t : ctx->kt)
    for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
  for (void* v : ctx->allocs) cudaFree(v);
  if (ctx->sc_h) cudaFreeHost(ctx->sc_h);
  if (ctx->status_h) cudaFreeHost(ctx->status_h);
  if (ctx->dscal_h) cudaFreeHost(ctx->dscal_h);
  delete ctx;
}

extern "C" const char* thermo_last_error(const thermo_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

extern "C" thermo_status thermo_set_density(thermo_ctx* ctx, const void* x, double p, double kmin, double kmax) {
  if (!ctx) return THERMO_EINVAL;
  if (!x) return fail(ctx, THERMO_EINVAL, "x is NULL");
  if (!(p >= 1.0) || !(kmin > 0.0) || !(kmax >= kmin) || !std::isfinite(kmax))
    return fail(ctx, THERMO_EINVAL, "need p >= 1 and 0 < kmin <= kmax");
  if (ctx->xf) {
    CK(cudaMemcpyAsync(ctx->xf, x, ctx->nelem * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    CK(simp_kappa<float>(ctx->g, ctx->xf, p, kmin, kmax, ctx->k64, ctx->k32, ctx->k16, ctx->klo, ctx->st));
  } else {
    CK(cudaMemcpyAsync(ctx->xd, x, ctx->nelem * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(simp_kappa<double>(ctx->g, ctx->xd, p, kmin, kmax, ctx->k64, ctx->k32, ctx->k16, ctx->klo, ctx->st));
  }
  // lifted right-hand side b = f - A_FD T_D (b_D = T_D)
  CK(dirichlet_rhs(ctx->g, ctx->bits, ctx->k64, ctx->f, ctx->TD, ctx->blift, ctx->st));
  ctx->sp = p;
  ctx->skmin = kmin;
  ctx->skmax = kmax;
  ctx->have_density = true;
  ctx->have_precond = false;
  return THERMO_OK;
}

extern "C" thermo_status thermo_update_density(thermo_ctx* ctx, const void* x, double p, double kmin, double kmax) {
  if (!ctx) return THERMO_EINVAL;
  const bool keep = ctx->have_precond;
  const thermo_status s = thermo_set_density(ctx, x, p, kmin, kmax);
  if (s == THERMO_OK) ctx->have_precond = keep;
  return s;
}

// ---------------------------------------------------------------------------
// preconditioner set-up (Sec. 3)
// operator of the outer CG loop: float-float (FP64-accurate on the FP32 pipes)
// or FP64 arithmetic, per opt.outer_apply
static bool use_ds(const thermo_ctx* ctx) {
  if (!fine_ds_supported(ctx->g)) return false;
  if (ctx->opt.outer_apply == 2) return true;
  if (ctx->opt.outer_apply == 1) return false;
  return ctx->opt.prec != THERMO_FP64;
}
extern "C" thermo_status thermo_setup_precond(thermo_ctx* ctx) {
  if (!ctx) return THERMO_EINVAL;
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "setup_precond before set_density");
  cudaStream_t st = ctx->st;
  const double t0 = now_ms();
  if (ctx->opt.pc != THERMO_PC_MMG) {
    ctx->have_precond = true;
    ctx->t_setup_ms = 0.0;
    return THERMO_OK;
  }
  const Geom& g = ctx->g;
  const int L1 = ctx->L1;
  CK(cudaMemsetAsync(ctx->status_dev, 0, 4 * sizeof(int), st));
  {
    // fine smoother coefficients
    const thermo_options& o = ctx->opt;
    if (o.smoother == 1) {
      // lmax(D^-1 A) by power iteration from the seeded start vector (FP64 vectors; the
      // operator in FP64 arithmetic for the FP64 form, else the FP64-accurate float-float apply)
      CK(power_start(g, ctx->bits, ctx->p, st));
      CK(vec_dot(g, ctx->p, ctx->p, 0, ctx->red, ctx->dscal, st));
      CK(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      CK(vec_scale(g, 1.0 / sqrt(ctx->dscal_h[0]), ctx->p, st));
      double lam = 0.0;
      for (int it = 0; it < o.power_iters; ++it) {
        if (use_ds(ctx))
          CK(fine_apply_ds(g, ctx->bits, ctx->k32, ctx->klo, ctx->p, ctx->q, nullptr, nullptr, nullptr, st));
        else
          CK(fine_apply_f64(g, ctx->bits, ctx->k64, ctx->p, ctx->q, nullptr, nullptr, nullptr, st));
        CK((fine_smooth<double, double>(g, ctx->bits, ctx->k64, ctx->q, nullptr, nullptr, ctx->p, 0.0, 1.0, st)));
        CK(vec_dot(g, ctx->p, ctx->p, 0, ctx->red, ctx->dscal, st));
        CK(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        lam = sqrt(ctx->dscal_h[0]);
        if (!(lam > 0.0) || !std::isfinite(lam)) {
          const thermo_status se = stage_check(ctx);  // a timed-out stage explains a bad estimate
          if (se != THERMO_OK) return se;
          return fail(ctx, THERMO_EINVAL, "power iteration failed (lmax = %g)", lam);
        }
        CK(vec_scale(g, 1.0 / lam, ctx->p, st));
      }
      ctx->lmax = lam;
      // Chebyshev on [lmax/ratio, 1.1 lmax]: three-term recurrence coefficients
      ctx->nsweep = o.cheb_degree;
      chebyshev_coefficients(lam, o.cheb_ratio, o.cheb_degree, ctx->sa, ctx->sb);
      CK(cudaMemsetAsync(ctx->p, 0, g.nsize * sizeof(double), st));
      CK(cudaMemsetAsync(ctx->q, 0, g.nsize * sizeof(double), st));
    } else {
      ctx->nsweep = o.nu_fine;
      for (int k = 0; k < o.nu_fine; ++k) {
        ctx->sa[k] = 0.0;
        ctx->sb[k] = o.omega;
      }
    }
  }
  Lev& l1 = ctx->lev[1];
  // lean: FP64 Phi shares the CG vectors' slab; clear it (padding nodes included)
  if (ctx->lean) CK(cudaMemsetAsync(ctx->phi64, 0, g.nsize * L1 * sizeof(double), st));
  // adaptive basis threshold of each level: tau / H_l^2, H_l the cell edge (b max(h), times the group sizes)
  auto thr_of = [&](int l) -> double {
    if (!(ctx->opt.eig_threshold > 0.0)) return 0.0;
    double H = ctx->opt.block * std::max(ctx->h[0], std::max(ctx->h[1], ctx->h[2]));
    for (int k = 2; k <= l; ++k) H *= ctx->lev[k].cl.g;
    return ctx->opt.eig_threshold / (H * H);
  };
  CK(level1_eigen(g, ctx->bits, ctx->k64, L1, ctx->phi64, l1.eig, l1.act, ctx->status_dev, thr_of(1), st));
  CK(level1_rowsum_corr(g, ctx->bits, ctx->k64, L1, ctx->phi64, l1.ntc, ctx->gcum_dev, l1.Dc, st));
  if (ctx->lean) {
    // FP32 hierarchy: every level but the coarsest is rounded once where it is
    // made; the next level is built (FP64 sums) from what is stored.  FP64 Phi
    // and Psi live in the CG vectors' slab, one at a time.
    const int top = ctx->nlev;
    if (top == 1) {
      CK(level1_rap<double>(g, ctx->bits, ctx->k64, L1, ctx->phi64, l1.T64, st));
      CK(fix_inactive<double>(l1.cl, l1.act, l1.T64, st));
    } else {
      CK(level1_rap<float>(g, ctx->bits, ctx->k64, L1, ctx->phi64, l1.T32, st));
      CK(fix_inactive<float>(l1.cl, l1.act, l1.T32, st));
    }
    CK(cvt_f64_f32(ctx->phi64, ctx->phi32, g.nsize * L1, st));
    for (int l = 2; l <= top; ++l) {
      Lev& pv = ctx->lev[l - 1];
      Lev& cu = ctx->lev[l];
      CK(group_eigen<float>(pv.cl, cu.cl, pv.T32, pv.Dc, pv.act, cu.Psi64, cu.eig, cu.act, ctx->status_dev, thr_of(l),
                            st));
      if (cu.ntc > 0) CK(group_project_corr(pv.cl, cu.cl, cu.Psi64, pv.Dc, cu.Dc, cu.ntc, st));
      if (l == top) {
        CK((group_rap<float, double>(pv.cl, cu.cl, cu.Psi64, pv.T32, cu.T64, st)));
        CK(fix_inactive<double>(cu.cl, cu.act, cu.T64, st));
      } else {
        CK((group_rap<float, float>(pv.cl, cu.cl, cu.Psi64, pv.T32, cu.T32, st)));
        CK(fix_inactive<float>(cu.cl, cu.act, cu.T32, st));
      }
      const long long np = cu.cl.ncell * (long long)cu.cl.g * cu.cl.g * cu.cl.g * pv.cl.L * cu.cl.L;
      CK(cvt_f64_f32(cu.Psi64, cu.Psi32, np, st));
    }
    for (int l = 1; l < top; ++l) CK(l1_inverse<float>(ctx->lev[l].cl, ctx->lev[l].T32, nullptr, ctx->lev[l].Di32, st));
    // the fine kernels read the padded layout's ghost nodes as zeros: clear what
    // set-up left in the vectors' memory
    CK(cudaMemsetAsync(ctx->slab64, 0, ctx->slab64_n * sizeof(double), st));
    CK(cudaMemsetAsync(ctx->slab32, 0, ctx->slab32_n * sizeof(float), st));
  } else {
    CK(level1_rap<double>(g, ctx->bits, ctx->k64, L1, ctx->phi64, l1.T64, st));
    CK(fix_inactive<double>(l1.cl, l1.act, l1.T64, st));
    for (int l = 2; l <= ctx->nlev; ++l) {
      Lev& pv = ctx->lev[l - 1];
      Lev& cu = ctx->lev[l];
      CK(group_eigen<double>(pv.cl, cu.cl, pv.T64, pv.Dc, pv.act, cu.Psi64, cu.eig, cu.act, ctx->status_dev,
                             thr_of(l), st));
      if (cu.ntc > 0) CK(group_project_corr(pv.cl, cu.cl, cu.Psi64, pv.Dc, cu.Dc, cu.ntc, st));
      CK((group_rap<double, double>(pv.cl, cu.cl, cu.Psi64, pv.T64, cu.T64, st)));
      CK(fix_inactive<double>(cu.cl, cu.act, cu.T64, st));
      const long long np = cu.cl.ncell * (long long)cu.cl.g * cu.cl.g * cu.cl.g * pv.cl.L * cu.cl.L;
      CK(cvt_f64_f32(cu.Psi64, cu.Psi32, np, st));
    }
    for (int l = 1; l < ctx->nlev; ++l) {
      Lev& lv = ctx->lev[l];
      CK(l1_inverse<double>(lv.cl, lv.T64, lv.Di64, lv.Di32, st));
      CK(cvt_f64_f32(lv.T64, lv.T32, lv.cl.ncell * 27 * lv.cl.L * lv.cl.L, st));
    }
    CK(cvt_f64_f32(ctx->phi64, ctx->phi32, g.nsize * L1, st));
  }
  CK(dense_assemble(ctx->lev[ctx->nlev].cl, ctx->lev[ctx->nlev].T64, ctx->cholA, st));
  CK(cholesky_inverse(ctx->ncoarse, ctx->cholA, ctx->Ainv, ctx->cholW, ctx->status_dev, st));
  CK(cudaMemcpyAsync(ctx->status_h, ctx->status_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->t_setup_ms = now_ms() - t0;
  {
    const thermo_status se = stage_check(ctx);
    if (se != THERMO_OK) return se;
  }
  if (ctx->status_h[0] != 0)
    return fail(ctx, THERMO_ESINGULAR, "coarsest Cholesky: non-positive pivot at %d", ctx->status_h[0] - 1);
  ctx->have_precond = true;
  return THERMO_OK;
}

// ---------------------------------------------------------------------------
// coarse part of the cycle on levels l..nlev, input lev[l].r, output lev[l].e
template <class T>
static T* lvr(Lev& l);
template <>
double* lvr<double>(Lev& l) { return l.r64; }
template <>
float* lvr<float>(Lev& l) { return l.r32; }
template <class T>
static T* lve(Lev& l);
template <>
double* lve<double>(Lev& l) { return l.e64; }
template <>
float* lve<float>(Lev& l) { return l.e32; }
template <class T>
static T* lvt(Lev& l);
template <>
double* lvt<double>(Lev& l) { return l.t64; }
template <>
float* lvt<float>(Lev& l) { return l.t32; }
template <class T>
static T* lvs(Lev& l);
template <>
double* lvs<double>(Lev& l) { return l.s64; }
template <>
float* lvs<float>(Lev& l) { return l.s32; }
template <class T>
static const T* lvT(Lev& l);
template <>
const double* lvT<double>(Lev& l) { return l.T64; }
template <>
const float* lvT<float>(Lev& l) { return l.T32; }
template <class T>
static const T* lvD(Lev& l);
template <>
const double* lvD<double>(Lev& l) { return l.Di64; }
template <>
const float* lvD<float>(Lev& l) { return l.Di32; }
template <class T>
static const T* lvP(Lev& l);
template <>
const double* lvP<double>(Lev& l) { return l.Psi64; }
template <>
const float* lvP<float>(Lev& l) { return l.Psi32; }

static cudaError_t outer_apply_dot(thermo_ctx* ctx, const double* p, double* q, double* dot) {
  const Geom& g = ctx->g;
  if (use_ds(ctx))
    return fine_apply_ds(g, ctx->bits, ctx->k32, ctx->klo, p, q, ctx->red.partial, ctx->red.counter, dot, ctx->st);
  return fine_apply_f64(g, ctx->bits, ctx->k64, p, q, ctx->red.partial, ctx->red.counter, dot, ctx->st);
}

// ---- kernel-class timers: begin/end bracket one launch on the context stream
static inline void kt_begin(thermo_ctx* ctx, int c) {
  if (!ctx->kt_on) return;
  KTimer& t = ctx->kt[c];
  if (t.used < KTimer::CAP) cudaEventRecord(t.ev[2 * t.used], ctx->st);
}
static inline void kt_end(thermo_ctx* ctx, int c, double bytes, double flops = 0.0) {
  if (!ctx->kt_on) return;
  KTimer& t = ctx->kt[c];
  if (t.used >= KTimer::CAP) return;
  cudaEventRecord(t.ev[2 * t.used + 1], ctx->st);
  ++t.used;
  t.pend_bytes += bytes;
  t.pend_flops += flops;
}
// after the stream has been synchronised: fold the recorded pairs into the totals
static void kt_fold(thermo_ctx* ctx) {
  if (!ctx->kt_on) return;
  for (KTimer& t : ctx->kt) {
    for (int i = 0; i < t.used; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]) == cudaSuccess) t.ms += ms;
    }
    t.launches += t.used;
    t.bytes += t.pend_bytes;
    t.flops += t.pend_flops;
    t.used = 0;
    t.pend_bytes = t.pend_flops = 0.0;
  }
}
// algorithmic DRAM bytes of the fine kernels: every array touched once
static double fine_bytes(const Geom& g, double s_node, double s_elem) {
  const double n = (double)(g.Nx + 1) * (g.Ny + 1) * (g.Nz + 1);
  const double m = (double)g.Nx * g.Ny * g.Nz;
  return n * s_node + m * s_elem + n / 8.0;  // + Dirichlet bitmask
}

// algorithmic bytes of the coarse kernels (each array once): tiles 27 L^2 per cell,
// l1 inverses L^2 per cell, vectors L per cell, group bases g^3 Lprev L per group
static double cb_tiles(const CLevel& c, double ts) { return (double)c.ncell * 27.0 * c.L * c.L * ts; }
static double cb_vec(const CLevel& c, double ts) { return (double)c.ncell * c.L * ts; }
static double cb_psi(const CLevel& f, const CLevel& c, double ts) {
  return (double)c.ncell * c.g * c.g * c.g * f.L * c.L * ts;
}
static inline void cb_add(thermo_ctx* ctx, double b) {
  if (ctx->kt_on) ctx->coarse_bytes += b;
}

template <class T>
static cudaError_t coarse_cycle(thermo_ctx* ctx, int l) {
  cudaStream_t st = ctx->st;
  Lev& lv = ctx->lev[l];
  cudaError_t e;
  const double ts = sizeof(T);
  if (l == ctx->nlev) {
    cb_add(ctx, (double)ctx->ncoarse * ctx->ncoarse * 8.0 + 2.0 * ctx->ncoarse * ts);  // FP64 inverse, x, y
    return dense_gemv<T>(ctx->ncoarse, ctx->Ainv, lvr<T>(lv), lve<T>(lv), st);
  }
  const CLevel& cl = lv.cl;
  const double b_smooth0 = (double)cl.ncell * cl.L * cl.L * ts + 2.0 * cb_vec(cl, ts);
  const double b_smooth = cb_tiles(cl, ts) + (double)cl.ncell * cl.L * cl.L * ts + 3.0 * cb_vec(cl, ts);
  const double b_resid = cb_tiles(cl, ts) + 3.0 * cb_vec(cl, ts);
  // sweeps on this level: nu_coarse, multiplied by nu_growth per level below level 1
  int nu = ctx->opt.nu_coarse;
  for (int k = 1; k < l && nu < 64; ++k) nu *= ctx->opt.nu_growth;
  if (nu > 64) nu = 64;
  T* E = lve<T>(lv);
  T* Tt = lvt<T>(lv);
  if ((e = coarse_smooth0<T>(lv.cl, lvD<T>(lv), lvr<T>(lv), E, st)) != cudaSuccess) return e;
  cb_add(ctx, b_smooth0);
  for (int s = 1; s < nu; ++s) {
    if ((e = coarse_smooth<T>(lv.cl, lvT<T>(lv), lvD<T>(lv), lvr<T>(lv), E, Tt, st)) != cudaSuccess) return e;
    cb_add(ctx, b_smooth);
    std::swap(E, Tt);
  }
  Lev& nx = ctx->lev[l + 1];
  // coarse corrections: two (W-cycle) on levels >= w_from, unless the next level is
  // the exact coarsest solve (a second Galerkin correction would be zero)
  const int reps = (ctx->opt.w_from > 0 && l >= ctx->opt.w_from && l + 1 < ctx->nlev) ? 2 : 1;
  for (int c = 0; c < reps; ++c) {
    if ((e = coarse_residual<T>(lv.cl, lvT<T>(lv), lvr<T>(lv), E, lvs<T>(lv), st)) != cudaSuccess) return e;
    cb_add(ctx, b_resid);
    if ((e = coarse_restrict<T>(lv.cl, nx.cl, lvP<T>(nx), lvs<T>(lv), lvr<T>(nx), st)) != cudaSuccess) return e;
    cb_add(ctx, cb_psi(cl, nx.cl, ts) + cb_vec(cl, ts) + cb_vec(nx.cl, ts));
    if ((e = coarse_cycle<T>(ctx, l + 1)) != cudaSuccess) return e;
    if ((e = coarse_prolong<T>(lv.cl, nx.cl, lvP<T>(nx), lve<T>(nx), E, st)) != cudaSuccess) return e;
    cb_add(ctx, cb_psi(cl, nx.cl, ts) + cb_vec(nx.cl, ts) + 2.0 * cb_vec(cl, ts));
  }
  for (int s = 0; s < nu; ++s) {
    if ((e = coarse_smooth<T>(lv.cl, lvT<T>(lv), lvD<T>(lv), lvr<T>(lv), E, Tt, st)) != cudaSuccess) return e;
    cb_add(ctx, b_smooth);
    std::swap(E, Tt);
  }
  if (E != lve<T>(lv)) {
    e = cudaMemcpyAsync(lve<T>(lv), E, lv.cl.ncell * lv.cl.L * sizeof(T), cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

// One V-cycle z = B r on the fine grid; S storage, C = compute, output To.
// Smoothing is the three-term sweep e' = e + a_k (e - e_prev) + b_k D^-1 (r - A e)
// (damped Jacobi: a_k = 0, b_k = omega; Chebyshev: the recurrence coefficients),
// applied from zero before restriction and from the prolonged iterate after.
template <class S, class To>
static cudaError_t vcycle_fine(thermo_ctx* ctx, const S* kap, const S* r, S* b0, S* b1, S* b2, To* z) {
  typedef typename Cv<S>::C C;
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  const int m = ctx->nsweep, L1 = ctx->L1;
  const double* sa = ctx->sa;
  const double* sb = ctx->sb;
  const C* phi = (sizeof(C) == 8) ? (const C*)ctx->phi64 : (const C*)ctx->phi32;
  Lev& l1 = ctx->lev[1];
  C* rc = (sizeof(C) == 8) ? (C*)l1.r64 : (C*)l1.r32;
  C* ec = (sizeof(C) == 8) ? (C*)l1.e64 : (C*)l1.e32;
  S* buf[3] = {b0, b1, b2};
  const double s = sizeof(S), c = sizeof(C);
  // algorithmic bytes of one sweep: r, kappa, mask, output; + iterate v, + previous iterate w
  auto sweep_bytes = [&](bool hv, bool hw, double so) {
    return ctx->kt_on ? fine_bytes(g, s + so + (hv ? s : 0.0) + (hw ? s : 0.0), s) : 0.0;
  };
  cudaError_t e;
  // pre-smoothing from e_0 = 0
  int cur = 0, prev = -1;
  kt_begin(ctx, THERMO_KT_SMOOTH);
  if ((e = fine_smooth<S, S>(g, ctx->bits, kap, r, nullptr, nullptr, buf[0], C(0), (C)sb[0], st)) != cudaSuccess)
    return e;
  kt_end(ctx, THERMO_KT_SMOOTH, sweep_bytes(false, false, s));
  for (int k = 1; k < m; ++k) {
    const int nxt = prev >= 0 ? 3 - cur - prev : (cur + 1) % 3;
    const S* w = (sa[k] != 0.0 && prev >= 0) ? buf[prev] : nullptr;
    kt_begin(ctx, THERMO_KT_SMOOTH);
    if ((e = fine_smooth<S, S>(g, ctx->bits, kap, r, buf[cur], w, buf[nxt], (C)sa[k], (C)sb[k], st)) != cudaSuccess)
      return e;
    kt_end(ctx, THERMO_KT_SMOOTH, sweep_bytes(true, w != nullptr, s));
    prev = cur;
    cur = nxt;
  }
  kt_begin(ctx, THERMO_KT_RESTRICT);
  if constexpr (sizeof(S) == 4 && sizeof(C) == 4) {
    // residual by the separable engine, then the block-strip restriction
    if (fine3_restrict_supported(g, L1))
      e = fine3_restrict(g, ctx->bits, (const float*)kap, (const float*)r, (const float*)buf[cur], (const float*)phi,
                         ctx->tmp32, (float*)rc, L1, st);
    else
      e = fine_restrict<S>(g, ctx->bits, kap, r, buf[cur], phi, rc, L1, st);
  } else {
    e = fine_restrict<S>(g, ctx->bits, kap, r, buf[cur], phi, rc, L1, st);
  }
  if (e != cudaSuccess) return e;
  kt_end(ctx, THERMO_KT_RESTRICT, ctx->kt_on ? fine_bytes(g, 2 * s + L1 * c, s) + (double)l1.cl.ncell * L1 * c : 0.0);
  kt_begin(ctx, THERMO_KT_COARSE);
  ctx->coarse_bytes = 0.0;
  if (sizeof(C) == 8)
    e = coarse_cycle<double>(ctx, 1);
  else
    e = coarse_cycle<float>(ctx, 1);
  if (e != cudaSuccess) return e;
  kt_end(ctx, THERMO_KT_COARSE, ctx->coarse_bytes);
  // prolongation (in place) and post-smoothing from the prolonged iterate
  kt_begin(ctx, THERMO_KT_PROLONG);
  if ((e = fine_prolong<S>(g, phi, ec, buf[cur], L1, st)) != cudaSuccess) return e;
  kt_end(ctx, THERMO_KT_PROLONG,
         (double)ctx->nnode * (2 * s + L1 * c) + (double)l1.cl.ncell * L1 * c);  // v in/out, Phi, e_c
  prev = -1;
  for (int k = 0; k < m; ++k) {
    const S* w = (k > 0 && sa[k] != 0.0) ? buf[prev] : nullptr;
    if (k == m - 1) {
      kt_begin(ctx, THERMO_KT_SMOOTH);
      e = fine_smooth<S, To>(g, ctx->bits, kap, r, buf[cur], w, z, (C)sa[k], (C)sb[k], st);
      kt_end(ctx, THERMO_KT_SMOOTH, sweep_bytes(true, w != nullptr, (double)sizeof(To)));
      return e;
    }
    const int nxt = prev >= 0 ? 3 - cur - prev : (cur + 1) % 3;
    kt_begin(ctx, THERMO_KT_SMOOTH);
    if ((e = fine_smooth<S, S>(g, ctx->bits, kap, r, buf[cur], w, buf[nxt], (C)sa[k], (C)sb[k], st)) != cudaSuccess)
      return e;
    kt_end(ctx, THERMO_KT_SMOOTH, sweep_bytes(true, w != nullptr, s));
    prev = cur;
    cur = nxt;
  }
  return cudaSuccess;
}

// z = B r where r is the FP64 residual already converted to the cycle's
// storage (mixed: ctx->r32 / r16); output: z64 (FP64 form) or z32.
static cudaError_t apply_precond(thermo_ctx* ctx) {
  const thermo_options& o = ctx->opt;
  const Geom& g = ctx->g;
  if (o.pc == THERMO_PC_NONE) return cudaMemcpyAsync(ctx->z64, ctx->r, g.nsize * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st);
  if (o.pc == THERMO_PC_JACOBI)
    return fine_smooth<double, double>(g, ctx->bits, ctx->k64, ctx->r, nullptr, nullptr, ctx->z64, 0.0, 1.0, ctx->st);
  if (o.prec == THERMO_FP64)
    return vcycle_fine<double, double>(ctx, ctx->k64, ctx->r, ctx->ea64, ctx->eb64, ctx->ec64, ctx->z64);
  if (o.prec == THERMO_MIXED)
    return vcycle_fine<float, float>(ctx, ctx->k32, ctx->r32, ctx->ea32, ctx->eb32, ctx->ec32, ctx->z32);
  return vcycle_fine<bf16, float>(ctx, ctx->k16, ctx->r16, ctx->ea16, ctx->eb16, ctx->ec16, ctx->z32);
}
static int zkind(const thermo_ctx* ctx) {
  return (ctx->opt.pc != THERMO_PC_MMG || ctx->opt.prec == THERMO_FP64) ? 0 : 1;
}
static const void* zptr(const thermo_ctx* ctx) { return zkind(ctx) == 0 ? (const void*)ctx->z64 : (const void*)ctx->z32; }
static int rkind(const thermo_ctx* ctx) {
  if (ctx->opt.pc != THERMO_PC_MMG || ctx->opt.prec == THERMO_FP64) return -1;
  return ctx->opt.prec == THERMO_MIXED ? 1 : 2;
}
static void* rptr(thermo_ctx* ctx) {
  const int k = rkind(ctx);
  return k == 1 ? (void*)ctx->r32 : (k == 2 ? (void*)ctx->r16 : nullptr);
}

// y = P A_L^-1 P^T v added to u (composite restriction / prolongation: FP64;
// the lean form has only the FP32 hierarchy and runs the chain in FP32 on a
// rounded copy of v, adding the FP64-summed prolongation to u)
static thermo_status coarse_correction(thermo_ctx* ctx, const double* v, double* u) {
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  Lev& l1 = ctx->lev[1];
  if (ctx->lean) {
    CK(vec_copy_cvt(g, v, ctx->r32, 1, st));
    CK(cudaMemsetAsync(ctx->ea32, 0, g.nsize * sizeof(float), st));
    CK(fine_restrict<float>(g, ctx->bits, ctx->k32, ctx->r32, ctx->ea32, ctx->phi32, l1.r32, ctx->L1, st));
    for (int l = 1; l < ctx->nlev; ++l) {
      Lev& a = ctx->lev[l];
      Lev& b = ctx->lev[l + 1];
      CK(coarse_restrict<float>(a.cl, b.cl, b.Psi32, a.r32, b.r32, st));
    }
    Lev& top = ctx->lev[ctx->nlev];
    CK(dense_gemv<float>(ctx->ncoarse, ctx->Ainv, top.r32, top.e32, st));
    for (int l = ctx->nlev - 1; l >= 1; --l) {
      Lev& a = ctx->lev[l];
      Lev& b = ctx->lev[l + 1];
      CK(cudaMemsetAsync(a.e32, 0, a.cl.ncell * a.cl.L * sizeof(float), st));
      CK(coarse_prolong<float>(a.cl, b.cl, b.Psi32, b.e32, a.e32, st));
    }
    CK(fine_prolong_add<float>(g, ctx->phi32, ctx->L1, l1.e32, u, st));
    return THERMO_OK;
  }
  CK(fine_restrict<double>(g, ctx->bits, ctx->k64, v, ctx->zero64, ctx->phi64, l1.r64, ctx->L1, st));
  for (int l = 1; l < ctx->nlev; ++l) {
    Lev& a = ctx->lev[l];
    Lev& b = ctx->lev[l + 1];
    CK(coarse_restrict<double>(a.cl, b.cl, b.Psi64, a.r64, b.r64, st));
  }
  Lev& top = ctx->lev[ctx->nlev];
  CK(dense_gemv<double>(ctx->ncoarse, ctx->Ainv, top.r64, top.e64, st));
  for (int l = ctx->nlev - 1; l >= 1; --l) {
    Lev& a = ctx->lev[l];
    Lev& b = ctx->lev[l + 1];
    CK(cudaMemsetAsync(a.e64, 0, a.cl.ncell * a.cl.L * sizeof(double), st));
    CK(coarse_prolong<double>(a.cl, b.cl, b.Psi64, b.e64, a.e64, st));
  }
  CK(fine_prolong_add<double>(g, ctx->phi64, ctx->L1, l1.e64, u, st));
  return THERMO_OK;
}

static thermo_status read_scalars(thermo_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->sc_h, ctx->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return THERMO_OK;
}

// true residual r = b - A u into ctx->r, ||r||^2 in sc->rr
static thermo_status true_residual(thermo_ctx* ctx, const double* b) {
  CK(fine_apply_f64(ctx->g, ctx->bits, ctx->k64, ctx->u, ctx->q, nullptr, nullptr, nullptr, ctx->st, true));
  CK(vec_residual(ctx->g, b, ctx->q, ctx->r, ctx->red, &ctx->sc->rr, ctx->st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_solve(thermo_ctx* ctx, const double* rhs, double* u, double tol,
                                      thermo_solve_info* info) {
  if (!ctx) return THERMO_EINVAL;
  if (!u) return fail(ctx, THERMO_EINVAL, "u is NULL");
  if (!(tol > 0.0)) return fail(ctx, THERMO_EINVAL, "tol must be > 0");
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "solve before set_density");
  if (!ctx->have_precond) return fail(ctx, THERMO_ESTATE, "solve before setup_precond");
  const thermo_options& o = ctx->opt;
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  thermo_solve_info inf;
  memset(&inf, 0, sizeof inf);
  inf.t_setup_ms = ctx->t_setup_ms;
  CK(cudaStreamSynchronize(st));
  const double t0 = now_ms();
  const double* b = ctx->blift;
  if (rhs) {
    CK(pack_nodes(g, rhs, ctx->bv, st));
    b = ctx->bv;
  }
  const int flexible = o.flexible < 0 ? (o.prec != THERMO_FP64 && o.pc == THERMO_PC_MMG) : o.flexible;
  const bool mmg = o.pc == THERMO_PC_MMG;
  // initial guess
  if (o.guess == THERMO_GUESS_GIVEN || o.guess == THERMO_GUESS_WARM_COARSE) {
    CK(pack_nodes(g, u, ctx->u, st));
  } else if (ctx->TD) {
    CK(cudaMemcpyAsync(ctx->u, ctx->TD, g.nsize * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemsetAsync(ctx->u, 0, g.nsize * sizeof(double), st));
  }
  // the Dirichlet rows are identities: every iterate carries u_D = b_D
  CK(vec_copy_dir(g, ctx->bits, b, ctx->u, st));
  if (mmg && (o.guess == THERMO_GUESS_COARSE || o.guess == THERMO_GUESS_WARM_COARSE)) {
    thermo_status s = true_residual(ctx, b);
    if (s != THERMO_OK) return s;
    s = coarse_correction(ctx, ctx->r, ctx->u);
    if (s != THERMO_OK) return s;
  }
  CK(vec_dot_free(g, ctx->bits, b, b, ctx->red, &ctx->sc->bb, st));
  {
    thermo_status s = true_residual(ctx, b);
    if (s != THERMO_OK) return s;
  }
  CK(cudaMemsetAsync(&ctx->sc->flag, 0, sizeof(int), st));
  thermo_status s = read_scalars(ctx);
  if (s != THERMO_OK) return s;
  const double bnorm = sqrt(ctx->sc_h->bb);
  double rn = sqrt(ctx->sc_h->rr);
  ctx->hist.clear();
  if (!std::isfinite(bnorm)) return fail(ctx, THERMO_EINVAL, "right-hand side is not finite");
  if (!std::isfinite(rn)) {
    const thermo_status se = stage_check(ctx);
    inf.status = se != THERMO_OK ? se : THERMO_EBREAKDOWN;
    if (se != THERMO_OK) {
      if (info) *info = inf;
      return se;
    }
    if (info) *info = inf;
    return fail(ctx, THERMO_EBREAKDOWN, "initial residual is not finite (check the density)");
  }
  int it = 0, restarts = 0, refinements = 0;
  thermo_status result = THERMO_OK;
  auto start_cycle = [&](void) -> thermo_status {
    // r (FP64) -> cycle storage, z = B r, rz = r.z, p = z
    if (rkind(ctx) > 0) CK(vec_copy_cvt(g, ctx->r, rptr(ctx), rkind(ctx), st));
    CK(apply_precond(ctx));
    CK(vec_dot(g, ctx->r, zptr(ctx), zkind(ctx), ctx->red, &ctx->sc->rz, st));
    CK(cg_pupdate(g, zptr(ctx), zkind(ctx), ctx->p, ctx->sc, 1, st));
    return THERMO_OK;
  };
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(ctx->u, 0, g.nsize * sizeof(double), st));
    rn = 0.0;
  } else if (rn > tol * bnorm) {
    s = start_cycle();
    if (s != THERMO_OK) return s;
    const int check = o.check_every < 1 ? 1 : o.check_every;
    // algorithmic bytes / flops of the loop's own kernels (timers only)
    const double zs = zkind(ctx) == 0 ? 8.0 : (zkind(ctx) == 1 ? 4.0 : 2.0);
    const double rs = rkind(ctx) == 0 ? 0.0 : (rkind(ctx) == 1 ? 4.0 : 2.0);
    const double apply_bytes = ctx->kt_on ? fine_bytes(g, 16.0, 8.0) : 0.0;
    const double apply_flops = 2.0 * (g.cube ? 21.0 : 27.0) * (double)ctx->nnode;
    const double nn = (double)ctx->nnode;
    // low-precision cycles limit how far one recurrence can reduce the residual:
    // restart from the true residual every restart_decades decades
    double anchor = rn;
    const double restart_factor = o.restart_decades > 0 ? pow(10.0, -o.restart_decades) : 0.0;
    while (true) {
      kt_begin(ctx, THERMO_KT_APPLY64);
      CK(outer_apply_dot(ctx, ctx->p, ctx->q, &ctx->sc->pq));
      kt_end(ctx, THERMO_KT_APPLY64, apply_bytes, apply_flops);
      kt_begin(ctx, THERMO_KT_CGVEC);
      CK(cg_update(g, ctx->u, ctx->r, ctx->p, ctx->q, flexible == 2 ? zptr(ctx) : nullptr, zkind(ctx), rptr(ctx),
                   rkind(ctx), ctx->sc, ctx->red, st));
      kt_end(ctx, THERMO_KT_CGVEC, nn * (4 * 8.0 + 2 * 8.0 + rs + (flexible == 2 ? zs : 0.0)));
      ++it;
      if (it % check == 0 || it >= o.max_iter) {
        s = read_scalars(ctx);
        if (s != THERMO_OK) return s;
        if (ctx->sc_h->flag) {
          result = fail(ctx, THERMO_EBREAKDOWN, "CG breakdown at iteration %d", it);
          break;
        }
        rn = sqrt(ctx->sc_h->rr);
        ctx->hist.push_back(bnorm > 0 ? rn / bnorm : 0.0);
        if (rn <= tol * bnorm) {
          s = true_residual(ctx, b);
          if (s != THERMO_OK) return s;
          s = read_scalars(ctx);
          if (s != THERMO_OK) return s;
          const double rt = sqrt(ctx->sc_h->rr);
          if (rt <= tol * bnorm || restarts >= 5) {
            if (rt > tol * bnorm) result = fail(ctx, THERMO_ENOTCONV, "true residual stagnates above tol");
            break;
          }
          ++restarts;
          s = start_cycle();
          if (s != THERMO_OK) return s;
          continue;
        }
        if (it >= o.max_iter) {
          result = fail(ctx, THERMO_ENOTCONV, "no convergence in %d iterations", it);
          break;
        }
        if (o.restart_decades > 0 && rn <= anchor * restart_factor) {
          // refinement step: true FP64 residual, fresh recurrence from z = B r
          s = true_residual(ctx, b);
          if (s != THERMO_OK) return s;
          s = read_scalars(ctx);
          if (s != THERMO_OK) return s;
          anchor = sqrt(ctx->sc_h->rr);
          ++refinements;
          s = start_cycle();
          if (s != THERMO_OK) return s;
          continue;
        }
      }
      CK(apply_precond(ctx));
      kt_begin(ctx, THERMO_KT_CGVEC);
      CK(cg_beta_dot(g, ctx->r, zptr(ctx), zkind(ctx), ctx->q, flexible, ctx->sc, ctx->red, st));
      kt_end(ctx, THERMO_KT_CGVEC, nn * (8.0 + zs + (flexible == 1 ? 8.0 : 0.0)));
      kt_begin(ctx, THERMO_KT_CGVEC);
      CK(cg_pupdate(g, zptr(ctx), zkind(ctx), ctx->p, ctx->sc, 0, st));
      kt_end(ctx, THERMO_KT_CGVEC, nn * (zs + 16.0));
    }
  }
  // final true residual (FP64)
  {
    thermo_status s2 = true_residual(ctx, b);
    if (s2 != THERMO_OK) return s2;
    s2 = read_scalars(ctx);
    if (s2 != THERMO_OK) return s2;
  }
  inf.rel_res_recursive = bnorm > 0 ? rn / bnorm : 0.0;
  inf.rel_res_true = bnorm > 0 ? sqrt(ctx->sc_h->rr) / bnorm : 0.0;
  CK(unpack_nodes(g, ctx->u, u, st));
  CK(cudaStreamSynchronize(st));
  kt_fold(ctx);
  {
    const thermo_status se = stage_check(ctx);
    if (se != THERMO_OK) result = se;
  }
  inf.iters = it;
  inf.restarts = restarts + refinements;
  inf.t_solve_ms = now_ms() - t0;
  inf.status = result;
  if (info) *info = inf;
  return result;
}

extern "C" thermo_status thermo_sensitivity(thermo_ctx* ctx, const double* u, double* dc) {
  if (!ctx) return THERMO_EINVAL;
  if (!u || !dc) return fail(ctx, THERMO_EINVAL, "NULL argument");
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "sensitivity before set_density");
  CK(pack_nodes(ctx->g, u, ctx->tmp, ctx->st));
  if (ctx->xf)
    CK(sensitivity<float>(ctx->g, ctx->tmp, ctx->xf, ctx->sp, ctx->skmin, ctx->skmax, dc, ctx->st));
  else
    CK(sensitivity<double>(ctx->g, ctx->tmp, ctx->xd, ctx->sp, ctx->skmin, ctx->skmax, dc, ctx->st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_compliance(thermo_ctx* ctx, const double* u, double* c) {
  if (!ctx) return THERMO_EINVAL;
  if (!u || !c) return fail(ctx, THERMO_EINVAL, "NULL argument");
  CK(pack_nodes(ctx->g, u, ctx->tmp, ctx->st));
  CK(vec_dot(ctx->g, ctx->f, ctx->tmp, 0, ctx->red, ctx->dscal, ctx->st));
  CK(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *c = ctx->dscal_h[0];
  return THERMO_OK;
}

extern "C" thermo_status thermo_apply(thermo_ctx* ctx, int precision, const double* u, double* y) {
  if (!ctx) return THERMO_EINVAL;
  if (!u || !y) return fail(ctx, THERMO_EINVAL, "NULL argument");
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "apply before set_density");
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  CK(pack_nodes(g, u, ctx->tmp, st));
  if (precision == THERMO_FP64) {
    CK(fine_apply_f64(g, ctx->bits, ctx->k64, ctx->tmp, ctx->q, nullptr, nullptr, nullptr, st, true));
  } else if (precision == THERMO_MIXED || precision == THERMO_MIXED_BF16S) {
    // the V-cycle's kernel: input zero on Gamma_D, rows there 0; identity rows restored below
    CK(vec_mask_dir(g, ctx->bits, ctx->tmp, st));
    if (precision == THERMO_MIXED) {
      CK(vec_copy_cvt(g, ctx->tmp, ctx->ea32, 1, st));
      CK(fine_apply_lp<float>(g, ctx->bits, ctx->k32, ctx->ea32, ctx->eb32, st, false));
      CK(vec_to_f64(g, ctx->eb32, 1, ctx->q, st));
    } else {
      bf16 *a16 = ctx->ea16, *b16 = ctx->eb16;
      if (!a16) return fail(ctx, THERMO_EINVAL, "BF16 buffers exist only for a MIXED_BF16S context");
      CK(vec_copy_cvt(g, ctx->tmp, a16, 2, st));
      CK(fine_apply_lp<bf16>(g, ctx->bits, ctx->k16, a16, b16, st, false));
      CK(vec_to_f64(g, b16, 2, ctx->q, st));
    }
    CK(pack_nodes(g, u, ctx->tmp, st));
    CK(vec_copy_dir(g, ctx->bits, ctx->tmp, ctx->q, st));
  } else {
    return fail(ctx, THERMO_EINVAL, "unknown precision %d", precision);
  }
  CK(unpack_nodes(g, ctx->q, y, st));
  return stage_check(ctx);
}

extern "C" thermo_status thermo_apply_dot(thermo_ctx* ctx, const double* p, double* q, double* pq) {
  if (!ctx) return THERMO_EINVAL;
  if (!p || !q || !pq) return fail(ctx, THERMO_EINVAL, "NULL argument");
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "apply before set_density");
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  CK(pack_nodes(g, p, ctx->tmp, st));
  CK(outer_apply_dot(ctx, ctx->tmp, ctx->q, ctx->dscal));
  CK(unpack_nodes(g, ctx->q, q, st));
  CK(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *pq = ctx->dscal_h[0];
  return stage_check(ctx);
}

extern "C" thermo_status thermo_vcycle(thermo_ctx* ctx, const double* r, double* z) {
  if (!ctx) return THERMO_EINVAL;
  if (!r || !z) return fail(ctx, THERMO_EINVAL, "NULL argument");
  if (!ctx->have_precond || ctx->opt.pc != THERMO_PC_MMG) return fail(ctx, THERMO_ESTATE, "no MMG preconditioner");
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  CK(pack_nodes(g, r, ctx->r, st));
  CK(vec_mask_dir(g, ctx->bits, ctx->r, st));  // the cycle assumes r = 0 on Gamma_D
  if (rkind(ctx) > 0) CK(vec_copy_cvt(g, ctx->r, rptr(ctx), rkind(ctx), st));
  CK(apply_precond(ctx));
  if (zkind(ctx) == 1) {
    CK(vec_to_f64(g, ctx->z32, 1, ctx->tmp, st));
    CK(unpack_nodes(g, ctx->tmp, z, st));
  } else {
    CK(unpack_nodes(g, ctx->z64, z, st));
  }
  return stage_check(ctx);
}

extern "C" thermo_status thermo_load_vector(thermo_ctx* ctx, double* f) {
  if (!ctx || !f) return THERMO_EINVAL;
  CK(unpack_nodes(ctx->g, ctx->f, f, ctx->st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_hierarchy(const thermo_ctx* ctx, int* nlevels, int* cells, int* nvec,
                                          long long* ndof) {
  if (!ctx) return THERMO_EINVAL;
  if (nlevels) *nlevels = ctx->nlev;
  for (int l = 1; l <= ctx->nlev; ++l) {
    const CLevel& c = ctx->lev[l].cl;
    if (cells) {
      cells[(l - 1) * 3 + 0] = c.mx;
      cells[(l - 1) * 3 + 1] = c.my;
      cells[(l - 1) * 3 + 2] = c.mz;
    }
    if (nvec) nvec[l - 1] = c.L;
    if (ndof) ndof[l - 1] = c.ncell * c.L;
  }
  return THERMO_OK;
}

extern "C" thermo_status thermo_export_level(thermo_ctx* ctx, int level, int what, double* out, long long count) {
  if (!ctx) return THERMO_EINVAL;
  if (!out || level < 1 || level > ctx->nlev) return fail(ctx, THERMO_EINVAL, "bad level / output");
  if (!ctx->have_precond || ctx->opt.pc != THERMO_PC_MMG) return fail(ctx, THERMO_ESTATE, "no hierarchy yet");
  Lev& lv = ctx->lev[level];
  const CLevel& c = lv.cl;
  cudaStream_t st = ctx->st;
  long long need = 0;
  const double* src = nullptr;
  if (what == 0) {
    if (level == 1) {
      need = ctx->nnode * ctx->L1;
      if (count < need) return fail(ctx, THERMO_EINVAL, "output too small (%lld < %lld)", count, need);
      if (ctx->lean)
        CK(phi_natural<float>(ctx->g, ctx->phi32, ctx->L1, out, st));
      else
        CK(phi_natural<double>(ctx->g, ctx->phi64, ctx->L1, out, st));
      return THERMO_OK;
    }
    need = c.ncell * (long long)c.g * c.g * c.g * ctx->lev[level - 1].cl.L * c.L;
    src = lv.Psi64;
    if (ctx->lean) {  // the FP32 copy, widened
      if (count < need) return fail(ctx, THERMO_EINVAL, "output too small (%lld < %lld)", count, need);
      CK(widen_f32(lv.Psi32, out, need, st));
      return THERMO_OK;
    }
  } else if (what == 1) {
    need = c.ncell * 27 * c.L * c.L;
    src = lv.T64;
    if (!src) {  // lean form: the FP32 tiles, widened
      if (count < need) return fail(ctx, THERMO_EINVAL, "output too small (%lld < %lld)", count, need);
      CK(widen_f32(lv.T32, out, need, st));
      return THERMO_OK;
    }
  } else if (what == 2) {
    need = c.ncell * c.L;
    src = lv.eig;
  } else if (what == 3) {
    if (level != ctx->nlev) return fail(ctx, THERMO_EINVAL, "inverse exists on the coarsest level only");
    need = (long long)ctx->ncoarse * ctx->ncoarse;
    src = ctx->Ainv;
  } else {
    return fail(ctx, THERMO_EINVAL, "unknown item %d", what);
  }
  if (count < need) return fail(ctx, THERMO_EINVAL, "output too small (%lld < %lld)", count, need);
  CK(cudaMemcpyAsync(out, src, need * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_resample(const int grid_c[3], const double* in, const int grid_f[3], double* out,
                                         int kind, void* stream) {
  if (!grid_c || !grid_f || !in || !out || in == out) return THERMO_EINVAL;
  if (kind < 0 || kind > 2) return THERMO_EINVAL;
  for (int k = 0; k < 3; ++k) {
    if (grid_c[k] < 1 || grid_f[k] < grid_c[k] || grid_f[k] % grid_c[k]) return THERMO_EINVAL;
    if (grid_f[k] > (1 << 20)) return THERMO_EINVAL;
  }
  const cudaError_t e = resample_field(grid_c, in, grid_f, out, kind, (cudaStream_t)stream);
  return e == cudaSuccess ? THERMO_OK : THERMO_ECUDA;
}

extern "C" thermo_status thermo_filter(thermo_ctx* ctx, const double* in, double* out, double rmin, int transpose) {
  if (!ctx) return THERMO_EINVAL;
  if (!in || !out || in == out || !(rmin > 0.0)) return fail(ctx, THERMO_EINVAL, "bad filter arguments");
  CK(density_filter(ctx->g.Nx, ctx->g.Ny, ctx->g.Nz, in, out, rmin, transpose, ctx->st));
  return THERMO_OK;
}

extern "C" thermo_status thermo_oc_update(thermo_ctx* ctx, double* x, const double* dc, const double* dv,
                                          double volfrac, double move, double rmin, double* change) {
  if (!ctx) return THERMO_EINVAL;
  if (!x || !dc || !dv || !(volfrac > 0.0) || !(move > 0.0)) return fail(ctx, THERMO_EINVAL, "bad OC arguments");
  const long long M = ctx->nelem;
  cudaStream_t st = ctx->st;
  if (!ctx->colsum) {
    CK(dalloc(ctx, &ctx->colsum, M));
    CK(dalloc(ctx, &ctx->xnew, M));
  }
  if (ctx->rmin_cs != rmin) {
    // column sums of the filter, colsum = H^T 1: the filtered volume is colsum . x / M
    CK(fill_const(ctx->xnew, M, 1.0, st));
    CK(density_filter(ctx->g.Nx, ctx->g.Ny, ctx->g.Nz, ctx->xnew, ctx->colsum, rmin, 1, st));
    ctx->rmin_cs = rmin;
  }
  double l1 = 0.0, l2 = 1e9, vol = 0.0;
  while ((l2 - l1) / (l1 + l2) > 1e-3) {
    const double lmid = 0.5 * (l1 + l2);
    CK(oc_candidate(M, x, dc, dv, ctx->colsum, lmid, move, ctx->xnew, ctx->red, ctx->dscal, st));
    CK(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    vol = ctx->dscal_h[0];
    if (vol > volfrac)
      l1 = lmid;
    else
      l2 = lmid;
  }
  if (change) {
    CK(max_abs_diff(M, x, ctx->xnew, ctx->red, ctx->dscal + 1, st));
    CK(cudaMemcpyAsync(ctx->dscal_h + 1, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *change = ctx->dscal_h[1];
  }
  CK(cudaMemcpyAsync(x, ctx->xnew, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return THERMO_OK;
}

extern "C" long long thermo_launch_count(void) { return thermo::launch_count(); }

extern "C" int thermo_residual_history(const thermo_ctx* ctx, double* out, int max) {
  if (!ctx) return 0;
  const int n = (int)ctx->hist.size();
  if (out)
    for (int i = 0; i < n && i < max; ++i) out[i] = ctx->hist[i];
  return n;
}

extern "C" thermo_status thermo_kernel_timers(thermo_ctx* ctx, int enable) {
  if (!ctx) return THERMO_EINVAL;
  if (!enable) {
    ctx->kt_on = false;
    return THERMO_OK;
  }
  CK(cudaStreamSynchronize(ctx->st));
  for (KTimer& t : ctx->kt) {
    if (t.ev.empty()) {
      t.ev.resize(2 * KTimer::CAP);
      for (cudaEvent_t& e : t.ev) CK(cudaEventCreate(&e));
    }
    t.used = 0;
    t.ms = t.bytes = t.flops = t.pend_bytes = t.pend_flops = 0.0;
    t.launches = 0;
  }
  ctx->kt_on = true;
  return THERMO_OK;
}

extern "C" thermo_status thermo_kernel_time(thermo_ctx* ctx, int kclass, double* ms, long long* launches,
                                            double* bytes, double* flops) {
  if (!ctx) return THERMO_EINVAL;
  if (kclass < 0 || kclass >= THERMO_KT_COUNT) return fail(ctx, THERMO_EINVAL, "kernel class %d out of range", kclass);
  const KTimer& t = ctx->kt[kclass];
  if (ms) *ms = t.ms;
  if (launches) *launches = t.launches;
  if (bytes) *bytes = t.bytes;
  if (flops) *flops = t.flops;
  return THERMO_OK;
}

// Time `reps` back-to-back launches of one internal kernel on the context's
// buffers with CUDA events on the context stream (see thermo.h).
extern "C" thermo_status thermo_bench_kernel(thermo_ctx* ctx, int which, int reps, double* ms_per_launch,
                                             double* bytes_per_launch) {
  if (!ctx || reps < 1 || !ms_per_launch) return THERMO_EINVAL;
  if (!ctx->have_density) return fail(ctx, THERMO_ESTATE, "bench before set_density");
  const bool needs_pc = which == 4 || which == 5 || which == 6 || which == 8 || which == 9;
  if (needs_pc && (!ctx->have_precond || ctx->opt.pc != THERMO_PC_MMG))
    return fail(ctx, THERMO_ESTATE, "kernel %d needs the MMG hierarchy", which);
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->st;
  const double n = (double)ctx->nnode, M = (double)ctx->nelem;
  Lev& l1 = ctx->lev[1];
  const double L1 = ctx->L1;
  double bytes = 0.0;
  auto run = [&]() -> cudaError_t {
    switch (which) {
      case 0:  // the outer CG loop's operator (float-float or FP64, per outer_apply)
        bytes = n * 16 + M * 8;
        return outer_apply_dot(ctx, ctx->p, ctx->q, &ctx->sc->pq);
      case 11:  // FP64-arithmetic apply + dot
        bytes = n * 16 + M * 8;
        return fine_apply_f64(g, ctx->bits, ctx->k64, ctx->p, ctx->q, ctx->red.partial, ctx->red.counter,
                              &ctx->sc->pq, st);
      case 12:  // float-float apply + dot
        bytes = n * 16 + M * 8;
        return fine_apply_ds(g, ctx->bits, ctx->k32, ctx->klo, ctx->p, ctx->q, ctx->red.partial, ctx->red.counter,
                             &ctx->sc->pq, st);
      case 1:
        bytes = n * 8 + M * 4;
        return fine_apply_lp<float>(g, ctx->bits, ctx->k32, ctx->ea32, ctx->eb32, st);
      case 2:
        if (!ctx->ea16) return cudaErrorInvalidValue;
        bytes = n * 4 + M * 2;
        return fine_apply_lp<bf16>(g, ctx->bits, ctx->k16, ctx->ea16, ctx->eb16, st);
      case 3:
        bytes = n * 16 + M * 4;
        return fine_smooth<float, float>(g, ctx->bits, ctx->k32, ctx->r32, ctx->ea32, ctx->ec32, ctx->eb32, 0.3f,
                                         0.6f, st);
      case 4:
        bytes = n * (8 + 4 * L1) + M * 4;
        if (fine3_restrict_supported(g, ctx->L1))
          return fine3_restrict(g, ctx->bits, ctx->k32, ctx->r32, ctx->ea32, ctx->phi32, ctx->tmp32, l1.r32, ctx->L1,
                                st);
        return fine_restrict<float>(g, ctx->bits, ctx->k32, ctx->r32, ctx->ea32, ctx->phi32, l1.r32, ctx->L1, st);
      case 5:
        bytes = n * (8 + 4 * L1);
        return fine_prolong<float>(g, ctx->phi32, l1.e32, ctx->ea32, ctx->L1, st);
      case 6:
        bytes = (double)l1.cl.ncell * (27.0 * l1.cl.L * l1.cl.L + 2.0 * l1.cl.L) * 4.0;
        return coarse_apply<float>(l1.cl, l1.T32, l1.e32, l1.s32, st);
      case 7:
        bytes = n * (8 * 4 + 4 + 8 * 2 + 4);
        return cg_update(g, ctx->tmp, ctx->bv, ctx->p, ctx->q, ctx->z32, 1, ctx->r32, 1, ctx->sc, ctx->red, st);
      case 8: {
        bytes = 0.0;
        const thermo_precision keep = ctx->opt.prec;
        ctx->opt.prec = THERMO_MIXED;
        cudaError_t e = apply_precond(ctx);
        ctx->opt.prec = keep;
        return e;
      }
      case 9: {
        bytes = 0.0;
        if (!ctx->z64 || !ctx->ea64) return cudaErrorInvalidValue;
        const thermo_precision keep = ctx->opt.prec;
        ctx->opt.prec = THERMO_FP64;
        cudaError_t e = apply_precond(ctx);
        ctx->opt.prec = keep;
        return e;
      }
      case 10:
        if (!ctx->ea64) return cudaErrorInvalidValue;
        bytes = n * 32 + M * 8;
        return fine_smooth<double, double>(g, ctx->bits, ctx->k64, ctx->r, ctx->ea64, ctx->ec64, ctx->eb64, 0.3, 0.6,
                                           st);
      default:
        return cudaErrorInvalidValue;
    }
  };
  CK(run());  // warm-up (also sets kernel attributes)
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  for (int i = 0; i < reps; ++i) CK(run());
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_launch = ms / reps;
  if (bytes_per_launch) *bytes_per_launch = bytes;
  return stage_check(ctx);
}

extern "C" thermo_status thermo_dense_spd_inverse(int n, const double* A, double* Ainv, void* stream, int* pivot,
                                                  char* msg, int msg_len) {
  auto say = [&](thermo_status s, const char* fmt, ...) {
    if (msg && msg_len > 0) {
      va_list ap;
      va_start(ap, fmt);
      vsnprintf(msg, (size_t)msg_len, fmt, ap);
      va_end(ap);
    }
    return s;
  };
  if (pivot) *pivot = 0;
  if (msg && msg_len > 0) msg[0] = 0;
  if (n < 1 || n > 20000 || !A || !Ainv) return say(THERMO_EINVAL, "need 1 <= n <= 20000 and device A, Ainv");
  cudaStream_t st = (cudaStream_t)stream;
  double *F = nullptr, *work = nullptr;
  int* status = nullptr;
  int hs = 0;
  thermo_status res = THERMO_OK;
  cudaError_t e = cudaMalloc(&F, (size_t)n * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&work, (size_t)cholesky_work_size(n) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e != cudaSuccess) {
    res = say(THERMO_ENOMEM, "scratch allocation failed: %s", cudaGetErrorString(e));
  } else {
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cholesky_inverse(n, F, Ainv, work, status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      res = say(THERMO_ECUDA, "%s", cudaGetErrorString(e));
    else if (hs != 0) {
      if (pivot) *pivot = hs - 1;
      res = say(THERMO_ESINGULAR, "non-positive pivot at row %d: the matrix is not positive definite", hs - 1);
    }
  }
  cudaFree(F);
  cudaFree(work);
  cudaFree(status);
  return res;
}

extern "C" thermo_status thermo_set_stage_wait(thermo_ctx* ctx, long long cycles) {
  if (!ctx) return THERMO_EINVAL;
  if (cycles < 0) return fail(ctx, THERMO_EINVAL, "the stage wait limit must be >= 0 (0 selects the default)");
  ctx->g.wait = cycles == 0 ? kStageWait : cycles;
  return THERMO_OK;
}

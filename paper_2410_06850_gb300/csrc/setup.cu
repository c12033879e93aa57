// Preconditioner set-up (Sec. 3): local spectral problems, Galerkin coarse
// operators, smoother inverses and the coarsest factorisation.
//
// * Eq. (8) on every level-1 block B (one CTA per block): the Neumann form of
//   the couplings internal to B, Ã_ij = A_ij (i != j in B),
//   Ã_ii = -sum_{j in B} A_ij, against the kappa-weighted lumped mass
//   m_i = sum_{e ∋ i} kappa_e |e|/8.  The L + 8 smallest eigenvectors of
//   C = M^-1/2 Ã M^-1/2 come from the FP32 solver of eigen.cuh (Householder,
//   bisection, inverse iteration); mapped to M^-1/2 v in FP64, M-orthonormalised
//   by Cholesky-QR (twice) and refined by an FP64 Rayleigh-Ritz step on the
//   sparse Ã, of which the L lowest Ritz vectors are kept.
// * Eq. (9) on every group G of g^3 cells of the previous level (one CTA per
//   group): Ã_G = (A_prev)_GG - blockdiag_c P_c^T diag(rho_G) P_c, i.e. the
//   Galerkin block of G minus the projected couplings that leave G (rho_G is
//   the fine row sum restricted to G); with M-orthonormal bases the mass is
//   the identity, so this is a standard eigenproblem over the group's active
//   dofs (same FP32 solver, FP64 Cholesky-QR and Rayleigh-Ritz on the tiles).
// * Galerkin operators A_l = R A_{l-1} R^T as 27-neighbour tiles (FP64).
// * l1-block-Jacobi inverses, dense FP64 Cholesky and explicit inverse of the
//   coarsest operator.
//
// Eigenvector sign convention: the entry of largest magnitude (lowest index
// on ties) is positive.  A cell with fewer admissible vectors than L keeps
// zero vectors in the remaining slots, flagged inactive.
#include <math.h>

#include "common.cuh"
#include "eigen.cuh"
#include "kernels.h"

namespace thermo {

// ---------------------------------------------------------------------------
// CTA-wide helpers (any blockDim that is a multiple of 32)
__device__ double cta_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sh[i];
    sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

// Parallel cyclic Jacobi (round-robin pairing) on a symmetric n2 x n2 matrix A
// (row-major, shared memory), n2 even; accumulates V (A_in = V diag(A_out) V^T).
// Rotation per pair (p, q): tau = (a_qq - a_pp)/(2 a_pq),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c;
// the 2x2 blocks of the pair grid are transformed independently.
template <class T>
__device__ int jacobi_eigen(T* A, T* V, int n2, T* cs, T* sn, int* pp, int* qq, double* sh, int max_sweeps,
                            double tol) {
  const int tid = threadIdx.x, nt = blockDim.x, m = n2 / 2;
  for (int i = tid; i < n2 * n2; i += nt) V[i] = (i / n2 == i % n2) ? T(1) : T(0);
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = tid; i < n2 * n2; i += nt) {
      const double v = (double)A[i];
      if (i / n2 != i % n2)
        off += v * v;
      else if (fabs(v) < 1e30)  // padding / inactive sentinels do not count
        tot += v * v;
    }
    off = cta_sum(off, sh);
    tot = cta_sum(tot, sh);
    if (off <= tol * tol * tot) break;
    for (int s = 0; s < n2 - 1; ++s) {
      for (int k = tid; k < m; k += nt) {
        int p, q;
        if (k == 0) {
          p = n2 - 1;
          q = s;
        } else {
          p = (s + k) % (n2 - 1);
          q = (s - k + n2 - 1) % (n2 - 1);
        }
        const T apq = A[p * n2 + q], app = A[p * n2 + p], aqq = A[q * n2 + q];
        T c = T(1), sv = T(0);
        if (apq != T(0) && fabs((double)apq) > 1e-30 * sqrt(fabs((double)app * (double)aqq))) {
          const T tau = (aqq - app) / (T(2) * apq);
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + t * t);
          sv = t * c;
        }
        cs[k] = c;
        sn[k] = sv;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      for (int w = tid; w < m * m; w += nt) {
        const int k = w / m, l = w - (w / m) * m;
        const int p = pp[k], q = qq[k], r = pp[l], s2 = qq[l];
        const T ck = cs[k], sk = sn[k], cl = cs[l], sl = sn[l];
        const T a_pr = A[p * n2 + r], a_ps = A[p * n2 + s2], a_qr = A[q * n2 + r], a_qs = A[q * n2 + s2];
        const T b_pr = ck * a_pr - sk * a_qr, b_ps = ck * a_ps - sk * a_qs;
        const T b_qr = sk * a_pr + ck * a_qr, b_qs = sk * a_ps + ck * a_qs;
        T c_pr = cl * b_pr - sl * b_ps, c_ps = sl * b_pr + cl * b_ps;
        T c_qr = cl * b_qr - sl * b_qs, c_qs = sl * b_qr + cl * b_qs;
        if (k == l) {
          c_ps = T(0);
          c_qr = T(0);
        }
        A[p * n2 + r] = c_pr;
        A[p * n2 + s2] = c_ps;
        A[q * n2 + r] = c_qr;
        A[q * n2 + s2] = c_qs;
      }
      for (int w = tid; w < n2 * m; w += nt) {
        const int i = w / m, l = w - (w / m) * m;
        const int r = pp[l], s2 = qq[l];
        const T cl = cs[l], sl = sn[l];
        const T vr = V[i * n2 + r], vs = V[i * n2 + s2];
        V[i * n2 + r] = cl * vr - sl * vs;
        V[i * n2 + s2] = sl * vr + cl * vs;
      }
      __syncthreads();
    }
  }
  return sweep;
}

// indices of the k smallest diagonal entries of A (ascending; ties -> lower index)
template <class T>
__device__ void select_smallest(const T* A, int n2, int k, int* sel) {
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    const T li = A[i * n2 + i];
    int rank = 0;
    for (int j = 0; j < n2; ++j) {
      const T lj = A[j * n2 + j];
      rank += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    if (rank < k) sel[rank] = i;
  }
  __syncthreads();
}

// Adaptive local basis (the GMsFEM-style alternative to a fixed L): of the k
// ascending Ritz values lam, the count with lam <= thr (thr = tau / H^2 of the
// level), at least one; thr <= 0 keeps k.  Every thread computes the same count
// from shared memory.
__device__ __forceinline__ int kept_count(const double* lam, int k, double thr) {
  if (!(thr > 0.0) || k == 0) return k;
  int c = 0;
  while (c < k && lam[c] <= thr) ++c;
  return c > 0 ? c : 1;
}

// Rayleigh-Ritz finish on an FP64 basis X[n][ld] (k columns, M-orthonormal):
// H = X^T W (W = Ã X) is diagonalised (FP64 Jacobi), X <- X Y sorted by
// eigenvalue, sign-fixed.  Scratch in shared memory.
__device__ void rr_finish(double* X, const double* W, int n, int ld, int k, double* H, double* Y, double* cs,
                          double* sn, int* pp, int* qq, double* sh, double* tmp, double* lam, int* sel) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int k2 = (k + 1) & ~1;
  for (int w = tid; w < k2 * k2; w += nt) {
    const int a = w / k2, b = w % k2;
    double s = 0.0;
    if (a < k && b < k) {
      for (int i = 0; i < n; ++i) s += X[i * ld + a] * W[i * ld + b];
    } else if (a == b) {
      s = 1e300;  // padding column, never selected
    }
    H[w] = s;
  }
  __syncthreads();
  // symmetrise
  for (int w = tid; w < k2 * k2; w += nt) {
    const int a = w / k2, b = w % k2;
    if (a < b && a < k && b < k) {
      const double v = 0.5 * (H[a * k2 + b] + H[b * k2 + a]);
      H[a * k2 + b] = v;
      H[b * k2 + a] = v;
    }
  }
  __syncthreads();
  jacobi_eigen<double>(H, Y, k2, cs, sn, pp, qq, sh, 30, 1e-15);
  select_smallest<double>(H, k2, k, sel);
  for (int w = tid; w < n * k; w += nt) {
    const int i = w / k, a = w % k;
    double s = 0.0;
    for (int b = 0; b < k; ++b) s += X[i * ld + b] * Y[b * k2 + sel[a]];
    tmp[i * ld + a] = s;
  }
  __syncthreads();
  for (int w = tid; w < n * k; w += nt) {
    const int i = w / k, a = w % k;
    X[i * ld + a] = tmp[i * ld + a];
  }
  if (tid < k) lam[tid] = H[sel[tid] * k2 + sel[tid]];
  __syncthreads();
  // sign: largest |entry| (lowest index on ties) positive
  if (tid < k) {
    double best = -1.0;
    int bi = 0;
    for (int i = 0; i < n; ++i) {
      const double v = fabs(X[i * ld + tid]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    tmp[tid] = X[bi * ld + tid] < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  for (int w = tid; w < n * k; w += nt) {
    const int i = w / k, a = w % k;
    X[i * ld + a] *= tmp[a];
  }
  __syncthreads();
}

// Cholesky-QR, twice, of the k columns of X[n][ld] in <a,b> = sum m_i a_i b_i
// (m == nullptr: Euclidean): G = X^T M X, G = R^T R (one thread, FP64),
// X <- X R^-1 (a thread per row).  Three barriers per pass instead of two per
// pair of columns; the columns come from an eigensolver and are nearly
// orthonormal, for which Cholesky-QR is stable.  A column whose pivot vanishes
// (numerically dependent) is set to zero.  G: k x k doubles of scratch.
__device__ void cholqr(double* X, const double* m, int n, int ld, int k, double* G) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int pass = 0; pass < 2; ++pass) {
    for (int w = tid; w < k * k; w += nt) {
      const int a = w / k, b = w % k;
      if (b < a) continue;
      double s = 0.0;
      for (int r = 0; r < n; ++r) s += (m ? m[r] : 1.0) * X[r * ld + a] * X[r * ld + b];
      G[a * k + b] = s;
    }
    __syncthreads();
    if (tid == 0) {
      for (int a = 0; a < k; ++a) {
        double dgn = G[a * k + a];
        for (int c = 0; c < a; ++c) dgn -= G[c * k + a] * G[c * k + a];
        const double ref = G[a * k + a];
        if (!(dgn > 1e-24 * (ref > 0.0 ? ref : 1.0))) {  // dependent column: zero it
          G[a * k + a] = 0.0;
          for (int b = a + 1; b < k; ++b) G[a * k + b] = 0.0;
          continue;
        }
        const double rd = sqrt(dgn);
        G[a * k + a] = rd;
        for (int b = a + 1; b < k; ++b) {
          double v = G[a * k + b];
          for (int c = 0; c < a; ++c) v -= G[c * k + a] * G[c * k + b];
          G[a * k + b] = v / rd;
        }
      }
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
      double* x = X + r * ld;
      for (int a = 0; a < k; ++a) {
        double v = x[a];
        for (int c = 0; c < a; ++c) v -= x[c] * G[c * k + a];
        x[a] = G[a * k + a] > 0.0 ? v / G[a * k + a] : 0.0;
      }
    }
    __syncthreads();
  }
}

// fine-grid coupling A_ij between node (x,y,z) and (x+ox, y+oy, z+oz), i != j
__device__ __forceinline__ double coupling(const Geom& g, const double* k64, int x, int y, int z, int ox, int oy,
                                           int oz) {
  double s = 0.0;
  const int exa = ox == 0 ? x - 1 : (ox < 0 ? x - 1 : x), exb = ox == 0 ? x : exa;
  const int eya = oy == 0 ? y - 1 : (oy < 0 ? y - 1 : y), eyb = oy == 0 ? y : eya;
  const int eza = oz == 0 ? z - 1 : (oz < 0 ? z - 1 : z), ezb = oz == 0 ? z : eza;
  for (int ez = eza; ez <= ezb; ++ez)
    for (int ey = eya; ey <= eyb; ++ey)
      for (int ex = exa; ex <= exb; ++ex) s += k64[eidx(g, ex, ey, ez)];
  const int pat = (ox != 0 ? 1 : 0) | (oy != 0 ? 2 : 0) | (oz != 0 ? 4 : 0);
  return g.c[pat] * s;
}
__device__ __forceinline__ double kappa_sum8(const Geom& g, const double* k64, int x, int y, int z) {
  double s = 0.0;
  for (int dz = -1; dz <= 0; ++dz)
    for (int dy = -1; dy <= 0; ++dy)
      for (int dx = -1; dx <= 0; ++dx) s += k64[eidx(g, x + dx, y + dy, z + dz)];
  return s;
}

// ---------------------------------------------------------------------------
// Eq. (8): level-1 bases.  Blocks are launched per class (last in x/y/z or
// not) so that the shared-memory footprint matches the block's node count.
constexpr int EIG_NT = 256;
constexpr int EIG_EXTRA = 8;  // Ritz vectors beyond L carried into the FP64 refinement

struct L1Smem {
  // offsets in bytes
  size_t C, Y, X, W, m, rs, A26, J26, H, Yr, cs64, sn64, pp, qq, sel, list, lmap, lam, lam32, scr, sh, total;
};
__host__ __device__ inline L1Smem l1_smem(int n2, int K, int nmap) {
  L1Smem s;
  size_t o = 0;
  auto al = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 15) & ~(size_t)15;
    return r;
  };
  const int k2 = (K + 1) & ~1;
  s.C = al((size_t)n2 * (n2 + 1) * 4);
  s.Y = al((size_t)K * n2 * 4);
  // X and W are contiguous: the FP32 eigensolver's factor storage aliases them
  s.X = al((size_t)n2 * K * 8);
  s.W = al((size_t)n2 * K * 8 + 8 * 64);
  s.m = al((size_t)n2 * 8);
  s.rs = al((size_t)n2 * 8);
  s.A26 = al((size_t)n2 * 26 * 8);
  s.J26 = al((size_t)n2 * 26);
  s.H = al((size_t)k2 * k2 * 8);
  s.Yr = al((size_t)k2 * k2 * 8);
  s.cs64 = al((size_t)k2 * 8);
  s.sn64 = al((size_t)k2 * 8);
  s.pp = al((size_t)k2 * 4);
  s.qq = al((size_t)k2 * 4);
  s.sel = al((size_t)k2 * 4);
  s.list = al((size_t)n2 * 4);
  s.lmap = al((size_t)nmap * 4);
  s.lam = al((size_t)k2 * 8);
  s.lam32 = al((size_t)k2 * 4);
  s.scr = al(eig_scratch_floats(n2) * 4);
  s.sh = al(40 * 8);
  s.total = o;
  return s;
}

// One CTA per block: assemble C = M^-1/2 Ã M^-1/2 (FP32) over the block's free
// nodes, take its K = L + 8 smallest eigenvectors with the FP32 solver of
// eigen.cuh, map them to phi = M^-1/2 v in FP64, M-orthonormalise (FP64 MGS)
// and refine by an FP64 Rayleigh-Ritz step on the sparse Ã; keep the L lowest.
__global__ void __launch_bounds__(EIG_NT) k_level1_eigen(Geom g, const uint32_t* __restrict__ bits,
                                                         const double* __restrict__ k64, int L, int lx, int ly, int lz,
                                                         int n2, double* __restrict__ phi, double* __restrict__ eig,
                                                         uint8_t* __restrict__ act, int* status, double thr) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = g.b;
  const int cxn = lx ? 1 : g.nbx - 1, cyn = ly ? 1 : g.nby - 1;
  int bid = blockIdx.x;
  const int ix = bid % cxn;
  bid /= cxn;
  const int iy = bid % cyn, iz = bid / cyn;
  const int bx = lx ? g.nbx - 1 : ix, by = ly ? g.nby - 1 : iy, bz = lz ? g.nbz - 1 : iz;
  const int wx = b + lx, wy = b + ly, wz = b + lz;  // nodes per axis of this block
  const int X0 = bx * b, Y0 = by * b, Z0 = bz * b;
  const int nmap = wx * wy * wz;
  const int Kmax = (L + EIG_EXTRA) < n2 ? (L + EIG_EXTRA) : n2;
  L1Smem S = l1_smem(n2, Kmax, nmap);
  const int lda = n2 + 1;
  float* C = (float*)(sm + S.C);
  float* Yf = (float*)(sm + S.Y);
  double* X = (double*)(sm + S.X);
  double* W = (double*)(sm + S.W);
  double* m = (double*)(sm + S.m);
  double* rs = (double*)(sm + S.rs);       // m^-1/2
  double* A26 = (double*)(sm + S.A26);     // couplings A_ij to the 26 neighbours (FP64), once per block
  signed char* J26 = (signed char*)(sm + S.J26);  // their compact indices (-1: outside / Dirichlet)
  double* H = (double*)(sm + S.H);
  double* Yr = (double*)(sm + S.Yr);
  double* cs64 = (double*)(sm + S.cs64);
  double* sn64 = (double*)(sm + S.sn64);
  int* pp = (int*)(sm + S.pp);
  int* qq = (int*)(sm + S.qq);
  int* sel = (int*)(sm + S.sel);
  int* list = (int*)(sm + S.list);
  int* lmap = (int*)(sm + S.lmap);
  double* lam = (double*)(sm + S.lam);
  float* lam32 = (float*)(sm + S.lam32);
  float* scr = (float*)(sm + S.scr);
  double* sh = (double*)(sm + S.sh);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long cell = bx + (long long)g.nbx * (by + (long long)g.nby * bz);

  // compact list of free nodes (natural order within the block), serial for determinism
  if (tid == 0) {
    int n = 0;
    for (int k = 0; k < nmap; ++k) {
      const int x = X0 + k % wx, y = Y0 + (k / wx) % wy, z = Z0 + k / (wx * wy);
      if (!is_dir(g, bits, x, y, z)) {
        lmap[k] = n;
        list[n++] = k;
      } else {
        lmap[k] = -1;
      }
    }
    sh[34] = (double)n;
  }
  __syncthreads();
  const int n = (int)sh[34];
  int kk = n < L ? n : L;
  const int K = n < Kmax ? n : Kmax;
  // mass, its inverse square root, and the couplings to the 26 neighbours (FP64, once)
  for (int i = tid; i < n; i += nt) {
    const int k = list[i];
    const int x = X0 + k % wx, y = Y0 + (k / wx) % wy, z = Z0 + k / (wx * wy);
    m[i] = kappa_sum8(g, k64, x, y, z) * g.vol * 0.125;
    rs[i] = 1.0 / sqrt(m[i]);
    int o = 0;
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          const int xx = x + ox - X0, yy = y + oy - Y0, zz = z + oz - Z0;
          int j = -1;
          if (xx >= 0 && yy >= 0 && zz >= 0 && xx < wx && yy < wy && zz < wz) j = lmap[xx + wx * (yy + wy * zz)];
          J26[i * 26 + o] = (signed char)j;
          A26[i * 26 + o] = j >= 0 ? coupling(g, k64, x, y, z, ox, oy, oz) : 0.0;
          ++o;
        }
  }
  for (int i = tid; i < n * lda; i += nt) C[i] = 0.f;
  __syncthreads();
  // the Neumann matrix scaled by M^-1/2 (FP32 entries from FP64 couplings and scales)
  for (int i = tid; i < n; i += nt) {
    double diag = 0.0;
    const float ri = (float)rs[i];
    for (int o = 0; o < 26; ++o) {
      const int j = J26[i * 26 + o];
      if (j < 0) continue;
      const double a = A26[i * 26 + o];
      diag -= a;
      C[i * lda + j] = (float)a * ri * (float)rs[j];
    }
    C[i * lda + i] = (float)(diag * rs[i] * rs[i]);
  }
  __syncthreads();
  if (n > 0) eig_lowest(C, lda, n, K, lam32, Yf, n2, scr, (float*)X, sh);
  // FP64 basis phi = M^-1/2 v over the K vectors, M-orthonormalised
  for (int w = tid; w < n * K; w += nt) {
    const int i = w / K, a = w % K;
    X[w] = (double)Yf[a * n2 + i] * rs[i];
  }
  __syncthreads();
  cholqr(X, m, n, K, K, H);
  // W = Ã X (difference form: (Ã x)_i = sum_{j in B} A_ij (x_j - x_i)), one (row, vector) item per thread
  for (int w = tid; w < n * K; w += nt) {
    const int i = w / K, a = w - (w / K) * K;
    const double xi = X[i * K + a];
    double acc = 0.0;
    for (int o = 0; o < 26; ++o) {
      const int j = J26[i * 26 + o];
      if (j < 0) continue;
      acc += A26[i * 26 + o] * (X[j * K + a] - xi);
    }
    W[w] = acc;
  }
  __syncthreads();
  // Rayleigh-Ritz on span(X): sorted Ritz pairs in X, lam (W reused as scratch)
  if (K > 0) rr_finish(X, W, n, K, K, H, Yr, cs64, sn64, pp, qq, sh, W, lam, sel);
  kk = kept_count(lam, kk, thr);
  // outputs: the L lowest (the adaptive count of them when thr > 0)
  for (int k = tid; k < nmap; k += nt) {
    const int x = X0 + k % wx, y = Y0 + (k / wx) % wy, z = Z0 + k / (wx * wy);
    const int i = lmap[k];
    const long long nd = nidx(g, x, y, z);
    for (int a = 0; a < L; ++a) phi[nd * L + a] = (i >= 0 && a < kk) ? X[i * K + a] : 0.0;
  }
  if (tid < L) {
    eig[cell * L + tid] = tid < kk ? lam[tid] : 0.0;
    act[cell * L + tid] = tid < kk ? 1 : 0;
  }
}

cudaError_t level1_eigen(const Geom& g, const uint32_t* bits, const double* k64, int L1, double* phi64, double* eig,
                         uint8_t* active, int* status, double thr, cudaStream_t st) {
  for (int lz = 0; lz < 2; ++lz)
    for (int ly = 0; ly < 2; ++ly)
      for (int lx = 0; lx < 2; ++lx) {
        const int cx = lx ? 1 : g.nbx - 1, cy = ly ? 1 : g.nby - 1, cz = lz ? 1 : g.nbz - 1;
        const long long nb = (long long)cx * cy * cz;
        if (nb <= 0) continue;
        const int nmap = (g.b + lx) * (g.b + ly) * (g.b + lz);
        const int n2 = (nmap + 1) & ~1;
        const int Kmax = (L1 + EIG_EXTRA) < n2 ? (L1 + EIG_EXTRA) : n2;
        const L1Smem S = l1_smem(n2, Kmax, nmap);
        if (S.total > 227 * 1024 || eig_lu_floats(n2, Kmax) * 4 > 2 * (size_t)n2 * Kmax * 8) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(k_level1_eigen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S.total);
        if (e != cudaSuccess) return e;
        note_launch(), k_level1_eigen<<<(unsigned)nb, EIG_NT, S.total, st>>>(g, bits, k64, L1, lx, ly, lz, n2, phi64,
                                                                             eig, active, status, thr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Row-sum corrections for the coarse-coarse problems (Eq. (9)):
// D[t][B] = sum_{i in B} rho_i^(t) phi_i phi_i^T, with rho_i^(t) the sum of the
// couplings of node i that leave its level-t cell or reach a Dirichlet node
// (= sum_{j in cell_t(i), j free} A_ij, since the Neumann rows sum to zero).
__global__ void k_level1_corr(Geom g, const uint32_t* __restrict__ bits, const double* __restrict__ k64, int L,
                              const double* __restrict__ phi, int nt_lv, const int* __restrict__ gcum,
                              double* __restrict__ D) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = g.b;
  const long long cell = blockIdx.x;
  const int bx = (int)(cell % g.nbx), by = (int)((cell / g.nbx) % g.nby), bz = (int)(cell / ((long long)g.nbx * g.nby));
  const int wx = b + (bx == g.nbx - 1), wy = b + (by == g.nby - 1), wz = b + (bz == g.nbz - 1);
  const int nmap = wx * wy * wz;
  double* contrib = (double*)sm;  // [nmap][L*L]
  for (int t = 0; t < nt_lv; ++t) {
    const int G = gcum[t];
    for (int k = threadIdx.x; k < nmap; k += blockDim.x) {
      const int x = bx * b + k % wx, y = by * b + (k / wx) % wy, z = bz * b + k / (wx * wy);
      double rho = 0.0;
      if (!is_dir(g, bits, x, y, z)) {
        const int cxi = bx / G, cyi = by / G, czi = bz / G;
        for (int oz = -1; oz <= 1; ++oz)
          for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
              if (!ox && !oy && !oz) continue;
              const int xx = x + ox, yy = y + oy, zz = z + oz;
              if (xx < 0 || yy < 0 || zz < 0 || xx > g.Nx || yy > g.Ny || zz > g.Nz) continue;
              const bool same = !is_dir(g, bits, xx, yy, zz) && blk_of(xx, b, g.nbx) / G == cxi &&
                                blk_of(yy, b, g.nby) / G == cyi && blk_of(zz, b, g.nbz) / G == czi;
              if (!same) rho -= coupling(g, k64, x, y, z, ox, oy, oz);
            }
      }
      const long long nd = nidx(g, x, y, z);
      for (int a = 0; a < L; ++a)
        for (int c = 0; c < L; ++c) contrib[k * L * L + a * L + c] = rho * phi[nd * L + a] * phi[nd * L + c];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < L * L; o += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < nmap; ++k) s += contrib[k * L * L + o];
      D[((long long)t * g.nbx * g.nby * g.nbz + cell) * L * L + o] = s;
    }
    __syncthreads();
  }
}
cudaError_t level1_rowsum_corr(const Geom& g, const uint32_t* bits, const double* k64, int L1, const double* phi64,
                               int nt, const int* gcum, double* D, cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  const int nmap = (g.b + 1) * (g.b + 1) * (g.b + 1);
  const size_t sm = (size_t)nmap * L1 * L1 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_level1_corr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  note_launch(), k_level1_corr<<<(unsigned)((long long)g.nbx * g.nby * g.nbz), 128, sm, st>>>(g, bits, k64, L1, phi64, nt, gcum, D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Level-1 Galerkin tiles: for block B, Y = A Phi_B on the one-node ring
// around B, then tile(B', B) = Phi_{B'}^T Y for the 27 neighbours B', stored
// in B''s row (its neighbour index points back at B).  FP64 sums; TO is the
// stored type (FP32 when the hierarchy is kept in FP32 only).
template <class TO>
__global__ void k_level1_rap(Geom g, const uint32_t* __restrict__ bits, const double* __restrict__ k64, int L,
                             const double* __restrict__ phi, TO* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = g.b;
  const long long cell = blockIdx.x;
  const int bx = (int)(cell % g.nbx), by = (int)((cell / g.nbx) % g.nby), bz = (int)(cell / ((long long)g.nbx * g.nby));
  const int wx = b + (bx == g.nbx - 1), wy = b + (by == g.nby - 1), wz = b + (bz == g.nbz - 1);
  const int X0 = bx * b, Y0 = by * b, Z0 = bz * b;
  const int rx = wx + 2, ry = wy + 2, rz = wz + 2, nreg = rx * ry * rz;
  double* Yv = (double*)sm;  // [nreg][L]
  for (int k = threadIdx.x; k < nreg; k += blockDim.x) {
    const int x = X0 - 1 + k % rx, y = Y0 - 1 + (k / rx) % ry, z = Z0 - 1 + k / (rx * ry);
    double acc[32];
    for (int a = 0; a < L; ++a) acc[a] = 0.0;
    const bool inside = x >= 0 && y >= 0 && z >= 0 && x <= g.Nx && y <= g.Ny && z <= g.Nz;
    if (inside && !is_dir(g, bits, x, y, z)) {
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int xx = x + ox, yy = y + oy, zz = z + oz;
            if (xx < X0 || yy < Y0 || zz < Z0 || xx >= X0 + wx || yy >= Y0 + wy || zz >= Z0 + wz) continue;
            if (is_dir(g, bits, xx, yy, zz)) continue;
            double aij;
            if (!ox && !oy && !oz)
              aij = g.c[0] * kappa_sum8(g, k64, x, y, z);
            else
              aij = coupling(g, k64, x, y, z, ox, oy, oz);
            const long long nd = nidx(g, xx, yy, zz);
            for (int a = 0; a < L; ++a) acc[a] += aij * phi[nd * L + a];
          }
    }
    for (int a = 0; a < L; ++a) Yv[k * L + a] = acc[a];
  }
  __syncthreads();
  // outputs: for each neighbour offset (dx,dy,dz) of B' relative to B
  for (int o = threadIdx.x; o < 27 * L * L; o += blockDim.x) {
    const int n = o / (L * L), a = (o / L) % L, kcol = o % L;
    const int dx = n % 3 - 1, dy = (n / 3) % 3 - 1, dz = n / 9 - 1;
    const int nbx = bx + dx, nby = by + dy, nbz = bz + dz;
    if (nbx < 0 || nby < 0 || nbz < 0 || nbx >= g.nbx || nby >= g.nby || nbz >= g.nbz) continue;
    // region positions belonging to B'
    const int xa = dx < 0 ? 0 : (dx == 0 ? 1 : rx - 1), xb = dx < 0 ? 1 : (dx == 0 ? rx - 1 : rx);
    const int ya = dy < 0 ? 0 : (dy == 0 ? 1 : ry - 1), yb = dy < 0 ? 1 : (dy == 0 ? ry - 1 : ry);
    const int za = dz < 0 ? 0 : (dz == 0 ? 1 : rz - 1), zb = dz < 0 ? 1 : (dz == 0 ? rz - 1 : rz);
    double s = 0.0;
    for (int zz = za; zz < zb; ++zz)
      for (int yy = ya; yy < yb; ++yy)
        for (int xx = xa; xx < xb; ++xx) {
          const int x = X0 - 1 + xx, y = Y0 - 1 + yy, z = Z0 - 1 + zz;
          const long long nd = nidx(g, x, y, z);
          s += phi[nd * L + a] * Yv[(xx + rx * (yy + ry * zz)) * L + kcol];
        }
    const long long nc = nbx + (long long)g.nbx * (nby + (long long)g.nby * nbz);
    const int back = (1 - dx) + 3 * (1 - dy) + 9 * (1 - dz);
    tiles[((nc * 27 + back) * L + a) * L + kcol] = (TO)s;
  }
}
template <class TO>
cudaError_t level1_rap(const Geom& g, const uint32_t* bits, const double* k64, int L1, const double* phi64,
                       TO* tiles, cudaStream_t st) {
  const int r = g.b + 3;
  const size_t sm = (size_t)r * r * r * L1 * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_level1_rap<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  note_launch(),
      k_level1_rap<TO><<<(unsigned)((long long)g.nbx * g.nby * g.nbz), 128, sm, st>>>(g, bits, k64, L1, phi64, tiles);
  return cudaGetLastError();
}
template cudaError_t level1_rap<double>(const Geom&, const uint32_t*, const double*, int, const double*, double*,
                                        cudaStream_t);
template cudaError_t level1_rap<float>(const Geom&, const uint32_t*, const double*, int, const double*, float*,
                                       cudaStream_t);

// ---------------------------------------------------------------------------
// Eq. (9): one CTA per group G of g^3 cells of the previous level.
struct GSmem {
  size_t C, Y, X, W, H, Yr, cs64, sn64, pp, qq, sel, alist, amap, lam, lam32, scr, sh, total;
};
__host__ __device__ inline GSmem g_smem(int n2, int K) {
  GSmem s;
  size_t o = 0;
  auto al = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 15) & ~(size_t)15;
    return r;
  };
  const int k2 = (K + 1) & ~1;
  s.C = al((size_t)n2 * (n2 + 1) * 4);
  s.Y = al((size_t)K * n2 * 4);
  s.X = al((size_t)n2 * K * 8);  // X, W contiguous (aliased by the FP32 solver's factors)
  s.W = al((size_t)n2 * K * 8 + 8 * 64);
  s.H = al((size_t)k2 * k2 * 8);
  s.Yr = al((size_t)k2 * k2 * 8);
  s.cs64 = al((size_t)k2 * 8);
  s.sn64 = al((size_t)k2 * 8);
  s.pp = al((size_t)k2 * 4);
  s.qq = al((size_t)k2 * 4);
  s.sel = al((size_t)k2 * 4);
  s.alist = al((size_t)n2 * 4);
  s.amap = al((size_t)n2 * 4);
  s.lam = al((size_t)k2 * 8);
  s.lam32 = al((size_t)k2 * 4);
  s.scr = al(eig_scratch_floats(n2) * 4);
  s.sh = al(40 * 8);
  s.total = o;
  return s;
}

__device__ __forceinline__ long long cell_of_local(const CLevel& prev, const CLevel& cur, long long G, int lc) {
  const int g = cur.g;
  const int gx = (int)(G % cur.mx), gy = (int)((G / cur.mx) % cur.my), gz = (int)(G / ((long long)cur.mx * cur.my));
  const int lx = lc % g, ly = (lc / g) % g, lz = lc / (g * g);
  return (gx * g + lx) + (long long)prev.mx * ((gy * g + ly) + (long long)prev.my * (gz * g + lz));
}
__device__ __forceinline__ int nbr_index(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }

// One CTA per group: Ã_G over the group's active dofs (FP32, symmetrised), its
// K = L + 8 smallest eigenvectors with the FP32 solver of eigen.cuh, FP64
// Gram-Schmidt and an FP64 Rayleigh-Ritz step on Ã_G from the FP64 tiles;
// the L lowest form Psi (mass = identity: the "mass trick" after Eq. (9)).
// TI: the stored type of the previous level's tiles (widened on load).
template <class TI>
__global__ void __launch_bounds__(EIG_NT) k_group_eigen(CLevel prev, CLevel cur, const TI* __restrict__ Tp,
                                                        const double* __restrict__ Dc, const uint8_t* __restrict__ actp,
                                                        int n2, double* __restrict__ Psi, double* __restrict__ eig,
                                                        uint8_t* __restrict__ actc, double thr) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int g = cur.g, Lp = prev.L, L = cur.L, ng = g * g * g, n = ng * Lp;
  const int Kmax = (L + EIG_EXTRA) < n2 ? (L + EIG_EXTRA) : n2;
  GSmem S = g_smem(n2, Kmax);
  const int lda = n2 + 1;
  float* C = (float*)(sm + S.C);
  float* Yf = (float*)(sm + S.Y);
  double* X = (double*)(sm + S.X);
  double* W = (double*)(sm + S.W);
  double* H = (double*)(sm + S.H);
  double* Yr = (double*)(sm + S.Yr);
  double* cs64 = (double*)(sm + S.cs64);
  double* sn64 = (double*)(sm + S.sn64);
  int* pp = (int*)(sm + S.pp);
  int* qq = (int*)(sm + S.qq);
  int* sel = (int*)(sm + S.sel);
  int* alist = (int*)(sm + S.alist);
  int* amap = (int*)(sm + S.amap);  // local dof -> compact active index (-1: inactive)
  double* lam = (double*)(sm + S.lam);
  float* lam32 = (float*)(sm + S.lam32);
  float* scr = (float*)(sm + S.scr);
  double* sh = (double*)(sm + S.sh);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long G = blockIdx.x;
  // compact list of active dofs (local dof order), serial for determinism
  if (tid == 0) {
    int na = 0;
    for (int d = 0; d < n; ++d) {
      const long long c = cell_of_local(prev, cur, G, d / Lp);
      amap[d] = -1;
      if (actp[c * Lp + d % Lp]) amap[d] = na, alist[na++] = d;
    }
    sh[34] = na;
  }
  __syncthreads();
  const int na = (int)sh[34];
  int kk = na < L ? na : L;
  const int K = na < Kmax ? na : Kmax;
  // row ia of Ã_G, one neighbouring cell lcj per thread item: the tile row and the
  // correction row are located once, then the Lp entries are read in order
  auto tile_row = [&](int di, int lcj, const TI*& T, const double*& D) {
    const int lci = di / Lp, i = di % Lp;
    const int dx = lcj % g - lci % g, dy = (lcj / g) % g - (lci / g) % g, dz = lcj / (g * g) - lci / (g * g);
    T = nullptr;
    D = nullptr;
    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return;
    const long long c = cell_of_local(prev, cur, G, lci);
    T = Tp + ((c * 27 + nbr_index(dx, dy, dz)) * Lp + i) * Lp;
    if (lci == lcj) D = Dc + (c * Lp + i) * Lp;
  };
  for (int w = tid; w < na * ng; w += nt) {
    const int ia = w / ng, lcj = w % ng;
    const TI* T;
    const double* D;
    tile_row(alist[ia], lcj, T, D);
    for (int j = 0; j < Lp; ++j) {
      const int ja = amap[lcj * Lp + j];
      if (ja < 0) continue;
      C[ia * lda + ja] = T ? (float)((double)T[j] - (D ? D[j] : 0.0)) : 0.f;
    }
  }
  __syncthreads();
  // symmetrise (the FP64 tiles are symmetric up to rounding)
  for (int w = tid; w < na * na; w += nt) {
    const int a = w / na, bcol = w % na;
    if (a < bcol) {
      const float v = 0.5f * (C[a * lda + bcol] + C[bcol * lda + a]);
      C[a * lda + bcol] = v;
      C[bcol * lda + a] = v;
    }
  }
  __syncthreads();
  if (na > 0) eig_lowest(C, lda, na, K, lam32, Yf, n2, scr, (float*)X, sh);
  for (int w = tid; w < na * K; w += nt) {
    const int i = w / K, a = w % K;
    X[w] = (double)Yf[a * n2 + i];
  }
  __syncthreads();
  cholqr(X, nullptr, na, K, K, H);
  // W = Ã_G X in FP64 from the tiles (active rows and columns)
  for (int w = tid; w < na * K; w += nt) {
    const int ia = w / K, a = w % K;
    const int di = alist[ia];
    double sacc = 0.0;
    for (int lcj = 0; lcj < ng; ++lcj) {
      const TI* T;
      const double* D;
      tile_row(di, lcj, T, D);
      if (!T) continue;
      for (int j = 0; j < Lp; ++j) {
        const int ja = amap[lcj * Lp + j];
        if (ja < 0) continue;
        sacc += ((double)T[j] - (D ? D[j] : 0.0)) * X[ja * K + a];
      }
    }
    W[w] = sacc;
  }
  __syncthreads();
  if (K > 0) rr_finish(X, W, na, K, K, H, Yr, cs64, sn64, pp, qq, sh, W, lam, sel);
  kk = kept_count(lam, kk, thr);
  // Psi rows in local dof order (inactive rows zero), the L lowest columns (adaptive count when thr > 0)
  double* out = Psi + G * (long long)n * L;
  for (int w = tid; w < n * L; w += nt) out[w] = 0.0;
  __syncthreads();
  for (int w = tid; w < na * L; w += nt) {
    const int ia = w / L, a = w % L;
    out[alist[ia] * L + a] = a < kk ? X[ia * K + a] : 0.0;
  }
  if (tid < L) {
    eig[G * L + tid] = tid < kk ? lam[tid] : 0.0;
    actc[G * L + tid] = tid < kk ? 1 : 0;
  }
}
template <class TI>
cudaError_t group_eigen(const CLevel& prev, const CLevel& cur, const TI* tiles_prev, const double* Dcorr,
                        const uint8_t* act_prev, double* Psi, double* eig, uint8_t* act_cur, int* status, double thr,
                        cudaStream_t st) {
  const int n = cur.g * cur.g * cur.g * prev.L;
  const int n2 = (n + 1) & ~1;
  const int Kmax = (cur.L + EIG_EXTRA) < n2 ? (cur.L + EIG_EXTRA) : n2;
  const GSmem S = g_smem(n2, Kmax);
  if (S.total > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_group_eigen<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total);
  if (e != cudaSuccess) return e;
  note_launch(), k_group_eigen<TI><<<(unsigned)cur.ncell, EIG_NT, S.total, st>>>(prev, cur, tiles_prev, Dcorr, act_prev,
                                                                                 n2, Psi, eig, act_cur, thr);
  return cudaGetLastError();
}
template cudaError_t group_eigen<double>(const CLevel&, const CLevel&, const double*, const double*, const uint8_t*,
                                         double*, double*, uint8_t*, int*, double, cudaStream_t);
template cudaError_t group_eigen<float>(const CLevel&, const CLevel&, const float*, const double*, const uint8_t*,
                                        double*, double*, uint8_t*, int*, double, cudaStream_t);

// D_G^(t) = Psi_G^T blockdiag_{c in G}(D_c^(t)) Psi_G for every later level t
__global__ void k_group_corr(CLevel prev, CLevel cur, const double* __restrict__ Psi, const double* __restrict__ Dp,
                             double* __restrict__ Dcur, int nt_lv) {
  const int g = cur.g, Lp = prev.L, L = cur.L, ng = g * g * g, n = ng * Lp;
  const long long G = blockIdx.x;
  const double* ps = Psi + G * (long long)n * L;
  for (int o = threadIdx.x; o < nt_lv * L * L; o += blockDim.x) {
    const int t = o / (L * L), a = (o / L) % L, bb = o % L;
    double s = 0.0;
    for (int lc = 0; lc < ng; ++lc) {
      const long long c = cell_of_local(prev, cur, G, lc);
      const double* D = Dp + ((long long)t * prev.ncell + c) * Lp * Lp;
      for (int i = 0; i < Lp; ++i) {
        double u = 0.0;
        for (int j = 0; j < Lp; ++j) u += D[i * Lp + j] * ps[(lc * Lp + j) * L + bb];
        s += ps[(lc * Lp + i) * L + a] * u;
      }
    }
    Dcur[((long long)t * cur.ncell + G) * L * L + a * L + bb] = s;
  }
}
cudaError_t group_project_corr(const CLevel& prev, const CLevel& cur, const double* Psi, const double* Dprev,
                               double* Dcur, int nt, cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  note_launch(), k_group_corr<<<(unsigned)cur.ncell, 128, 0, st>>>(prev, cur, Psi, Dprev + prev.ncell * prev.L * prev.L, Dcur, nt);
  return cudaGetLastError();
}

// A_l tiles: tile(G, G') = sum_{c in G, c' in G' adjacent} Psi_G[c]^T T(c,c') Psi_G'[c']
// (FP64 sums; TI / TO: stored types of the previous and the new tiles)
template <class TI, class TO>
__global__ void k_group_rap(CLevel prev, CLevel cur, const double* __restrict__ Psi, const TI* __restrict__ Tp,
                            TO* __restrict__ T) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int g = cur.g, Lp = prev.L, L = cur.L, ng = g * g * g, n = ng * Lp;
  double* out = (double*)sm;       // [27][L][L]
  double* Wt = out + 27 * L * L;   // [Lp][L]
  const long long G = blockIdx.x;
  const int gx = (int)(G % cur.mx), gy = (int)((G / cur.mx) % cur.my), gz = (int)(G / ((long long)cur.mx * cur.my));
  for (int i = threadIdx.x; i < 27 * L * L; i += blockDim.x) out[i] = 0.0;
  __syncthreads();
  const double* psG = Psi + G * (long long)n * L;
  for (int lc = 0; lc < ng; ++lc) {
    const int lx = lc % g, ly = (lc / g) % g, lz = lc / (g * g);
    const int cx = gx * g + lx, cy = gy * g + ly, cz = gz * g + lz;
    const long long c = cx + (long long)prev.mx * (cy + (long long)prev.my * cz);
    for (int nn = 0; nn < 27; ++nn) {
      const int dx = nn % 3 - 1, dy = (nn / 3) % 3 - 1, dz = nn / 9 - 1;
      const int ncx = cx + dx, ncy = cy + dy, ncz = cz + dz;
      if (ncx < 0 || ncy < 0 || ncz < 0 || ncx >= prev.mx || ncy >= prev.my || ncz >= prev.mz) continue;
      const int Gx = ncx / g, Gy = ncy / g, Gz = ncz / g;
      const long long G2 = Gx + (long long)cur.mx * (Gy + (long long)cur.my * Gz);
      const int lc2 = (ncx % g) + g * ((ncy % g) + g * (ncz % g));
      const int gn = nbr_index(Gx - gx, Gy - gy, Gz - gz);
      const TI* Tc = Tp + (c * 27 + nn) * Lp * Lp;
      const double* ps2 = Psi + G2 * (long long)n * L + (long long)lc2 * Lp * L;
      for (int w = threadIdx.x; w < Lp * L; w += blockDim.x) {
        const int i = w / L, bb = w % L;
        double s = 0.0;
        for (int j = 0; j < Lp; ++j) s += (double)Tc[i * Lp + j] * ps2[j * L + bb];
        Wt[w] = s;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < L * L; w += blockDim.x) {
        const int a = w / L, bb = w % L;
        double s = 0.0;
        for (int i = 0; i < Lp; ++i) s += psG[(lc * Lp + i) * L + a] * Wt[i * L + bb];
        out[gn * L * L + w] += s;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < 27 * L * L; i += blockDim.x) T[G * 27 * L * L + i] = (TO)out[i];
}
template <class TI, class TO>
cudaError_t group_rap(const CLevel& prev, const CLevel& cur, const double* Psi, const TI* tiles_prev, TO* tiles,
                      cudaStream_t st) {
  const size_t sm = (27 * (size_t)cur.L * cur.L + (size_t)prev.L * cur.L) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_group_rap<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  note_launch(), k_group_rap<TI, TO><<<(unsigned)cur.ncell, 256, sm, st>>>(prev, cur, Psi, tiles_prev, tiles);
  return cudaGetLastError();
}
#define INST_GRAP(TI, TO)                                                                                     \
  template cudaError_t group_rap<TI, TO>(const CLevel&, const CLevel&, const double*, const TI*, TO*, cudaStream_t);
INST_GRAP(double, double)
INST_GRAP(float, float)
INST_GRAP(float, double)

// inactive dofs (zero basis vectors) get an identity row in the centre tile
template <class TT>
__global__ void k_fix_inactive(CLevel lv, const uint8_t* __restrict__ act, TT* __restrict__ T) {
  const long long nd = lv.ncell * lv.L;
  for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < nd; d += (long long)gridDim.x * blockDim.x) {
    if (act[d]) continue;
    const long long c = d / lv.L;
    const int i = (int)(d % lv.L);
    T[((c * 27 + 13) * lv.L + i) * lv.L + i] = (TT)1;
  }
}
template <class TT>
cudaError_t fix_inactive(const CLevel& lv, const uint8_t* act, TT* tiles, cudaStream_t st) {
  const long long nd = lv.ncell * lv.L;
  note_launch(), k_fix_inactive<TT><<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(lv, act, tiles);
  return cudaGetLastError();
}
template cudaError_t fix_inactive<double>(const CLevel&, const uint8_t*, double*, cudaStream_t);
template cudaError_t fix_inactive<float>(const CLevel&, const uint8_t*, float*, cudaStream_t);

// l1-block-Jacobi: inverse of (A_cc + diag(sum_{off-cell} |a_ij|)), FP64 Gauss-Jordan
// (TT: the stored tile type, widened on load; Di64 may be NULL)
template <class TT>
__global__ void k_l1inv(CLevel lv, const TT* __restrict__ T, double* __restrict__ Di64, float* __restrict__ Di32) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int L = lv.L;
  double* M = (double*)sm + threadIdx.x * 2 * L * L;  // [L][2L] augmented
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= lv.ncell) return;
  for (int i = 0; i < L; ++i) {
    double off = 0.0;
    for (int n = 0; n < 27; ++n) {
      if (n == 13) continue;
      const TT* row = T + ((c * 27 + n) * L + i) * L;
      for (int j = 0; j < L; ++j) off += fabs((double)row[j]);
    }
    const TT* row = T + ((c * 27 + 13) * L + i) * L;
    for (int j = 0; j < L; ++j) {
      M[i * 2 * L + j] = (double)row[j] + (i == j ? off : 0.0);
      M[i * 2 * L + L + j] = i == j ? 1.0 : 0.0;
    }
  }
  for (int k = 0; k < L; ++k) {
    int piv = k;
    for (int i = k + 1; i < L; ++i)
      if (fabs(M[i * 2 * L + k]) > fabs(M[piv * 2 * L + k])) piv = i;
    if (piv != k)
      for (int j = 0; j < 2 * L; ++j) {
        const double t = M[k * 2 * L + j];
        M[k * 2 * L + j] = M[piv * 2 * L + j];
        M[piv * 2 * L + j] = t;
      }
    const double d = M[k * 2 * L + k];
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (int j = 0; j < 2 * L; ++j) M[k * 2 * L + j] *= inv;
    for (int i = 0; i < L; ++i) {
      if (i == k) continue;
      const double f = M[i * 2 * L + k];
      if (f != 0.0)
        for (int j = 0; j < 2 * L; ++j) M[i * 2 * L + j] -= f * M[k * 2 * L + j];
    }
  }
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      const double v = M[i * 2 * L + L + j];
      if (Di64) Di64[(c * L + i) * L + j] = v;
      Di32[(c * L + i) * L + j] = (float)v;
    }
}
template <class TT>
cudaError_t l1_inverse(const CLevel& lv, const TT* tiles, double* Dinv64, float* Dinv32, cudaStream_t st) {
  int nt = 64;
  size_t per = 2 * (size_t)lv.L * lv.L * sizeof(double);
  while (nt > 1 && per * nt > 96 * 1024) nt >>= 1;
  const size_t sm = per * nt;
  cudaError_t e = cudaFuncSetAttribute(k_l1inv<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  note_launch(), k_l1inv<TT><<<(unsigned)((lv.ncell + nt - 1) / nt), nt, sm, st>>>(lv, tiles, Dinv64, Dinv32);
  return cudaGetLastError();
}
template cudaError_t l1_inverse<double>(const CLevel&, const double*, double*, float*, cudaStream_t);
template cudaError_t l1_inverse<float>(const CLevel&, const float*, double*, float*, cudaStream_t);

// dense coarsest operator A[(c,i)][(c',j)]
__global__ void k_dense(CLevel lv, const double* __restrict__ T, double* __restrict__ A) {
  const long long N = lv.ncell * lv.L;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < N * N; w += (long long)gridDim.x * blockDim.x) {
    const long long r = w / N, col = w % N;
    const long long c = r / lv.L, c2 = col / lv.L;
    const int i = (int)(r % lv.L), j = (int)(col % lv.L);
    const int cx = (int)(c % lv.mx), cy = (int)((c / lv.mx) % lv.my), cz = (int)(c / ((long long)lv.mx * lv.my));
    const int dx = (int)(c2 % lv.mx) - cx, dy = (int)((c2 / lv.mx) % lv.my) - cy,
              dz = (int)(c2 / ((long long)lv.mx * lv.my)) - cz;
    double v = 0.0;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1)
      v = T[((c * 27 + nbr_index(dx, dy, dz)) * lv.L + i) * lv.L + j];
    A[w] = v;
  }
}
cudaError_t dense_assemble(const CLevel& lv, const double* tiles, double* A, cudaStream_t st) {
  const long long N = lv.ncell * lv.L;
  long long nb = (N * N + 255) / 256;
  if (nb > 152 * 64) nb = 152 * 64;
  note_launch(), k_dense<<<(unsigned)nb, 256, 0, st>>>(lv, tiles, A);
  return cudaGetLastError();
}

__global__ void k_cvt(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
cudaError_t cvt_f64_f32(const double* a, float* b, long long n, cudaStream_t st) {
  long long nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  if (nb < 1) nb = 1;
  note_launch(), k_cvt<<<(unsigned)nb, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

template <class C>
__global__ void k_phi_nat(Geom g, const C* __restrict__ phi, int L, double* __restrict__ out) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const long long t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const long long nd = nidx(g, x, y, z);
    for (int a = 0; a < L; ++a) out[i * L + a] = (double)phi[nd * L + a];
  }
}
template <class C>
cudaError_t phi_natural(const Geom& g, const C* phi_pad, int L1, double* out, cudaStream_t st) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  note_launch(), k_phi_nat<C><<<(unsigned)nb, 256, 0, st>>>(g, phi_pad, L1, out);
  return cudaGetLastError();
}
template cudaError_t phi_natural<double>(const Geom&, const double*, int, double*, cudaStream_t);
template cudaError_t phi_natural<float>(const Geom&, const float*, int, double*, cudaStream_t);

}  // namespace thermo

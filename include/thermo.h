/*
 * thermo.h — C ABI of libthermo: preconditioned CG for the 3-D steady heat
 * equation with SIMP conductivity on a structured grid of trilinear (Q1)
 * elements, preconditioned by the multiscale multigrid (MMG) of
 * "A robust solver for large-scale heat transfer topology optimization"
 * (arXiv 2410.06850), and the adjoint compliance sensitivity.
 *
 * Paper anchors
 *   Sec. 2.1 Eq. (1)   SIMP law  kappa_e = kmin + x_e^p (kmax - kmin)
 *   Sec. 2.2 Eq. (5)   SPD system A t = f (here: Q1 nodal elements)
 *   Sec. 2.3 Eqs. (6)-(7)  objective and adjoint sensitivity
 *   Sec. 3  Eq. (8)    local spectral problem on each coarse block
 *   Sec. 3  Eq. (9)    spectral problem on coarse-coarse blocks in W_c
 *   Sec. 3  Algorithm 1  smoothed multigrid cycle (generalised to Q grids)
 *   Sec. 4             PETSc CG with the preconditioner; set-up / LS1 / LS2
 *
 * Conventions (all entry points)
 *   - Grid: Nx x Ny x Nz box elements of size hx x hy x hz.  Nodes
 *     n = i + (Nx+1)*(j + (Ny+1)*k) (x fastest); elements
 *     e = ex + Nx*(ey + Ny*ez).  Element e's local node a = ax+2ay+4az is
 *     node (ex+ax, ey+ay, ez+az).
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous in
 *     the layout above, unless a parameter says "host".  The library copies
 *     into its own padded device layout and owns every internal buffer.
 *   - All device work is enqueued on the CUDA stream given to thermo_create.
 *     Calls return after enqueueing, except those that launch TMA-staged
 *     fine-grid kernels (setup_precond, solve, vcycle, apply, apply_dot,
 *     bench_kernel), which synchronise the stream to read the context's
 *     stage time-out word (and, for solve, once per convergence check), and
 *     thermo_compliance (returns a host scalar).
 *   - Every call returns a thermo_status; none aborts, asserts or traps.  On
 *     failure the context stays valid and thermo_last_error() describes it.
 *   - Call order: create -> set_density -> setup_precond -> solve (any number
 *     of times) -> sensitivity.  set_density invalidates the preconditioner;
 *     solve before setup_precond (with pc = MMG) returns THERMO_ESTATE.
 *   - The context is not thread-safe; use one context per host thread.
 */
#ifndef THERMO_H
#define THERMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thermo_ctx thermo_ctx; /* opaque, owned by the library */

typedef enum {
  THERMO_OK = 0,
  THERMO_EINVAL = -1,      /* bad argument (sizes, NULL, empty Dirichlet set) */
  THERMO_ENOMEM = -2,      /* device or host allocation failed */
  THERMO_ECUDA = -3,       /* a CUDA call or kernel launch failed */
  THERMO_ENOTCONV = -4,    /* max_iter reached; u holds the last iterate */
  THERMO_EBREAKDOWN = -5,  /* CG breakdown: p^T A p <= 0 or NaN/Inf */
  THERMO_ESINGULAR = -6,   /* non-positive pivot in the coarsest Cholesky */
  THERMO_ESTATE = -7       /* call out of order (e.g. solve before setup) */
} thermo_status;

typedef enum {
  THERMO_FP64 = 0,         /* everything FP64 (V-cycle included), standard PCG */
  THERMO_MIXED = 1,        /* FP32 V-cycle inside FP64 flexible CG */
  THERMO_MIXED_BF16S = 2   /* as MIXED, fine-grid smoother data stored as BF16 */
} thermo_precision;

typedef enum {
  THERMO_PC_MMG = 0,       /* the multiscale multigrid V-cycle (Algorithm 1) */
  THERMO_PC_NONE = 1,      /* plain CG (comparison mode) */
  THERMO_PC_JACOBI = 2     /* point-Jacobi PCG (comparison mode) */
} thermo_pc;

typedef enum {
  THERMO_GUESS_ZERO = 0,        /* u0 = 0 (Dirichlet values on Gamma_D) */
  THERMO_GUESS_GIVEN = 1,       /* u0 = u on entry */
  THERMO_GUESS_COARSE = 2,      /* u0 = P A_L^-1 P^T b: coarsest solution interpolated */
  THERMO_GUESS_WARM_COARSE = 3  /* u0 = u + P A_L^-1 P^T (b - A u) */
} thermo_guess;

#define THERMO_MAX_LEVELS 8

/* Hierarchy and solver options.  Level 1 cells are blocks of block^3 fine
 * elements carrying nvec[0] local eigenvectors (Eq. (8)); level l >= 2 cells
 * are groups of group[l-1]^3 level-(l-1) cells carrying nvec[l-1] vectors
 * (Eq. (9)).  The last level is solved by dense FP64 Cholesky. */
typedef struct {
  int levels;                       /* number of coarse levels, 1..THERMO_MAX_LEVELS */
  int block;                        /* b (fine elements per block edge) */
  int group[THERMO_MAX_LEVELS];     /* group[l-1] = g_l for l >= 2 (group[0] unused) */
  int nvec[THERMO_MAX_LEVELS];      /* nvec[l-1] = L_l, 1 <= L_l <= 32 */
  int nu_fine;                      /* damped-Jacobi sweeps before and after (>= 1) */
  int nu_coarse;                    /* l1-block-Jacobi sweeps on coarse levels (>= 1) */
  double omega;                     /* fine Jacobi damping (default 2/3) */
  thermo_precision prec;
  thermo_pc pc;
  int guess;                        /* a thermo_guess value */
  int max_iter;                     /* default 10000 */
  int flexible;                     /* -1 auto (1 iff prec != FP64); 0 standard PCG;
                                       1 flexible CG, new direction A-orthogonalised
                                       against the last one (robust to the FP32 cycle);
                                       2 flexible CG with the Polak-Ribiere beta */
  int check_every;                  /* host convergence check every k iterations (>= 1) */
  int smoother;                     /* fine smoother: 0 damped Jacobi (nu_fine sweeps, omega),
                                       1 Chebyshev-accelerated Jacobi (default) */
  int cheb_degree;                  /* Chebyshev: operator applications per smoothing (>= 1) */
  double cheb_ratio;                /* Chebyshev interval [lmax/ratio, 1.1 lmax] of D^-1 A */
  int power_iters;                  /* power iterations estimating lmax(D^-1 A) in set-up */
  int outer_apply;                  /* operator of the outer CG loop: 0 auto (float-float for the
                                       mixed forms when the grid allows it: cubic elements,
                                       Nx a multiple of 64), 1 FP64 arithmetic, 2 float-float
                                       (FP64-accurate sums of two floats on the FP32 pipes;
                                       falls back to 1 where the grid does not allow it) */
  int nu_growth;                    /* coarse sweeps on level l: nu_coarse * nu_growth^(l-1),
                                       capped at 64 (1: the same on every coarse level;
                                       default 2) */
  int w_from;                       /* 0: V-cycle; k > 0: levels >= k make two coarse
                                       corrections per visit (W-cycle below level k), except
                                       just above the direct coarsest solve (default 3) */
  double restart_decades;           /* > 0: restart the recurrence from the true FP64
                                       residual each time the recursive residual has
                                       dropped by this many decades (iterative refinement
                                       around the low-precision cycle); 0: never */
  int density_fp32;                 /* 0: thermo_set_density's x is double[M]; 1: float[M]
                                       (stored as given, widened where it is used;
                                       default 0) */
  int fine_engine;                  /* FP32 fine sweeps and applies on cubic elements:
                                       0 (default) the separable engine (box sums of the
                                       Q1 operator, one x column per warp, rows in
                                       registers); 1 the two-nodes-per-lane engine
                                       (grids with Nx a multiple of 64) */
  int lean;                         /* 0 (default): FP64 and FP32 copies of the hierarchy.
                                       1 (mixed forms only): the hierarchy is stored once,
                                       in FP32 (Phi, Psi, the tiles of every level but the
                                       coarsest, the l1 inverses); each level's tiles and
                                       bases are computed in FP64 arithmetic from the
                                       stored FP32 tiles of the level below and rounded
                                       once; the FP64 set-up intermediates (Phi before
                                       rounding, Psi, the row-sum corrections) live in the
                                       memory of the CG and cycle vectors, which set-up
                                       does not use; the coarse initial guess runs the FP32
                                       chain.  Roughly halves the context's device memory. */
  double eig_threshold;             /* 0 (default): every cell of level l keeps nvec[l-1]
                                       local eigenvectors (the paper's fixed L_c, L_cc).
                                       tau > 0: adaptive count (the GMsFEM-style
                                       alternative): a cell keeps its eigenpairs with
                                       lambda H_l^2 <= tau, at most nvec[l-1] (the slot
                                       capacity), at least one; H_l = block max(h) times
                                       the group sizes of levels 2..l; lambda of Eq. (8)
                                       (kappa-mass generalised) or Eq. (9).  Unused slots
                                       are inactive (identity rows in A_l). */
} thermo_options;

typedef struct {
  int iters;                        /* A p products = preconditioner applications */
  int restarts;                     /* residual replacements after a failed true-residual check */
  double rel_res_recursive;         /* ||r_k|| / ||b_F|| of the recurrence at exit */
  double rel_res_true;              /* ||b - A u|| / ||b_F|| recomputed in FP64 at exit */
  double t_setup_ms;                /* last thermo_setup_precond wall time */
  double t_solve_ms;                /* this solve's wall time */
  int status;                       /* thermo_status of the solve */
} thermo_solve_info;

/* Fill *opt with the defaults for an Nx x Ny x Nz grid: b = 4, L_1 = 4, then
 * groups of 2^3 cells down to a coarsest level of 4^3 cells (8^3 cells when
 * the smallest axis has more than 32 level-1 cells, i.e. grids above 128 per
 * axis: an exact coarse-coarse solve of 8,704 unknowns) with L = 17 (the
 * second level keeps 8 vectors when there are more than two coarse levels),
 * Chebyshev fine smoother of degree 5 on [lmax/30, 1.1 lmax] (15 power
 * iterations), nu_fine = 2 / omega = 2/3 for the Jacobi alternative,
 * nu_coarse = 1, MIXED, MMG, coarse guess, max_iter = 10000, flexible auto,
 * check_every = 1.  Returns EINVAL if the
 * grid is not a multiple of 4 in each axis. */
thermo_status thermo_default_options(const int grid[3], thermo_options *opt);

/* Create a solver context for the steady heat problem of Sec. 2.1 (Dirichlet
 * data on Gamma_D, adiabatic elsewhere, element heat source) discretised as the
 * linear system of Sec. 2.2 Eq. (5).
 *   grid[3]          host: Nx, Ny, Nz (each a multiple of opt->block and
 *                    Nx/b etc. a multiple of the product of the group sizes)
 *   h[3]             host: element edge lengths (> 0)
 *   dirichlet_mask   device, uint8[(Nx+1)(Ny+1)(Nz+1)]: 1 = node on Gamma_D.
 *                    Must be non-empty (else the operator is singular: EINVAL).
 *   dirichlet_value  device, double[nodes] or NULL (= 0): T_D on Gamma_D
 *   source           device, double[Nx*Ny*Nz]: element heat source q_e; the
 *                    load is f_i = sum_{e contains i} q_e |e| / 8
 *   cuda_stream      a cudaStream_t (NULL = legacy default stream)
 *   opt              host, or NULL for thermo_default_options(grid)
 *   out              host: receives the context
 */
thermo_status thermo_create(const int grid[3], const double h[3],
                            const uint8_t *dirichlet_mask,
                            const double *dirichlet_value,
                            const double *source, void *cuda_stream,
                            const thermo_options *opt, thermo_ctx **out);

/* Device bytes thermo_create would allocate for this grid and these options
 * (opt NULL = defaults; has_dirichlet_value: whether a dirichlet_value array
 * will be given), without touching a GPU: the same allocation plan run
 * without allocating.  Counts the context's own buffers (each rounded up to
 * 512 bytes), not the caller's inputs or the CUDA context.  Returns EINVAL
 * for grids or options thermo_create rejects. */
thermo_status thermo_plan_bytes(const int grid[3], const thermo_options *opt,
                                int has_dirichlet_value, long long *bytes);

/* Set the design (Sec. 2.1 Eq. (1)): x device double[M] (float[M] when
 * opt.density_fp32 = 1, kept in FP32 as given) in [0,1] (not checked), p >= 1,
 * 0 < kmin <= kmax.  The context copies x (the caller's array may be freed).
 * kappa is evaluated once per element here and kept in FP64, FP32 plus the
 * float-float low part, and BF16 for the MIXED_BF16S form.  Marks the
 * preconditioner stale. */
thermo_status thermo_set_density(thermo_ctx *ctx, const void *x, double p,
                                 double kmin, double kmax);

/* As thermo_set_density (Sec. 2.1 Eq. (1)), but a preconditioner built for an
 * earlier design stays in use: the operator, the load lifting and the fine
 * smoother's conductivities follow the new design, while the coarse spaces,
 * Galerkin operators and the smoother's spectral interval are the old ones.
 * CG then solves the new system with the old preconditioner, which stays
 * effective for small design changes (a finite-difference perturbation of a
 * few elements, a damped design step).  If no preconditioner exists yet this
 * is thermo_set_density.  Same arguments and errors. */
thermo_status thermo_update_density(thermo_ctx *ctx, const void *x, double p, double kmin, double kmax);

/* Build the MMG hierarchy for the current design (Sec. 3): local spectral
 * problems (Eq. (8)) on every block, M-orthonormal bases, Galerkin operators,
 * spectral problems on groups (Eq. (9)), l1-block-Jacobi inverses and the
 * dense FP64 Cholesky of the coarsest operator.  ESINGULAR on a non-positive
 * pivot.  Synchronises the stream.  With pc = NONE/JACOBI this only records
 * that the context is ready. */
thermo_status thermo_setup_precond(thermo_ctx *ctx);

/* Solve the system of Sec. 2.2 Eq. (5) with CG preconditioned by the cycle of
 * Sec. 3 Algorithm 1 (the state solve LS1 of Sec. 4), started from the
 * interpolated coarse solution (opt.guess).
 * Solve A u = b to ||b - A u||_2 <= tol ||b_F||_2, where b_F is b on the free
 * (non-Dirichlet) nodes; the Dirichlet rows are identities satisfied exactly
 * by every iterate.  Checked on the recursive residual, confirmed on the true
 * FP64 residual at exit.
 *   rhs   device double[nodes] (natural layout), or NULL for the assembled
 *         load f (with Dirichlet lifting b_F = f_F - A_FD T_D, b_D = T_D)
 *   u     device double[nodes]: initial guess if opt.guess is GIVEN or
 *         WARM_COARSE; the solution on return (also on ENOTCONV)
 *   info  host, may be NULL
 * Synchronises the stream once per convergence check. */
thermo_status thermo_solve(thermo_ctx *ctx, const double *rhs, double *u,
                           double tol, thermo_solve_info *info);

/* Adjoint sensitivity of the compliance c = f^T u for homogeneous Dirichlet
 * data (adjoint = state, Sec. 2.3):
 *   dc[e] = -p x_e^(p-1) (kmax - kmin) u_e^T K0 u_e
 * u device double[nodes], dc device double[M]. */
thermo_status thermo_sensitivity(thermo_ctx *ctx, const double *u, double *dc);

/* result = x . y (FP64), a context-free variant of the CG reduction that
 * allocates no memory.  The paper has no counterpart: this is a service
 * entry point for callers that must not allocate device memory during the
 * call, e.g. code running under a caller-managed memory budget, or a loop
 * that cannot afford the device-wide synchronisation an allocation may imply;
 * such a caller may also hold no thermo_ctx (creating one allocates).
 * Scratch: a file-scope device array in the library (partial sums of fixed
 * 8192-element chunks plus an arrival counter), hence n <= 134,217,728;
 * larger n is rejected with THERMO_EINVAL and a message.  The counter must
 * start at zero: it is zero when the library loads, zeroed again at the
 * first call on each device, and every completed call leaves it at zero.
 *   x, y    device double[n] (may be NULL when n == 0)
 *   result  device double, written by the kernel (0 for n == 0)
 *   stream  a cudaStream_t (NULL = legacy default stream); the call only
 *           enqueues work, except the first call on each device, which
 *           resolves the scratch address and zeroes the counter
 *           synchronously: make it before any stream capture
 *   msg     host buffer of msg_len bytes for an error message, may be NULL
 * Deterministic: fixed chunking and tree order, bitwise repeatable for
 * equal inputs.  Calls on one device share the scratch: two calls whose
 * kernels overlap in time (different streams, or host threads) race and give
 * wrong results; serialise them (same stream, or events).
 * Errors: EINVAL (bad arguments, n over the limit), ECUDA (no device, symbol
 * lookup or launch failure). */
thermo_status thermo_dot_noalloc(const double *x, const double *y, long long n, double *result,
                                 void *stream, char *msg, int msg_len);

/* c = f^T u (Sec. 2.3 Eq. (6) with q = 1: the mean temperature).
 * u device double[nodes]; c host double*.  Synchronises the stream. */
thermo_status thermo_compliance(thermo_ctx *ctx, const double *u, double *c);

/* Ainv = A^-1 for a dense symmetric positive definite A with the library's
 * blocked FP64 Cholesky factorisation and explicit inverse: the routine of
 * the direct coarsest-level solve of Sec. 3 Algorithm 1 (A_cc^-1; the paper's
 * Sec. 4 uses a sparse LU), exposed on caller-supplied matrices so that it
 * can be checked on its own.  Context-free.
 *   n       order, 1 <= n <= 20000
 *   A       device double[n][n], row-major; symmetrised as (A + A^T)/2, not modified
 *   Ainv    device double[n][n], row-major, written (symmetric)
 *   stream  a cudaStream_t (NULL = legacy default stream); synchronised
 *   pivot   host int or NULL: on THERMO_ESINGULAR the 0-based row of the
 *           first non-positive (or non-finite) pivot
 *   msg     host buffer of msg_len bytes for an error message, may be NULL
 * Allocates and frees its scratch (about 2 n^2 doubles) on the current device.
 * Errors: EINVAL (arguments), ENOMEM, ECUDA, ESINGULAR (A not positive
 * definite; Ainv then holds no useful values). */
thermo_status thermo_dense_spd_inverse(int n, const double *A, double *Ainv, void *stream, int *pivot,
                                       char *msg, int msg_len);

/* Stage wait limit of the TMA-staged fine-grid kernels (robustness support,
 * no counterpart in the paper).  Each kernel stages its input planes into a
 * shared-memory ring through asynchronous tensor copies and waits for them
 * with a bounded wait: after a first non-blocking test it polls for at most
 * `cycles` clock64 cycles (0 restores the default, 2^31 cycles, about one
 * second).  A wait that runs out marks the launch's results invalid in a
 * per-context device word, stops the kernel from issuing further copies and
 * lets it drain the copies already in flight before it exits; every entry
 * point that launches such a kernel (set-up, solve, cycle, applies, kernel
 * benchmark) reads and clears the word and then returns THERMO_ECUDA.  The
 * context stays usable.  A tiny limit (1 cycle) makes the waits run out on
 * purpose, which is how the time-out path is tested.  EINVAL if cycles < 0. */
thermo_status thermo_set_stage_wait(thermo_ctx *ctx, long long cycles);

/* Last error message of this context (never NULL).  Context management: no
 * counterpart in the paper. */
const char *thermo_last_error(const thermo_ctx *ctx);

/* Release every device and host resource of the context (NULL is a no-op).
 * Context management: no counterpart in the paper. */
void thermo_destroy(thermo_ctx *ctx);

/* ---- Inspection and building blocks (tests, benchmarks, the SIMP harness) */

/* y = A u with the Dirichlet-eliminated operator of Sec. 2.2 Eq. (5) (identity rows on Gamma_D,
 * no coupling to Gamma_D columns), in the given arithmetic:
 * THERMO_FP64 (FP64), THERMO_MIXED (FP32 data and math) or
 * THERMO_MIXED_BF16S (BF16 data, FP32 math).  u, y: device double[nodes].
 * Synchronises the stream to read the stage time-out word (see
 * thermo_set_stage_wait); THERMO_ECUDA if a kernel gave up waiting. */
thermo_status thermo_apply(thermo_ctx *ctx, int precision, const double *u, double *y);

/* q = A p and pq = p^T A p with the fused kernel of the outer CG loop (the
 * operator of Sec. 2.2 Eq. (5) and the CG reduction of Sec. 4): FP64
 * arithmetic or the FP64-accurate float-float kernel, as opt.outer_apply
 * selects.  p, q device double[nodes]; p must vanish on Gamma_D (as CG
 * directions do); pq host.  Deterministic (fixed reduction order).
 * Synchronises the stream. */
thermo_status thermo_apply_dot(thermo_ctx *ctx, const double *p, double *q, double *pq);

/* z = B r: one MMG V-cycle (Algorithm 1) in the context's precision.
 * r, z: device double[nodes]; entries of r on Gamma_D are ignored (treated as
 * zero) and z vanishes there.  Requires setup_precond (THERMO_ESTATE
 * otherwise).  Synchronises the stream; THERMO_ECUDA if a fine-grid kernel gave
 * up waiting for one of its staged planes (bounded wait; the context stays
 * usable). */
thermo_status thermo_vcycle(thermo_ctx *ctx, const double *r, double *z);

/* The assembled load vector f, the right-hand side of Sec. 2.2 Eq. (5) before
 * the Dirichlet lifting (device double[nodes]). */
thermo_status thermo_load_vector(thermo_ctx *ctx, double *f);

/* The coarse spaces of Sec. 3 (Eq. (8) on level 1, Eq. (9) above), one entry
 * per coarse level.  Hierarchy description (host outputs, any may be NULL):
 * nlevels (coarse levels), cells[l*3+k] cells per axis of level l+1,
 * nvec[l], ndof[l] = cells * nvec. */
thermo_status thermo_hierarchy(const thermo_ctx *ctx, int *nlevels, int *cells,
                               int *nvec, long long *ndof);

/* Copy level data of Sec. 3 out (bases of Eq. (8) / Eq. (9), Galerkin
 * operators, local eigenvalues, the coarsest inverse of Algorithm 1's direct
 * solve) (device double outputs, FP64 masters):
 *   what = 0: basis of level `level` — level 1: Phi as double[nodes][L_1]
 *             (natural node order); level l >= 2: Psi as
 *             double[cells_l][g^3 L_{l-1}][L_l] (rows in the group's local
 *             cell order lx + g ly + g^2 lz, then vector index)
 *   what = 1: Galerkin operator tiles double[cells][27][L][L], neighbour
 *             n = (dx+1) + 3(dy+1) + 9(dz+1); row dofs of the cell, column
 *             dofs of the neighbour
 *   what = 2: local eigenvalues double[cells][L]
 *   what = 3: (coarsest level only) dense inverse A_L^-1 double[n][n]
 * `count` is the capacity of `out` in doubles; EINVAL if too small. */
thermo_status thermo_export_level(thermo_ctx *ctx, int level, int what,
                                  double *out, long long count);

/* Resolution change of a field between two grids of the same box (the
 * interpolation technique of Sec. 3: a design optimised at low resolution is
 * carried to the next resolution as its start, 128^3 -> 256^3 -> 512^3 in
 * Sec. 4.1; the solution can be carried alongside as a warm start).
 *   grid_c, grid_f  host int[3]; grid_f[k] = r_k grid_c[k], integer r_k >= 1
 *   in              device double[]: the coarse field (x fastest)
 *   out             device double[]: the fine field (in != out)
 *   kind 0          element field, piecewise constant (each coarse element's
 *                   value on its r_x r_y r_z children; mean preserved)
 *   kind 1          element field, trilinear between cell centres (fine centre
 *                   at (i + 1/2)/r - 1/2 in coarse-centre units), constant beyond
 *                   the outermost centres; stays within the input's range
 *   kind 2          nodal field (grid + 1 values per axis): the coarse trilinear
 *                   (Q1) function evaluated at the fine nodes
 * Products and sums are rounded separately, x then y then z.  Needs no
 * context; enqueued on `stream`.  EINVAL for non-integer ratios, kind out of
 * range or in == out; ECUDA if the launch fails. */
thermo_status thermo_resample(const int grid_c[3], const double *in,
                              const int grid_f[3], double *out, int kind,
                              void *stream);

/* The paper's own discretisation (Sec. 2.2 Eqs. (4)-(5)): the cell-centred
 * two-point flux approximation, one temperature per element in natural cell
 * order c = i + Nx (j + Ny k), FP64.  An internal face between cells a and b
 * has the transmissibility kappa_F |F| / h with the harmonic mean
 * kappa_F = 2 / (1/kappa_a + 1/kappa_b); a face on Gamma_D reaches the
 * prescribed T_D over half a cell (2 kappa_c |F| / h); other boundary faces
 * are adiabatic.  dirichlet_faces: device uint8[M], bit 0/1 the -x/+x face of
 * the cell, 2/3 -y/+y, 4/5 -z/+z (set only on the box boundary).  These are
 * context-free kernels on caller-owned device arrays, enqueued on `stream`;
 * EINVAL for NULL arrays, non-positive sizes or p < 1, ECUDA if a launch fails.
 *
 *   thermo_tpfa_conductivity  kappa_c = kmin + x_c^p (kmax - kmin)   (Eq. (1))
 *   thermo_tpfa_apply         y = A t   (t != y)
 *   thermo_tpfa_rhs           b = f0 (1 - x^p) |K| + tau_D T_D      (Eq. (1) source)
 *   thermo_tpfa_sensitivity   dc/dx_e = u^T (df/dx_e - dA/dx_e t + db/dx_e) for the
 *                             mean temperature c = sum(t) / M (Eq. (6)), with t the
 *                             state (A t = b) and u the adjoint, A u = 1/M (Eq. (7)) */
thermo_status thermo_tpfa_conductivity(long long M, const double *x, double p,
                                       double kmin, double kmax, double *kappa,
                                       void *stream);
thermo_status thermo_tpfa_apply(const int grid[3], const double h[3],
                                const double *kappa,
                                const uint8_t *dirichlet_faces,
                                const double *t, double *y, void *stream);
thermo_status thermo_tpfa_rhs(const int grid[3], const double h[3],
                              const double *x, double p, double f0,
                              const double *kappa,
                              const uint8_t *dirichlet_faces, double TD,
                              double *b, void *stream);
thermo_status thermo_tpfa_sensitivity(const int grid[3], const double h[3],
                                      const double *x, double p, double kmin,
                                      double kmax, double f0,
                                      const double *kappa,
                                      const uint8_t *dirichlet_faces,
                                      double TD, const double *t,
                                      const double *u, double *dc,
                                      void *stream);

/* Density filter (textbook SIMP harness, not in the paper):
 * out_e = sum_j w_ej in_j / sum_j w_ej with w_ej = max(0, rmin - |c_e - c_j|)
 * in element units, truncated at the domain boundary; transpose = 1 applies
 * the transpose (gradient chain rule).  in/out device double[M], in != out. */
thermo_status thermo_filter(thermo_ctx *ctx, const double *in, double *out,
                            double rmin, int transpose);

/* Optimality-criteria update (textbook SIMP harness; the paper's Sec. 2.3
 * uses MMA) with bisection on the multiplier so that the
 * filtered volume fraction hits volfrac: x (device double[M], in/out),
 * dc, dv device double[M].  change (host, may be NULL) receives
 * max |x_new - x_old|. */
thermo_status thermo_oc_update(thermo_ctx *ctx, double *x, const double *dc,
                               const double *dv, double volfrac, double move,
                               double rmin, double *change);

/* Convergence history of the CG iteration of Sec. 4.
 * Relative recursive residuals ||r_k|| / ||b_F|| of the last thermo_solve, one
 * per convergence check (every opt.check_every iterations); copies at most
 * max of them to out (host, may be NULL) and returns how many exist. */
int thermo_residual_history(const thermo_ctx *ctx, double *out, int max);

/* Number of kernel launches this library has issued in the process (host
 * counter; for launch accounting in benchmarks; measurement support, no
 * counterpart in the paper). */
long long thermo_launch_count(void);

/* Measurement support (no counterpart in the paper).
 * Benchmark one internal kernel: `reps` back-to-back launches on the
 * context's own buffers, timed with CUDA events on the context stream.
 *   which: 0 the outer CG loop's apply (+ fused p.Ap; float-float or FP64
 *          per opt.outer_apply), 1 FP32 apply, 2 BF16 apply,
 *          3 FP32 fine smoother sweep, 4 FP32 fused residual + restriction,
 *          5 FP32 prolongation, 6 level-1 block-sparse apply,
 *          7 FP64 CG update, 8 one mixed V-cycle, 9 one FP64 V-cycle,
 *          10 FP64 fine smoother sweep, 11 FP64-arithmetic apply + p.Ap,
 *          12 float-float apply + p.Ap (EINVAL-like CUDA error where the
 *          grid does not allow it)
 *   ms_per_launch (host): average duration; bytes_per_launch (host, may be
 *   NULL): algorithmic DRAM bytes of one launch (0 for whole cycles).
 * Kernels 4-6, 8, 9 need setup_precond; 2 needs a MIXED_BF16S context and 9
 * an FP64 context.  Buffer contents are overwritten. */
thermo_status thermo_bench_kernel(thermo_ctx *ctx, int which, int reps, double *ms_per_launch,
                                  double *bytes_per_launch);

/* Kernel-class timers (no counterpart in the paper: measurement support).
 * When enabled, every launch of the classes below issued by thermo_solve is
 * bracketed by a pair of CUDA events recorded on the context stream; the
 * pairs are folded into per-class totals when thermo_solve returns (it
 * synchronises there).  At most 4096 launches per class and solve are timed;
 * later ones are counted in neither total.
 *   THERMO_KT_APPLY64  fine FP64 operator apply with the fused p.Ap (CG loop)
 *   THERMO_KT_SMOOTH   fine smoother sweeps of the V-cycle (all variants)
 *   THERMO_KT_RESTRICT fine fused residual + restriction
 *   THERMO_KT_PROLONG  fine prolongation
 *   THERMO_KT_COARSE   everything below the fine grid in one V-cycle
 *   THERMO_KT_CGVEC    CG vector kernels (update, beta, direction, conversion)
 * bytes/flops are the algorithmic DRAM bytes and floating-point operations of
 * the timed launches: compulsory traffic of each array once per launch (for
 * THERMO_KT_COARSE: every coarse launch of the cycle, tiles 27 L^2 and l1
 * inverses L^2 per cell, vectors, group bases, the coarsest FP64 inverse;
 * levels small enough to stay in L2 are counted all the same). */
enum {
  THERMO_KT_APPLY64 = 0,
  THERMO_KT_SMOOTH = 1,
  THERMO_KT_RESTRICT = 2,
  THERMO_KT_PROLONG = 3,
  THERMO_KT_COARSE = 4,
  THERMO_KT_CGVEC = 5,
  THERMO_KT_COUNT = 6
};
/* enable != 0 creates the events (once) and zeroes the totals; 0 stops timing. */
thermo_status thermo_kernel_timers(thermo_ctx *ctx, int enable);
/* Totals since the last enable: summed event time (ms), timed launches,
 * algorithmic bytes and flops.  Any output may be NULL. */
thermo_status thermo_kernel_time(thermo_ctx *ctx, int kclass, double *ms, long long *launches, double *bytes,
                                 double *flops);

#ifdef __cplusplus
}
#endif
#endif /* THERMO_H */

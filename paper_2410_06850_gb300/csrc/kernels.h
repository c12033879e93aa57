// Host-side launchers of the libthermo kernels (internal, C++ linkage).
#pragma once
#include "common.cuh"

namespace thermo {

// ---- fine.cu
unsigned fine_num_ctas(const Geom& g);
cudaError_t fine_apply_f64(const Geom& g, const uint32_t* mask, const double* kap, const double* u, double* y,
                           double* partial, unsigned* counter, double* dot, cudaStream_t st, bool mask_input = false);
template <class S>
cudaError_t fine_apply_lp(const Geom& g, const uint32_t* mask, const S* kap, const S* u, S* y, cudaStream_t st,
                          bool mask_input = false);
template <class S, class To>
cudaError_t fine_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e, const S* w,
                        To* out, typename Cv<S>::C cA, typename Cv<S>::C cB, cudaStream_t st);
template <class S>
cudaError_t fine_restrict(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e,
                          const typename Cv<S>::C* phi, typename Cv<S>::C* rc, int L1, cudaStream_t st);
template <class S>
cudaError_t fine_prolong(const Geom& g, const typename Cv<S>::C* phi, const typename Cv<S>::C* ec, S* e, int L1,
                         cudaStream_t st);

// ---- vec.cu : device scalars of the Krylov loop
struct CgScalars {
  double pq, rr, rz, rzo, rzn, alpha, beta, bb, tmp;
  int flag;  // 1: breakdown (p.Ap <= 0 or not finite)
  int pad;
};

struct Reducer {  // deterministic multi-CTA reduction scratch
  double* partial;
  unsigned* counter;
  int nblocks;
};

cudaError_t pack_nodes(const Geom& g, const double* nat, double* pad, cudaStream_t st);
cudaError_t unpack_nodes(const Geom& g, const double* pad, double* nat, cudaStream_t st);
cudaError_t mask_to_bits(const Geom& g, const uint8_t* nat, uint32_t* bits, cudaStream_t st);
cudaError_t count_mask(const Geom& g, const uint8_t* nat, long long n, int* out, cudaStream_t st);
template <class X>  // X: stored design type (double or float)
cudaError_t simp_kappa(const Geom& g, const X* x, double p, double kmin, double kmax, double* k64,
                       float* k32, bf16* k16, float* klo, cudaStream_t st);
cudaError_t load_vector(const Geom& g, const double* q, double* f, cudaStream_t st);
cudaError_t widen_f32(const float* a, double* b, long long n, cudaStream_t st);
cudaError_t dirichlet_rhs(const Geom& g, const uint32_t* bits, const double* k64, const double* f,
                          const double* TDpad, double* b, cudaStream_t st);
// y = a*x + b*y style helpers on padded FP64 vectors (interior rows)
cudaError_t vec_residual(const Geom& g, const double* b, const double* Ax, double* r, const Reducer& red,
                         double* rr, cudaStream_t st);
cudaError_t vec_dot(const Geom& g, const double* a, const void* b, int b_is_float, const Reducer& red, double* out,
                    cudaStream_t st);
cudaError_t vec_dot_free(const Geom& g, const uint32_t* bits, const double* a, const double* b, const Reducer& red,
                         double* out, cudaStream_t st);
cudaError_t vec_copy_cvt(const Geom& g, const double* src, void* dst, int dst_kind, cudaStream_t st);  // 0 f64,1 f32,2 bf16
cudaError_t cg_update(const Geom& g, double* u, double* r, const double* p, const double* q, const void* z_old,
                      int z_kind, void* r_lp, int r_lp_kind, CgScalars* sc, const Reducer& red, cudaStream_t st);
cudaError_t cg_beta_dot(const Geom& g, const double* r, const void* z, int zk, const double* q, int flexible,
                        CgScalars* sc, const Reducer& red, cudaStream_t st);
cudaError_t cg_pupdate(const Geom& g, const void* z, int z_kind, double* p, const CgScalars* sc, int first,
                       cudaStream_t st);
cudaError_t vec_to_f64(const Geom& g, const void* src, int kind, double* dst, cudaStream_t st);
template <class C>  // u += Phi ec with Phi, ec stored as C (double or float), FP64 sums
cudaError_t fine_prolong_add(const Geom& g, const C* phi, int L1, const C* ec, double* u, cudaStream_t st);
// two-nodes-per-lane FP32-compute fine sweeps / applies (fine2.cu): cubic
// elements, Nx a multiple of 64
bool fine2_supported(const Geom& g);
int fine2_tiles_xy(const Geom& g);  // CTAs per z chunk
int fine2_ctas_per_sm();            // resident CTAs per SM of the FP32 sweep
template <class S, class To>
cudaError_t fine2_smooth(const Geom& g, const uint32_t* mask, const S* kap, const S* r, const S* e, const S* w, To* out,
                         float cA, float cB, cudaStream_t st);
template <class S>
cudaError_t fine2_apply(const Geom& g, const uint32_t* mask, const S* kap, const S* u, S* y, cudaStream_t st);
// separable FP32 fine sweeps / applies (fine3.cu): cubic elements, any grid
bool fine3_supported(const Geom& g);
int fine3_tiles_x(const Geom& g);
int fine3_tiles_y(const Geom& g);
int fine3_ctas_per_sm();
template <class To>
cudaError_t fine3_smooth(const Geom& g, const uint32_t* mask, const float* kap, const float* r, const float* e,
                         const float* w, To* out, float cA, float cB, cudaStream_t st);
cudaError_t fine3_apply(const Geom& g, const uint32_t* mask, const float* kap, const float* u, float* y,
                        cudaStream_t st);
bool fine3_restrict_supported(const Geom& g, int L1);
cudaError_t fine3_restrict(const Geom& g, const uint32_t* mask, const float* kap, const float* r, const float* e,
                           const float* phi, float* res, float* rc, int L1, cudaStream_t st);
// float-float FP64-accurate fine apply (+ fused p.q when dot != NULL); see fine_ds.cu
bool fine_ds_supported(const Geom& g);
unsigned fine_ds_num_ctas(const Geom& g);
int fine_ds_tiles_xy(const Geom& g);
int fine_ds_ctas_per_sm();
cudaError_t fine_apply_ds(const Geom& g, const uint32_t* mask, const float* khi, const float* klo, const double* u,
                          double* y, double* partial, unsigned* counter, double* dot, cudaStream_t st);
cudaError_t vec_mask_dir(const Geom& g, const uint32_t* bits, double* v, cudaStream_t st);
cudaError_t vec_copy_dir(const Geom& g, const uint32_t* bits, const double* src, double* dst, cudaStream_t st);
cudaError_t power_start(const Geom& g, const uint32_t* bits, double* v, cudaStream_t st);
cudaError_t vec_scale(const Geom& g, double a, double* v, cudaStream_t st);
cudaError_t fill_const(double* a, long long n, double v, cudaStream_t st);
cudaError_t vec_axpy_pad(const Geom& g, double a, const double* x, double* y, cudaStream_t st);
template <class X>
cudaError_t sensitivity(const Geom& g, const double* upad, const X* x, double p, double kmin, double kmax,
                        double* dc, cudaStream_t st);
cudaError_t resample_field(const int gc[3], const double* in, const int gf[3], double* out, int kind,
                           cudaStream_t st);
cudaError_t density_filter(int Nx, int Ny, int Nz, const double* in, double* out, double rmin, int transpose,
                           cudaStream_t st);
cudaError_t oc_candidate(long long M, const double* x, const double* dc, const double* dv, const double* colsum,
                         double lmid, double move, double* xnew, const Reducer& red, double* vol, cudaStream_t st);
cudaError_t max_abs_diff(long long M, const double* a, const double* b, const Reducer& red, double* out,
                         cudaStream_t st);

// ---- coarse.cu : block-sparse levels (27 neighbour tiles of L x L per cell)
struct CLevel {
  int mx, my, mz;   // cells per axis
  int L;            // vectors per cell
  int g;            // group edge that formed this level from the previous one (l >= 2)
  long long ncell;  // mx*my*mz
};
template <class T>
cudaError_t coarse_smooth0(const CLevel& lv, const T* Dinv, const T* r, T* e, cudaStream_t st);
template <class T>
cudaError_t coarse_smooth(const CLevel& lv, const T* tiles, const T* Dinv, const T* r, const T* e, T* out,
                          cudaStream_t st);
template <class T>
cudaError_t coarse_residual(const CLevel& lv, const T* tiles, const T* r, const T* e, T* res, cudaStream_t st);
template <class T>
cudaError_t coarse_restrict(const CLevel& fine, const CLevel& crs, const T* Psi, const T* res, T* rc,
                            cudaStream_t st);
template <class T>
cudaError_t coarse_prolong(const CLevel& fine, const CLevel& crs, const T* Psi, const T* ec, T* e, cudaStream_t st);
template <class T>
cudaError_t coarse_apply(const CLevel& lv, const T* tiles, const T* x, T* y, cudaStream_t st);
template <class T>
cudaError_t dense_gemv(int n, const double* Ainv, const T* x, T* y, cudaStream_t st);

// ---- setup.cu
struct SetupWork;
// thr > 0: adaptive count of basis vectors per cell (eigenvalues <= thr kept, at least one)
cudaError_t level1_eigen(const Geom& g, const uint32_t* bits, const double* k64, int L1, double* phi64,
                         double* eig, uint8_t* active, int* status, double thr, cudaStream_t st);
cudaError_t level1_rowsum_corr(const Geom& g, const uint32_t* bits, const double* k64, int L1,
                               const double* phi64, int nt, const int* gcum, double* D, cudaStream_t st);
template <class TO>  // TO: stored tile type (double or float); sums in FP64
cudaError_t level1_rap(const Geom& g, const uint32_t* bits, const double* k64, int L1, const double* phi64,
                       TO* tiles, cudaStream_t st);
template <class TI>  // TI: stored type of the previous level's tiles
cudaError_t group_eigen(const CLevel& prev, const CLevel& cur, const TI* tiles_prev, const double* Dcorr,
                        const uint8_t* act_prev, double* Psi, double* eig, uint8_t* act_cur, int* status,
                        double thr, cudaStream_t st);
cudaError_t group_project_corr(const CLevel& prev, const CLevel& cur, const double* Psi, const double* Dprev,
                               double* Dcur, int nt, cudaStream_t st);
template <class TI, class TO>  // (double, double), (float, float), (float, double)
cudaError_t group_rap(const CLevel& prev, const CLevel& cur, const double* Psi, const TI* tiles_prev,
                      TO* tiles, cudaStream_t st);
template <class TT>
cudaError_t fix_inactive(const CLevel& lv, const uint8_t* act, TT* tiles, cudaStream_t st);
template <class TT>  // Dinv64 may be NULL
cudaError_t l1_inverse(const CLevel& lv, const TT* tiles, double* Dinv64, float* Dinv32, cudaStream_t st);
cudaError_t dense_assemble(const CLevel& lv, const double* tiles, double* A, cudaStream_t st);
// ---- dense.cu : blocked FP64 Cholesky + explicit inverse of the coarsest operator
long long cholesky_work_size(int n);  // doubles of scratch cholesky_inverse needs
cudaError_t cholesky_inverse(int n, double* A, double* Ainv, double* work, int* status, cudaStream_t st);
cudaError_t cvt_f64_f32(const double* a, float* b, long long n, cudaStream_t st);
template <class C>
cudaError_t phi_natural(const Geom& g, const C* phi_pad, int L1, double* out, cudaStream_t st);

}  // namespace thermo

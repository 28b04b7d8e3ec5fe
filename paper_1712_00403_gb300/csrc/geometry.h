// Mapped-geometry kernels: quadrature-point geometry, separable fit, weighted
// pressure-mass diagonal, CSR structure / assembly / SpMV.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdst.h"

namespace fdst {

// Geometry at the tensor grid of quadrature points (q1 fastest); device arrays.
struct GeoPoints {
  int nq[3] = {0, 0, 0};
  const double *pts[3] = {}, *wts[3] = {};
  int64_t Q = 0;
  double *jinv = nullptr;   // 9 x Q, (J^{-1})_{ij} at [(3i + j) Q + q]
  double *det = nullptr;    // Q
  double *nu = nullptr;     // Q
};

// Per-direction element tables (device arrays) for TH velocity (degree p+1,
// interior indices) and pressure (degree p).
struct MeshTables {
  int ne[3] = {0, 0, 0}, nq = 0, p = 0, np[3] = {0, 0, 0};
  const int *v_first[3] = {}, *p_first[3] = {};   // first global function index nonzero on element e
  const int *p_elo[3] = {}, *p_ehi[3] = {};       // element range of pressure function l
  const double *vtab[3] = {};   // [(e (p+2) + i) nq + a] * 2 + der : value / derivative of local velocity fn i
  const double *ptab[3] = {};   // [(e (p+1) + l) nq + a]
};

// CSR layout tables: velocity row (r, i): [3 velocity boxes][pressure box];
// pressure row l: [3 velocity boxes]; boxes are products of per-direction ranges.
struct CsrTables {
  int64_t off[5] = {0, 0, 0, 0, 0};
  int nv[3] = {0, 0, 0}, np[3] = {0, 0, 0};
  const int64_t *row_ptr = nullptr;
  const int *vv_lo[3] = {}, *vv_w[3] = {};
  const int *vp_lo[3] = {}, *vp_w[3] = {};
  const int *pv_lo[3] = {}, *pv_w[3] = {};
};

struct CsrDev {
  const int64_t *row_ptr = nullptr;
  const int *col = nullptr;
  const double *val = nullptr;
  const float2 *val_df = nullptr;   // the values as FP32 pairs (double-float SpMV), or nullptr
  int64_t nrows = 0, nnz = 0;
};

// kind: kGeoSineBump or kGeoAnnulus (the values of FDST_GEOM_SINE_BUMP / FDST_GEOM_ANNULUS)
constexpr int kGeoSineBump = 1, kGeoAnnulus = 2;
void launch_geo_points(const GeoPoints &gp, int kind, double amp, double contrast, cudaStream_t s);
void launch_logc(const GeoPoints &gp, double *L, cudaStream_t s);
void launch_fit_sweep(const double *L, double *f, int d, const GeoPoints &gp, int fstride, cudaStream_t s);
void launch_diag_q(const GeoPoints &gp, const MeshTables &mt, double *dq, cudaStream_t s);
void launch_csr_cols(const CsrTables &ct, int *col, cudaStream_t s);
size_t assemble_smem_bytes(int p);
fdst_status launch_assemble(const GeoPoints &gp, const MeshTables &mt, const CsrTables &ct, double *val,
                            cudaStream_t s);
// y_j = A x_j in double-float arithmetic (x pre-split into FP32 pairs, FP64 result).
void launch_spmv_df(const CsrDev &A, const float2 *x2, double *y, int64_t stride, int nrhs, const int *done,
                    cudaStream_t s);
void launch_spmv(const CsrDev &A, const double *x, double *y, int64_t stride, int nrhs, const int *done,
                 cudaStream_t s);
void launch_csr_diag(const CsrDev &A, double *d, cudaStream_t s);
// Matrix-free mapped operator, the point stage: fields G[r][a] (3 r + a) and P (9) of each
// right-hand side (Q entries each, fstride apart per right-hand side) replaced by the fluxes
// F[r][a] and the pressure test field E (FP64, or FP32 pairs with the geometry as pairs).
// mode 0: the operator; 1: B^T only (P in, F out: sigma = -P I); 2: B only (G in, E out).
void launch_mf_points_f64(double *F, int64_t Q, int64_t fstride, int nrhs, const GeoPoints &gp, const int *done,
                          int mode, cudaStream_t s);
void launch_mf_points_df(float2 *F, int64_t Q, int64_t fstride, int nrhs, const float2 *jd, const float2 *wdd,
                         const float2 *nud, const int *done, int mode, cudaStream_t s);
// Coefficient fields of diag(A) (18 fields: velocity component r, direction pair (a <= b)).
void launch_mf_diag_coef(double *C, const GeoPoints &gp, cudaStream_t s);
void launch_mf_geo_df(const GeoPoints &gp, float2 *jd, float2 *wdd, float2 *nud, cudaStream_t s);
// Rows [r0, r0 + nr) restricted to columns [c_lo, c_hi): cnt[q] = entries of row r0 + q
// kept; the copy writes them (in order) at out_ptr[q] of the new arrays.
void launch_csr_count_range(const CsrDev &A, int64_t r0, int64_t nr, int c_lo, int c_hi, int64_t *cnt,
                            cudaStream_t s);
void launch_csr_copy_range(const CsrDev &A, int64_t r0, int64_t nr, int c_lo, int c_hi, const int64_t *out_ptr,
                           int *ocol, double *oval, float2 *oval_df, cudaStream_t s);

}  // namespace fdst

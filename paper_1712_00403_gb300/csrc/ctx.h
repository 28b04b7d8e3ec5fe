// The handle (fdst_ctx) and allocation helpers shared by the C ABI files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "geometry.h"
#include "internal.h"
#include "kernels.h"
#include "kernels_tc.h"

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return FDST_CUDA_ERROR;                                                         \
    }                                                                                 \
  } while (0)

namespace fdst {

// ------------------------------------------------------------------ handle

struct FdChain {
  int nsteps = 0;
  int div_step = -1;
  const double *B[6] = {};
  const uint8_t *Bt[6] = {};   // tensor-core operand image of the same step (pre-split, padded)
  std::vector<double> Bh[6];   // host copy of B (K x N row-major) for the packing
  int R[6] = {}, K[6] = {}, N[6] = {};
  double *lam_row = nullptr, *lam_col = nullptr;
  float *lam_row_f = nullptr, *lam_col_f = nullptr;
  const double *scale = nullptr;  // D^{-1/2} of P^G (nullptr: identity)
  int64_t off = 0, size = 0;
};

struct BandDev {
  int rows, cols, w;
  double *vals;
  int *lo;
  float2 *vals_df;   // the same values split into FP32 pairs (double-float matvec)
  std::vector<double> hvals;   // host copy of vals (rows x w)
  std::vector<double> hdiag;   // host copy of the diagonal A(i, i), i < min(rows, cols)
};

// One Kronecker term of the operator: block dst += coef (F2 x F1 x F0) block src.
struct Term {
  int dst, src;
  double coef;
  int f[3];  // band ids (mode order); -1 for the unused mode in 2D
};

struct PlanOp {
  int stage;
  int in_kind, in_id;    // kind: 0 = user x block, 1 = T1 buffer, 2 = G buffer
  int out_kind, out_id;  // kind: 1 = T1, 2 = G, 3 = user y block
  int band;
  int mode;
  int dims[3];           // input dims
  double coef;
  int accumulate;
  const float2 *vals_df;  // coef x band values as FP32 pairs (double-float matvec)
  int swap;               // output written with its two slow coordinates exchanged
};

}  // namespace fdst

struct fdst_ctx {
  fdst_desc desc{};
  int dim = 0, p = 0;
  std::vector<std::vector<double>> knots;
  std::vector<fdst::Space1D> pres;
  std::vector<std::vector<fdst::Space1D>> vel;
  int nblocks = 0;
  int shape[4][3] = {};
  int64_t off[5] = {};
  int64_t n_total = 0;
  int max_rhs = 1;
  std::vector<void *> allocs;
  int64_t device_bytes = 0;
  // FD
  std::vector<fdst::FdChain> chains;
  double *work[2] = {nullptr, nullptr};
  float *work_f[2] = {nullptr, nullptr};
  std::vector<int64_t> f_off;   // per-chain offset in the padded FP32 workspace
  int64_t f_total = 0;          // padded FP32 workspace per right-hand side
  uint8_t *tmaps = nullptr;     // TMA descriptors (128 B each), chain-major, tmap_steps per chain
  int tmap_steps = 0;
  // matvec
  std::vector<fdst::BandDev> bands;
  std::vector<fdst::PlanOp> plan;
  // the same ops for the double-float matvec: in 3D the T1 buffers hold (l1, l2, i0)
  // with l1 slowest, so that the stage-2 products contract the slowest index
  std::vector<fdst::PlanOp> plan_df;
  std::vector<fdst::Term> terms;   // the operator's Kronecker terms (identity map)
  // the B and B^T parts of the operator alone (block preconditioners P_T, P_C), built
  // with the GMRES workspace on first use
  struct SubPlan {
    std::vector<fdst::PlanOp> ops, ops_df;
    std::vector<int64_t> t1_size, g_size;
    std::vector<double *> t1, g;
  } plan_b, plan_bt;
  // GMRES: Krylov basis of gm_cap + 1 block vectors (max_rhs right-hand sides each),
  // three work vectors, device scalars
  int gm_cap = 0, gm_zcap = 0;
  double *gm_V = nullptr, *gm_Z = nullptr, *gm_w = nullptr, *gm_t = nullptr, *gm_u = nullptr;
  double *gm_coef = nullptr, *gm_part = nullptr, *gm_scal = nullptr;
  int *gm_mask = nullptr;
  std::vector<double *> t1, g;
  std::vector<int64_t> t1_size, g_size;
  float2 *x2 = nullptr, *y2 = nullptr;   // double-float copies of the matvec input / output
  // MINRES
  double *v = nullptr, *v_old = nullptr, *z = nullptr, *z_new = nullptr, *Az = nullptr, *w = nullptr,
         *w_old = nullptr;
  double *partials = nullptr, *dots = nullptr;
  unsigned *counters = nullptr;
  fdst::MinresState *state = nullptr;
  int *done = nullptr, *n_stopped = nullptr;
  int *h_n_stopped = nullptr;
  double *h_dots = nullptr;
  double *hb = nullptr, *hx = nullptr;  // device buffers for the host-pointer entry points
  // mapped geometry (CSR operator, weighted pencils of P_D^G)
  bool mapped = false;
  fdst::CsrDev csr;
  fdst::CsrDev csr_b, csr_bt;   // its B and B^T blocks (built with the GMRES workspace)
  fdst::GeoPoints gp;           // geometry at the quadrature points
  // matrix-free mapped operator (sum factorization): fields at the points (10 per
  // right-hand side: G[r][a] then P, Q entries each), the plans from the solution to
  // the fields and back, the geometry as FP32 pairs
  bool mf = false;
  int64_t mf_Q = 0;
  int64_t mf_foff[10] = {};
  std::vector<fdst::PlanOp> mf_fwd, mf_fwd_df, mf_bwd, mf_bwd_df;
  std::vector<int64_t> mf_fwd_t1s, mf_fwd_gs, mf_bwd_t1s, mf_bwd_gs;
  std::vector<double *> mf_fwd_t1, mf_fwd_g, mf_bwd_t1, mf_bwd_g;
  double *mf_F = nullptr;
  float2 *mf_Fw = nullptr, *mf_jd = nullptr, *mf_wd = nullptr, *mf_nu = nullptr;
  std::vector<fdst::Term> mf_fwd_terms, mf_bwd_terms;
  // the B^T and B parts (pressure -> P -> fluxes -> velocity; velocity -> G -> E -> pressure)
  struct MfPart {
    std::vector<fdst::PlanOp> fwd, fwd_df, bwd, bwd_df;
    std::vector<int64_t> fwd_t1s, fwd_gs, bwd_t1s, bwd_gs;
    std::vector<double *> fwd_t1, fwd_g, bwd_t1, bwd_g;
  } mf_bt, mf_b;
  bool mf_parts = false;
  int mf_bv[3] = {}, mf_dv[3] = {};   // band ids of the velocity point-basis values / derivatives
  std::vector<std::vector<fdst::Mat>> geo_K, geo_M;   // [component][direction]
  std::vector<std::vector<double>> geo_scale;          // D^{-1/2} per block (P_D^G)
  // timing
  int timing = 0;
  double ms_matvec = 0, ms_prec = 0, ms_vector = 0;
  int64_t n_matvec = 0, n_prec = 0;
  // events around the matvec's compute launches alone (banded mode products or CSR SpMV,
  // without the FP64 <-> FP32-pair conversions), resolved at the end of fdst_solve
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> kev;
  double ms_kernel = 0;
  int64_t n_kernel = 0;
};

namespace fdst {

// Host-side allocation-failure injection (fdst_inject_alloc_failure): the
// status this allocation must fail with, or FDST_OK when it is not the one
// armed to fail.
fdst_status injected_alloc_failure();

template <typename T>
inline fdst_status dalloc(fdst_ctx *h, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (const fdst_status inj = injected_alloc_failure()) {
    set_error(inj == FDST_OUT_OF_MEMORY ? "cudaMalloc: out of memory (injected by fdst_inject_alloc_failure)"
                                        : "cudaMalloc: CUDA error (injected by fdst_inject_alloc_failure)");
    return inj;
  }
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? FDST_OUT_OF_MEMORY : FDST_CUDA_ERROR;
  }
  h->allocs.push_back((void *)*p);
  h->device_bytes += (int64_t)(count * sizeof(T));
  return FDST_OK;
}

template <typename T>
inline fdst_status upload(fdst_ctx *h, T **p, const std::vector<T> &v) {
  fdst_status st = dalloc(h, p, v.size());
  if (st != FDST_OK) return st;
  CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FDST_OK;
}

#define TRY(x)                           \
  do {                                   \
    fdst_status s_ = (x);                \
    if (s_ != FDST_OK) return s_;        \
  } while (0)

// Preconditioner apply and matvec of one handle (fdst.cu); exact = true forces FP64.
// s = P_D^{-1} r on the blocks in block_mask (bit b: block b; velocity 0..dim-1, pressure dim).
// B and B^T blocks of the assembled mapped operator (csr_b, csr_bt).
fdst_status build_coupling_csr(fdst_ctx *h);
// D_V^{-1/2} of P_D^G (h->geo_scale[0..2]) from diag(A) over the block vector.
void set_velocity_scaling(fdst_ctx *h, const std::vector<double> &diagA);
fdst_status run_apply(fdst_ctx *h, const double *r, double *s, int nrhs, const int *done, cudaStream_t st,
                      unsigned block_mask = ~0u);
fdst_status run_matvec(fdst_ctx *h, const double *x, double *y, int nrhs, const int *done, cudaStream_t st,
                       bool exact = false);

// What to do with a right-hand side whose recurrence estimate met its
// threshold, given its FP64 true relative residual now and at its previous
// check (negative: none). The first time the true residual is above tol the
// recurrence is resumed with a tighter threshold (its state intact: the
// estimate is a P^{-1}-norm residual, the target an l2 one). If that is not
// enough, the recurrence has drifted from the true residual (rounding in the
// iterations' arithmetic, loss of orthogonality over long runs), and MINRES
// is restarted from the current iterate with an FP64 residual, at most
// kMaxRestarts times before the solve is reported as stagnated.
enum { kKeepStopped = 0, kResume = 1, kRestart = 2, kStagnated = 3 };
constexpr int kMaxRestarts = 8;
// Lowest estimate threshold |eta_j| / |eta_0| the MINRES recurrence is asked to
// reach: below about this the recurrence runs on rounding noise (its Lanczos
// vectors are divided by tiny beta) and the iterate can be driven away from the
// solution. A check that would need a lower threshold restarts from the current
// iterate instead, and a tolerance below reach ends in FDST_STAGNATION.
constexpr double kTauFloor = 1e-14;
int resume_action(const MinresState &S, double true_rel, double prev_true, int restarts, double tol, int maxit);

// Restarts MINRES for the right-hand sides listed in `which` from the current
// iterate x: v = b - A x (FP64), z = P^{-1} v / gamma, direction vectors
// zeroed; their state keeps eta0 and the iteration count, and the estimate
// threshold becomes the one that corresponds to tol at the restart point.
// Leaves h->done[j] = 0 for the listed ones and 1 for every other one;
// hs (host copy of the states) is updated and uploaded.
// vecs: the (v, v_old, w, w_old) buffers in their current roles (default: the handle's).
fdst_status minres_restart(fdst_ctx *h, const double *b, double *x, int nrhs, const std::vector<int> &which,
                           const std::vector<double> &true_rel, double tol, std::vector<MinresState> &hs,
                           cudaStream_t st, double *const *vecs = nullptr);

}  // namespace fdst

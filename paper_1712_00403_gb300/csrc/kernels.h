// Device kernel launchers (host-callable) used by the C ABI implementation.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fdst {

constexpr int kMaxGroup = 8;

// process-wide count of kernel launches issued by this library
void count_launch(long long n);
long long launch_count();

// One mode contraction of the FD method written as a GEMM with a transposed
// store: C(r, n) = sum_k A[r*K + k] * B[k*N + n], stored at C[n*R + r].
// The contracted index is the fastest of the input, so the output's fastest
// index is the next one to contract (Algorithm 1 steps 2 and 4 as a chain of
// such steps). Optional: the input scaled by scale_in[r*K + k], the output
// divided by (lam_row[r] + lam_col[n]) (Algorithm 1 step 3) and scaled by
// scale_out[n*R + r].
struct GemmProb {
  const double *A = nullptr;
  double *C = nullptr;
  const double *B = nullptr;
  int64_t a_rhs_stride = 0, c_rhs_stride = 0;
  int R = 0, K = 0, N = 0;
  const double *lam_row = nullptr, *lam_col = nullptr;
  const double *scale_in = nullptr, *scale_out = nullptr;
  const int *done_flag = nullptr;   // skipped when *done_flag != 0 (batched solves)
};
// Up to kMaxGroup problems by value, or any number from a device table.
struct GemmGroup {
  GemmProb p[kMaxGroup];
  int nprob = 0;
  const GemmProb *table = nullptr;
  int maxR = 0, maxN = 0, tn = 0;   // with a table: largest R, N; tn: forced column tile (0 = pick)
};
void launch_gemm_f64(const GemmGroup &g, int nrhs, const int *done, cudaStream_t s);

// Banded mode product: Y = coef * (X x_mode Bd) (or Y += ...), X with dims
// (d0, d1, d2) (d0 fastest), Bd rows x d_mode banded: row i has entries
// vals[i*w + j] at columns lo[i] + j.
struct BandOp {
  const double *X = nullptr;
  double *Y = nullptr;
  const double *vals = nullptr;
  const int *lo = nullptr;
  int w = 0, rows = 0;
  int d0 = 1, d1 = 1, d2 = 1, mode = 0;
  double coef = 1.0;
  int accumulate = 0;
  int64_t x_rhs_stride = 0, y_rhs_stride = 0;
  const int *done_flag = nullptr;
};
struct BandGroup {
  BandOp op[kMaxGroup];
  int nop = 0;
  const BandOp *table = nullptr;
  int64_t maxt = 0;                 // with a table: largest output size
  int threads = 256;
};
void launch_band(const BandGroup &g, int nrhs, const int *done, cudaStream_t s);

// Double-float variant: tensors and band values are FP32 pairs (hi, lo) with
// hi + lo the value (48-bit significand); products and sums use error-free
// transformations (FMA-based exact product, Knuth's TwoSum). Same operation
// as BandOp with coef folded into vals: Y = X x_mode Bd (or Y += ...), X, Y,
// vals hold float2. With swap, Y is written with its two slow coordinates
// exchanged: the output (c0, c1, c2) with extents (e0, e1, e2) (c0 fastest,
// e_mode = rows) goes to c0 + e0 (c2 + e2 c1).
struct BandOpDF {
  const float2 *X = nullptr;
  float2 *Y = nullptr;
  double *Y64 = nullptr;            // set: the result (after accumulating Y) is written as FP64 here, same offsets
                                    // (the last product into a block writes the joined value; Y is not written)
  const float2 *vals = nullptr;
  const int *lo = nullptr;
  int w = 0, rows = 0;
  int d0 = 1, d1 = 1, d2 = 1, mode = 0;
  int accumulate = 0;
  int swap = 0;
  int64_t x_rhs_stride = 0, y_rhs_stride = 0;
  const int *done_flag = nullptr;
};
struct BandGroupDF {
  BandOpDF op[kMaxGroup];
  int nop = 0;
  const BandOpDF *table = nullptr;
  int64_t maxt = 0;
  int threads = 128;                // at most 256
  int w = 0;                        // with a table: the band width every op shares (0: mixed or unknown)
  int row_pairs = 1;                // with a shared width: modes 1/2 take band rows in pairs where they can
};
void launch_band_df(const BandGroupDF &g, int nrhs, const int *done, cudaStream_t s);
// Element-wise conversions: kind 0 double -> float (nearest), 1 double -> FP32 pair,
// 2 FP32 pair -> double, 3 float -> double.
void launch_convert(int kind, const void *in, void *out, int64_t n, cudaStream_t s);
// y2 = split(x) (double -> FP32 pair) and x = join(y2) over n entries per right-hand side.
void launch_split_df(const double *x, float2 *y, int64_t n, int64_t stride, int nrhs, const int *done,
                     cudaStream_t s);
void launch_join_df(const float2 *x, double *y, int64_t n, int64_t stride, int nrhs, const int *done,
                    cudaStream_t s);

// ---- MINRES (per right-hand side state, all device resident)
struct MinresState {
  double gamma, gamma_old, delta, c, c_old, s, s_old, eta, eta0;
  double inv_a1, a2, a3, coef_x, inv_gamma_new, tau;
  int iters, status, stop, pad;
};

// dot products <a_j, b_j> over n elements for every right-hand side j
// (vectors at stride `stride`), reduced deterministically into out[j].
void launch_dot(const double *a, const double *b, int64_t n, int64_t stride, int nrhs, double *partials,
                unsigned *counters, double *out, const int *done, cudaStream_t s);

// GMRES basis operations; basis vector k of right-hand side r at V + k * vstride + r * stride,
// rows with skip[r] != 0 left alone.
// out[r * ldo + k0 + k] = <V_{k0+k}, w> for k < kc (fixed-order reductions; part: 8 * 304 * nrhs doubles).
void launch_basis_dots(const double *V, int64_t vstride, int k0, int kc, const double *w, int64_t n,
                       int64_t stride, int nrhs, double *part, double *out, int ldo, const int *skip,
                       cudaStream_t s);
// w_r += sign * sum_{k < kc} c[r * ldc + k] V_k, kc <= 256.
void launch_basis_axpy(const double *V, int64_t vstride, int kc, const double *c, int ldc, double sign, double *w,
                       int64_t n, int64_t stride, int nrhs, const int *skip, cudaStream_t s);
// dst_r = src_r / sqrt(nrm2[r]).
void launch_scale_by_norm(const double *src, double *dst, const double *nrm2, int64_t n, int64_t stride, int nrhs,
                          const int *skip, cudaStream_t s);

// *flag = 1 when some x[i], 0 <= i < n, differs from zero (NaN counts as nonzero), else 0.
void launch_any_nonzero(const double *x, int64_t n, int *flag, cudaStream_t s);

// y_j = alpha * x_j + beta * y_j for all j (elementwise, deterministic).
void launch_axpby(const double *x, double *y, double alpha, double beta, int64_t n, int64_t stride, int nrhs,
                  cudaStream_t s);

// MINRES init after v = b - A x0, z_new = P^{-1} v and dot g = <v, z_new>.
void launch_minres_init(MinresState *st, const double *g, int *done, int nrhs, int *n_stopped, double tol,
                        cudaStream_t s);
// t = Az - (delta/gamma) v - (gamma/gamma_old) v_old; v_old <- v; v <- t (delta = <Az, z>).
// rotate: v_old <- t only (v untouched); the caller then exchanges the v and v_old pointers.
void launch_minres_lanczos(const double *Az, double *v, double *v_old, const MinresState *st,
                           const double *delta, int64_t n, int64_t stride, int nrhs, const int *done,
                           cudaStream_t s, bool rotate = false);
// a[i] <-> b[i], i < n.
void launch_swap(double *a, double *b, int64_t n, cudaStream_t s);

// scalar QR update from gamma_new^2 = <v_new, z_new> (one thread per right-hand side).
// The estimate |eta|/eta0 is compared with the per-right-hand-side threshold st.tau.
void launch_minres_scalars(MinresState *st, const double *delta, const double *g2, int nrhs, int maxit,
                           const int *done, int *n_stopped, cudaStream_t s);
// w_new = (z - a3 w_old - a2 w)/a1; w_old <- w; w <- w_new; x += coef_x w_new; z <- z_new / gamma_new;
// with z_df set, also z_df <- the double-float split of the new z (the next matvec's input).
// rotate: w_old <- w_new only (w untouched); the caller then exchanges the w and w_old pointers.
void launch_minres_update(double *w_old, double *w, double *x, double *z, const double *z_new,
                          MinresState *st, int64_t n, int64_t stride, int nrhs, int *done, cudaStream_t s,
                          float2 *z_df = nullptr, bool rotate = false);
void launch_minres_commit(MinresState *st, int *done, int nrhs, cudaStream_t s);
// v = b - Ax, v_old = w = w_old = 0 for the right-hand sides with done[j] == 0.
void launch_restart_vectors(const double *b, const double *Ax, double *v, double *v_old, double *w, double *w_old,
                            int64_t n, int64_t stride, int nrhs, const int *done, cudaStream_t s);
// z <- z / gamma (per right-hand side) used at start.
void launch_scale_by_inv_gamma(double *z, const MinresState *st, int64_t n, int64_t stride, int nrhs,
                               const int *done, cudaStream_t s);

}  // namespace fdst

/*
 * fdst.h - C ABI of the GB300 library for Fast-Diagonalization (FD)
 * preconditioned MINRES on the isogeometric Stokes system
 * (Montardini, Sangalli, Tani, arXiv 1712.00403).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Unknowns are ordered as the block system of Sec. 3 (eq. Stokes_system):
 *   [u_1; u_2; (u_3;) p]. Each block is vec-ordered with i1 fastest (Sec. 2.3,
 *   vec operator): index i1 + n1*(i2 + n2*i3). Velocity blocks hold interior
 *   (Dirichlet-free) functions only (Taylor-Hood: eq. V_TH_0_basis1;
 *   Raviart-Thomas: eq. basisRT_V1); the pressure block holds all functions.
 * - Several right-hand sides are stored back to back: vector j starts at
 *   j * n_total doubles.
 * - Pointers named d_* are device pointers owned by the caller; pointers named
 *   h_* are host pointers owned by the caller. Device work is enqueued on the
 *   given stream (NULL = legacy default stream) and is asynchronous unless a
 *   function says otherwise. Input and output vectors must not alias.
 * - Every function returns an fdst_status; nothing throws across the ABI.
 *   fdst_last_error() returns a thread-local text for the last failure.
 */
#ifndef FDST_H
#define FDST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-compatible with cudaStream_t; callers need not include CUDA headers. */
typedef struct CUstream_st *fdst_stream;
typedef struct fdst_ctx *fdst_handle;

typedef enum {
  FDST_OK = 0,
  FDST_INVALID_ARGUMENT = 1, /* bad knots (not open, decreasing, multiplicity > p), sizes, flags */
  FDST_NOT_SPD = 2,          /* Cholesky of a univariate mass matrix failed */
  FDST_OUT_OF_MEMORY = 3,    /* device allocation failed */
  FDST_CUDA_ERROR = 4,       /* a CUDA runtime call failed */
  FDST_MAXIT = 5,            /* MINRES hit maxit before the tolerance */
  FDST_STAGNATION = 6,       /* MINRES residual estimate stopped decreasing */
  FDST_BREAKDOWN = 7,        /* Lanczos breakdown: preconditioner not positive on a Krylov vector */
  FDST_TIMEOUT = 8,          /* a bounded device-side wait expired */
  FDST_NAN_DETECTED = 9,     /* NaN/Inf in a MINRES inner product */
  FDST_ADMISSION_REJECTED = 10,
  FDST_NOT_SUPPORTED = 11,   /* combination of options not implemented */
  FDST_CANCELLED = 12        /* a server request cancelled before it finished (fdst_server_cancel) */
} fdst_status;

enum { FDST_TH = 0, FDST_RT = 1 };                          /* discretization (Sec. 2.2) */
/* FD contraction arithmetic: FP64 (DFMA); split-TF32 (each operand = TF32 hi +
 * lo, products hi*hi + hi*lo + lo*hi on tcgen05); split-BF16 (each operand =
 * three bf16 pieces, the six products with piece indices i + j <= 2). Both
 * split forms accumulate in FP32 and keep FP32 intermediates. */
enum { FDST_FD_F64 = 0, FDST_FD_TF32X3 = 1, FDST_FD_BF16X6 = 2 };
/* Geometry map G of the parametric cube (3D Taylor-Hood): the identity; the sine
 * bump x = eta + a sin(pi eta1) sin(pi eta2) sin(pi eta3) (1,1,1); or the eighth
 * of a thick annulus of Sec. 7 (inner radius 1, outer 2, height 1) in polar form
 * x = (r cos t, r sin t, eta3), r = 1 + eta1, t = pi eta2 / 4. */
enum { FDST_GEOM_IDENTITY = 0, FDST_GEOM_SINE_BUMP = 1, FDST_GEOM_ANNULUS = 2 };
/* P_D (Sec. 5) or P_D^G (Sec. 6): P_D^G needs a mapped geometry (3D TH) or the
 * viscosity family on the identity map (3D TH or RT); with a constant viscosity
 * on the identity map it equals P_D and setup returns FDST_NOT_SUPPORTED. */
enum { FDST_VARIANT_PD = 0, FDST_VARIANT_PD_GEO = 1 };
/* Matvec arithmetic: FP64 (DFMA), or double-float (each value an unevaluated
 * sum of two floats, 48-bit significand, error-free FMA products and TwoSum
 * additions on the FP32 units). fdst_solve ends on a true residual computed
 * with the FP64 matvec. */
enum { FDST_MV_F64 = 0, FDST_MV_DF64 = 1 };
enum { FDST_MATVEC_ASSEMBLED = 0, FDST_MATVEC_MATRIX_FREE = 1 };
/* Block preconditioners for GMRES (Sec. 4): P_T = [[P_V, B^T], [0, -P_Q]] (block
 * triangular) and P_C = [[P_V, B^T], [B, B P_V^{-1} B^T - P_Q]] (constraint). */
enum { FDST_PREC_PT = 0, FDST_PREC_PC = 1 };
/* GMRES form: left-preconditioned (Arnoldi on P^{-1} A), flexible right-preconditioned
 * (Arnoldi on A with z_j = P^{-1} v_j kept: exact Arnoldi relation whatever the
 * precision of P^{-1}), or AUTO (left with the FP64 FD apply, flexible with the split ones). */
enum { FDST_GMRES_LEFT = 0, FDST_GMRES_FLEXIBLE = 1, FDST_GMRES_AUTO = 2 };

typedef struct {
  int dim;                 /* 2 or 3 */
  int discretization;      /* FDST_TH or FDST_RT */
  int degree;              /* pressure spline degree p >= 1; velocity degree is p+1 (Sec. 2.2) */
  const double *h_knots[3];/* open pressure knot vector of each direction on [0,1] (Sec. 2.1) */
  int nknots[3];           /* its length m + p + 1 */
  double viscosity;        /* constant nu > 0 (identity geometry); ignored on the mapped geometries */
  int geometry;            /* FDST_GEOM_* */
  int variant;             /* FDST_VARIANT_* */
  int fd_precision;        /* FDST_FD_* */
  double cpen;             /* Nitsche penalty C_pen (RT); <= 0 selects 5(alpha+1) (Sec. 7) */
  int max_rhs;             /* most right-hand sides one call will pass (workspace sizing), >= 1 */
  int matvec_precision;    /* FDST_MV_F64 or FDST_MV_DF64 */
  double geometry_amplitude;  /* sine-bump amplitude a, in (0, 0.25]; <= 0 selects 0.1; ignored by the annulus */
  double viscosity_contrast;  /* k >= 1 selects nu(x) = 1 + (k - 1)(1 - cos(2 pi x1)) / 2 (values in
                                 [1, k]); <= 0: on a mapped geometry the map's own field (nu(x) = 1 +
                                 0.5 sin(2 pi x1) cos(2 pi x2) on the sine bump, nu = 1 on the annulus),
                                 on the identity map the constant `viscosity`. On the identity map (3D,
                                 TH or RT) the family depends on eta_1 alone: the operator stays a sum of
                                 Kronecker products, each A-block term's direction-1 factor weighted by
                                 nu (the RT Nitsche faces included), and FDST_VARIANT_PD_GEO builds the
                                 Appendix's weighted pencils for it (RT: K~ with tau(0), tau(1)).
                                 0 < k < 1 is FDST_INVALID_ARGUMENT; k >= 1 in 2D FDST_NOT_SUPPORTED */
  int matvec_form;         /* mapped geometry: FDST_MATVEC_ASSEMBLED (CSR) or FDST_MATVEC_MATRIX_FREE
                              (no CSR: the operator, its B and B^T parts and diag(A) by sum
                              factorization at the quadrature points, FP64 for the true residual);
                              ignored on the identity map (Kronecker operator) */
} fdst_desc;

typedef struct {
  int dim;
  int64_t n_total;         /* length of one block vector */
  int nblocks;             /* dim velocity blocks + 1 pressure block */
  int64_t block_offset[4];
  int block_shape[4][3];   /* (n1, n2, n3) of each block; n3 = 1 in 2D */
  int64_t device_bytes;    /* device memory held by the handle */
  double flops_apply;      /* algorithmic flops of one preconditioner apply (one right-hand side):
                              velocity 4 N sum_d n_d (Algorithm 1 steps 2 and 4), pressure 2 N sum_d n_d */
  double flops_matvec;     /* algorithmic flops of one matvec: 2 x (band entries used) over the
                              banded Kronecker factors of the evaluation plan (identity map, or
                              the matrix-free plans of the mapped operator without their point
                              stage), or 2 x nonzeros of the assembled CSR */
} fdst_sizes;

typedef struct {
  int iterations;
  int status;              /* FDST_OK (converged), FDST_MAXIT, FDST_BREAKDOWN, FDST_NAN_DETECTED, ... */
  double eta_rel;          /* final ||r||_{P^-1} / ||r_0||_{P^-1} from the MINRES recurrence */
  double true_rel_res;     /* ||b - A x||_2 / ||b||_2 computed in FP64 after the solve */
  int iterations_estimate; /* iteration at which the recurrence estimate first met tol (a stopping
                              rule on the estimate alone); iterations continue until the FP64 true
                              residual meets tol */
} fdst_solve_info;

/*
 * fdst_setup - build the spaces, univariate matrices, eigen-factors and
 * device data of one Stokes problem (Sec. 2.1-2.2, Sec. 5, eq. eig_dec,
 * Algorithm 1 step 1; Sec. 6 and the Appendix for FDST_VARIANT_PD_GEO).
 * Host arrays in *desc are copied; the caller keeps them. Blocks the host
 * until the device data are uploaded. On failure *out is NULL.
 * Errors: FDST_INVALID_ARGUMENT, FDST_NOT_SPD, FDST_OUT_OF_MEMORY,
 * FDST_CUDA_ERROR, FDST_NOT_SUPPORTED.
 */
fdst_status fdst_setup(const fdst_desc *desc, fdst_handle *out);

/* Release every device and host resource of the handle (NULL is accepted). */
fdst_status fdst_destroy(fdst_handle h);

/* Sizes and layout of the block vectors of the handle. */
fdst_status fdst_get_sizes(fdst_handle h, fdst_sizes *out);

/*
 * fdst_apply_prec - s = P^{-1} r for nrhs stacked vectors, with P = P_D =
 * diag(P_V, P_Q) (eq. P_D) or P_D^G (Sec. 6). Velocity blocks by the FD method
 * (Algorithm 1: s = (U3 x U2 x U1) Delta^{-1} (U3 x U2 x U1)^T r with
 * Delta = sum_d c_d Lambda_d, c_k = 2 for component k, eq. prec3D_TH),
 * pressure by P_Q^{-1} = M3^{-1} x M2^{-1} x M1^{-1} (eq. precQ).
 * d_r, d_s: device, nrhs * n_total doubles each, not aliased.
 * Uses the handle's workspace: calls on one handle must not overlap in time.
 * Errors: FDST_INVALID_ARGUMENT (nrhs < 1 or > max_rhs), FDST_CUDA_ERROR.
 */
fdst_status fdst_apply_prec(fdst_handle h, const double *d_r, double *d_s, int nrhs, fdst_stream stream);

/*
 * fdst_matvec - y = A x with A the Stokes matrix of eq. Stokes_system:
 * matrix-free Kronecker form on the identity map (blocks A_rs, B_r of Sec. 3
 * with nu constant), assembled CSR on a mapped geometry; arithmetic as set by
 * desc.matvec_precision.
 * d_x, d_y: device, nrhs * n_total doubles each, not aliased.
 */
fdst_status fdst_matvec(fdst_handle h, const double *d_x, double *d_y, int nrhs, fdst_stream stream);

/*
 * fdst_solve - P-preconditioned MINRES (Paige-Saunders; Sec. 4, Sec. 7: tol
 * 1e-8, x0 = 0) on nrhs independent right-hand sides at once. Every
 * right-hand side keeps its own recurrence and stops on its own when
 * ||r_j||_{P^-1} <= tol ||r_0||_{P^-1}. d_x holds the initial guesses on entry
 * and the solutions on exit (an all-zero d_x is detected and r_0 = b taken
 * without a matvec). The true residual ||b - A x||_2 / ||b||_2 is checked in
 * FP64 when the estimates meet their thresholds. info: host
 * array of nrhs entries, filled when the call returns (the call synchronizes
 * the stream). Returns FDST_OK when every right-hand side converged,
 * otherwise the first non-OK per-RHS status. Per-RHS statuses: FDST_OK,
 * FDST_MAXIT (maxit reached), FDST_STAGNATION (the true residual stayed
 * above tol through the restarts), FDST_BREAKDOWN (<P^-1 v, v> < 0: the
 * preconditioner is not positive definite on a Krylov vector),
 * FDST_NAN_DETECTED (NaN/Inf in an inner product, e.g. from a non-finite
 * right-hand side), FDST_TIMEOUT (a bounded wait in a tensor-core kernel
 * expired during the solve; the iterates are not trustworthy).
 */
fdst_status fdst_solve(fdst_handle h, const double *d_b, double *d_x, int nrhs, double tol, int maxit,
                       fdst_solve_info *info, fdst_stream stream);

/*
 * fdst_apply_block_prec - s = P^{-1} r for P = P_T (back substitution: q =
 * -P_Q^{-1} r_q, u = P_V^{-1}(r_u - B^T q)) or P = P_C (the paper's product
 * form: z = P_V^{-1} r_u, q = -P_Q^{-1}(r_q - B z), u = z - P_V^{-1} B^T q),
 * Sec. 4; P_V^{-1}, P_Q^{-1} the handle's FD applies, B and B^T in its matvec
 * precision: Kronecker plans on the identity map, the B and B^T blocks of the
 * assembled CSR on a mapped handle, the velocity-only / pressure-only parts of
 * the sum-factorization plans on a matrix-free mapped handle (there P_V, P_Q
 * are the P_D^G blocks when the handle's variant is P_D^G). Device vectors of
 * nrhs block vectors; r and s must not alias. Asynchronous on stream (the
 * first call builds the B / B^T plans and the GMRES work vectors).
 */
fdst_status fdst_apply_block_prec(fdst_handle h, int prec, const double *d_r, double *d_s, int nrhs,
                                  fdst_stream stream);

/*
 * fdst_solve_gmres - GMRES (Saad-Schultz) with P_T or P_C (Sec. 4; eq. P_T,
 * eq. P_C, applied through the product form of P_C^{-1}), their P_V, P_Q
 * blocks the handle's FD applies and B, B^T the Kronecker parts of the
 * operator (identity map) or of the mapped operator, as fdst_apply_block_prec.
 *   form:    FDST_GMRES_LEFT, FDST_GMRES_FLEXIBLE or FDST_GMRES_AUTO (above).
 *   b, x:    device block vectors (nrhs back to back), x the initial guess in and
 *            the solution out, as fdst_solve; an all-zero x (the paper's start)
 *            is detected on the device and the first residual taken as b.
 *   restart: Krylov basis size m in [1, 255]; the handle keeps a basis of
 *            (m + 1) x max_rhs block vectors (and m more for the flexible form),
 *            allocated on first use and grown when a larger m is asked for, and
 *            restarts from the current iterate when it is full.
 * Arnoldi with classical Gram-Schmidt applied twice, Givens rotations on the
 * Hessenberg matrix; the estimate is ||P^{-1}(b - A x_j)|| / ||P^{-1} b||
 * (left) or ||b - A x_j|| / ||b|| (flexible). When
 * it meets the threshold (tol at first) x_j is formed and its FP64 true
 * residual ||b - A x_j|| / ||b|| computed: <= tol ends that right-hand side,
 * otherwise the threshold drops to 0.5 tau tol / true and the Arnoldi process
 * continues. info[r]: iterations, status, eta_rel (the estimate),
 * true_rel_res, iterations_estimate (first iteration with estimate <= tol).
 * Synchronizes the stream. Matvecs in the iterations use the handle's matvec
 * precision.
 */
fdst_status fdst_solve_gmres(fdst_handle h, int prec, int form, const double *d_b, double *d_x, int nrhs,
                             double tol, int maxit, int restart, fdst_solve_info *info, fdst_stream stream);

/*
 * fdst_solve_host - fdst_solve with host vectors: copies h_b (and h_x as the
 * initial guess) to handle-owned device buffers, solves, copies the
 * solutions back to h_x. Pinned host memory makes the copies asynchronous.
 */
fdst_status fdst_solve_host(fdst_handle h, const double *h_b, double *h_x, int nrhs, double tol, int maxit,
                            fdst_solve_info *info, fdst_stream stream);

/*
 * fdst_solve_host_zero - fdst_solve_host from the zero initial guess (the
 * paper's x0 = 0, Sec. 7): h_x is output only (never read), the device
 * iterate is cleared on the device, so only h_b travels to the GPU and only
 * the solutions come back. Same arguments, errors and info as fdst_solve_host.
 */
fdst_status fdst_solve_host_zero(fdst_handle h, const double *h_b, double *h_x, int nrhs, double tol, int maxit,
                                 fdst_solve_info *info, fdst_stream stream);

/* fdst_apply_prec_host - fdst_apply_prec with host vectors (copies in and out). */
fdst_status fdst_apply_prec_host(fdst_handle h, const double *h_r, double *h_s, int nrhs, fdst_stream stream);

/*
 * fdst_set_timing - when on, fdst_solve records CUDA events around its
 * phases (Stokes matvec, preconditioner, vector updates) on its stream and
 * accumulates their durations; fdst_get_timing returns the sums (ms) and the
 * number of matvec and preconditioner launches since the last reset.
 */
fdst_status fdst_set_timing(fdst_handle h, int on);
fdst_status fdst_get_timing(fdst_handle h, double *ms_matvec, double *ms_prec, double *ms_vector,
                            int64_t *n_matvec, int64_t *n_prec);

/*
 * fdst_get_kernel_timing - with timing on, the matvecs inside the MINRES
 * iterations also record CUDA events around their compute launches alone (the
 * banded Kronecker mode products of the Cartesian operator, or the CSR SpMV on
 * mapped geometry; not the FP64 <-> FP32-pair conversions around them). Returns
 * the summed duration (ms, resolved when fdst_solve returns) and the number of
 * launches inside those spans since the last fdst_set_timing. FDST_INVALID_ARGUMENT
 * for a NULL handle; NULL outputs are skipped.
 */
fdst_status fdst_get_kernel_timing(fdst_handle h, double *ms, int64_t *launches);

/*
 * fdst_convert - the element-wise precision conversions of the mixed-precision
 * paths, done on the integer units from the IEEE 754 binary64/binary32
 * encodings (GB300's conversion instructions run on its small FP64 unit):
 *   kind 0: double -> float, rounded to nearest (ties to even);
 *   kind 1: double -> double-float pair (hi, lo) as 2 floats per entry, hi the
 *           truncated leading 24 bits, hi + lo within 2^-48 |x|;
 *   kind 2: double-float pair (2 floats per entry) -> double (hi + lo, rounded);
 *   kind 3: float -> double (exact).
 * d_in, d_out: device buffers of n entries (caller-owned, not overlapping).
 * Asynchronous on stream. FDST_INVALID_ARGUMENT for a kind outside 0..3,
 * n < 0 or a NULL buffer with n > 0.
 */
fdst_status fdst_convert(int kind, const void *d_in, void *d_out, int64_t n, fdst_stream stream);

/*
 * fdst_fd_apply_static - allocation-free FD solve of one Kronecker-sum block:
 *   s = (U_d x ... x U_1) Delta^{-1} (U_d x ... x U_1)^T r,
 *   Delta[i1, i2, (i3)] = sum_d coef[d] * lam_d[i_d],
 * i.e. the solution of sum_d coef[d] (x)_e (K_e if e == d else M_e) s = r for
 * pencils K_d U_d = M_d U_d diag(lam_d), U_d^T M_d U_d = I. The paper has no
 * counterpart of this entry point: it exists for callers that cannot call
 * cudaMalloc (code inside another framework's memory pool or allocator lock,
 * hosts that forbid device allocation after start-up, call sites that must
 * not trigger an allocation). It needs no handle and allocates nothing.
 *   dim: 2 or 3; n[d]: univariate sizes, 1 <= n[d] <= 256, prod n[d] <= 2359296
 *   (larger sizes return FDST_INVALID_ARGUMENT with a message);
 *   d_U[d]: device, n[d] x n[d] row-major eigenvector matrix U_d (U[i][a] =
 *   component i of eigenvector a); d_lam[d]: device, n[d] eigenvalues;
 *   coef: host, dim coefficients; d_r, d_s: device, prod n[d] doubles each,
 *   vec-ordered with i1 fastest. d_s is also used as intermediate storage
 *   during the call. r and s must not overlap, and neither may lie inside the
 *   static scratch array (FDST_INVALID_ARGUMENT otherwise). The library cannot
 *   see buffer lengths: U_d, lam_d, r and s must hold the sizes above.
 *   Asynchronous on `stream`.
 * Scratch: one file-scope __device__ array of 2359296 + 4*256*256 + 256
 * doubles (about 21 MB) that every GPU which loads the library holds until
 * the process exits. All calls on a device share it and it keeps the last
 * call's contents (every call overwrites what it reads), so calls whose
 * device work overlaps in time (different streams, threads or processes
 * sharing the context) race and must be serialized by the caller.
 * Every call looks up the array's device address (cudaGetSymbolAddress) on
 * the current device instead of caching it, so the address stays right after
 * the context is reset and re-created. The first call on a device also loads
 * the library's device code there; make that first call before any stream
 * capture.
 */
fdst_status fdst_fd_apply_static(int dim, const int n[3], const double *const d_U[3], const double *const d_lam[3],
                                 const double coef[3], const double *d_r, double *d_s, fdst_stream stream);

/*
 * Batched solves: many independent problems of uneven sizes, one right-hand
 * side each, advanced together. Every phase of a MINRES iteration (Stokes
 * matvec rounds, each FD contraction step, inner products, vector updates)
 * is one grouped launch over all problems, and one iteration is replayed from
 * a CUDA graph. The handles must share fd_precision and matvec_precision and
 * use the identity geometry; a handle may belong to one batch at a time and
 * must not be used on its own while the batch solves (the batch uses the
 * handle's workspace). autotune != 0 times, on the batch's own shapes at
 * creation, how each contraction step's tensor-core launch is fed (B streamed
 * with A at each ring depth that fits, B resident in shared memory, A's TF32
 * pieces in tensor memory) and the banded-kernel block size, and keeps the
 * fastest of each (fdst_batch_info, fdst_batch_tuning report them); without it
 * B is streamed at the deepest ring that fits.
 */
typedef struct fdst_batch_ctx *fdst_batch;
fdst_status fdst_batch_create(const fdst_handle *handles, int n, int autotune, fdst_batch *out);
/* d_b[i], d_x[i]: device vectors of handle i (x: initial guess in, solution out);
 * info: n entries. Same stopping rule as fdst_solve; synchronizes the stream. */
fdst_status fdst_batch_solve(fdst_batch b, const double *const *d_b, double *const *d_x, double tol, int maxit,
                             fdst_solve_info *info, fdst_stream stream);
fdst_status fdst_batch_info(fdst_batch b, int *tc_ring, int *band_threads, double *ms_apply, double *ms_matvec);
/* The autotuner's choice per contraction step: *nsteps = the number of steps;
 * for the first min(cap, *nsteps) steps modes[i] = 1 (B streamed), 2 (B
 * resident, A in shared memory) or 3 (B resident, A in tensor memory) and
 * rings[i] = the ring depth (0 = as deep as fits); both 0 for an FP64 batch.
 * Arrays are caller-owned host memory of cap entries (cap = 0 queries nsteps). */
fdst_status fdst_batch_tuning(fdst_batch b, int cap, int *nsteps, int *modes, int *rings);
/* Sets the feeding mode and ring depth of every contraction step (n = the
 * number of steps, modes and rings as above, host arrays read during the call).
 * FDST_NOT_SUPPORTED (nothing changed) when a mode does not fit a step's shapes
 * or the batch is FP64; FDST_INVALID_ARGUMENT for other values. */
fdst_status fdst_batch_set_tuning(fdst_batch b, int n, const int *modes, const int *rings);
fdst_status fdst_batch_destroy(fdst_batch b);

/*
 * Request server (continuous batching). Requests queue on submission; each
 * fdst_server_step finishes the active problems whose recurrence stopped and
 * whose FP64 true residual is <= tol (their solution is copied to host memory
 * and their device handle returns to an idle cache keyed by problem shape),
 * admits queued requests while fewer than max_active are active and the
 * device memory held stays within hbm_budget_bytes (evicting idle handles
 * least-recently-used first), and advances every active problem by
 * iters_per_step MINRES iterations with grouped launches. Times are in the
 * caller's clock (t_arrival given at submission, `now` at each step).
 * A request whose device handle, once set up, needs more than the whole
 * budget can never be admitted: it finishes with FDST_ADMISSION_REJECTED.
 * A request whose handle set-up fails finishes with that status
 * (FDST_OUT_OF_MEMORY when a device allocation failed); the server goes on
 * with the others. If a bounded wait in a tensor-core kernel expires during a
 * step, every request active in that step finishes with FDST_TIMEOUT.
 */
typedef struct {
  int64_t hbm_budget_bytes;  /* device bytes the server may hold in handles; <= 0: 90% of free memory */
  int max_active;            /* most problems advanced together (>= 1) */
  int fd_precision;          /* FDST_FD_* for every request */
  int matvec_precision;      /* FDST_MV_* for every request */
  double tol;                /* MINRES tolerance (true relative residual) */
  int maxit;
  int iters_per_step;        /* MINRES iterations per fdst_server_step (>= 1) */
} fdst_server_opts;
typedef struct fdst_server_ctx *fdst_server;
fdst_status fdst_server_create(const fdst_server_opts *opts, fdst_server *out);
/* problem: as for fdst_setup (max_rhs and precisions are the server's); h_b: host
 * right-hand side of the problem's n_total entries, copied. */
fdst_status fdst_server_submit(fdst_server s, const fdst_desc *problem, const double *h_b, double t_arrival,
                               int64_t *id);
fdst_status fdst_server_step(fdst_server s, double now, int *n_active, int *n_queued, int64_t *n_finished);
/* *finished = 1 once the request is done; then h_x (n_total doubles, may be NULL) and info are filled. */
fdst_status fdst_server_result(fdst_server s, int64_t id, int *finished, double *h_x, fdst_solve_info *info,
                               double *t_arrival, double *t_admit, double *t_done);
fdst_status fdst_server_stats(fdst_server s, int64_t *handles_created, int64_t *handles_reused,
                              int64_t *handles_evicted, int64_t *bytes_held, int *max_active_seen);
/*
 * fdst_server_cancel - withdraws request `id`. A queued request finishes at
 * once with status FDST_CANCELLED (a device handle still being set up for it
 * in the background goes to the idle cache when ready); an active one is
 * retired at the start of the next fdst_server_step with FDST_CANCELLED, its
 * handle returned to the idle cache. A cancelled request returns no solution
 * (h_x of fdst_server_result is left as it is). A finished request is left
 * as it is. FDST_INVALID_ARGUMENT for an unknown id or a NULL server.
 */
fdst_status fdst_server_cancel(fdst_server s, int64_t id);
fdst_status fdst_server_destroy(fdst_server s);

/* Number of CUDA kernels this library has launched in the process so far
 * (diagnostics: lets a caller count the kernels inside a timed region). */
int64_t fdst_kernel_launches(void);

/*
 * fdst_check_bounded_wait - self-test of the failure detection, without a fault:
 * launches one thread that waits, through the bounded mbarrier wait of the
 * tensor-core kernel, on a barrier nothing arrives on. *gave_up = 1 when the
 * wait expired after its limit (about 2 s) and raised its abort flag, and the
 * kernel returned; *seconds = the launch's duration. The device stays usable.
 * Returns FDST_TIMEOUT (the status a real expiry gives) when the wait expired
 * as designed, FDST_OK if it did not expire (the test failed);
 * FDST_INVALID_ARGUMENT for NULL outputs; synchronous.
 */
fdst_status fdst_check_bounded_wait(int *gave_up, double *seconds);

/* *flag = 1 when a bounded device-side wait in a tensor-core kernel expired
 * (the kernel then skipped its output and returned) since the library loaded;
 * synchronizes the device. */
fdst_status fdst_device_error(int *flag);

/*
 * fdst_inject_alloc_failure - host-side fault injection for tests: the nth
 * device allocation the library makes for a handle from now on (nth >= 1,
 * counted across threads) fails without calling cudaMalloc, with `status`:
 * FDST_OUT_OF_MEMORY (as when device memory runs out) or FDST_CUDA_ERROR (as
 * when the runtime reports another error). fdst_setup then returns that
 * status (a server request finishes with it). nth <= 0 disarms. Nothing on
 * the GPU is touched. FDST_INVALID_ARGUMENT for another status.
 */
fdst_status fdst_inject_alloc_failure(int64_t nth, int status);

/* Thread-local description of the last error on this thread. */
const char *fdst_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FDST_H */

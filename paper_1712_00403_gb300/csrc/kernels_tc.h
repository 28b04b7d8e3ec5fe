// Split-TF32 tensor-core (tcgen05) mode contraction: launcher interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/fdst.h"

namespace fdst {

// Same contraction as GemmProb (C(r, n) = sum_k A(r, k) B(k, n) stored at
// C[n*R + r]) with FP32 intermediates; B is pre-split into TF32 hi/lo parts.
// A is read by TMA from the FP32 array A32 (row r at r*lda, lda a multiple of
// 4, right-hand sides a_rhs_stride apart) through the tensor map `tmap`
// (device memory, made by tc_encode_map). When A64 is set (first step of a
// chain) the group's launch first writes A32 = (float)(A64 * scale_in)
// (A64 rows at r*K, right-hand sides a64_rhs_stride apart). C(r, n) with
// r = u*out_nv + v is stored at (n*(R/out_nv) + u)*ldc + v: the output's rows
// (n, u) hold the next contracted index v, padded to ldc (a multiple of 32
// for FP32 outputs; out_nv = ldc = R writes C[n*R + r]); the last step writes
// FP64 (C64, times scale_out).
struct TcProb {
  const double *A64 = nullptr;
  const float *A32 = nullptr;
  const void *tmap = nullptr;
  double *C64 = nullptr;
  float *C32 = nullptr;
  const float *Bt = nullptr;
  int64_t a_rhs_stride = 0, a64_rhs_stride = 0, c_rhs_stride = 0;
  int R = 0, K = 0, N = 0;
  int lda = 0, out_nv = 0, ldc = 0;
  const float *lam_row = nullptr, *lam_col = nullptr;
  const double *scale_in = nullptr, *scale_out = nullptr;
  const int *done_flag = nullptr;   // the problem is skipped when *done_flag != 0 (batched solves)
};
// Up to 8 problems by value, or any number from a device table (table != nullptr).
struct TcGroup {
  TcProb p[8];
  int nprob = 0;
  const TcProb *table = nullptr;
  int maxR = 0, maxN = 0;           // with a table: largest tc_padded_rows and N among its problems
  int convert = 0;                  // 1: convert A64 into A32 first (problems with A64 set)
};
// Writes the TMA descriptor (128 bytes, host memory) that reads boxes of
// 32 columns x 32 rows of one row run of A32 into the K-major SWIZZLE_128B
// shared-memory image of the tensor-core operand. A32 rows r = u*nv + v
// (v < nv, u < nu) hold K values at pitch lda floats; right-hand sides are
// rhs_stride floats apart. Columns at or beyond K and rows v at or beyond nv
// read as zero.
fdst_status tc_encode_map(void *map128, const float *A32, int K, int nv, int nu, int lda, int64_t rhs_stride, int nrhs);
// Rows a contraction occupies in the kernel's row-group grid: R / out_nv runs
// of out_nv rows, each padded to a multiple of 32 (TcGroup.maxR in table mode).
int tc_padded_rows(int R, int out_nv);
// Row pitch (floats) of the FP32 operands and intermediates: K rounded up to 32.
inline int tc_ld(int K) { return (K + 31) & ~31; }
// ring: shared-memory stages (0 = as many as fit, capped at 4).
fdst_status launch_gemm_tc(const TcGroup &g, int nrhs, const int *done, cudaStream_t s, int ring = 0);
// number of stages that fit for the widest column tile of g
int tc_max_ring(const TcGroup &g);

// Host packing of B (K x N row-major FP64) into the kernel's per-stage
// shared-memory image (TF32 hi/lo, SWIZZLE_32B K-major); size in floats.
size_t tc_packed_floats(int K, int N);
void tc_pack(const double *B, int K, int N, std::vector<float> &out);
// 1 when a bounded wait inside the tensor-core kernel expired since start.
fdst_status tc_error_flag(int *value);

}  // namespace fdst

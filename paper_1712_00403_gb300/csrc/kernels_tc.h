// Split-TF32 tensor-core (tcgen05) mode contraction: launcher interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/fdst.h"

namespace fdst {

// Same contraction as GemmProb (C(r, n) = sum_k A(r, k) B(k, n) stored at
// C[n*R + r]) with FP32 intermediates: the first step reads the FP64 input,
// the last writes FP64; B is pre-split into TF32 hi/lo parts.
// Row r of A starts at r*lda (lda = K for the FP64 input, a multiple of 4
// for FP32 intermediates). C(r, n) with r = u*out_nv + v is stored at
// (n*(R/out_nv) + u)*ldc + v: the output's rows (n, u) hold the next
// contracted index v, padded to ldc (out_nv = ldc = R writes C[n*R + r]).
struct TcProb {
  const double *A64 = nullptr;
  const float *A32 = nullptr;
  double *C64 = nullptr;
  float *C32 = nullptr;
  const float *Bt = nullptr;
  int64_t a_rhs_stride = 0, c_rhs_stride = 0;
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
  int maxR = 0, maxN = 0;           // with a table: largest R and N among its problems
};
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

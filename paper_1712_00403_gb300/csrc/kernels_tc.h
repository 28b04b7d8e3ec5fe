// Split-TF32 tensor-core (tcgen05) mode contraction: launcher interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/fdst.h"

namespace fdst {

// Same contraction as GemmProb (C(r, n) = sum_k A(r, k) B(k, n)) with FP32
// intermediates; B is pre-split into TF32 hi/lo parts. A is read by TMA from
// the FP32 array A32 (row r at r*lda, lda a multiple of 8; right-hand sides
// a_rhs_stride apart) through the tensor map `tmap` (device memory, made by
// tc_encode_map). When A64 is set (first step of a chain) the group's launch
// first writes A32 = (float)(A64 * scale_in) (A64 rows at r*K, right-hand
// sides a64_rhs_stride apart). Rows r = u*out_nv + v (out_nv = size of the
// next contracted index): on intermediate steps C(r, n) goes in FP32 to
// n*c_cs + u*ldv + v (the next step's rows, pitch ldv = its lda, c_cs =
// (R/out_nv)*ldv); on the last step in FP64, times scale_out, to n*R + r.
struct TcProb {
  const double *A64 = nullptr;
  const float *A32 = nullptr;
  const void *tmap = nullptr;
  double *C64 = nullptr;
  float *C32 = nullptr;
  const uint8_t *Bt = nullptr;      // B image (tc_pack) of the group's split mode
  int64_t a_rhs_stride = 0, a64_rhs_stride = 0, c_rhs_stride = 0;
  int64_t c_cs = 0;
  int R = 0, K = 0, N = 0;
  int lda = 0, out_nv = 0, ldv = 0;
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
  int convert = 0;                  // 1: convert A64 into A32 first (problems with A64 set)
  int split = 0;                    // 0: split-TF32 (hi/lo, 3 products); 1: split-BF16 (3 pieces, 6 products)
  int rhs0 = 0;                     // the launch covers right-hand sides rhs0 .. rhs0 + nrhs - 1
  int bmax = 0;                     // with a table: largest B image of one (problem, column tile) in bytes
                                    // (tc_b_tile_bytes; 0 = unknown: B is streamed)
  int mode = 0;                     // how B and A are fed: 0 the launcher's choice (B resident in shared
                                    // memory when it fits beside two A stages; for split-TF32 A's pieces
                                    // in tensor memory when they fit too), 1 B streamed with A, 2 B resident
                                    // with A in shared memory, 3 B resident with A in tensor memory; a mode
                                    // that does not fit returns FDST_NOT_SUPPORTED
};
// Largest B image of one column tile of a K x N factor (the resident-B footprint).
int tc_b_tile_bytes(int K, int N, int split);
// Layout of one contraction step of a chain (rows R, contracted size K,
// out_nv = size of the next contracted index): lda = K rounded up to 8 (TMA
// pitch), ldv = out_nv rounded up to 8 (the next step's lda), c_cs = output
// slice pitch (R for the last step's unpadded FP64 result).
struct TcLayout {
  int lda, ldv, nu;
  int64_t c_cs;
};
inline int tc_round(int x, int m) { return (x + m - 1) / m * m; }
inline TcLayout tc_layout(int R, int K, int out_nv, bool last) {
  TcLayout L;
  L.nu = R / out_nv;
  L.lda = tc_round(K, 8);
  L.ldv = tc_round(out_nv, 8);
  L.c_cs = last ? R : (int64_t)L.nu * L.ldv;
  return L;
}
// Writes the TMA descriptor (128 bytes, host memory) that reads boxes of
// 32 columns x 128 rows of A32 (dims K, R, nrhs; row pitch lda floats;
// right-hand-side pitch rhs_stride floats) into the K-major SWIZZLE_128B
// shared-memory image of the tensor-core operand. Columns at or beyond K and
// rows at or beyond R read as zero.
fdst_status tc_encode_map(void *map128, const float *A32, int K, int R, int lda, int64_t rhs_stride, int nrhs);
// ring: shared-memory stages (0 = as many as fit, capped at 4).
fdst_status launch_gemm_tc(const TcGroup &g, int nrhs, const int *done, cudaStream_t s, int ring = 0);
// number of stages that fit for the widest column tile of g
int tc_max_ring(const TcGroup &g);
// FDST_OK when a launch of g with this ring depth (0 = as deep as fits) and g.mode fits
// (host-only; the launch would return the same status).
fdst_status tc_mode_fits(const TcGroup &g, int ring);

// Host packing of B (K x N row-major FP64) into the kernel's per-stage
// shared-memory image (SWIZZLE_32B K-major; TF32 hi/lo or three bf16 pieces
// by split); size in bytes.
size_t tc_packed_bytes(int K, int N, int split);
void tc_pack(const double *B, int K, int N, int split, std::vector<uint8_t> &out);
// 1 when a bounded wait inside the tensor-core kernel expired since start.
fdst_status tc_error_flag(int *value);
// How many tensor-core CTAs gave up on an expired bounded wait since start
// (read synchronously; compare two readings to see whether a span of work had one).
fdst_status tc_error_count(int *value);
// Runs the bounded-wait self-test kernel: *gave_up = 1 when the wait expired and
// reported it; *seconds = its duration.
fdst_status tc_wait_selftest(int *gave_up, double *seconds);

}  // namespace fdst

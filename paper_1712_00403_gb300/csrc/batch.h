// Batch internals shared with the request server.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/fdst.h"

struct fdst_ctx;

namespace fdst {
// x0_zero: the caller knows hx = 0, so v = b without the FP64 matvec.
fdst_status member_init(fdst_ctx *h, int *n_stopped, double tol, cudaStream_t st, bool x0_zero = false);
fdst_status member_residual(fdst_ctx *h, cudaStream_t st);
// Writes the FP32 pairs of the member's z (double-float batches) after z was set anew.
void member_split_z(fdst_ctx *h, cudaStream_t st);
fdst_status batch_new(const std::vector<fdst_ctx *> &hs, int ring, int threads, fdst_batch *out);
fdst_status batch_step(fdst_batch b, int maxit, cudaStream_t st);
int *batch_stop_counter(fdst_batch b);
}  // namespace fdst

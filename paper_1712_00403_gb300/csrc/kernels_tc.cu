// Split-TF32 tcgen05 mode contraction (placeholder until the kernel lands).
#include "internal.h"
#include "kernels_tc.h"

namespace fdst {
fdst_status launch_gemm_tc(const TcGroup &, int, const int *, cudaStream_t) {
  set_error("split-TF32 FD contraction not built");
  return FDST_NOT_SUPPORTED;
}
}  // namespace fdst

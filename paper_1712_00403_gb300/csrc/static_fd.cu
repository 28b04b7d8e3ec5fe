// Allocation-free FD solve of one Kronecker-sum block.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator lock, a plugin whose host forbids
// device allocation after start-up, or a call site that must not trigger an
// allocation (and its implicit synchronization) in the middle of a stream.
// fdst_fd_apply_static serves them: it needs no handle and allocates nothing.
// The intermediate tensor, the transposed eigenvector matrices and the
// eigenvalue sums live in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "kernels.h"

namespace fdst {

namespace {
constexpr int64_t kStaticMaxN = 2359296;   // block entries (>= 129^3)
constexpr int kStaticMaxDim = 256;          // univariate size n_d
constexpr int64_t kStaticDoubles =
    kStaticMaxN + 3 * (int64_t)kStaticMaxDim * kStaticMaxDim + (int64_t)kStaticMaxDim * kStaticMaxDim + kStaticMaxDim;
}  // namespace

// Scratch shared by every call on a device: [intermediate tensor | U_1^T U_2^T U_3^T | lam_row | lam_col].
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// Device address of the scratch on the current device. Looked up on every
// call (not cached), so a context that was reset and re-created since the
// last call gets its own address.
static fdst_status static_scratch(double **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("fdst_fd_apply_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return FDST_CUDA_ERROR;
  }
  *out = static_cast<double *>(p);
  return FDST_OK;
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
static bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

__global__ void k_static_transpose(const double *U, double *Ut, int n) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && j < n) Ut[(int64_t)j * n + i] = U[(int64_t)i * n + j];
}

// lam_row[b*n1 + a] = c1 lam1[a] + c2 lam2[b] (3D) or c1 lam1[a] (2D); lam_col[c] = c_d lam_d[c].
__global__ void k_static_lambda(const double *l1, const double *l2, const double *l3, double c1, double c2, double c3,
                                int dim, int n1, int n2, int n3, double *lam_row, double *lam_col) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (dim == 3) {
    if (t < (int64_t)n1 * n2) lam_row[t] = c1 * l1[t % n1] + c2 * l2[t / n1];
    if (t < n3) lam_col[t] = c3 * l3[t];
  } else {
    if (t < n1) lam_row[t] = c1 * l1[t];
    if (t < n2) lam_col[t] = c2 * l2[t];
  }
}

}  // namespace fdst

using namespace fdst;

extern "C" fdst_status fdst_fd_apply_static(int dim, const int n[3], const double *const d_U[3],
                                            const double *const d_lam[3], const double coef[3], const double *d_r,
                                            double *d_s, fdst_stream stream) {
  if (!n || !d_U || !d_lam || !coef || !d_r || !d_s) {
    set_error("fdst_fd_apply_static: NULL argument");
    return FDST_INVALID_ARGUMENT;
  }
  if (dim != 2 && dim != 3) {
    set_error("fdst_fd_apply_static: dim must be 2 or 3");
    return FDST_INVALID_ARGUMENT;
  }
  int64_t N = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1 || n[d] > kStaticMaxDim) {
      set_error("fdst_fd_apply_static: n_d must lie in [1, 256]");
      return FDST_INVALID_ARGUMENT;
    }
    if (!d_U[d] || !d_lam[d]) {
      set_error("fdst_fd_apply_static: NULL factor");
      return FDST_INVALID_ARGUMENT;
    }
    N *= n[d];
  }
  if (N > kStaticMaxN) {
    set_error("fdst_fd_apply_static: block has " + std::to_string(N) + " entries, more than the static maximum " +
              std::to_string(kStaticMaxN));
    return FDST_INVALID_ARGUMENT;
  }
  double *base = nullptr;
  fdst_status st = static_scratch(&base);
  if (st != FDST_OK) return st;
  const size_t bytes = (size_t)N * sizeof(double), scratch_bytes = (size_t)kStaticDoubles * sizeof(double);
  if (ranges_overlap(d_r, bytes, d_s, bytes)) {
    set_error("fdst_fd_apply_static: r and s overlap");
    return FDST_INVALID_ARGUMENT;
  }
  if (ranges_overlap(d_r, bytes, base, scratch_bytes) || ranges_overlap(d_s, bytes, base, scratch_bytes)) {
    set_error("fdst_fd_apply_static: r or s lies inside the library's static scratch array");
    return FDST_INVALID_ARGUMENT;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *buf = base;
  double *Ut[3] = {base + kStaticMaxN, base + kStaticMaxN + (int64_t)kStaticMaxDim * kStaticMaxDim,
                   base + kStaticMaxN + 2 * (int64_t)kStaticMaxDim * kStaticMaxDim};
  double *lam_row = base + kStaticMaxN + 3 * (int64_t)kStaticMaxDim * kStaticMaxDim;
  double *lam_col = lam_row + (int64_t)kStaticMaxDim * kStaticMaxDim;
  const int n1 = n[0], n2 = n[1], n3 = dim == 3 ? n[2] : 1;
  for (int d = 0; d < dim; ++d) {
    dim3 grid((n[d] + 127) / 128, n[d]);
    count_launch(1);
    k_static_transpose<<<grid, 128, 0, s>>>(d_U[d], Ut[d], n[d]);
  }
  {
    const int64_t m = (int64_t)n1 * n2 > n3 ? (int64_t)n1 * n2 : n3;
    count_launch(1);
    k_static_lambda<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_lam[0], d_lam[1], dim == 3 ? d_lam[2] : d_lam[1],
                                                             coef[0], coef[1], dim == 3 ? coef[2] : 0.0, dim, n1, n2,
                                                             n3, lam_row, lam_col);
  }
  // Algorithm 1 steps 2-4 as the rotation-GEMM chain; the intermediates
  // alternate between the static buffer and the caller's output vector.
  int nsteps, Rs[6], Ns[6], div_step;
  const double *Bs[6];
  if (dim == 3) {
    nsteps = 6;
    div_step = 2;
    int R[6] = {n2 * n3, n1 * n3, n1 * n2, n2 * n3, n1 * n3, n1 * n2};
    int Nn[6] = {n1, n2, n3, n1, n2, n3};
    for (int j = 0; j < 6; ++j) {
      Rs[j] = R[j];
      Ns[j] = Nn[j];
      Bs[j] = j < 3 ? d_U[j] : Ut[j - 3];
    }
  } else {
    nsteps = 4;
    div_step = 1;
    int R[4] = {n2, n1, n2, n1};
    int Nn[4] = {n1, n2, n1, n2};
    for (int j = 0; j < 4; ++j) {
      Rs[j] = R[j];
      Ns[j] = Nn[j];
      Bs[j] = j < 2 ? d_U[j] : Ut[j - 2];
    }
  }
  for (int j = 0; j < nsteps; ++j) {
    GemmGroup g;
    g.nprob = 1;
    GemmProb &P = g.p[0];
    // even steps write the static buffer, odd steps the caller's output (the last step is odd)
    P.A = j == 0 ? d_r : (j % 2 == 1 ? buf : d_s);
    P.C = j % 2 == 0 ? buf : d_s;
    P.B = Bs[j];
    P.R = Rs[j];
    P.K = P.N = Ns[j];
    if (j == div_step) {
      P.lam_row = lam_row;
      P.lam_col = lam_col;
    }
    launch_gemm_f64(g, 1, nullptr, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("fdst_fd_apply_static: ") + cudaGetErrorString(e));
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
}

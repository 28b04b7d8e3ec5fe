// Split-TF32 tensor-core mode contraction for the FD preconditioner apply
// (Algorithm 1 steps 2-4), written for sm_103a with tcgen05:
//
//   C(r, n) = sum_k A(r, k) B(k, n)   stored transposed at C[n*R + r]
//
// A is the tensor being contracted (its contracted index is the fastest, see
// kernels.h), B a univariate factor U_d, U_d^T or M_d^{-1}. Both operands are
// split into TF32 pairs x = x_hi + x_lo and the three leading products
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in FP32 in tensor memory.
//
// One CTA (4 warps) computes a 128-row x NT-column tile (NT <= 256, a
// multiple of 16; wider N uses several column tiles). K runs in stages of 32
// through a two-stage shared-memory ring:
//   * B stages are pre-split and pre-swizzled on the host, so one bulk async
//     copy (cp.async.bulk, mbarrier transaction count) brings each in;
//   * A stages are read with coalesced loads, split in registers and stored in
//     the same K-major SWIZZLE_32B layout;
//   * thread 0 issues tcgen05.mma (kind::tf32, M=128, N=NT, K=8) and commits
//     to a per-stage mbarrier that releases the stage for reuse;
//   * the epilogue reads the accumulator with tcgen05.ld, applies the fused
//     Algorithm 1 step 3 divide (lam_row[r] + lam_col[n]) and the optional
//     D^{-1/2} scaling, and writes the transposed FP32 (or final FP64) tensor.
// Every mbarrier wait is bounded (about 2 s of %globaltimer); on expiry the
// kernel raises a device error flag, waits (bounded) for its own in-flight
// work, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "kernels_tc.h"

namespace fdst {

namespace {
constexpr int kM = 128;          // tile rows = TMEM lanes
constexpr int kKC = 32;          // K per pipeline stage (4 MMA k-steps of 8)
constexpr int kThreads = 128;
constexpr int kNTMax = 256;
constexpr int kAStageBytes = 2 * 4 * kM * 32;   // hi/lo x 4 k-steps x 128 rows x 32 B
constexpr unsigned long long kWaitNs = 2000000000ull;
}  // namespace

int tc_npad(int N) { return (N + 15) & ~15; }
int tc_kpad(int K) { return (K + 7) & ~7; }
static int tile_nt(int npad, int t) {
  int rest = npad - t * kNTMax;
  return rest < kNTMax ? rest : kNTMax;
}

size_t tc_packed_floats(int K, int N) { return 2 * (size_t)tc_kpad(K) * tc_npad(N); }

static inline float tf32_trunc(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u &= 0xFFFFE000u;
  std::memcpy(&x, &u, 4);
  return x;
}

// Packs B (K x N row-major, FP64) into the per-stage shared-memory image the
// kernel copies: for column tile t, stage s (k in [32 s, 32 s + 32)):
// [part hi|lo][k-step j][row n of the tile][8 TF32 values, 16-byte chunks
// swizzled by bit 2 of n (SWIZZLE_32B)].
void tc_pack(const double *B, int K, int N, std::vector<float> &out) {
  const int kp = tc_kpad(K), np = tc_npad(N);
  out.assign(2 * (size_t)kp * np, 0.0f);
  size_t tile_base = 0;
  for (int t = 0; t * kNTMax < np; ++t) {
    const int NT = tile_nt(np, t), n0 = t * kNTMax;
    for (int k0 = 0; k0 < kp; k0 += kKC) {
      const int ks = (kp - k0) / 8 < 4 ? (kp - k0) / 8 : 4;
      const size_t sb = tile_base + 2 * (size_t)NT * k0;
      for (int part = 0; part < 2; ++part)
        for (int j = 0; j < ks; ++j)
          for (int nn = 0; nn < NT; ++nn)
            for (int e = 0; e < 8; ++e) {
              const int k = k0 + 8 * j + e, n = n0 + nn;
              const double v = (k < K && n < N) ? B[(size_t)k * N + n] : 0.0;
              const float hi = tf32_trunc((float)v);
              const float lo = (float)(v - (double)hi);
              const int c = (e >> 2) ^ ((nn >> 2) & 1), w = e & 3;
              out[sb + ((size_t)(part * ks + j) * NT + nn) * 8 + c * 4 + w] = part ? lo : hi;
            }
    }
    tile_base += 2 * (size_t)NT * kp;
  }
}

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_32B (8-row atoms of 32 B,
// 256 B between atoms along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw32(const void *p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr >> 4) & 0x3FFFull;
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major): 16 B
  d |= (uint64_t)(256 >> 4) << 32;        // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)6 << 61;                 // SWIZZLE_32B
  return d;
}

// Instruction descriptor: D f32, A/B tf32, K-major both, N = nt, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int nt) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

// ------------------------------------------------------------------ kernel

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(TcGroup g, int nrhs, const int *done, int *err) {
  const int prob = blockIdx.z % g.nprob, rhs = blockIdx.z / g.nprob;
  if (done && done[rhs]) return;
  const TcProb &P = g.p[prob];
  const int R = P.R, K = P.K, N = P.N;
  const int row0 = blockIdx.x * kM;
  const int npad = (N + 15) & ~15;
  const int n0 = blockIdx.y * kNTMax;
  if (row0 >= R || n0 >= npad) return;
  const int NT = npad - n0 < kNTMax ? npad - n0 : kNTMax;
  const int kp = (K + 7) & ~7;
  const int nstages = (kp + kKC - 1) / kKC;
  const uint32_t ncols = NT <= 32 ? 32 : NT <= 64 ? 64 : NT <= 128 ? 128 : 256;
  const int stage_bytes = kAStageBytes + 2 * 4 * NT * 32;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);  // [0,1] copy, [2,3] mma
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 4);
  volatile int *sh_ok = reinterpret_cast<volatile int *>(bar + 5);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t roff = (int64_t)rhs * P.rhs_stride;
  const double *A64 = P.A64 ? P.A64 + roff : nullptr;
  const float *A32 = P.A32 ? P.A32 + roff : nullptr;
  // packed B of this column tile
  size_t btile = 0;
  for (int t = 0; t < (int)blockIdx.y; ++t) btile += 2 * (size_t)kNTMax * kp;
  const float *Bt = P.Bt + btile;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sh_ok = 1;
  }
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(NT);
  int last_commit = -1;

  for (int s = 0; s < nstages; ++s) {
    const int b = s & 1;
    const int k0 = s * kKC;
    const int ks = (kp - k0) / 8 < 4 ? (kp - k0) / 8 : 4;
    uint8_t *sA = smem + b * stage_bytes;
    uint8_t *sB = sA + kAStageBytes;
    const uint32_t bbytes = 2u * ks * NT * 32u;
    if (tid == 0) {
      bool ok = *sh_ok != 0;
      if (ok && s >= 2) ok = mbar_wait(&bar[2 + b], ((s - 2) >> 1) & 1);   // stage buffer free again
      if (ok) {
        mbar_expect_tx(&bar[b], bbytes);
        bulk_g2s(sB, Bt + 2 * (size_t)NT * k0, bbytes, &bar[b]);
      }
      *sh_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!*sh_ok) break;
    // A stage: a warp covers 4 rows x one k-step of 8 (32-byte sectors, conflict-free stores)
    for (int it = 0; it < 32; ++it) {
      const int idx = tid + kThreads * it;
      const int e = idx & 7, rq = (idx >> 3) & 3, rest = idx >> 5;
      const int rg = rest & 31, j = rest >> 5;
      if (j >= ks) continue;
      const int rr = rg * 4 + rq, r = row0 + rr, k = k0 + 8 * j + e;
      float a = 0.0f;
      if (r < R && k < K) {
        const int64_t ai = (int64_t)r * K + k;
        double v = A64 ? A64[ai] : (double)A32[ai];
        if (P.scale_in) v *= P.scale_in[ai];
        a = (float)v;
      }
      const float hi = __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
      const float lo = a - hi;
      const int c = (e >> 2) ^ ((rr >> 2) & 1);
      const uint32_t off = j * (kM * 32) + rr * 32 + c * 16 + (e & 3) * 4;
      *reinterpret_cast<float *>(sA + off) = hi;
      *reinterpret_cast<float *>(sA + 4 * kM * 32 + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      bool ok = mbar_wait(&bar[b], (s >> 1) & 1);   // B stage landed
      if (ok) {
        tc_fence_after();
        for (int j = 0; j < ks; ++j) {
          const uint64_t ah = sdesc_sw32(sA + j * kM * 32);
          const uint64_t al = sdesc_sw32(sA + 4 * kM * 32 + j * kM * 32);
          const uint64_t bh = sdesc_sw32(sB + (size_t)j * NT * 32);
          const uint64_t bl = sdesc_sw32(sB + (size_t)(ks + j) * NT * 32);
          mma_tf32(tmem, ah, bh, idesc, (s > 0 || j > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        mma_commit(&bar[2 + b]);
        last_commit = s;
      }
      *sh_ok = ok ? 1 : 0;
    }
  }
  // wait for the last committed group of MMAs (it covers every earlier one)
  if (tid == 0) {
    bool ok = *sh_ok != 0;
    if (last_commit >= 0) {
      const bool fin = mbar_wait(&bar[2 + (last_commit & 1)], (last_commit >> 1) & 1);
      ok = ok && fin && last_commit == nstages - 1;
    } else {
      ok = false;
    }
    if (!ok) atomicExch(err, 1);
    *sh_ok = ok ? 1 : 0;
  }
  __syncthreads();
  tc_fence_after();
  if (*sh_ok) {
    const int r = row0 + warp * 32 + lane;
    const float lr = (P.lam_row && r < R) ? P.lam_row[r] : 0.0f;
    const int64_t coff = roff;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < R) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = n0 + c0 + q;
          if (n >= N) break;
          float x = __uint_as_float(v[q]);
          if (P.lam_row) x = x / (lr + P.lam_col[n]);
          const int64_t ci = (int64_t)n * R + r;
          if (P.C64) {
            double y = (double)x;
            if (P.scale_out) y *= P.scale_out[ci];
            P.C64[coff + ci] = y;
          } else {
            P.C32[coff + ci] = x;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

static int *g_err_flag = nullptr;

fdst_status launch_gemm_tc(const TcGroup &g, int nrhs, const int *done, cudaStream_t s) {
  int maxR = 0, maxN = 0;
  for (int i = 0; i < g.nprob; ++i) {
    if (g.p[i].N > maxN) maxN = g.p[i].N;
    if (g.p[i].R > maxR) maxR = g.p[i].R;
  }
  const int npad = tc_npad(maxN);
  const int ntiles = (npad + kNTMax - 1) / kNTMax;
  const int nt = npad < kNTMax ? npad : kNTMax;
  const int smem = 2 * (kAStageBytes + 2 * 4 * nt * 32) + 64 + 1024;
  static int configured = 0;
  if (!g_err_flag) {
    if (cudaMalloc(&g_err_flag, sizeof(int)) != cudaSuccess || cudaMemset(g_err_flag, 0, sizeof(int)) != cudaSuccess) {
      set_error("tensor-core error flag allocation failed");
      return FDST_CUDA_ERROR;
    }
  }
  if (smem > configured) {
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
      set_error("cudaFuncSetAttribute(k_gemm_tc) failed");
      return FDST_CUDA_ERROR;
    }
    configured = smem;
  }
  dim3 grid((maxR + kM - 1) / kM, ntiles, g.nprob * nrhs);
  count_launch(1);
  k_gemm_tc<<<grid, kThreads, smem, s>>>(g, nrhs, done, g_err_flag);
  return FDST_OK;
}

fdst_status tc_error_flag(int *value) {
  *value = 0;
  if (!g_err_flag) return FDST_OK;
  if (cudaMemcpy(value, g_err_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("reading the tensor-core error flag failed");
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
}

}  // namespace fdst

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
// Persistent, warp-specialized kernel (one CTA per SM, 17 warps). A tile is
// 128 rows x NT columns (NT <= 256, a multiple of 16); K runs in stages of 32
// through a ring of 2-4 shared-memory stages:
//   * warps 0-7 (producers) read A with 16-byte loads two stages ahead
//     (register double buffer; FP32 intermediates have rows padded to a
//     multiple of 4), split to TF32 hi/lo and store the K-major SWIZZLE_32B
//     image with 16-byte shared stores; producer thread 0 also brings the
//     stage's B image
//     (pre-split and pre-swizzled on the host) with one bulk async copy
//     (cp.async.bulk, mbarrier transaction count);
//   * warp 16 allocates tensor memory and its lane 0 issues tcgen05.mma
//     (kind::tf32, M=128, N=NT, K=8), releasing each stage with
//     tcgen05.commit; accumulators are double-buffered in tensor memory;
//   * warps 8-15 (two per TMEM lane quarter, alternating 16-column chunks)
//     drain the other accumulator with tcgen05.ld (the next chunk's load in
//     flight while the current one is stored) while the next tile's MMAs
//     run, apply the fused
//     Algorithm 1 step 3 divide (lam_row[r] + lam_col[n]) and the optional
//     D^{-1/2} scaling, and write the transposed FP32 (or final FP64) tensor.
// Every mbarrier wait is bounded (about 2 s of %globaltimer) and also gives
// up when another role has aborted; on expiry the kernel raises a device
// error flag, waits (bounded) for its own in-flight work, frees its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <mutex>

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
constexpr int kProducers = 256;  // warps 0-7
constexpr int kEpiWarp0 = 8;     // warps 8-15 (two per TMEM lane quarter)
constexpr int kMmaWarp = 16;
constexpr int kThreads = 544;
constexpr int kQuads = kM * kKC / 4 / kProducers;  // 4-element quads per producer thread per stage
constexpr int kNTMax = 256;
constexpr int kAStageBytes = 2 * 4 * kM * 32;   // hi/lo x 4 k-steps x 128 rows x 32 B
constexpr int kSmemBudget = 227 * 1024;
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

// Bounded wait for the phase with the given parity to complete; gives up
// after about 2 s or as soon as *abort is set by another role.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > kWaitNs) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Wait for outstanding tcgen05.ld; v's registers are operands so that no read
// of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15])
               :
               : "memory");
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

struct TileInfo {
  int prob, rhs, row0, n0, NT, nstages, kp;
  bool valid;
};

__device__ __forceinline__ const TcProb &prob_of(const TcGroup &g, int i) { return g.table ? g.table[i] : g.p[i]; }

__device__ __forceinline__ TileInfo decode_tile(const TcGroup &g, int T, int nrt, int ntn, const int *done) {
  TileInfo t;
  const int rt = T % nrt;
  const int rest = T / nrt;
  const int nt = rest % ntn;
  const int z = rest / ntn;
  t.prob = z % g.nprob;
  t.rhs = z / g.nprob;
  const TcProb &P = prob_of(g, t.prob);
  const int npad = (P.N + 15) & ~15;
  t.row0 = rt * kM;
  t.n0 = nt * kNTMax;
  t.valid = t.row0 < P.R && t.n0 < npad && !(done && done[t.rhs]) && !(P.done_flag && *P.done_flag);
  t.NT = npad - t.n0 < kNTMax ? npad - t.n0 : kNTMax;
  t.kp = (P.K + 7) & ~7;
  t.nstages = (t.kp + kKC - 1) / kKC;
  return t;
}

// Next valid tile index after T (T = -1: the first of this CTA); total if none.
__device__ __forceinline__ int next_tile(const TcGroup &g, int T, int total, int nrt, int ntn, const int *done) {
  T = T < 0 ? (int)blockIdx.x : T + (int)gridDim.x;
  while (T < total && !decode_tile(g, T, nrt, ntn, done).valid) T += gridDim.x;
  return T;
}

struct Cursor {
  int T, s;
  TileInfo t;
};

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(TcGroup g, int nrhs, const int *done, int *err, int nrt, int ntn, int nstage_ring, int ntc,
              int ntmax_smem) {
  const int total = nrt * ntn * g.nprob * nrhs;
  // ntmax_smem: widest column tile of the launch (B region); ntc: TMEM columns per accumulator
  const int stage_bytes = kAStageBytes + 2 * 4 * ntmax_smem * 32;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + nstage_ring * stage_bytes);
  uint64_t *full = bars, *empty = bars + 4, *tfull = bars + 8, *tempty = bars + 10;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 12);
  volatile int *abort = reinterpret_cast<volatile int *>(bars + 13);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < nstage_ring; ++i) {
      mbar_init(&full[i], kProducers + 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, 2 * ntc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ producers
    const int ptid = tid;
    // quad it of this thread: rows 4g..4g+3 of a warp, lane -> (row rq, 16-byte chunk cc, k-step j);
    // a quarter-warp stores 8 distinct 16-byte slots (conflict-free)
    int q_rr[kQuads], q_kk[kQuads];
    uint32_t q_off[kQuads];
#pragma unroll
    for (int it = 0; it < kQuads; ++it) {
      const int qd = ptid + kProducers * it;
      const int gq = qd >> 5, l = qd & 31;
      const int rq = l & 3, cc = (l >> 2) & 1, j = l >> 3;
      q_rr[it] = gq * 4 + rq;
      q_kk[it] = j * 8 + cc * 4;
      q_off[it] = j * (kM * 32) + q_rr[it] * 32 + ((cc ^ ((q_rr[it] >> 2) & 1)) * 16);
    }
    auto load = [&](const Cursor &c, float4 (&reg)[kQuads]) {
      const TcProb &P = prob_of(g, c.t.prob);
      const int k0 = c.s * kKC;
      if (P.A32) {
        const float *A32 = P.A32 + (int64_t)c.t.rhs * P.a_rhs_stride;
#pragma unroll
        for (int it = 0; it < kQuads; ++it) {
          const int r = c.t.row0 + q_rr[it], k = k0 + q_kk[it];
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
          if (r < P.R && k < P.K) {
            a = *reinterpret_cast<const float4 *>(A32 + (int64_t)r * P.lda + k);
            if (k + 1 >= P.K) a.y = 0.f;
            if (k + 2 >= P.K) a.z = 0.f;
            if (k + 3 >= P.K) a.w = 0.f;
          }
          reg[it] = a;
        }
      } else {
        const double *A64 = P.A64 + (int64_t)c.t.rhs * P.a_rhs_stride;
#pragma unroll
        for (int it = 0; it < kQuads; ++it) {
          const int r = c.t.row0 + q_rr[it], k = k0 + q_kk[it];
          float v[4] = {0.f, 0.f, 0.f, 0.f};
          if (r < P.R) {
            const int64_t base = (int64_t)r * P.lda + k;
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (k + e < P.K) {
                double x = A64[base + e];
                if (P.scale_in) x *= P.scale_in[(int64_t)r * P.K + k + e];
                v[e] = (float)x;
              }
          }
          reg[it] = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
    };
    auto advance = [&](Cursor &c) -> bool {
      if (++c.s < c.t.nstages) return true;
      c.s = 0;
      c.T = next_tile(g, c.T, total, nrt, ntn, done);
      if (c.T >= total) return false;
      c.t = decode_tile(g, c.T, nrt, ntn, done);
      return true;
    };
    int q = 0;
    auto split_hi = [](float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); };
    auto produce = [&](const Cursor &c, const float4 (&reg)[kQuads]) -> bool {
      const int slot = q % nstage_ring, u = q / nstage_ring;
      if (u > 0 && !mbar_wait(&empty[slot], (u - 1) & 1, abort)) return false;
      uint8_t *sA = smem + slot * stage_bytes;
      uint8_t *sB = sA + kAStageBytes;
      if (ptid == 0) {
        const int k0 = c.s * kKC;
        const int ks = (c.t.kp - k0) / 8 < 4 ? (c.t.kp - k0) / 8 : 4;
        const uint32_t bbytes = 2u * ks * c.t.NT * 32u;
        const size_t btile = 2 * (size_t)kNTMax * c.t.kp * (size_t)(c.t.n0 / kNTMax);
        mbar_expect_tx(&full[slot], bbytes);
        bulk_g2s(sB, prob_of(g, c.t.prob).Bt + btile + 2 * (size_t)c.t.NT * k0, bbytes, &full[slot]);
      }
#pragma unroll
      for (int it = 0; it < kQuads; ++it) {
        const float4 a = reg[it];
        const float4 hi = make_float4(split_hi(a.x), split_hi(a.y), split_hi(a.z), split_hi(a.w));
        const float4 lo = make_float4(a.x - hi.x, a.y - hi.y, a.z - hi.z, a.w - hi.w);
        *reinterpret_cast<float4 *>(sA + q_off[it]) = hi;
        *reinterpret_cast<float4 *>(sA + 4 * kM * 32 + q_off[it]) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&full[slot]);
      ++q;
      return true;
    };
    float4 ra[kQuads], rb[kQuads];
    Cursor c0;
    c0.T = next_tile(g, -1, total, nrt, ntn, done);
    c0.s = 0;
    bool has0 = c0.T < total;
    if (has0) {
      c0.t = decode_tile(g, c0.T, nrt, ntn, done);
      load(c0, ra);
    }
    Cursor c1 = c0;
    bool has1 = has0 && advance(c1);
    if (has1) load(c1, rb);
    while (has0) {
      if (!produce(c0, ra)) break;
      Cursor c2 = c1;
      bool has2 = has1 && advance(c2);
      if (has2) load(c2, ra);
      if (!has1) break;
      if (!produce(c1, rb)) break;
      Cursor c3 = c2;
      bool has3 = has2 && advance(c3);
      if (has3) load(c3, rb);
      c0 = c2;
      has0 = has2;
      c1 = c3;
      has1 = has3;
    }
  } else if (warp < kMmaWarp) {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3, half = (warp - kEpiWarp0) >> 2;
    int v = 0;
    for (int T = next_tile(g, -1, total, nrt, ntn, done); T < total; T = next_tile(g, T, total, nrt, ntn, done)) {
      const TileInfo t = decode_tile(g, T, nrt, ntn, done);
      const TcProb &P = prob_of(g, t.prob);
      const int acc = v & 1;
      if (!mbar_wait(&tfull[acc], (v >> 1) & 1, abort)) break;
      tc_fence_after();
      const int r = t.row0 + quarter * 32 + lane;
      const bool rok = r < P.R;
      const float lr = (P.lam_row && rok) ? P.lam_row[r] : 0.0f;
      const float *lc = P.lam_col;
      const int nu = P.R / P.out_nv, uu = r / P.out_nv, vv0 = r - uu * P.out_nv;
      // output address of column n: base + n * cstride (row-major over (n, u), padded v)
      const int64_t cstride = (int64_t)nu * P.ldc;
      const int64_t base = (int64_t)t.rhs * P.c_rhs_stride + (int64_t)uu * P.ldc + vv0;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * ntc);
      const int nchunks = t.NT / 16;
      auto store_chunk = [&](const uint32_t (&vals)[16], int c) {
        const int nb = t.n0 + 16 * c;
        if (!rok) return;
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) {
          const int n = nb + qq;
          if (n < P.N) {
            float x = __uint_as_float(vals[qq]);
            if (lc) x = x / (lr + lc[n]);
            if (P.C64) {
              double y = (double)x;
              if (P.scale_out) y *= P.scale_out[(int64_t)n * P.R + r];
              P.C64[base + n * cstride] = y;
            } else {
              P.C32[base + n * cstride] = x;
            }
          }
        }
      };
      // chunks half, half+2, ...: the next chunk's TMEM load is in flight while one is stored
      uint32_t va[16], vb[16];
      int c = half;
      if (c < nchunks) tmem_ld16_nowait(taddr + 16 * c, va);
      while (c < nchunks) {
        tmem_wait_ld_regs(va);
        if (c + 2 < nchunks) tmem_ld16_nowait(taddr + 16 * (c + 2), vb);
        store_chunk(va, c);
        c += 2;
        if (c >= nchunks) break;
        tmem_wait_ld_regs(vb);
        if (c + 2 < nchunks) tmem_ld16_nowait(taddr + 16 * (c + 2), va);
        store_chunk(vb, c);
        c += 2;
      }
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      ++v;
    }
  } else {
    // ------------------------------------------------------------ MMA issuer (one thread)
    if (lane == 0) {
      int q = 0, v = 0, last_slot = -1, last_par = 0;
      bool ok = true;
      for (int T = next_tile(g, -1, total, nrt, ntn, done); ok && T < total;
           T = next_tile(g, T, total, nrt, ntn, done)) {
        const TileInfo t = decode_tile(g, T, nrt, ntn, done);
        const int acc = v & 1, u = v >> 1;
        if (u > 0 && !mbar_wait(&tempty[acc], (u - 1) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * ntc);
        const uint32_t idesc = idesc_tf32(t.NT);
        for (int s = 0; s < t.nstages; ++s) {
          const int slot = q % nstage_ring;
          if (!mbar_wait(&full[slot], (q / nstage_ring) & 1, abort)) { ok = false; break; }
          tc_fence_after();
          uint8_t *sA = smem + slot * stage_bytes;
          uint8_t *sB = sA + kAStageBytes;
          const int k0 = s * kKC;
          const int ks = (t.kp - k0) / 8 < 4 ? (t.kp - k0) / 8 : 4;
          for (int j = 0; j < ks; ++j) {
            const uint64_t ah = sdesc_sw32(sA + j * kM * 32);
            const uint64_t al = sdesc_sw32(sA + 4 * kM * 32 + j * kM * 32);
            const uint64_t bh = sdesc_sw32(sB + (size_t)j * t.NT * 32);
            const uint64_t bl = sdesc_sw32(sB + (size_t)(ks + j) * t.NT * 32);
            mma_tf32(d, ah, bh, idesc, (s > 0 || j > 0) ? 1u : 0u);
            mma_tf32(d, ah, bl, idesc, 1u);
            mma_tf32(d, al, bh, idesc, 1u);
          }
          mma_commit(&empty[slot]);
          last_slot = slot;
          last_par = (q / nstage_ring) & 1;
          ++q;
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
        ++v;
      }
      if (!ok) {
        atomicExch(err, 1);
        *abort = 1;
      }
      // drain: the last commit covers every MMA issued before it (bounded wait, ignoring abort)
      if (last_slot >= 0) {
        volatile int never = 0;
        mbar_wait(&empty[last_slot], last_par, &never);
      }
    }
    __syncwarp();
  }
  if (*abort && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * ntc);
  }
}

static int *g_err_flag = nullptr;

static void tc_dims(const TcGroup &g, int &maxR, int &maxN) {
  maxR = g.maxR;
  maxN = g.maxN;
  if (!g.table)
    for (int i = 0; i < g.nprob; ++i) {
      if (g.p[i].N > maxN) maxN = g.p[i].N;
      if (g.p[i].R > maxR) maxR = g.p[i].R;
    }
}

int tc_max_ring(const TcGroup &g) {
  int maxR, maxN;
  tc_dims(g, maxR, maxN);
  const int npad = tc_npad(maxN);
  const int nt = npad < kNTMax ? npad : kNTMax;
  const int stage_bytes = kAStageBytes + 2 * 4 * nt * 32;
  int nring = (kSmemBudget - 2048) / stage_bytes;
  return nring > 4 ? 4 : nring;
}

fdst_status launch_gemm_tc(const TcGroup &g, int nrhs, const int *done, cudaStream_t s, int ring) {
  int maxR, maxN;
  tc_dims(g, maxR, maxN);
  const int npad = tc_npad(maxN);
  const int ntn = (npad + kNTMax - 1) / kNTMax;
  const int nt = npad < kNTMax ? npad : kNTMax;
  const int ntc = nt <= 32 ? 32 : nt <= 64 ? 64 : nt <= 128 ? 128 : 256;   // TMEM columns per accumulator
  const int stage_bytes = kAStageBytes + 2 * 4 * nt * 32;
  int nring = tc_max_ring(g);
  if (ring > 0 && ring < nring) nring = ring;
  if (nring < 2) {
    set_error("tensor-core contraction: shared memory too small for two stages");
    return FDST_NOT_SUPPORTED;
  }
  const int smem = nring * stage_bytes + 1024 + 1024;
  static int configured = 0, nsm = 0;
  static std::mutex init_mutex;
  std::lock_guard<std::mutex> lock(init_mutex);
  if (!g_err_flag) {
    if (cudaMalloc(&g_err_flag, sizeof(int)) != cudaSuccess || cudaMemset(g_err_flag, 0, sizeof(int)) != cudaSuccess) {
      set_error("tensor-core error flag allocation failed");
      return FDST_CUDA_ERROR;
    }
  }
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm < 1) nsm = 1;
  }
  if (smem > configured) {
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
      set_error("cudaFuncSetAttribute(k_gemm_tc) failed");
      return FDST_CUDA_ERROR;
    }
    configured = smem;
  }
  const int nrt = (maxR + kM - 1) / kM;
  const long long total = (long long)nrt * ntn * g.nprob * nrhs;
  const int grid = total < nsm ? (int)total : nsm;
  count_launch(1);
  k_gemm_tc<<<grid, kThreads, smem, s>>>(g, nrhs, done, g_err_flag, nrt, ntn, nring, ntc, nt);
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

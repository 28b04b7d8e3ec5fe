// Split-TF32 tensor-core mode contraction for the FD preconditioner apply
// (Algorithm 1 steps 2-4), written for sm_103a with tcgen05:
//
//   C(r, n) = sum_k A(r, k) B(k, n)   stored transposed at C[n*R + r]
//
// A is the tensor being contracted (its contracted index is the fastest, see
// kernels.h), B a univariate factor U_d, U_d^T or M_d^{-1}. Both operands are
// split into TF32 pairs x = x_hi + x_lo (both rounded to nearest) and the three leading products
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in FP32 in tensor memory.
//
// Persistent, warp-specialized kernel (one CTA per SM, 18 warps). A tile is
// 128 rows x NT columns (NT <= 256, a multiple of 16); K runs in stages of 32
// through a ring of 2-4 shared-memory stages:
//   * warp 17 (lane 0) issues, per stage, one TMA tensor load of A (box 32
//     FP32 columns x 128 rows, SWIZZLE_128B K-major, straight into the
//     operand image's hi half; rows and columns past the tensor read as
//     zero) and, when B streams, one bulk async copy of the stage's B image
//     (pre-split and pre-swizzled on the host, SWIZZLE_32B K-major), all on
//     one mbarrier transaction count, as soon as the MMA has released the
//     slot. When the B image of a (problem, column tile) fits beside two A
//     stages it stays resident instead: it is copied once into its own
//     region and again only when the CTA's next tile needs another B (after
//     every MMA issued so far has completed); tiles are ordered row tile
//     fastest, then right-hand side, so a CTA keeps one B for long runs;
//   * warps 0-7 split the landed FP32 tile in place into TF32 hi (kept where
//     it landed) and lo (written to the lo half at the same offsets) with
//     conflict-free 16-byte shared-memory accesses;
//   * warp 16 allocates tensor memory and its lane 0 issues tcgen05.mma
//     (kind::tf32, M=128, N=NT, K=8), releasing each stage with
//     tcgen05.commit; accumulators are double-buffered in tensor memory;
//   * warps 8-15 (two halves of one warp per TMEM lane quarter, alternating
//     16-column chunks) drain the other accumulator with tcgen05.ld (the next
//     chunk's load in flight) while the next tile's MMAs run, apply the fused
//     Algorithm 1 step 3 divide (lam_row[r] + lam_col[n]) and the optional
//     D^{-1/2} scaling, and write the transposed FP32 (or final FP64) tensor.
// The first contraction of a chain reads FP64: a grouped elementwise kernel
// converts it (times the optional D^{-1/2} scaling) to the FP32 layout first.
// Every mbarrier wait is bounded (about 2 s of %globaltimer) and also gives
// up when another role has aborted; on expiry the kernel raises a device
// error flag, waits (bounded) for its own in-flight copies and MMAs, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "fp_bits.cuh"
#include "internal.h"
#include "kernels.h"
#include "kernels_tc.h"

namespace fdst {

namespace {
constexpr int kM = 128;          // tile rows = TMEM lanes
constexpr int kKC = 32;          // K per pipeline stage (4 MMA k-steps of 8)
constexpr int kConv = 256;       // warps 0-7: TF32 split of the landed A tile
constexpr int kEpiWarp0 = 8;     // warps 8-15 (two per TMEM lane quarter)
constexpr int kMmaWarp = 16;
constexpr int kTmaWarp = 17;
constexpr int kThreads = 576;
constexpr int kAHalfBytes = kM * kKC * 4;   // 128 rows x 32 FP32 (hi or lo half of a stage's A)
constexpr int kNTMax = 256;
// A part of a stage: split-TF32: the landed FP32 tile turned into hi in place
// plus a lo copy (2 x 16 KB); split-BF16: the landed tile plus three bf16
// planes of 2 k-steps of 16 (16 KB + 3 x 8 KB). B part: bytes per K element
// and column: 8 (two TF32 parts) or 6 (three bf16 parts).
template <int SPLIT> struct SplitTraits;
template <> struct SplitTraits<0> {
  static constexpr int kAStage = 2 * 4 * kM * 32, kBPE = 8, kKStep = 8;
};
template <> struct SplitTraits<1> {
  static constexpr int kAStage = 4 * kM * 32 + 3 * 2 * kM * 32, kBPE = 6, kKStep = 16;
};
constexpr int kSmemBudget = 227 * 1024;
constexpr int kMaxRhsLaunch = 640;   // stop flags copied into the barrier region (bytes 192..831)
constexpr unsigned long long kWaitNs = 2000000000ull;
}  // namespace

int tc_npad(int N) { return (N + 15) & ~15; }
int tc_kpad(int K, int split) { return split ? (K + 15) & ~15 : (K + 7) & ~7; }
static int tile_nt(int npad, int t) {
  int rest = npad - t * kNTMax;
  return rest < kNTMax ? rest : kNTMax;
}

int tc_b_tile_bytes(int K, int N, int split) {
  const int kp = tc_kpad(K, split), np = tc_npad(N), bpe = split ? SplitTraits<1>::kBPE : SplitTraits<0>::kBPE;
  int b = 0;
  for (int t = 0; t * kNTMax < np; ++t) b = std::max(b, bpe * tile_nt(np, t) * kp);
  return b;
}

size_t tc_packed_bytes(int K, int N, int split) { return (split ? 6 : 8) * (size_t)tc_kpad(K, split) * tc_npad(N); }

// Three bf16 pieces of a float by truncation: x = b0 + b1 + b2 up to the last
// 8 bits of x's 24-bit significand (each difference is exact in FP32).
static inline void bf16_split3_host(float x, uint16_t &b0, uint16_t &b1, uint16_t &b2) {
  uint32_t u, v;
  std::memcpy(&u, &x, 4);
  u &= 0xFFFF0000u;
  float h;
  std::memcpy(&h, &u, 4);
  const float r1 = x - h;
  std::memcpy(&v, &r1, 4);
  v &= 0xFFFF0000u;
  float h1;
  std::memcpy(&h1, &v, 4);
  const float r2 = r1 - h1;
  uint32_t w;
  std::memcpy(&w, &r2, 4);
  b0 = (uint16_t)(u >> 16);
  b1 = (uint16_t)(v >> 16);
  b2 = (uint16_t)(w >> 16);
}

// Nearest TF32 value of a float (10 stored mantissa bits; ties away from zero),
// on the encoding: adding half a TF32 ulp to the magnitude bits and clearing
// the 13 low bits rounds the magnitude to nearest (a carry moves into the
// exponent as it should).
static inline float tf32_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  std::memcpy(&x, &u, 4);
  return x;
}

// Packs B (K x N row-major, FP64) into the per-stage shared-memory image the
// kernel copies: for column tile t, stage s (k in [32 s, 32 s + 32)):
// [part][k-step j][row n of the tile][one k-step of values, 16-byte chunks
// swizzled by bit 2 of n (SWIZZLE_32B)]; split-TF32: parts hi|lo, k-steps of
// 8 TF32 values; split-BF16: parts b0|b1|b2, k-steps of 16 bf16 values.
void tc_pack(const double *B, int K, int N, int split, std::vector<uint8_t> &out) {
  const int kp = tc_kpad(K, split), np = tc_npad(N), bpe = split ? 6 : 8, kst = split ? 16 : 8;
  const int nparts = split ? 3 : 2;
  out.assign((size_t)bpe * kp * np, 0);
  size_t tile_base = 0;
  for (int t = 0; t * kNTMax < np; ++t) {
    const int NT = tile_nt(np, t), n0 = t * kNTMax;
    for (int k0 = 0; k0 < kp; k0 += kKC) {
      const int ks = (kp - k0) / kst < kKC / kst ? (kp - k0) / kst : kKC / kst;
      const size_t sb = tile_base + (size_t)bpe * NT * k0;
      for (int j = 0; j < ks; ++j)
        for (int nn = 0; nn < NT; ++nn)
          for (int e = 0; e < kst; ++e) {
            const int k = k0 + kst * j + e, n = n0 + nn;
            const double v = (k < K && n < N) ? B[(size_t)k * N + n] : 0.0;
            const int ebytes = split ? 2 : 4, per_chunk = 16 / ebytes;
            const int c = (e / per_chunk) ^ ((nn >> 2) & 1), w = e % per_chunk;
            for (int part = 0; part < nparts; ++part) {
              uint8_t *dst = out.data() + sb + ((size_t)(part * ks + j) * NT + nn) * 32 + c * 16 + w * ebytes;
              if (split) {
                uint16_t b[3];
                bf16_split3_host((float)v, b[0], b[1], b[2]);
                std::memcpy(dst, &b[part], 2);
              } else {
                const float hi = tf32_rn((float)v);
                const float lo = tf32_rn((float)(v - (double)hi));
                std::memcpy(dst, part ? &lo : &hi, 4);
              }
            }
          }
    }
    tile_base += (size_t)bpe * NT * kp;
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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
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

// TMA tensor load of one box (coordinates innermost first) into shared memory,
// completing as transaction bytes on the mbarrier.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
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

// The same MMA with the A operand in tensor memory (lane = row of A, one 32-bit
// column per TF32 element along K).
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                   taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
               "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
               : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B (8-row atoms of
// 128 B, 1024 B between atoms along M), descriptor version 1. The k-steps of
// a 32-wide stage start 32 B apart inside the atom; the hardware applies the
// swizzle to the address bits, so the start address alone selects one.
__device__ __forceinline__ uint64_t sdesc_sw128(const void *p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr >> 4) & 0x3FFFull;
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major): 16 B
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D f32, A/B bf16 (kind::f16), K-major both, N = nt, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int nt) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Three bf16 pieces (truncation) of each of 8 floats, packed per piece.
__device__ __forceinline__ void bf16_split3x8(const float (&x)[8], uint4 &p0, uint4 &p1, uint4 &p2) {
  uint32_t h[8], m[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint32_t u = __float_as_uint(x[e]) & 0xFFFF0000u;
    const float r1 = x[e] - __uint_as_float(u);
    const uint32_t v = __float_as_uint(r1) & 0xFFFF0000u;
    const float r2 = r1 - __uint_as_float(v);
    h[e] = u >> 16;
    m[e] = v >> 16;
    l[e] = __float_as_uint(r2) >> 16;
  }
  p0 = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
  p1 = make_uint4(m[0] | (m[1] << 16), m[2] | (m[3] << 16), m[4] | (m[5] << 16), m[6] | (m[7] << 16));
  p2 = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16), l[6] | (l[7] << 16));
}

// Nearest TF32 value (ties away from zero) on the encoding, as tf32_rn on the host.
__device__ __forceinline__ float tf32_rn_dev(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

// Instruction descriptor: D f32, A/B tf32, K-major both, N = nt, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int nt) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

// ------------------------------------------------------------------ kernel

// A tile is 128 consecutive rows r0..r0+127 of A (one TMA box per stage) by
// NT columns.
struct TileInfo {
  int prob, rhs, r0, n0, NT, nstages, kp;
  bool valid;
};

__device__ __forceinline__ const TcProb &prob_of(const TcGroup &g, int i) { return g.table ? g.table[i] : g.p[i]; }

// `done` here is the launch's copy of the per-right-hand-side stop flags in
// shared memory (index rhs - rhs0), read once when the CTA starts.
template <int SPLIT>
__device__ __forceinline__ TileInfo decode_tile(const TcGroup &g, int T, int nrt, int ntn, int nrhs,
                                                const uint8_t *done) {
  // row tile fastest, then right-hand side, then column tile, then problem: the
  // tiles a CTA takes (gridDim.x apart) share one B operand for long runs
  TileInfo t;
  const int rt = T % nrt;
  int rest = T / nrt;
  t.rhs = g.rhs0 + rest % nrhs;
  rest /= nrhs;
  const int nt = rest % ntn;
  t.prob = rest / ntn;
  const TcProb &P = prob_of(g, t.prob);
  const int npad = (P.N + 15) & ~15;
  t.r0 = rt * kM;
  t.n0 = nt * kNTMax;
  t.valid = t.r0 < P.R && t.n0 < npad && !done[t.rhs - g.rhs0] && !(P.done_flag && *P.done_flag);
  t.NT = npad - t.n0 < kNTMax ? npad - t.n0 : kNTMax;
  t.kp = SPLIT ? (P.K + 15) & ~15 : (P.K + 7) & ~7;
  t.nstages = (t.kp + kKC - 1) / kKC;
  return t;
}

// Next valid tile index after T (T = -1: the first of this CTA); total if none.
__device__ __forceinline__ int next_tile(const TcGroup &g, int T, int total, int nrt, int ntn, int nrhs,
                                         const uint8_t *done) {
  T = T < 0 ? (int)blockIdx.x : T + (int)gridDim.x;
  while (T < total && !decode_tile<0>(g, T, nrt, ntn, nrhs, done).valid) T += gridDim.x;
  return T;
}

struct Cursor {
  int T, s;
  TileInfo t;
};

template <int SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(TcGroup g, int nrhs, const int *done, int *err, int nrt, int ntn, int nstage_ring, int ntc,
              int ntmax_smem, int bres, int amode, int tmem_cols) {
  using TR = SplitTraits<SPLIT>;
  const int total = nrt * ntn * g.nprob * nrhs;
  // Two ways to feed B. Streaming (bres == 0): every stage carries its slice of
  // B next to A (ntmax_smem: widest column tile of the launch). Resident
  // (bres > 0): the whole B image of the current (problem, column tile) sits in
  // a region of bres bytes after the ring and is copied again only when a
  // CTA's next tile needs another one, so the ring moves A alone.
  // ntc: TMEM columns per accumulator (the second starts at column ntc).
  // amode 1 (split-TF32 with resident B): the split warps write A's TF32 hi/lo
  // pieces into tensor memory (two stages of 64 columns from column 2 ntc: hi
  // in the first 32, lo in the next 32) and release the landed shared-memory
  // slot as soon as they have read it, so a ring slot holds only the 16 KB the
  // TMA lands and the MMAs read A from tensor memory.
  const bool resident = bres > 0;
  const bool atm = amode != 0;
  const int stage_bytes = atm ? kAHalfBytes : resident ? TR::kAStage : TR::kAStage + TR::kBPE * ntmax_smem * kKC;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *Bres = smem + nstage_ring * stage_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(Bres + (resident ? bres : 0));
  uint64_t *landed = bars, *split = bars + 4, *empty = bars + 8, *tfull = bars + 12, *tempty = bars + 14;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 16);
  volatile int *abort = reinterpret_cast<volatile int *>(bars + 17);
  uint64_t *bfull = bars + 18;
  uint64_t *a_empty = bars + 19;                              // amode 1: TMEM A stage free (MMA commit)
  uint64_t *bfree = bars + 21;   // amode 1: every MMA on the resident B done before a tile needing another B
  uint8_t *done_s = reinterpret_cast<uint8_t *>(bars + 24);   // nrhs <= kMaxRhsLaunch flags

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < nrhs; i += kThreads) done_s[i] = done ? (done[g.rhs0 + i] != 0) : 0;
  if (tid == 0) {
    for (int i = 0; i < nstage_ring; ++i) {
      mbar_init(&landed[i], 1);
      mbar_init(&split[i], kConv / 32);
      mbar_init(&empty[i], atm ? kConv / 32 : 1);
    }
    for (int i = 0; i < 2; ++i) mbar_init(&a_empty[i], 1);
    mbar_init(bfree, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
    }
    mbar_init(bfull, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kTmaWarp) {
    // ------------------------------------------------------------ TMA issuer (one thread)
    if (lane == 0) {
      int q = 0, last_q = -1, bkey = -1, nb = 0;
      int last_par[4] = {-1, -1, -1, -1};
      bool ok = true;
      for (int T = next_tile(g, -1, total, nrt, ntn, nrhs, done_s); ok && T < total;
           T = next_tile(g, T, total, nrt, ntn, nrhs, done_s)) {
        const TileInfo t = decode_tile<SPLIT>(g, T, nrt, ntn, nrhs, done_s);
        const TcProb &P = prob_of(g, t.prob);
        const size_t btile = (size_t)TR::kBPE * kNTMax * t.kp * (size_t)(t.n0 / kNTMax);
        const int key = t.prob * ntn + t.n0 / kNTMax;
        if (resident && key != bkey) {
          // the resident B is overwritten only after every MMA issued so far has
          // completed: the commit of the last stage issued covers them all
          // (amode 1: the MMA thread commits bfree once before each change of B, so the
          // nb-th reload waits for phase nb - 1 and no phase can be skipped or aliased)
          if (last_q >= 0 && !(atm ? mbar_wait(bfree, (uint32_t)((nb - 1) & 1), abort)
                                   : mbar_wait(&empty[last_q % nstage_ring], (last_q / nstage_ring) & 1, abort))) {
            ok = false;
            break;
          }
          const uint32_t bb = (uint32_t)TR::kBPE * t.NT * t.kp;
          mbar_expect_tx(bfull, bb);
          for (uint32_t o = 0; o < bb; o += 32768u)
            bulk_g2s(Bres + o, P.Bt + btile + o, bb - o < 32768u ? bb - o : 32768u, bfull);
          bkey = key;
          ++nb;
        }
        for (int s = 0; s < t.nstages; ++s, ++q) {
          const int slot = q % nstage_ring, u = q / nstage_ring;
          if (u > 0 && !mbar_wait(&empty[slot], (u - 1) & 1, abort)) { ok = false; break; }
          uint8_t *sA = smem + slot * stage_bytes;
          const int k0 = s * kKC;
          const uint32_t bbytes =
              resident ? 0u : (uint32_t)TR::kBPE * t.NT * (t.kp - k0 < kKC ? t.kp - k0 : kKC);
          mbar_expect_tx(&landed[slot], kAHalfBytes + bbytes);
          tma_load_3d(sA, P.tmap, k0, t.r0, t.rhs, &landed[slot]);
          if (!resident) bulk_g2s(sA + TR::kAStage, P.Bt + btile + (size_t)TR::kBPE * t.NT * k0, bbytes, &landed[slot]);
          last_par[slot] = u & 1;
          last_q = q;
        }
      }
      if (!ok) *abort = 1;
      // every copy issued has landed before the CTA may exit (bounded, ignoring abort)
      volatile int never = 0;
      for (int i = 0; i < nstage_ring; ++i)
        if (last_par[i] >= 0) mbar_wait(&landed[i], (uint32_t)last_par[i], &never);
      if (nb > 0) mbar_wait(bfull, (uint32_t)((nb - 1) & 1), &never);
    }
    __syncwarp();
  } else if (warp < kEpiWarp0 && atm) {
    // ------------------------------------------------------------ TF32 split into tensor memory
    // Warps w and w + 4 share TMEM lane quarter w % 4 (rows 32 (w % 4) + lane) and take
    // K columns 0-15 and 16-31 of the stage.
    const int quarter = warp & 3, khalf = warp >> 2, r = quarter * 32 + lane;
    const uint32_t tlane = (uint32_t)(quarter * 32) << 16;
    int q = 0;
    bool ok = true;
    for (int T = next_tile(g, -1, total, nrt, ntn, nrhs, done_s); ok && T < total;
         T = next_tile(g, T, total, nrt, ntn, nrhs, done_s)) {
      const TileInfo t = decode_tile<SPLIT>(g, T, nrt, ntn, nrhs, done_s);
      for (int s = 0; s < t.nstages; ++s, ++q) {
        const int slot = q % nstage_ring, as = q & 1, au = q >> 1;
        if (!mbar_wait(&landed[slot], (q / nstage_ring) & 1, abort)) { ok = false; break; }
        // the row's 16 FP32 values: chunks 4 khalf .. 4 khalf + 3 of the SWIZZLE_128B row
        const uint8_t *row = smem + slot * stage_bytes + (r >> 3) * 1024 + (r & 7) * 128;
        float x[16];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 v = *reinterpret_cast<const float4 *>(row + (((4 * khalf + c) ^ (r & 7)) << 4));
          x[4 * c] = v.x;
          x[4 * c + 1] = v.y;
          x[4 * c + 2] = v.z;
          x[4 * c + 3] = v.w;
        }
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float h = tf32_rn_dev(x[e]);
          hi[e] = __float_as_uint(h);
          lo[e] = __float_as_uint(tf32_rn_dev(x[e] - h));
        }
        // the slot's values are consumed (in registers) before it is handed back to
        // the TMA: order these generic-proxy reads before its async-proxy writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);   // the slot may be landed again
        if (au > 0 && !mbar_wait(&a_empty[as], (au - 1) & 1, abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t ta = tmem + tlane + (uint32_t)(2 * ntc + 64 * as + 16 * khalf);
        tmem_st16(ta, hi);
        tmem_st16(ta + 32, lo);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&split[as]);
      }
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ TF32 split of the landed tile
    int q = 0;
    bool ok = true;
    for (int T = next_tile(g, -1, total, nrt, ntn, nrhs, done_s); ok && T < total;
         T = next_tile(g, T, total, nrt, ntn, nrhs, done_s)) {
      const TileInfo t = decode_tile<SPLIT>(g, T, nrt, ntn, nrhs, done_s);
      for (int s = 0; s < t.nstages; ++s, ++q) {
        const int slot = q % nstage_ring;
        if (!mbar_wait(&landed[slot], (q / nstage_ring) & 1, abort)) { ok = false; break; }
        uint8_t *sA = smem + slot * stage_bytes;
        if (SPLIT == 0) {
          for (int c = tid; c < kAHalfBytes / 16; c += kConv) {
            float4 *ph = reinterpret_cast<float4 *>(sA + c * 16);
            const float4 a = *ph;
            // hi = nearest TF32 value of a, lo = nearest TF32 value of the exact
            // remainder a - hi (at most 12 significant bits): a = hi + lo to 2^-24 |a|
            float4 hi, lo;
            hi.x = tf32_rn_dev(a.x);
            hi.y = tf32_rn_dev(a.y);
            hi.z = tf32_rn_dev(a.z);
            hi.w = tf32_rn_dev(a.w);
            lo = make_float4(tf32_rn_dev(a.x - hi.x), tf32_rn_dev(a.y - hi.y), tf32_rn_dev(a.z - hi.z),
                             tf32_rn_dev(a.w - hi.w));
            *ph = hi;
            *reinterpret_cast<float4 *>(sA + kAHalfBytes + c * 16) = lo;
          }
        } else {
          // 128 rows x 4 groups of 8 k: read the landed FP32 (SWIZZLE_128B: 16-byte chunk
          // c of row r at (r/8)*1024 + (r%8)*128 + ((c ^ r%8) * 16)), write the three bf16
          // pieces into their planes (k-steps of 16, SWIZZLE_32B: chunk c of row r at
          // r*32 + ((c ^ (r/4)%2) * 16))
          for (int it = tid; it < kM * 4; it += kConv) {
            const int r = it >> 2, kq = it & 3;
            const uint8_t *row = sA + (r >> 3) * 1024 + (r & 7) * 128;
            const float4 x0 = *reinterpret_cast<const float4 *>(row + (((2 * kq) ^ (r & 7)) << 4));
            const float4 x1 = *reinterpret_cast<const float4 *>(row + (((2 * kq + 1) ^ (r & 7)) << 4));
            const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            uint4 p0, p1, p2;
            bf16_split3x8(xs, p0, p1, p2);
            const int j = kq >> 1, c = kq & 1;
            const int off = j * (kM * 32) + r * 32 + ((c ^ ((r >> 2) & 1)) << 4);
            uint8_t *planes = sA + kAHalfBytes;
            *reinterpret_cast<uint4 *>(planes + off) = p0;
            *reinterpret_cast<uint4 *>(planes + 2 * kM * 32 + off) = p1;
            *reinterpret_cast<uint4 *>(planes + 4 * kM * 32 + off) = p2;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&split[slot]);
      }
    }
  } else if (warp < kMmaWarp) {
    // ------------------------------------------------------------ epilogue
    // Each half (4 warps, one per TMEM lane quarter) takes every other 16-column
    // chunk; a lane owns one row and stores its 16 columns (consecutive lanes
    // write consecutive positions of a column).
    const int quarter = warp & 3, half = (warp - kEpiWarp0) >> 2;
    int v = 0;
    for (int T = next_tile(g, -1, total, nrt, ntn, nrhs, done_s); T < total; T = next_tile(g, T, total, nrt, ntn, nrhs, done_s)) {
      const TileInfo t = decode_tile<SPLIT>(g, T, nrt, ntn, nrhs, done_s);
      const TcProb &P = prob_of(g, t.prob);
      const int acc = v & 1;
      if (!mbar_wait(&tfull[acc], (v >> 1) & 1, abort)) break;
      tc_fence_after();
      // every field the stores need, in registers (no reloads between stores)
      const int r = t.r0 + quarter * 32 + lane, R = P.R, Ncols = P.N;
      const bool rok = r < R;
      const float lr = (P.lam_row && rok) ? P.lam_row[r] : 0.0f;
      const float *__restrict__ lc = P.lam_col;
      const double *__restrict__ so = P.scale_out;
      const int64_t cs = P.c_cs;
      // row r = u*out_nv + v goes to n*cs + u*ldv + v (FP32) or n*R + r (FP64 result)
      const int uu = r / P.out_nv;
      const int64_t pos = P.C64 ? (int64_t)r : (int64_t)uu * P.ldv + (r - uu * P.out_nv);
      double *__restrict__ c64 = P.C64 ? P.C64 + (int64_t)t.rhs * P.c_rhs_stride + pos : nullptr;
      float *__restrict__ c32 = P.C32 ? P.C32 + (int64_t)t.rhs * P.c_rhs_stride + pos : nullptr;
      const double *__restrict__ sor = so ? so + r : nullptr;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * ntc);
      const int nchunks = t.NT / 16;
      // Stores walk a pointer down the columns (c_cs or R apart); the divide's
      // 16 column eigenvalue sums are loaded once per chunk (lane l holds column
      // nb + l % 16) and broadcast by shuffles; the divide is x * (1/Delta) with
      // the fast reciprocal (2 ulp in FP32, far below the split products' error).
      auto store_chunk = [&](const uint32_t (&vals)[16], int c) {
        const int nb = t.n0 + 16 * c;
        float lcv = 0.0f;
        if (lc) lcv = nb + (lane & 15) < Ncols ? lc[nb + (lane & 15)] : 1.0f;
        if (c64) {
          double *p = c64 + (int64_t)nb * cs;
          const double *ps = sor ? sor + (int64_t)nb * R : nullptr;
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) {
            float x = __uint_as_float(vals[qq]);
            if (lc) x = __fdividef(x, lr + __shfl_sync(0xffffffffu, lcv, qq));
            if (rok && nb + qq < Ncols) {
              double y = f32_to_f64(x);
              if (ps) y *= ps[(int64_t)qq * R];
              *p = y;
            }
            p += cs;
          }
        } else if (lc) {
          float *p = c32 + (int64_t)nb * cs;
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) {
            const float lq = __shfl_sync(0xffffffffu, lcv, qq);
            if (rok && nb + qq < Ncols) *p = __fdividef(__uint_as_float(vals[qq]), lr + lq);
            p += cs;
          }
        } else {
          float *p = c32 + (int64_t)nb * cs;
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) {
            if (rok && nb + qq < Ncols) *p = __uint_as_float(vals[qq]);
            p += cs;
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
      int q = 0, v = 0, last_slot = -1, last_par = 0, bkey = -1, nb = 0;
      bool ok = true;
      for (int T = next_tile(g, -1, total, nrt, ntn, nrhs, done_s); ok && T < total;
           T = next_tile(g, T, total, nrt, ntn, nrhs, done_s)) {
        const TileInfo t = decode_tile<SPLIT>(g, T, nrt, ntn, nrhs, done_s);
        const int acc = v & 1, u = v >> 1;
        if (u > 0 && !mbar_wait(&tempty[acc], (u - 1) & 1, abort)) { ok = false; break; }
        const int key = t.prob * ntn + t.n0 / kNTMax;
        if (resident && key != bkey) {
          if (!mbar_wait(bfull, (uint32_t)(nb & 1), abort)) { ok = false; break; }
          bkey = key;
          ++nb;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * ntc);   // accumulator columns [acc ntc, acc ntc + NT)
        const uint32_t idesc = SPLIT ? idesc_bf16(t.NT) : idesc_tf32(t.NT);
        for (int s = 0; s < t.nstages; ++s) {
          const int slot = q % nstage_ring;
          if (atm) {
            const int as = q & 1;
            if (!mbar_wait(&split[as], (q >> 1) & 1, abort)) { ok = false; break; }
            tc_fence_after();
            const int k0 = s * kKC;
            const int ks = (t.kp - k0) / 8 < 4 ? (t.kp - k0) / 8 : 4;
            const uint8_t *sB = Bres + (size_t)8 * t.NT * k0;
            const uint64_t bh0 = sdesc_sw32(sB), bl0 = sdesc_sw32(sB + (size_t)ks * t.NT * 32);
            const uint64_t bstep = (uint64_t)t.NT * 2;
            const uint32_t ah0 = tmem + (uint32_t)(2 * ntc + 64 * as);
            const uint32_t acc0 = s > 0 ? 1u : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (j < ks) {
                const uint32_t ah = ah0 + 8u * j, al = ah + 32u;
                const uint64_t bh = bh0 + bstep * j, bl = bl0 + bstep * j;
                mma_tf32_ta(d, ah, bh, idesc, j > 0 ? 1u : acc0);
                mma_tf32_ta(d, ah, bl, idesc, 1u);
                mma_tf32_ta(d, al, bh, idesc, 1u);
              }
            }
            mma_commit(&a_empty[as]);
            last_slot = as;
            last_par = (q >> 1) & 1;
            ++q;
            continue;
          }
          if (!mbar_wait(&split[slot], (q / nstage_ring) & 1, abort)) { ok = false; break; }
          tc_fence_after();
          uint8_t *sA = smem + slot * stage_bytes;
          const int k0 = s * kKC;
          uint8_t *sB = resident ? Bres + (size_t)TR::kBPE * t.NT * k0 : sA + TR::kAStage;
          const int ks = (t.kp - k0) / TR::kKStep < kKC / TR::kKStep ? (t.kp - k0) / TR::kKStep : kKC / TR::kKStep;
          // Descriptors are built once per stage; a k-step moves the start address
          // field (16-byte units, bits 0-13) by a constant, so the issue loop is a
          // few adds per MMA (one thread must keep the tensor pipe fed)
          const uint32_t acc0 = s > 0 ? 1u : 0u;
          if (SPLIT == 0) {
            const uint64_t ah0 = sdesc_sw128(sA), al0 = sdesc_sw128(sA + kAHalfBytes);
            const uint64_t bh0 = sdesc_sw32(sB), bl0 = sdesc_sw32(sB + (size_t)ks * t.NT * 32);
            const uint64_t bstep = (uint64_t)t.NT * 2;   // NT rows x 32 B per k-step
#pragma unroll
            for (int j = 0; j < kKC / TR::kKStep; ++j) {
              if (j < ks) {
                const uint64_t ah = ah0 + 2u * j, al = al0 + 2u * j;   // 32 B per k-step inside the atom
                const uint64_t bh = bh0 + bstep * j, bl = bl0 + bstep * j;
                mma_tf32(d, ah, bh, idesc, j > 0 ? 1u : acc0);
                mma_tf32(d, ah, bl, idesc, 1u);
                mma_tf32(d, al, bh, idesc, 1u);
              }
            }
          } else {
            // 6 leading products of (a0 + a1 + a2)(b0 + b1 + b2): pieces i + j <= 2
            const uint64_t a00 = sdesc_sw32(sA + kAHalfBytes), b00 = sdesc_sw32(sB);
            const uint64_t apart = (uint64_t)(2 * kM * 32) >> 4, astep = (uint64_t)(kM * 32) >> 4;
            const uint64_t bstep = (uint64_t)t.NT * 2, bpart = bstep * ks;
#pragma unroll
            for (int j = 0; j < kKC / TR::kKStep; ++j) {
              if (j < ks) {
                const uint64_t a0 = a00 + astep * j, a1 = a0 + apart, a2 = a1 + apart;
                const uint64_t b0 = b00 + bstep * j, b1 = b0 + bpart, b2 = b1 + bpart;
                mma_bf16(d, a0, b0, idesc, j > 0 ? 1u : acc0);
                mma_bf16(d, a0, b1, idesc, 1u);
                mma_bf16(d, a1, b0, idesc, 1u);
                mma_bf16(d, a0, b2, idesc, 1u);
                mma_bf16(d, a1, b1, idesc, 1u);
                mma_bf16(d, a2, b0, idesc, 1u);
              }
            }
          }
          mma_commit(&empty[slot]);
          last_slot = slot;
          last_par = (q / nstage_ring) & 1;
          ++q;
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
        ++v;
        if (atm) {
          // the TMA may overwrite the resident B only once every MMA on it has completed
          const int T2 = next_tile(g, T, total, nrt, ntn, nrhs, done_s);
          if (T2 < total) {
            const TileInfo t2 = decode_tile<SPLIT>(g, T2, nrt, ntn, nrhs, done_s);
            if (t2.prob * ntn + t2.n0 / kNTMax != key) mma_commit(bfree);
          }
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        *abort = 1;
      }
      // drain: the last commit covers every MMA issued before it (bounded wait, ignoring abort)
      if (last_slot >= 0) {
        volatile int never = 0;
        mbar_wait(atm ? &a_empty[last_slot] : &empty[last_slot], last_par, &never);
      }
    }
    __syncwarp();
  }
  if (*abort && tid == 0) atomicAdd(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

// FP64 first-step input (times the optional scaling) to the FP32 layout the
// TMA reads: A32[r*lda + k] = (float)(A64[r*K + k] * scale_in[r*K + k]).
__global__ void k_tc_convert(TcGroup g, const int *done) {
  const int rhs = g.rhs0 + (int)blockIdx.y;
  if (done && done[rhs]) return;
  const TcProb &P = prob_of(g, blockIdx.z);
  if (!P.A64 || (P.done_flag && *P.done_flag)) return;
  const double *src = P.A64 + rhs * P.a64_rhs_stride;
  float *dst = const_cast<float *>(P.A32) + rhs * P.a_rhs_stride;
  // a warp per row (lanes along k, coalesced FP64 loads and FP32 stores), four
  // loads per lane in flight before the conversions
  const int K = P.K, R = P.R, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + (threadIdx.x >> 5); r < R; r += gridDim.x * nw) {
    const double *s = src + (size_t)r * K;
    const double *sc = P.scale_in ? P.scale_in + (size_t)r * K : nullptr;
    float *d = dst + (size_t)r * P.lda;
    for (int k0 = 0; k0 < K; k0 += 128) {
      double x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + 32 * u + lane;
        x[u] = k < K ? s[k] : 0.0;
      }
      if (sc) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 32 * u + lane;
          if (k < K) x[u] *= sc[k];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + 32 * u + lane;
        if (k < K) d[k] = f64_to_f32_rn(x[u]);
      }
    }
  }
}

fdst_status tc_encode_map(void *map128, const float *A32, int K, int R, int lda, int64_t rhs_stride, int nrhs) {
  using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  static std::mutex m;
  {
    std::lock_guard<std::mutex> lock(m);
    if (!encode) {
      void *fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
              cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return FDST_CUDA_ERROR;
      }
      encode = reinterpret_cast<Encode>(fn);
    }
  }
  if ((reinterpret_cast<uintptr_t>(A32) & 15) || (lda & 3) || (rhs_stride & 3) || K < 1 || R < 1 || nrhs < 1) {
    set_error("tensor map: FP32 operand must be 16-byte aligned with row and right-hand-side pitches of 4 floats");
    return FDST_INVALID_ARGUMENT;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)nrhs};
  const cuuint64_t strides[2] = {(cuuint64_t)lda * 4, (cuuint64_t)rhs_stride * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)kM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(reinterpret_cast<CUtensorMap *>(map128), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            const_cast<float *>(A32), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
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
  const int stage_bytes = g.split ? SplitTraits<1>::kAStage + SplitTraits<1>::kBPE * nt * kKC
                                  : SplitTraits<0>::kAStage + SplitTraits<0>::kBPE * nt * kKC;
  int nring = (kSmemBudget - 2048) / stage_bytes;
  return nring > 4 ? 4 : nring;
}

// The launch's shape: column tiles, tensor-memory columns, feeding mode (B
// streamed or resident, A in shared or tensor memory), ring depth and shared
// memory. Host-only; FDST_NOT_SUPPORTED when the requested mode does not fit.
struct TcPlan {
  int maxR, ntn, nt, ntc, bres, amode, tmem_cols, nring, smem;
};

static fdst_status tc_plan(const TcGroup &g, int ring, TcPlan &P) {
  int maxR, maxN;
  tc_dims(g, maxR, maxN);
  const int npad = tc_npad(maxN);
  const int ntn = (npad + kNTMax - 1) / kNTMax;
  const int nt = npad < kNTMax ? npad : kNTMax;
  int ntc = nt <= 32 ? 32 : nt <= 64 ? 64 : nt <= 128 ? 128 : 256;   // TMEM columns per accumulator
  const int astage = g.split ? SplitTraits<1>::kAStage : SplitTraits<0>::kAStage;
  const int bpe = g.split ? SplitTraits<1>::kBPE : SplitTraits<0>::kBPE;
  int stage_bytes = astage + bpe * nt * kKC;
  int nring = tc_max_ring(g);
  // resident B when the largest (problem, column tile) image fits beside two A stages
  int bres = 0;
  int bmax = g.table ? g.bmax : 0;
  if (!g.table)
    for (int i = 0; i < g.nprob; ++i) bmax = std::max(bmax, tc_b_tile_bytes(g.p[i].K, g.p[i].N, g.split));
  if (bmax > 0 && g.mode != 1) {
    const int nr = std::min(4, (kSmemBudget - 2048 - bmax) / astage);
    if (nr >= 2) {
      bres = (bmax + 1023) & ~1023;
      nring = std::min(4, (kSmemBudget - 2048 - bres) / astage);
      stage_bytes = astage;
    }
  }
  if ((g.mode == 2 || g.mode == 3) && bres == 0) {
    set_error("tensor-core contraction: the resident B operand does not fit in shared memory");
    return FDST_NOT_SUPPORTED;
  }
  // split-TF32 with resident B: A's pieces go to tensor memory when both accumulators
  // (32-column multiples) and two 64-column A stages fit in its 512 columns
  int amode = 0, tmem_cols = 2 * ntc;
  if (bres > 0 && !g.split && 2 * ((nt + 31) & ~31) + 128 <= 512 && g.mode != 2) {
    amode = 1;
    ntc = (nt + 31) & ~31;
    tmem_cols = 512;
    stage_bytes = kAHalfBytes;
    nring = std::min(4, (kSmemBudget - 2048 - bres) / kAHalfBytes);
  }
  if (g.mode == 3 && !amode) {
    set_error("tensor-core contraction: A in tensor memory needs split-TF32, resident B and N <= 192");
    return FDST_NOT_SUPPORTED;
  }
  if (ring > 0 && ring < nring) nring = ring;
  if (nring < 2) {
    set_error("tensor-core contraction: shared memory too small for two stages");
    return FDST_NOT_SUPPORTED;
  }
  P.maxR = maxR;
  P.ntn = ntn;
  P.nt = nt;
  P.ntc = ntc;
  P.bres = bres;
  P.amode = amode;
  P.tmem_cols = tmem_cols;
  P.nring = nring;
  P.smem = nring * stage_bytes + bres + 1024 + 1024;
  return FDST_OK;
}

fdst_status tc_mode_fits(const TcGroup &g, int ring) {
  TcPlan P;
  return tc_plan(g, ring, P);
}

fdst_status launch_gemm_tc(const TcGroup &g, int nrhs, const int *done, cudaStream_t s, int ring) {
  if (nrhs > kMaxRhsLaunch) {
    // the kernel keeps the stop flags of its right-hand sides in shared memory
    TcGroup h = g;
    for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsLaunch) {
      h.rhs0 = g.rhs0 + r0;
      const fdst_status st = launch_gemm_tc(h, std::min(kMaxRhsLaunch, nrhs - r0), done, s, ring);
      if (st != FDST_OK) return st;
    }
    return FDST_OK;
  }
  TcPlan P;
  {
    const fdst_status st = tc_plan(g, ring, P);
    if (st != FDST_OK) return st;
  }
  const int maxR = P.maxR, ntn = P.ntn, nt = P.nt, ntc = P.ntc, bres = P.bres, amode = P.amode;
  const int tmem_cols = P.tmem_cols, nring = P.nring;
  const int smem = P.smem;
  static int configured[2] = {0, 0}, nsm = 0;
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
  const int sp = g.split ? 1 : 0;
  if (smem > configured[sp]) {
    const cudaError_t e = sp ? cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                             : cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute(k_gemm_tc) failed");
      return FDST_CUDA_ERROR;
    }
    configured[sp] = smem;
  }
  if (g.convert) {
    long long blocks = ((long long)maxR + 7) / 8;   // 8 rows (warps) per block
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    count_launch(1);
    k_tc_convert<<<dim3((unsigned)blocks, nrhs, g.nprob), 256, 0, s>>>(g, done);
  }
  const int nrt = (maxR + kM - 1) / kM;
  const long long total = (long long)nrt * ntn * g.nprob * nrhs;
  const int grid = total < nsm ? (int)total : nsm;
  count_launch(1);
  if (sp)
    k_gemm_tc<1><<<grid, kThreads, smem, s>>>(g, nrhs, done, g_err_flag, nrt, ntn, nring, ntc, nt, bres, amode,
                                              tmem_cols);
  else
    k_gemm_tc<0><<<grid, kThreads, smem, s>>>(g, nrhs, done, g_err_flag, nrt, ntn, nring, ntc, nt, bres, amode,
                                              tmem_cols);
  return FDST_OK;
}

// Self-test of the failure detection: one thread waits, through the same bounded
// wait the contraction kernel uses, on an mbarrier nothing ever arrives on; the
// wait must give up after its limit and raise the abort flag, and the kernel
// must then return normally.
__global__ void k_wait_selftest(int *out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool completed = mbar_wait(&bar, 0, &abort_flag);
    out[0] = completed ? 1 : 0;
    out[1] = abort_flag;
  }
}

fdst_status tc_wait_selftest(int *gave_up, double *seconds) {
  int *d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) {
    set_error("self-test allocation failed");
    return FDST_OUT_OF_MEMORY;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  count_launch(1);
  k_wait_selftest<<<1, 32>>>(d);
  cudaEventRecord(e1, 0);
  int h[2] = {1, 0};
  const cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error(std::string("self-test: ") + cudaGetErrorString(e));
    return FDST_CUDA_ERROR;
  }
  *gave_up = (h[0] == 0 && h[1] == 1) ? 1 : 0;
  *seconds = ms * 1e-3;
  return FDST_OK;
}

fdst_status tc_error_count(int *value) {
  *value = 0;
  if (!g_err_flag) return FDST_OK;
  if (cudaMemcpy(value, g_err_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("reading the tensor-core error flag failed");
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
}

fdst_status tc_error_flag(int *value) {
  const fdst_status st = tc_error_count(value);
  if (st != FDST_OK) return st;
  *value = *value > 0 ? 1 : 0;
  return FDST_OK;
}

}  // namespace fdst

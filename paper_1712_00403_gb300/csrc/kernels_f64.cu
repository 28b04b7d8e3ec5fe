// FP64 device kernels: FD mode contractions (rotation GEMM with the
// Algorithm 1 step 3 divide fused into the epilogue), banded Kronecker mode
// products of the Stokes matvec, deterministic dot products and the MINRES
// vector / scalar updates. On GB300 the FP64 pipe (~1.2 TFLOP/s measured) is
// the bound of every kernel here that does arithmetic; the vector kernels
// are HBM-bound.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <type_traits>

#include "df_arith.cuh"
#include "fp_bits.cuh"
#include "kernels.h"

namespace fdst {

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ rotation GEMM

namespace {
constexpr int kBR = 64;   // rows per tile
constexpr int kBK = 16;   // k per smem stage
constexpr int kThreads = 256;
}  // namespace

template <int TN>
__global__ void __launch_bounds__(kThreads) k_gemm_f64(GemmGroup g, int nrhs, const int *done) {
  constexpr int BN = 16 * TN;
  const int prob = blockIdx.z % g.nprob;
  const int rhs = blockIdx.z / g.nprob;
  if (done && done[rhs]) return;
  const GemmProb &P = g.table ? g.table[prob] : g.p[prob];
  if (P.done_flag && *P.done_flag) return;
  const int R = P.R, K = P.K, N = P.N;
  const int r0 = blockIdx.x * kBR, n0 = blockIdx.y * BN;
  if (r0 >= R || n0 >= N) return;
  const double *A = P.A + rhs * P.a_rhs_stride;
  double *C = P.C + rhs * P.c_rhs_stride;
  const double *B = P.B;

  __shared__ double As[kBK][kBR + 1];
  __shared__ double Bs[kBK][BN];
  const int tid = threadIdx.x, tr = tid & 15, tn = tid >> 4;
  double acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kBK) {
#pragma unroll
    for (int e = 0; e < (kBR * kBK) / kThreads; ++e) {
      int idx = tid + e * kThreads;
      int kk = idx % kBK, rr = idx / kBK;
      int r = r0 + rr, k = k0 + kk;
      double v = 0.0;
      if (r < R && k < K) {
        int64_t ai = (int64_t)r * K + k;
        v = A[ai];
        if (P.scale_in) v *= P.scale_in[ai];
      }
      As[kk][rr] = v;
    }
#pragma unroll
    for (int e = 0; e < (BN * kBK) / kThreads; ++e) {
      int idx = tid + e * kThreads;
      int nn = idx % BN, kk = idx / BN;
      int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? B[(int64_t)k * N + n] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double a[4], b[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = r0 + tr + 16 * i;
    if (r >= R) continue;
    double lr = P.lam_row ? P.lam_row[r] : 0.0;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tn + 16 * j;
      if (n >= N) continue;
      double v = acc[i][j];
      if (P.lam_row) v = v / (lr + P.lam_col[n]);
      int64_t ci = (int64_t)n * R + r;
      if (P.scale_out) v *= P.scale_out[ci];
      C[ci] = v;
    }
  }
}

void launch_gemm_f64(const GemmGroup &g, int nrhs, const int *done, cudaStream_t s) {
  int maxR = g.maxR, maxN = g.maxN;
  if (!g.table)
    for (int i = 0; i < g.nprob; ++i) {
      maxR = g.p[i].R > maxR ? g.p[i].R : maxR;
      maxN = g.p[i].N > maxN ? g.p[i].N : maxN;
    }
  // column tile: forced (tuned), else the one that wastes the fewest padded columns
  int best = g.tn, bestpad = 1 << 30;
  if (!best) {
    best = 4;
    for (int tn = 2; tn <= 4; ++tn) {
      int bn = 16 * tn;
      long long pad = 0;
      if (g.table) pad = (long long)((maxN + bn - 1) / bn * bn - maxN);
      else
        for (int i = 0; i < g.nprob; ++i) pad += (long long)(((g.p[i].N + bn - 1) / bn) * bn - g.p[i].N) * g.p[i].R;
      if (pad < bestpad || (pad == bestpad && tn > best)) { bestpad = (int)pad; best = tn; }
    }
  }
  dim3 grid((maxR + kBR - 1) / kBR, (maxN + 16 * best - 1) / (16 * best), g.nprob * nrhs);
  count_launch(1);
  if (best == 2) k_gemm_f64<2><<<grid, kThreads, 0, s>>>(g, nrhs, done);
  else if (best == 3) k_gemm_f64<3><<<grid, kThreads, 0, s>>>(g, nrhs, done);
  else k_gemm_f64<4><<<grid, kThreads, 0, s>>>(g, nrhs, done);
}

// ------------------------------------------------------------------ banded mode product

__global__ void __launch_bounds__(512) k_band(BandGroup g, int nrhs, const int *done) {
  const int rhs = blockIdx.y;
  if (done && done[rhs]) return;
  const BandOp &op = g.table ? g.table[blockIdx.z] : g.op[blockIdx.z];
  if (op.done_flag && *op.done_flag) return;
  const int mode = op.mode;
  const unsigned od0 = mode == 0 ? op.rows : op.d0, od1 = mode == 1 ? op.rows : op.d1,
                 od2 = mode == 2 ? op.rows : op.d2;
  const int64_t total = (int64_t)od0 * od1 * od2;
  const int64_t stride_in = mode == 0 ? 1 : (mode == 1 ? (int64_t)op.d0 : (int64_t)op.d0 * op.d1);
  const double *X = op.X + rhs * op.x_rhs_stride;
  double *Y = op.Y + rhs * op.y_rhs_stride;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const unsigned ou = (unsigned)o;            // a block has fewer than 2^32 entries
    const unsigned t = ou / od0;
    const int o0 = (int)(ou - t * od0);
    const unsigned o2u = t / od1;
    const int o1 = (int)(t - o2u * od1), o2 = (int)o2u;
    const int i = mode == 0 ? o0 : (mode == 1 ? o1 : o2);
    int64_t base;
    if (mode == 0) base = ((int64_t)o2 * op.d1 + o1) * op.d0;
    else if (mode == 1) base = (int64_t)o2 * op.d1 * op.d0 + o0;
    else base = (int64_t)o1 * op.d0 + o0;
    const double *v = op.vals + (int64_t)i * op.w;
    const int l = op.lo[i];
    double acc = 0.0;
    for (int j = 0; j < op.w; ++j) acc = fma(v[j], X[base + (int64_t)(l + j) * stride_in], acc);
    acc *= op.coef;
    Y[o] = op.accumulate ? Y[o] + acc : acc;
  }
}

void launch_band(const BandGroup &g, int nrhs, const int *done, cudaStream_t s) {
  int64_t maxt = g.maxt;
  if (!g.table)
    for (int i = 0; i < g.nop; ++i) {
      const auto &o = g.op[i];
      int64_t t = (int64_t)(o.mode == 0 ? o.rows : o.d0) * (o.mode == 1 ? o.rows : o.d1) * (o.mode == 2 ? o.rows : o.d2);
      maxt = t > maxt ? t : maxt;
    }
  const int thr = g.threads > 0 ? g.threads : 256;
  int64_t blocks = (maxt + thr - 1) / thr;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  dim3 grid((unsigned)blocks, nrhs, g.nop);
  count_launch(1);
  k_band<<<grid, thr, 0, s>>>(g, nrhs, done);
}

// ------------------------------------------------------------------ double-float banded mode product
// GB300's FP64 pipe runs at 1/62 of its FP32 rate, so the matvec can also be
// evaluated in double-float arithmetic on the FP32 units: a value is an
// unevaluated sum hi + lo of two floats. Products use the exact FMA residual
// (p = a*b, e = fma(a, b, -p)), sums use Knuth's branch-free TwoSum.

// Each thread computes T outputs that share one band row i (so one V row and
// one lo[i]). Mode 0 (contracted index fastest): T consecutive lines, lanes
// over the flattened (line group, row) pairs, so that no lane idles when the
// row count is not a multiple of the warp width. Modes 1 and 2: T entries of
// the flattened (outer, fastest) index strided by the warp width, lanes over
// consecutive entries (coalesced X and Y); when a warp's 32 T entries lie in
// one outer slab (always in mode 2 but for the tail) they sit at one base
// address plus constant offsets. Work items run row-fastest so that warps in
// flight share their X windows in L1/L2.
// At most 256 threads per block and 64 registers per thread (4 blocks of 256 per SM).
// W > 0: every op of the launch has band width W (the band loops unroll fully,
// so the loads take immediate offsets from a few base pointers); W = 0: any width.
// PAIRS (with W > 0): modes 1/2 take band rows in pairs where they can (below).
template <int T, int W, bool PAIRS>
__global__ void __launch_bounds__(256, 4) k_band_df(BandGroupDF g, int nrhs, const int *done) {
  const int rhs = blockIdx.y;
  if (done && done[rhs]) return;
  const BandOpDF &op = g.table ? g.table[blockIdx.z] : g.op[blockIdx.z];
  if (op.done_flag && *op.done_flag) return;
  const float2 *X = op.X + rhs * op.x_rhs_stride;
  float2 *Y = op.Y + rhs * op.y_rhs_stride;
  const unsigned lane = threadIdx.x & 31;
  // (one operand of one right-hand side holds fewer than 2^32 entries: 32-bit offsets and work indices)
  const unsigned warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  const int w = op.w;
  const unsigned rows = (unsigned)op.rows;
  // the op's coefficient is folded into vals: store (or add) the renormalized sum.
  // With accumulation the T old values of Y are loaded together before the first
  // store, so that their latencies overlap.
  const bool acc = op.accumulate != 0;
  double *y64 = op.Y64 ? op.Y64 + rhs * op.y_rhs_stride : nullptr;
  auto finish = [&](float sh, float sl, float2 yo, float2 *dst) {
    if (acc) df_add(sh, sl, yo.x, yo.y);
    const float2 r = df_norm(sh, sl);
    if (y64) y64[dst - Y] = f64_join(r);
    else *dst = r;
  };
  const bool swap = op.swap != 0;
  const unsigned d0 = (unsigned)op.d0, d1 = (unsigned)op.d1, d2 = (unsigned)op.d2;
  if (op.mode == 0) {
    const unsigned lines = d1 * d2;
    const unsigned groups = (lines + T - 1) / T;
    const unsigned nq = groups * rows;          // (line group, row) pairs
    const unsigned chunks = (nq + 31) >> 5;
    for (unsigned u = warp0; u < chunks; u += nwarps) {
      const unsigned q = u * 32u + lane;
      if (q >= nq) continue;
      const unsigned grp = q / rows;
      const unsigned i = q - grp * rows;
      const unsigned L0 = grp * T;
      const float2 *xp = X + ((size_t)L0 * d0 + op.lo[i]);
      const float2 *vp = op.vals + (size_t)i * w;
      // output offsets of lines L0 + t: (L0 + t) rows + i, or with the slow coordinates
      // swapped i + rows (l2 + d2 l1) for line l1 + d1 l2
      unsigned yoff[T];
      if (!swap) {
#pragma unroll
        for (int t = 0; t < T; ++t) yoff[t] = (L0 + t) * rows + i;
      } else {
        unsigned l2 = L0 / d1, l1 = L0 - l2 * d1;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          yoff[t] = i + rows * (l2 + d2 * l1);
          if (++l1 == d1) { l1 = 0; ++l2; }
        }
      }
      float sh[T], sl[T];
#pragma unroll
      for (int t = 0; t < T; ++t) sh[t] = sl[t] = 0.0f;
      if (L0 + T <= lines) {
        if constexpr (W > 0) {
          const float2 *xt[T];
#pragma unroll
          for (int t = 0; t < T; ++t) xt[t] = xp + t * d0;
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const float2 v = vp[j];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, xt[t][j], sh[t], sl[t]);
          }
        } else {
#pragma unroll 2
          for (int j = 0; j < w; ++j) {
            const float2 v = vp[j];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, xp[t * d0 + j], sh[t], sl[t]);
          }
        }
        float2 yo[T];
#pragma unroll
        for (int t = 0; t < T; ++t) yo[t] = acc ? Y[yoff[t]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < T; ++t) finish(sh[t], sl[t], yo[t], Y + yoff[t]);
      } else {
        const unsigned nt = lines - L0;
        for (int j = 0; j < w; ++j) {
          const float2 v = vp[j];
#pragma unroll
          for (int t = 0; t < T; ++t)
            if (t < nt) df_fma_acc(v, xp[t * d0 + j], sh[t], sl[t]);
        }
        float2 yo[T];
#pragma unroll
        for (int t = 0; t < T; ++t) yo[t] = acc && t < nt ? Y[yoff[t]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < T; ++t)
          if (t < nt) finish(sh[t], sl[t], yo[t], Y + yoff[t]);
      }
    }
  } else {
    // Y[(o * rows + i) * P + p], X[(o * din + l) * P + p], m = o * P + p over outer * P entries
    const unsigned P = op.mode == 1 ? d0 : d0 * d1;
    const unsigned outer = op.mode == 1 ? d2 : 1, din = op.mode == 1 ? d1 : d2;
    // output offset of entry (o, p) of row i: (o rows + i) P + p, or with the slow
    // coordinates swapped p + P (o + outer i) (mode 1) and c0 + d0 (i + rows c1) for
    // p = c0 + d0 c1 (mode 2)
    auto out12 = [&](unsigned o, unsigned pp, unsigned i) -> unsigned {
      if (!swap) return (o * rows + i) * P + pp;
      if (op.mode == 1) return pp + P * (o + outer * i);
      const unsigned c1 = pp / d0;
      return (pp - c1 * d0) + d0 * (i + rows * c1);
    };
    const unsigned M = outer * P;
    const unsigned mb = (M + 32 * T - 1) / (32 * T);
    // band row i over the 32 T entries of chunk cb
    auto row_unit = [&](unsigned cb, unsigned i) {
      const unsigned c0 = cb * (32 * T);     // first entry of this warp's chunk
      const unsigned l = op.lo[i];
      const float2 *vp = op.vals + (size_t)i * w;
      float sh[T], sl[T];
#pragma unroll
      for (int t = 0; t < T; ++t) sh[t] = sl[t] = 0.0f;
      const unsigned o0 = c0 / P;
      if (c0 + 32 * T <= M && c0 + 32 * T <= (o0 + 1) * P) {
        // the whole chunk in one outer slab (warp-uniform): offsets 32 t from one base
        const unsigned p0 = c0 - o0 * P + lane;
        const float2 *xp = X + ((size_t)(o0 * din + l) * P + p0);
        if constexpr (W > 0) {
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const float2 v = vp[j];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, xp[32 * t], sh[t], sl[t]);
            xp += P;
          }
        } else {
#pragma unroll 4
          for (int j = 0; j < w; ++j) {
            const float2 v = vp[j];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, xp[32 * t], sh[t], sl[t]);
            xp += P;
          }
        }
        unsigned yoff[T];
        if (!swap || op.mode == 1) {
          const unsigned y0 = out12(o0, p0, i);
#pragma unroll
          for (int t = 0; t < T; ++t) yoff[t] = y0 + 32 * t;
        } else {
          // mode 2, swapped: step c0 by 32 per t, carrying into c1
          unsigned c1 = p0 / d0, c0 = p0 - c1 * d0;
#pragma unroll
          for (int t = 0; t < T; ++t) {
            yoff[t] = c0 + d0 * (i + rows * c1);
            c0 += 32;
            while (c0 >= d0) { c0 -= d0; ++c1; }
          }
        }
        float2 yo[T];
#pragma unroll
        for (int t = 0; t < T; ++t) yo[t] = acc ? Y[yoff[t]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < T; ++t) finish(sh[t], sl[t], yo[t], Y + yoff[t]);
      } else {
        const unsigned m0 = c0 + lane;
        unsigned xo[T], yo[T];
        bool ok[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const unsigned m = m0 + 32 * t;
          ok[t] = m < M;
          const unsigned o = ok[t] ? m / P : 0, pp = ok[t] ? m - o * P : 0;
          xo[t] = (o * din + l) * P + pp;
          yo[t] = out12(o, pp, i);
        }
        // unrolled by 4: the loads of four band columns are in flight together
#pragma unroll 4
        for (int j = 0; j < w; ++j) {
          const float2 v = vp[j];
#pragma unroll
          for (int t = 0; t < T; ++t) {
            if (ok[t]) df_fma_acc(v, X[xo[t]], sh[t], sl[t]);
            xo[t] += P;
          }
        }
        float2 yv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) yv[t] = acc && ok[t] ? Y[yo[t]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < T; ++t)
          if (ok[t]) finish(sh[t], sl[t], yv[t], Y + yo[t]);
      }
    };
    if constexpr (W > 0 && PAIRS) {
      // Rows in pairs (i, i + 1): when lo[i + 1] = lo[i] + D for D <= 2 and the chunk lies
      // in one outer slab, the two rows read one window of W + D input rows, so each
      // loaded X entry feeds both rows' sums (each sum still runs over its own band in
      // column order, so every output equals the one-row evaluation bit for bit). Other
      // pairs run row by row. (Pairs in mode 0, where the lanes run over rows, spread a
      // warp's loads over twice the columns and were slower. Launches of many small
      // products with one right-hand side each, as in a batch, run without pairs:
      // halving their warps lengthened each launch's tail.)
      auto pair_unit = [&](auto dc, unsigned cb, unsigned i, unsigned o0) {
        constexpr int D = decltype(dc)::value;
        const unsigned c0 = cb * (32 * T);
        const unsigned p0 = c0 - o0 * P + lane;
        const float2 *va = op.vals + (size_t)i * W, *vb = va + W;
        const float2 *xp = X + ((size_t)(o0 * din + (unsigned)op.lo[i]) * P + p0);
        float ah[T], al[T], bh[T], bl[T];
#pragma unroll
        for (int t = 0; t < T; ++t) ah[t] = al[t] = bh[t] = bl[t] = 0.0f;
#pragma unroll
        for (int j = 0; j < W + D; ++j) {
          float2 x[T];
#pragma unroll
          for (int t = 0; t < T; ++t) x[t] = xp[32 * t];
          if (j < W) {
            const float2 v = va[j];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, x[t], ah[t], al[t]);
          }
          if (j >= D) {
            const float2 v = vb[j - D];
#pragma unroll
            for (int t = 0; t < T; ++t) df_fma_acc(v, x[t], bh[t], bl[t]);
          }
          xp += P;
        }
        // output offsets of both rows: row i + 1 sits one row stride after row i
        unsigned ya[T];
        unsigned rstride;
        if (!swap || op.mode == 1) {
          const unsigned y0 = out12(o0, p0, i);
#pragma unroll
          for (int t = 0; t < T; ++t) ya[t] = y0 + 32 * t;
          rstride = out12(o0, p0, i + 1) - y0;
        } else {
          unsigned c1 = p0 / d0, e0 = p0 - c1 * d0;
#pragma unroll
          for (int t = 0; t < T; ++t) {
            ya[t] = e0 + d0 * (i + rows * c1);
            e0 += 32;
            while (e0 >= d0) { e0 -= d0; ++c1; }
          }
          rstride = d0;
        }
        // the old values of both rows are loaded together before the first store
        float2 yo[2 * T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
          yo[t] = acc ? Y[ya[t]] : make_float2(0.f, 0.f);
          yo[T + t] = acc ? Y[ya[t] + rstride] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < T; ++t) finish(ah[t], al[t], yo[t], Y + ya[t]);
#pragma unroll
        for (int t = 0; t < T; ++t) finish(bh[t], bl[t], yo[T + t], Y + ya[t] + rstride);
      };
      const unsigned npairs = (rows + 1) >> 1;
      for (unsigned u = warp0; u < mb * npairs; u += nwarps) {
        const unsigned cb = u / npairs;
        const unsigned i = 2 * (u - cb * npairs);
        const unsigned c0 = cb * (32 * T);
        const unsigned o0 = c0 / P;
        const bool slab = c0 + 32 * T <= M && c0 + 32 * T <= (o0 + 1) * P;
        const int D = i + 1 < rows ? op.lo[i + 1] - op.lo[i] : -1;
        if (slab && D == 0) pair_unit(std::integral_constant<int, 0>{}, cb, i, o0);
        else if (slab && D == 1) pair_unit(std::integral_constant<int, 1>{}, cb, i, o0);
        else if (slab && D == 2) pair_unit(std::integral_constant<int, 2>{}, cb, i, o0);
        else {
          row_unit(cb, i);
          if (i + 1 < rows) row_unit(cb, i + 1);
        }
      }
    } else {
      for (unsigned u = warp0; u < mb * rows; u += nwarps) {
        const unsigned cb = u / rows;
        row_unit(cb, u - cb * rows);
      }
    }
  }
}

void launch_band_df(const BandGroupDF &g, int nrhs, const int *done, cudaStream_t s) {
  int64_t maxt = g.maxt;
  if (!g.table)
    for (int i = 0; i < g.nop; ++i) {
      const auto &o = g.op[i];
      int64_t t = (int64_t)(o.mode == 0 ? o.rows : o.d0) * (o.mode == 1 ? o.rows : o.d1) * (o.mode == 2 ? o.rows : o.d2);
      maxt = t > maxt ? t : maxt;
    }
  constexpr int T = 4;
  const int thr = g.threads > 0 && g.threads <= 256 ? g.threads : 128;
  int64_t blocks = (maxt / T + thr - 1) / thr;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  dim3 grid((unsigned)blocks, nrhs, g.nop);
  count_launch(1);
  // the band width shared by every op of the launch (by value: from the ops; from a
  // table: as the caller states), dispatched to a fully unrolled instantiation
  int w = g.w;
  if (!g.table) {
    w = g.nop > 0 ? g.op[0].w : 0;
    for (int i = 1; i < g.nop; ++i)
      if (g.op[i].w != w) w = 0;
  }
  switch (w) {
#define FDST_BAND_W(WW)                                                 \
    case WW:                                                            \
      if (g.row_pairs) k_band_df<T, WW, true><<<grid, thr, 0, s>>>(g, nrhs, done);  \
      else k_band_df<T, WW, false><<<grid, thr, 0, s>>>(g, nrhs, done); \
      break;
    // the widths of the banded factors at degrees 1..8 (Kronecker plans and point-basis tables)
    FDST_BAND_W(2) FDST_BAND_W(3) FDST_BAND_W(4) FDST_BAND_W(5) FDST_BAND_W(6) FDST_BAND_W(7)
    FDST_BAND_W(8) FDST_BAND_W(9) FDST_BAND_W(10) FDST_BAND_W(11) FDST_BAND_W(12) FDST_BAND_W(13)
    FDST_BAND_W(14) FDST_BAND_W(15) FDST_BAND_W(16) FDST_BAND_W(17) FDST_BAND_W(19) FDST_BAND_W(20)
#undef FDST_BAND_W
    default: k_band_df<T, 0, false><<<grid, thr, 0, s>>>(g, nrhs, done); break;
  }
}

// Two entries per thread with 16-byte accesses where the row start allows it
// (an odd leading entry on its own), so that each request moves twice the bytes.
__global__ void k_split_df(const double *x, float2 *y, int64_t n, int64_t stride, const int *done) {
  const int j = blockIdx.y;
  if (done && done[j]) return;
  const double *xr = x + j * stride;
  float2 *yr = y + j * stride;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  const uintptr_t ax = reinterpret_cast<uintptr_t>(xr) & 15, ay = reinterpret_cast<uintptr_t>(yr) & 15;
  if (ax != ay) {   // rows not aligned alike: one entry per thread
    for (int64_t i = t0; i < n; i += ts) yr[i] = f64_split(xr[i]);
    return;
  }
  const int64_t head = ax != 0 && n > 0 ? 1 : 0;   // both 8 mod 16: one leading entry aligns both
  if (head && t0 == 0) yr[0] = f64_split(xr[0]);
  const int64_t pairs = (n - head) >> 1;
  const double2 *x2 = reinterpret_cast<const double2 *>(xr + head);
  float4 *y4 = reinterpret_cast<float4 *>(yr + head);
  for (int64_t i = t0; i < pairs; i += ts) {
    const double2 v = x2[i];
    const float2 a = f64_split(v.x), b = f64_split(v.y);
    y4[i] = make_float4(a.x, a.y, b.x, b.y);
  }
  if (((n - head) & 1) && t0 == 0) yr[n - 1] = f64_split(xr[n - 1]);
}
__global__ void k_join_df(const float2 *x, double *y, int64_t n, int64_t stride, const int *done) {
  const int j = blockIdx.y;
  if (done && done[j]) return;
  const float2 *xr = x + j * stride;
  double *yr = y + j * stride;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  const uintptr_t ax = reinterpret_cast<uintptr_t>(xr) & 15, ay = reinterpret_cast<uintptr_t>(yr) & 15;
  if (ax != ay) {   // rows not aligned alike: one entry per thread
    for (int64_t i = t0; i < n; i += ts) yr[i] = f64_join(xr[i]);
    return;
  }
  const int64_t head = ax != 0 && n > 0 ? 1 : 0;   // both 8 mod 16: one leading entry aligns both
  if (head && t0 == 0) yr[0] = f64_join(xr[0]);
  const int64_t pairs = (n - head) >> 1;
  const float4 *x4 = reinterpret_cast<const float4 *>(xr + head);
  double2 *y2 = reinterpret_cast<double2 *>(yr + head);
  for (int64_t i = t0; i < pairs; i += ts) {
    const float4 v = x4[i];
    y2[i] = make_double2(f64_join(make_float2(v.x, v.y)), f64_join(make_float2(v.z, v.w)));
  }
  if (((n - head) & 1) && t0 == 0) yr[n - 1] = f64_join(xr[n - 1]);
}

// Element-wise precision conversions (the integer-unit forms above) over n entries.
__global__ void k_convert(int kind, const void *in, void *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    switch (kind) {
      case 0: static_cast<float *>(out)[i] = f64_to_f32_rn(static_cast<const double *>(in)[i]); break;
      case 1: static_cast<float2 *>(out)[i] = f64_split(static_cast<const double *>(in)[i]); break;
      case 2: static_cast<double *>(out)[i] = f64_join(static_cast<const float2 *>(in)[i]); break;
      default: static_cast<double *>(out)[i] = f32_to_f64(static_cast<const float *>(in)[i]); break;
    }
  }
}

void launch_convert(int kind, const void *in, void *out, int64_t n, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_convert<<<(unsigned)blocks, 256, 0, s>>>(kind, in, out, n);
}

void launch_split_df(const double *x, float2 *y, int64_t n, int64_t stride, int nrhs, const int *done,
                     cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_split_df<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(x, y, n, stride, done);
}

void launch_join_df(const float2 *x, double *y, int64_t n, int64_t stride, int nrhs, const int *done,
                    cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_join_df<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(x, y, n, stride, done);
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-level partial sums, then the last block to finish (atomic ticket)
// adds the partials in index order: the result does not depend on timing.
__global__ void __launch_bounds__(256) k_dot(const double *a, const double *b, int64_t n, int64_t stride,
                                             double *partials, unsigned *counters, double *out,
                                             const int *done) {
  const int rhs = blockIdx.y;
  if (done && done[rhs]) return;
  const double *x = a + rhs * stride;
  const double *y = b + rhs * stride;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  __shared__ double ws[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    partials[(int64_t)rhs * gridDim.x + blockIdx.x] = t;
    __threadfence();
    unsigned ticket = atomicAdd(&counters[rhs], 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    double t = 0.0;
    const volatile double *pp = partials + (int64_t)rhs * gridDim.x;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += 32) t += pp[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      out[rhs] = t;
      counters[rhs] = 0u;
    }
  }
}

void launch_dot(const double *a, const double *b, int64_t n, int64_t stride, int nrhs, double *partials,
                unsigned *counters, double *out, const int *done, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 304) blocks = 304;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_dot<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(a, b, n, stride, partials, counters, out, done);
}

__global__ void k_any_nonzero(const double *x, int64_t n, int *flag) {
  bool nz = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    nz |= !(x[i] == 0.0);
  if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

void launch_any_nonzero(const double *x, int64_t n, int *flag, cudaStream_t s) {
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_any_nonzero<<<(unsigned)blocks, 256, 0, s>>>(x, n, flag);
}

__global__ void k_axpby(const double *x, double *y, double alpha, double beta, int64_t n, int64_t stride) {
  const double *xr = x + blockIdx.y * stride;
  double *yr = y + blockIdx.y * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    yr[i] = alpha * xr[i] + (beta == 0.0 ? 0.0 : beta * yr[i]);
}

void launch_axpby(const double *x, double *y, double alpha, double beta, int64_t n, int64_t stride, int nrhs,
                  cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_axpby<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(x, y, alpha, beta, n, stride);
}

// ------------------------------------------------------------------ MINRES

__global__ void k_minres_init(MinresState *st, const double *g, int *done, int nrhs, int *n_stopped, double tol) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  MinresState S = {};
  S.tau = tol > 1e-14 ? tol : 1e-14;   // the recurrence's floor (kTauFloor)
  double g2 = g[j];
  S.iters = 0;
  S.status = 0;
  S.stop = 0;
  if (!(g2 >= 0.0) || isinf(g2)) {
    S.status = isnan(g2) || isinf(g2) ? 9 : 7;  // FDST_NAN_DETECTED : FDST_BREAKDOWN
    done[j] = 1;
    atomicAdd(n_stopped, 1);
  } else {
    double gamma = sqrt(g2);
    S.gamma = gamma;
    S.gamma_old = 1.0;
    S.c = S.c_old = 1.0;
    S.s = S.s_old = 0.0;
    S.eta = S.eta0 = gamma;
    S.inv_gamma_new = gamma > 0.0 ? 1.0 / gamma : 0.0;
    done[j] = gamma == 0.0;
    if (gamma == 0.0) atomicAdd(n_stopped, 1);
  }
  st[j] = S;
}

void launch_minres_init(MinresState *st, const double *g, int *done, int nrhs, int *n_stopped, double tol,
                        cudaStream_t s) {
  count_launch(1);
  k_minres_init<<<(nrhs + 63) / 64, 64, 0, s>>>(st, g, done, nrhs, n_stopped, tol);
}

__global__ void k_scale_inv_gamma(double *z, const MinresState *st, int64_t n, int64_t stride, const int *done) {
  const int j = blockIdx.y;
  if (done && done[j]) return;
  const double f = st[j].inv_gamma_new;
  double *zr = z + j * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    zr[i] *= f;
}

void launch_scale_by_inv_gamma(double *z, const MinresState *st, int64_t n, int64_t stride, int nrhs,
                               const int *done, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_scale_inv_gamma<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(z, st, n, stride, done);
}

// Lanczos step in place, per right-hand side: t = Az - (delta/gamma) v - (gamma/gamma_old) v_old,
// then v_old <- v, v <- t (no buffer-role swaps: frozen right-hand sides keep their state).
// The elementwise MINRES kernels take two entries per thread with 16-byte
// accesses when every row they touch starts at the same 16-byte phase (the
// handle's vectors always do; a caller's x may not), one otherwise.
__device__ __forceinline__ bool same_phase(const void *a, const void *b) {
  return ((reinterpret_cast<uintptr_t>(a) ^ reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

// ROT: the new Lanczos vector is written over v_old and v is left as it is (the
// caller exchanges the two roles), so the pass writes one vector instead of two.
template <bool ROT>
__global__ void k_minres_lanczos(const double *Az, double *v, double *v_old, const MinresState *st,
                                 const double *delta, int64_t n, int64_t stride, const int *done) {
  const int j = blockIdx.y;
  if (done[j]) return;
  const double gamma = st[j].gamma, gamma_old = st[j].gamma_old;
  const double f1 = delta[j] / gamma, f2 = gamma / gamma_old;
  const double *a = Az + j * stride;
  double *vv = v + j * stride, *vo = v_old + j * stride;
  // one entry: returns the new Lanczos value t, stores it (and, without ROT, shifts v into v_old)
  auto one = [&](int64_t i) {
    const double vi = vv[i], t = a[i] - f1 * vi - f2 * vo[i];
    if (ROT) {
      vo[i] = t;
    } else {
      vo[i] = vi;
      vv[i] = t;
    }
  };
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  if (!(same_phase(a, vv) && same_phase(a, vo))) {
    for (int64_t i = t0; i < n; i += ts) one(i);
    return;
  }
  const int64_t head = (reinterpret_cast<uintptr_t>(a) & 15) && n > 0 ? 1 : 0;
  if (head && t0 == 0) one(0);
  const int64_t pairs = (n - head) >> 1;
  const double2 *a2 = reinterpret_cast<const double2 *>(a + head);
  double2 *v2 = reinterpret_cast<double2 *>(vv + head), *o2 = reinterpret_cast<double2 *>(vo + head);
  for (int64_t i = t0; i < pairs; i += ts) {
    const double2 ai = a2[i], vi = v2[i], oi = o2[i];
    const double2 t = make_double2(ai.x - f1 * vi.x - f2 * oi.x, ai.y - f1 * vi.y - f2 * oi.y);
    if (ROT) {
      o2[i] = t;
    } else {
      o2[i] = vi;
      v2[i] = t;
    }
  }
  if (((n - head) & 1) && t0 == 0) one(n - 1);
}

void launch_minres_lanczos(const double *Az, double *v, double *v_old, const MinresState *st,
                           const double *delta, int64_t n, int64_t stride, int nrhs, const int *done,
                           cudaStream_t s, bool rotate) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  if (rotate)
    k_minres_lanczos<true><<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(Az, v, v_old, st, delta, n, stride, done);
  else
    k_minres_lanczos<false><<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(Az, v, v_old, st, delta, n, stride, done);
}

__global__ void k_swap(double *a, double *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = a[i];
    a[i] = b[i];
    b[i] = t;
  }
}

void launch_swap(double *a, double *b, int64_t n, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_swap<<<(unsigned)blocks, 256, 0, s>>>(a, b, n);
}

// One thread per right-hand side: Givens QR update of the Lanczos tridiagonal
// matrix and the residual estimate eta (the QR recurrences of MINRES).
__global__ void k_minres_scalars(MinresState *st, const double *delta, const double *g2v, int nrhs, int maxit,
                                 const int *done, int *n_stopped) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs || done[j]) return;
  MinresState S = st[j];
  const double d = delta[j], g2 = g2v[j];
  S.iters += 1;
  if (isnan(d) || isinf(d) || isnan(g2) || isinf(g2)) {
    S.status = 9;  // FDST_NAN_DETECTED
    S.stop = 1;
    S.inv_a1 = 0.0; S.a2 = 0.0; S.a3 = 0.0; S.coef_x = 0.0; S.inv_gamma_new = 0.0;
    st[j] = S;
    atomicAdd(n_stopped, 1);
    return;
  }
  const bool breakdown = g2 < 0.0;
  const double gn = breakdown ? 0.0 : sqrt(g2);
  const double a0 = S.c * d - S.c_old * S.s * S.gamma;
  const double a1 = sqrt(a0 * a0 + gn * gn);
  const double a2 = S.s * d + S.c_old * S.c * S.gamma;
  const double a3 = S.s_old * S.gamma;
  const double cn = a1 > 0.0 ? a0 / a1 : 1.0, sn = a1 > 0.0 ? gn / a1 : 0.0;
  S.inv_a1 = a1 > 0.0 ? 1.0 / a1 : 0.0;
  S.a2 = a2;
  S.a3 = a3;
  S.coef_x = cn * S.eta;
  S.eta = -sn * S.eta;
  S.inv_gamma_new = gn > 0.0 ? 1.0 / gn : 0.0;
  S.gamma_old = S.gamma;
  S.gamma = gn;
  S.c_old = S.c;
  S.c = cn;
  S.s_old = S.s;
  S.s = sn;
  const double rel = fabs(S.eta) / S.eta0;
  if (breakdown) { S.status = 7; S.stop = 1; }
  else if (rel <= S.tau || gn == 0.0) { S.status = 0; S.stop = 1; }
  else if (S.iters >= maxit) { S.status = 5; S.stop = 1; }
  if (S.stop) atomicAdd(n_stopped, 1);
  st[j] = S;
}

void launch_minres_scalars(MinresState *st, const double *delta, const double *g2, int nrhs, int maxit,
                           const int *done, int *n_stopped, cudaStream_t s) {
  count_launch(1);
  k_minres_scalars<<<(nrhs + 63) / 64, 64, 0, s>>>(st, delta, g2, nrhs, maxit, done, n_stopped);
}

// w_new = (z - a3 w_old - a2 w)/a1; w_old <- w; w <- w_new; x += coef_x w_new;
// z <- z_new / gamma_new (the next normalized Lanczos vector), all in place; with z_df
// set, also the double-float pairs of the new z (the next banded matvec reads them
// instead of a separate split pass).
// ROT: the new direction is written over w_old and w is left as it is (the caller
// exchanges the two roles), so the pass writes one direction vector instead of two.
template <bool ROT>
__global__ void k_minres_update(double *w_old, double *w, double *x, double *z, const double *z_new,
                                const MinresState *st, int64_t n, int64_t stride, const int *done, float2 *z_df) {
  const int j = blockIdx.y;
  if (done[j]) return;
  const MinresState &S = st[j];
  const double ia1 = S.inv_a1, a2 = S.a2, a3 = S.a3, cx = S.coef_x, ig = S.inv_gamma_new;
  double *wo = w_old + j * stride, *ww = w + j * stride, *xx = x + j * stride, *zz = z + j * stride;
  const double *zn = z_new + j * stride;
  float2 *zd = z_df ? z_df + j * stride : nullptr;
  auto step = [&](double wi, double woi, double zi, double xi, double zni, double &wo_out, double &w_out,
                  double &x_out, double &z_out) {
    const double wn = (zi - a3 * woi - a2 * wi) * ia1;
    if (ROT) {
      wo_out = wn;
    } else {
      wo_out = wi;
      w_out = wn;
    }
    x_out = fma(cx, wn, xi);
    z_out = zni * ig;
  };
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ts = (int64_t)gridDim.x * blockDim.x;
  const bool zd_ok = !zd || (((reinterpret_cast<uintptr_t>(zd) >> 3) ^ (reinterpret_cast<uintptr_t>(ww) >> 3)) & 1) == 0;
  if (!(same_phase(ww, wo) && same_phase(ww, xx) && same_phase(ww, zz) && same_phase(ww, zn) && zd_ok)) {
    for (int64_t i = t0; i < n; i += ts) {
      step(ww[i], wo[i], zz[i], xx[i], zn[i], wo[i], ww[i], xx[i], zz[i]);
      if (zd) zd[i] = f64_split(zz[i]);
    }
    return;
  }
  const int64_t head = (reinterpret_cast<uintptr_t>(ww) & 15) && n > 0 ? 1 : 0;
  if (head && t0 == 0) {
    step(ww[0], wo[0], zz[0], xx[0], zn[0], wo[0], ww[0], xx[0], zz[0]);
    if (zd) zd[0] = f64_split(zz[0]);
  }
  const int64_t pairs = (n - head) >> 1;
  double2 *w2 = reinterpret_cast<double2 *>(ww + head), *o2 = reinterpret_cast<double2 *>(wo + head);
  double2 *x2 = reinterpret_cast<double2 *>(xx + head), *z2 = reinterpret_cast<double2 *>(zz + head);
  const double2 *n2 = reinterpret_cast<const double2 *>(zn + head);
  for (int64_t i = t0; i < pairs; i += ts) {
    const double2 wi = w2[i], oi = o2[i], zi = z2[i], xi = x2[i], ni = n2[i];
    double2 no, nw, nx, nz;
    step(wi.x, oi.x, zi.x, xi.x, ni.x, no.x, nw.x, nx.x, nz.x);
    step(wi.y, oi.y, zi.y, xi.y, ni.y, no.y, nw.y, nx.y, nz.y);
    o2[i] = no;
    if (!ROT) w2[i] = nw;
    x2[i] = nx;
    z2[i] = nz;
    if (zd) {
      const float2 a = f64_split(nz.x), b = f64_split(nz.y);
      reinterpret_cast<float4 *>(zd + head)[i] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  if (((n - head) & 1) && t0 == 0) {
    step(ww[n - 1], wo[n - 1], zz[n - 1], xx[n - 1], zn[n - 1], wo[n - 1], ww[n - 1], xx[n - 1], zz[n - 1]);
    if (zd) zd[n - 1] = f64_split(zz[n - 1]);
  }
}

void launch_minres_update(double *w_old, double *w, double *x, double *z, const double *z_new,
                          MinresState *st, int64_t n, int64_t stride, int nrhs, int *done, cudaStream_t s,
                          float2 *z_df, bool rotate) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  if (rotate)
    k_minres_update<true><<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(w_old, w, x, z, z_new, st, n, stride, done,
                                                                     z_df);
  else
    k_minres_update<false><<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(w_old, w, x, z, z_new, st, n, stride, done,
                                                                      z_df);
}

__global__ void k_minres_commit(MinresState *st, int *done, int nrhs) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs && !done[j] && st[j].stop) done[j] = 1;
}

void launch_minres_commit(MinresState *st, int *done, int nrhs, cudaStream_t s) {
  count_launch(1);
  k_minres_commit<<<(nrhs + 63) / 64, 64, 0, s>>>(st, done, nrhs);
}

// Restart vectors of the right-hand sides with done[j] == 0: v = b - Ax (Ax
// precomputed), v_old = w = w_old = 0.
__global__ void k_restart_vectors(const double *b, const double *Ax, double *v, double *v_old, double *w,
                                  double *w_old, int64_t n, int64_t stride, const int *done) {
  const int j = blockIdx.y;
  if (done[j]) return;
  const int64_t o = j * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    v[o + i] = b[o + i] - Ax[o + i];
    v_old[o + i] = 0.0;
    w[o + i] = 0.0;
    w_old[o + i] = 0.0;
  }
}

void launch_restart_vectors(const double *b, const double *Ax, double *v, double *v_old, double *w, double *w_old,
                            int64_t n, int64_t stride, int nrhs, const int *done, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_restart_vectors<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(b, Ax, v, v_old, w, w_old, n, stride, done);
}

// ------------------------------------------------------------------ GMRES basis operations
// Basis vector k of right-hand side r at V + k * vstride + r * stride; rows are
// skipped where skip[r] != 0. Reductions run in a fixed order (per-block
// partial sums, then the blocks in index order): results do not depend on timing.

constexpr int kDotChunk = 8;       // basis vectors per dot launch
constexpr int kDotBlocks = 304;    // 2 blocks per SM

__global__ void __launch_bounds__(256) k_mdot_part(const double *V, int64_t vstride, int kc, const double *w,
                                                   int64_t n, int64_t stride, double *part, const int *skip) {
  const int r = blockIdx.y;
  if (skip && skip[r]) return;
  const double *wr = w + r * stride;
  const double *vr = V + r * stride;
  double acc[kDotChunk];
#pragma unroll
  for (int k = 0; k < kDotChunk; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = wr[i];
#pragma unroll
    for (int k = 0; k < kDotChunk; ++k)
      if (k < kc) acc[k] = fma(vr[k * vstride + i], wi, acc[k]);
  }
  __shared__ double ws[kDotChunk][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDotChunk; ++k) {
    const double t = warp_sum(acc[k]);
    if (lane == 0) ws[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < kc) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += ws[threadIdx.x][q];
    part[((int64_t)r * kDotChunk + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_mdot_final(const double *part, int nblk, int kc, double *out, int ldo, int k0, int nrhs,
                             const int *skip) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = t / kDotChunk, k = t % kDotChunk;
  if (r >= nrhs || k >= kc || (skip && skip[r])) return;
  const double *pp = part + ((int64_t)r * kDotChunk + k) * nblk;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += pp[b];
  out[(int64_t)r * ldo + k0 + k] = s;
}

void launch_basis_dots(const double *V, int64_t vstride, int k0, int kc, const double *w, int64_t n,
                       int64_t stride, int nrhs, double *part, double *out, int ldo, const int *skip,
                       cudaStream_t s) {
  for (int k = 0; k < kc; k += kDotChunk) {
    const int c = kc - k < kDotChunk ? kc - k : kDotChunk;
    count_launch(2);
    k_mdot_part<<<dim3(kDotBlocks, nrhs), 256, 0, s>>>(V + (int64_t)(k0 + k) * vstride, vstride, c, w, n,
                                                       stride, part, skip);
    k_mdot_final<<<(nrhs * kDotChunk + 127) / 128, 128, 0, s>>>(part, kDotBlocks, c, out, ldo, k0 + k, nrhs, skip);
  }
}

// w_r += sign * sum_{k < kc} c[r * ldc + k] * V_k (one pass over the kc vectors and w)
__global__ void k_basis_axpy(const double *V, int64_t vstride, int kc, const double *c, int ldc, double sign,
                             double *w, int64_t n, int64_t stride, const int *skip) {
  const int r = blockIdx.y;
  if (skip && skip[r]) return;
  __shared__ double cs[256];
  for (int k = threadIdx.x; k < kc; k += blockDim.x) cs[k] = sign * c[(int64_t)r * ldc + k];
  __syncthreads();
  double *wr = w + r * stride;
  const double *vr = V + r * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = wr[i];
    for (int k = 0; k < kc; ++k) a = fma(cs[k], vr[k * vstride + i], a);
    wr[i] = a;
  }
}

void launch_basis_axpy(const double *V, int64_t vstride, int kc, const double *c, int ldc, double sign, double *w,
                       int64_t n, int64_t stride, int nrhs, const int *skip, cudaStream_t s) {
  if (kc <= 0) return;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_basis_axpy<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(V, vstride, kc, c, ldc, sign, w, n, stride, skip);
}

// dst_r = src_r / sqrt(nrm2[r]) (0 where the norm is 0)
__global__ void k_scale_by_norm(const double *src, double *dst, const double *nrm2, int64_t n, int64_t stride,
                                const int *skip) {
  const int r = blockIdx.y;
  if (skip && skip[r]) return;
  const double q = nrm2[r] > 0.0 ? 1.0 / sqrt(nrm2[r]) : 0.0;
  const double *a = src + r * stride;
  double *b = dst + r * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i] * q;
}

void launch_scale_by_norm(const double *src, double *dst, const double *nrm2, int64_t n, int64_t stride, int nrhs,
                          const int *skip, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  count_launch(1);
  k_scale_by_norm<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(src, dst, nrm2, n, stride, skip);
}

}  // namespace fdst

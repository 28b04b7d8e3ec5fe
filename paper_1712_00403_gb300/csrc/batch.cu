// Batched FD-preconditioned MINRES on many independent Stokes problems of
// uneven sizes (one right-hand side each). Every phase of an iteration is one
// grouped launch over all problems, driven by device tables built once:
//   * FD apply: for each contraction step, one tensor-core (or FP64) launch
//     whose problem table holds every problem's chains (Algorithm 1 steps 2-4);
//   * Stokes matvec: the problems' banded-Kronecker plans merged stage by
//     stage into rounds of ops with distinct outputs and one band width (one
//     launch per round); in double-float the update writes the FP32 pairs of
//     the next z and the last product into each result block writes FP64, so
//     no split or join pass runs;
//   * MINRES vector updates and inner products: one launch per operation over
//     a table of per-problem segments.
// Pointers never change between iterations (in-place Lanczos/direction
// shifts), so one iteration is captured into a CUDA graph and replayed. An
// autotuner times, per contraction step, how the tensor-core kernel is fed (B
// streamed with A at each ring depth, B resident in shared memory, A's TF32
// pieces in tensor memory) and the banded-kernel block size on the batch's own
// shapes and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "batch.h"
#include "ctx.h"
#include "fp_bits.cuh"

namespace fdst {

enum { kB = 0, kX, kV, kVOld, kZ, kZNew, kAz, kW, kWOld, kNVec };

struct BatchSeg {
  double *vec[kNVec];
  float2 *x2, *y2;
  MinresState *st;
  int *done;
  double *partials, *dots;   // dots: [0] residual/g, [1] delta, [2] g2, [3] |b|^2
  unsigned *counter;
  int64_t n;
};

namespace {
constexpr int kDotBlocks = 128;

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

__global__ void __launch_bounds__(256) k_bdot(const BatchSeg *segs, int ia, int ib, int slot) {
  const BatchSeg &S = segs[blockIdx.y];
  if (*S.done) return;
  const double *x = S.vec[ia], *y = S.vec[ib];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  __shared__ double ws[8];
  __shared__ bool last;
  s = bwarp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    S.partials[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(S.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    const volatile double *pp = S.partials;
    double t = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += 32) t += pp[i];
    t = bwarp_sum(t);
    if (threadIdx.x == 0) {
      S.dots[slot] = t;
      *S.counter = 0u;
    }
  }
}

__global__ void k_blanczos(const BatchSeg *segs) {
  const BatchSeg &S = segs[blockIdx.y];
  if (*S.done) return;
  const double gamma = S.st->gamma, gamma_old = S.st->gamma_old;
  const double f1 = S.dots[1] / gamma, f2 = gamma / gamma_old;
  const double *a = S.vec[kAz];
  double *v = S.vec[kV], *vo = S.vec[kVOld];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = v[i];
    const double t = a[i] - f1 * vi - f2 * vo[i];
    vo[i] = vi;
    v[i] = t;
  }
}

// Givens QR update of each problem's MINRES recurrence (same recurrence as
// k_minres_scalars, one thread per problem).
__global__ void k_bscalars(const BatchSeg *segs, int n, int maxit, int *n_stopped) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const BatchSeg &B = segs[j];
  if (*B.done) return;
  MinresState S = *B.st;
  const double d = B.dots[1], g2 = B.dots[2];
  S.iters += 1;
  if (isnan(d) || isinf(d) || isnan(g2) || isinf(g2)) {
    S.status = 9;
    S.stop = 1;
    S.inv_a1 = S.a2 = S.a3 = S.coef_x = S.inv_gamma_new = 0.0;
    *B.st = S;
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
  *B.st = S;
}

// with df, also the FP32 pairs of the new z (the next matvec's input) into x2
__global__ void k_bupdate(const BatchSeg *segs, int df) {
  const BatchSeg &B = segs[blockIdx.y];
  if (*B.done) return;
  const MinresState &S = *B.st;
  const double ia1 = S.inv_a1, a2 = S.a2, a3 = S.a3, cx = S.coef_x, ig = S.inv_gamma_new;
  double *wo = B.vec[kWOld], *w = B.vec[kW], *x = B.vec[kX], *z = B.vec[kZ];
  const double *zn = B.vec[kZNew];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    const double wn = (z[i] - a3 * wo[i] - a2 * wi) * ia1;
    wo[i] = wi;
    w[i] = wn;
    x[i] = fma(cx, wn, x[i]);
    const double znew = zn[i] * ig;
    z[i] = znew;
    if (df) B.x2[i] = f64_split(znew);
  }
}

__global__ void k_bcommit(const BatchSeg *segs, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && !*segs[j].done && segs[j].st->stop) *segs[j].done = 1;
}

__global__ void k_bjoin(const BatchSeg *segs, int dst) {
  const BatchSeg &B = segs[blockIdx.y];
  if (*B.done) return;
  double *y = B.vec[dst];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x) {
    y[i] = f64_join(B.y2[i]);
  }
}

}  // namespace fdst

using namespace fdst;

struct fdst_batch_ctx {
  std::vector<fdst_ctx *> hs;
  int n = 0;
  bool tc = false, df = false;
  bool join = false;   // double-float results joined by a pass of their own (else by the last products)
  std::vector<BatchSeg> hsegs;
  BatchSeg *segs = nullptr;
  int *n_stopped = nullptr, *h_n_stopped = nullptr;
  struct Step {
    void *tab = nullptr;
    int count = 0, maxR = 0, maxN = 0;
    int bmax = 0;            // largest resident-B image among the step's problems
    int mode = 1, ring = 0;  // feeding mode (TcGroup::mode; B streamed unless the autotuner picked
                             // another) and ring depth (0: as many stages as fit)
  };
  std::vector<Step> steps;
  struct Round {
    void *tab = nullptr;
    int count = 0;
    int64_t maxt = 0;
    int w = 0;               // band width shared by the round's ops (double-float rounds)
  };
  std::vector<Round> rounds;
  int ring = 0, threads = 256;
  double ms_apply = 0.0, ms_matvec = 0.0;
  int64_t maxn = 0;
  std::vector<void *> allocs;
  cudaStream_t bs = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_maxit = -1;
  bool use_graph = true;
};

namespace fdst {

static fdst_status balloc(fdst_batch b, void **p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    set_error("batch: cudaMalloc failed");
    return FDST_OUT_OF_MEMORY;
  }
  b->allocs.push_back(*p);
  return FDST_OK;
}

template <typename T>
static fdst_status bupload(fdst_batch b, T **p, const std::vector<T> &v) {
  TRY(balloc(b, (void **)p, sizeof(T) * std::max<size_t>(1, v.size())));
  if (!v.empty() && cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("batch: table upload failed");
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
}

static dim3 seg_grid(const fdst_batch b) {
  int64_t blocks = (b->maxn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  return dim3((unsigned)blocks, (unsigned)b->n);
}

static TcGroup step_group(fdst_batch b, const fdst_batch_ctx::Step &S, int mode) {
  TcGroup g;
  g.split = b->hs[0]->desc.fd_precision == FDST_FD_BF16X6 ? 1 : 0;
  g.table = static_cast<const TcProb *>(S.tab);
  g.nprob = S.count;
  g.maxR = S.maxR;
  g.maxN = S.maxN;
  g.bmax = S.bmax;
  g.mode = mode;
  g.convert = &S == &b->steps[0];
  return g;
}

static fdst_status batch_step_apply(fdst_batch b, const fdst_batch_ctx::Step &S, cudaStream_t st, int mode, int ring) {
  return launch_gemm_tc(step_group(b, S, mode), 1, nullptr, st, ring);
}

// ring < 0: each step's own autotuned mode and ring depth.
static fdst_status batch_apply(fdst_batch b, cudaStream_t st, int ring) {
  for (auto &S : b->steps) {
    if (S.count == 0) continue;
    if (b->tc) {
      TRY(ring < 0 ? batch_step_apply(b, S, st, S.mode, S.ring) : batch_step_apply(b, S, st, 1, ring));
    } else {
      GemmGroup g;
      g.table = static_cast<const GemmProb *>(S.tab);
      g.nprob = S.count;
      g.maxR = S.maxR;
      g.maxN = S.maxN;
      launch_gemm_f64(g, 1, nullptr, st);
    }
  }
  return FDST_OK;
}

static void batch_matvec(fdst_batch b, cudaStream_t st, int threads) {
  const dim3 sg = seg_grid(b);
  // (double-float: x2 holds the pairs of z, written by member_init, the update and restarts)
  for (auto &R : b->rounds) {
    if (b->df) {
      BandGroupDF g;
      g.table = static_cast<const BandOpDF *>(R.tab);
      g.nop = R.count;
      g.maxt = R.maxt;
      g.threads = threads;
      g.w = R.w;
      g.row_pairs = 0;   // many small products per launch: one band row per warp
      launch_band_df(g, 1, nullptr, st);
    } else {
      BandGroup g;
      g.table = static_cast<const BandOp *>(R.tab);
      g.nop = R.count;
      g.maxt = R.maxt;
      g.threads = threads;
      launch_band(g, 1, nullptr, st);
    }
  }
  if (b->join) {
    count_launch(1);
    k_bjoin<<<sg, 256, 0, st>>>(b->segs, kAz);
  }
}

static fdst_status batch_iterate(fdst_batch b, int maxit, cudaStream_t st) {
  const dim3 sg = seg_grid(b);
  const dim3 dg(kDotBlocks, b->n);
  const int tb = (b->n + 63) / 64;
  batch_matvec(b, st, b->threads);
  count_launch(4);
  k_bdot<<<dg, 256, 0, st>>>(b->segs, kAz, kZ, 1);
  k_blanczos<<<sg, 256, 0, st>>>(b->segs);
  TRY(batch_apply(b, st, -1));
  k_bdot<<<dg, 256, 0, st>>>(b->segs, kV, kZNew, 2);
  k_bscalars<<<tb, 64, 0, st>>>(b->segs, b->n, maxit, b->n_stopped);
  count_launch(2);
  k_bupdate<<<sg, 256, 0, st>>>(b->segs, b->df ? 1 : 0);
  k_bcommit<<<tb, 64, 0, st>>>(b->segs, b->n);
  return FDST_OK;
}

// Times candidate tensor-core ring depths and banded-kernel block sizes on the
// batch's own tables and keeps the fastest of each: per contraction step the
// feeding mode of B and A and the ring depth, and the banded block size.
static fdst_status batch_autotune(fdst_batch b) {
  cudaStream_t st = b->bs;
  for (auto *h : b->hs) {
    CK(cudaMemsetAsync(h->done, 0, sizeof(int), st));
    CK(cudaMemsetAsync(h->v, 0, sizeof(double) * h->n_total, st));
    CK(cudaMemsetAsync(h->z, 0, sizeof(double) * h->n_total, st));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto &&fn) -> float {
    fn();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r) fn();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 2.0f;
  };
  if (b->tc) {
    // per contraction step: B streamed with A at each ring depth that fits, B resident
    // with A in shared memory, B resident with A's TF32 pieces in tensor memory; a
    // mode that does not fit the step's shapes is skipped
    double total = 0.0;
    int ring_min = 4;
    for (auto &S : b->steps) {
      if (S.count == 0) continue;
      const TcGroup g0 = step_group(b, S, 1);
      float best = 1e30f;
      auto consider = [&](int mode, int ring) {
        if (tc_mode_fits(step_group(b, S, mode), ring) != FDST_OK) return;
        const float ms = timed([&] { batch_step_apply(b, S, st, mode, ring); });
        if (ms < best) { best = ms; S.mode = mode; S.ring = ring; }
      };
      for (int ring = 2; ring <= tc_max_ring(g0); ++ring) consider(1, ring);
      consider(2, 0);
      consider(3, 0);
      total += best;
      if (S.mode == 1) ring_min = std::min(ring_min, S.ring);
    }
    b->ring = ring_min;
    b->ms_apply = total;
  } else {
    b->ms_apply = timed([&] { batch_apply(b, st, 0); });
  }
  float best = 1e30f;
  for (int thr : {128, 256}) {
    float ms = timed([&] { batch_matvec(b, st, thr); });
    if (ms < best) { best = ms; b->threads = thr; }
  }
  b->ms_matvec = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  return FDST_OK;
}

static fdst_status build_batch(fdst_batch b) {
  const int n = b->n;
  // ---- segments (rhs 0 of every handle; b and x live in the handle's host-call buffers)
  b->hsegs.resize(n);
  for (int i = 0; i < n; ++i) {
    fdst_ctx *h = b->hs[i];
    if (!h->hb) {
      TRY(dalloc(h, &h->hb, (size_t)h->n_total * h->max_rhs));
      TRY(dalloc(h, &h->hx, (size_t)h->n_total * h->max_rhs));
    }
    BatchSeg &S = b->hsegs[i];
    S.vec[kB] = h->hb;
    S.vec[kX] = h->hx;
    S.vec[kV] = h->v;
    S.vec[kVOld] = h->v_old;
    S.vec[kZ] = h->z;
    S.vec[kZNew] = h->z_new;
    S.vec[kAz] = h->Az;
    S.vec[kW] = h->w;
    S.vec[kWOld] = h->w_old;
    S.x2 = h->x2;
    S.y2 = h->y2;
    S.st = h->state;
    S.done = h->done;
    S.partials = h->partials;
    S.dots = h->dots;
    S.counter = h->counters;
    S.n = h->n_total;
    b->maxn = std::max(b->maxn, h->n_total);
  }
  TRY(bupload(b, &b->segs, b->hsegs));
  // ---- FD step tables
  int maxsteps = 0;
  for (auto *h : b->hs)
    for (auto &c : h->chains) maxsteps = std::max(maxsteps, c.nsteps);
  b->steps.assign(maxsteps, fdst_batch_ctx::Step());
  for (int j = 0; j < maxsteps; ++j) {
    std::vector<TcProb> tcp;
    std::vector<GemmProb> gp;
    auto &S = b->steps[j];
    for (auto *h : b->hs)
      for (size_t ci = 0; ci < h->chains.size(); ++ci) {
        const FdChain &c = h->chains[ci];
        if (j >= c.nsteps) continue;
        const bool first = j == 0, last = j == c.nsteps - 1;
        const TcLayout L = tc_layout(c.R[j], c.K[j], c.K[(j + 1) % c.nsteps], last);
        S.maxR = std::max(S.maxR, c.R[j]);
        S.maxN = std::max(S.maxN, c.N[j]);
        if (b->tc) {
          TcProb P;
          if (first) { P.A64 = h->v + c.off; P.a64_rhs_stride = h->n_total; }
          P.A32 = h->work_f[(j + 1) % 2] + h->f_off[ci];
          P.a_rhs_stride = h->f_total;
          P.lda = L.lda;
          P.tmap = h->tmaps + 128 * (ci * h->tmap_steps + j);
          P.out_nv = c.K[(j + 1) % c.nsteps];
          P.ldv = L.ldv;
          P.c_cs = L.c_cs;
          if (last) P.C64 = h->z_new + c.off;
          else P.C32 = h->work_f[j % 2] + h->f_off[ci];
          P.Bt = c.Bt[j];
          P.R = c.R[j]; P.K = c.K[j]; P.N = c.N[j];
          if (j == c.div_step) { P.lam_row = c.lam_row_f; P.lam_col = c.lam_col_f; }
          P.scale_in = first ? c.scale : nullptr;
          P.scale_out = last ? c.scale : nullptr;
          P.done_flag = h->done;
          S.bmax = std::max(S.bmax, tc_b_tile_bytes(P.K, P.N, h->desc.fd_precision == FDST_FD_BF16X6 ? 1 : 0));
          tcp.push_back(P);
        } else {
          GemmProb P;
          P.A = first ? h->v + c.off : h->work[(j - 1) % 2] + c.off;
          P.C = last ? h->z_new + c.off : h->work[j % 2] + c.off;
          P.B = c.B[j];
          P.R = c.R[j]; P.K = c.K[j]; P.N = c.N[j];
          if (j == c.div_step) { P.lam_row = c.lam_row; P.lam_col = c.lam_col; }
          P.scale_in = first ? c.scale : nullptr;
          P.scale_out = last ? c.scale : nullptr;
          P.done_flag = h->done;
          gp.push_back(P);
        }
      }
    if (b->tc) {
      S.count = (int)tcp.size();
      TcProb *d = nullptr;
      TRY(bupload(b, &d, tcp));
      S.tab = d;
    } else {
      S.count = (int)gp.size();
      GemmProb *d = nullptr;
      TRY(bupload(b, &d, gp));
      S.tab = d;
    }
  }
  // ---- matvec rounds: (stage, k-th op on the same output) merged across problems
  // keyed by (stage, k-th op on the same output, band width): a double-float launch
  // then shares one width and runs the kernel's fully unrolled instantiation
  std::map<std::tuple<int, int, int>, std::vector<BandOpDF>> rdf;
  std::map<std::tuple<int, int, int>, std::vector<BandOp>> rf;
  std::map<std::tuple<int, int, int>, int64_t> rmax;
  // double-float: the last product into each result block writes Az in FP64 itself
  // (when every problem's plan writes all of its blocks), so no join pass runs
  bool all_joined = b->df;
  for (auto *h : b->hs) {
    std::map<int, int> blocks;
    for (const PlanOp &op : h->plan_df)
      if (op.out_kind == 3) blocks[op.out_id] = 1;
    if ((int)blocks.size() != h->dim + 1) all_joined = false;
  }
  b->join = b->df && !all_joined;
  for (auto *h : b->hs) {
    std::map<std::tuple<int, int, int>, int> seen;   // (stage, out_kind, out_id) -> ops so far
    const auto &plan = b->df ? h->plan_df : h->plan;
    std::map<int, size_t> last;
    for (size_t k = 0; k < plan.size(); ++k)
      if (plan[k].out_kind == 3) last[plan[k].out_id] = k;
    for (size_t opi = 0; opi < plan.size(); ++opi) {
      const PlanOp &op = plan[opi];
      const int round = seen[std::make_tuple(op.stage, op.out_kind, op.out_id)]++;
      const auto key = std::make_tuple(op.stage, round, b->df ? h->bands[op.band].w : 0);
      const BandDev &bd = h->bands[op.band];
      int od[3] = {op.dims[0], op.dims[1], op.dims[2]};
      od[op.mode] = bd.rows;
      rmax[key] = std::max(rmax[key], (int64_t)od[0] * od[1] * od[2]);
      if (b->df) {
        BandOpDF o;
        o.vals = op.vals_df; o.lo = bd.lo; o.w = bd.w; o.rows = bd.rows;
        o.d0 = op.dims[0]; o.d1 = op.dims[1]; o.d2 = op.dims[2]; o.mode = op.mode;
        o.accumulate = op.accumulate;
        o.swap = op.swap;
        if (op.in_kind == 0) o.X = h->x2 + h->off[op.in_id];
        else if (op.in_kind == 1) o.X = reinterpret_cast<const float2 *>(h->t1[op.in_id]);
        else o.X = reinterpret_cast<const float2 *>(h->g[op.in_id]);
        if (op.out_kind == 3) {
          o.Y = h->y2 + h->off[op.out_id];
          if (all_joined && last[op.out_id] == opi) o.Y64 = h->Az + h->off[op.out_id];
        }
        else if (op.out_kind == 1) o.Y = reinterpret_cast<float2 *>(h->t1[op.out_id]);
        else o.Y = reinterpret_cast<float2 *>(h->g[op.out_id]);
        o.done_flag = h->done;
        rdf[key].push_back(o);
      } else {
        BandOp o;
        o.vals = bd.vals; o.lo = bd.lo; o.w = bd.w; o.rows = bd.rows;
        o.d0 = op.dims[0]; o.d1 = op.dims[1]; o.d2 = op.dims[2]; o.mode = op.mode;
        o.coef = op.coef;
        o.accumulate = op.accumulate;
        if (op.in_kind == 0) o.X = h->z + h->off[op.in_id];
        else if (op.in_kind == 1) o.X = h->t1[op.in_id];
        else o.X = h->g[op.in_id];
        if (op.out_kind == 3) o.Y = h->Az + h->off[op.out_id];
        else if (op.out_kind == 1) o.Y = h->t1[op.out_id];
        else o.Y = h->g[op.out_id];
        o.done_flag = h->done;
        rf[key].push_back(o);
      }
    }
  }
  for (auto &kv : rmax) {
    fdst_batch_ctx::Round R;
    R.maxt = kv.second;
    R.w = std::get<2>(kv.first);
    if (b->df) {
      auto &v = rdf[kv.first];
      R.count = (int)v.size();
      BandOpDF *d = nullptr;
      TRY(bupload(b, &d, v));
      R.tab = d;
    } else {
      auto &v = rf[kv.first];
      R.count = (int)v.size();
      BandOp *d = nullptr;
      TRY(bupload(b, &d, v));
      R.tab = d;
    }
    if (R.count > 65535) {
      set_error("batch: too many matvec ops in one round");
      return FDST_NOT_SUPPORTED;
    }
    b->rounds.push_back(R);
  }
  TRY(balloc(b, (void **)&b->n_stopped, sizeof(int)));
  if (cudaMallocHost((void **)&b->h_n_stopped, sizeof(int)) != cudaSuccess) {
    set_error("batch: pinned allocation failed");
    return FDST_CUDA_ERROR;
  }
  return FDST_OK;
}

// Start of one member's MINRES (right-hand side 0 of its handle, b and x in
// the handle's hb / hx): v = b - A x0 (v = b when x0 = 0), z = P^{-1} v / gamma_1,
// |b|^2 in dots[3].
fdst_status member_init(fdst_ctx *h, int *n_stopped, double tol, cudaStream_t st, bool x0_zero) {
  const int64_t m = h->n_total;
  CK(cudaMemsetAsync(h->done, 0, sizeof(int), st));
  launch_axpby(h->hb, h->v, 1.0, 0.0, m, m, 1, st);
  if (!x0_zero) {
    TRY(run_matvec(h, h->hx, h->Az, 1, nullptr, st, true));
    launch_axpby(h->Az, h->v, -1.0, 1.0, m, m, 1, st);
  }
  CK(cudaMemsetAsync(h->v_old, 0, sizeof(double) * m, st));
  CK(cudaMemsetAsync(h->w, 0, sizeof(double) * m, st));
  CK(cudaMemsetAsync(h->w_old, 0, sizeof(double) * m, st));
  TRY(run_apply(h, h->v, h->z, 1, nullptr, st));
  launch_dot(h->v, h->z, m, m, 1, h->partials, h->counters, h->dots, nullptr, st);
  launch_minres_init(h->state, h->dots, h->done, 1, n_stopped, tol, st);
  launch_scale_by_inv_gamma(h->z, h->state, m, m, 1, h->done, st);
  launch_dot(h->hb, h->hb, m, m, 1, h->partials, h->counters, h->dots + 3, nullptr, st);
  member_split_z(h, st);
  return FDST_OK;
}

// Double-float batches read the FP32 pairs of z (x2); the update keeps them current,
// and this writes them after the member's z was set anew (start, restart).
void member_split_z(fdst_ctx *h, cudaStream_t st) {
  if (h->desc.matvec_precision == FDST_MV_DF64 && h->x2)
    launch_split_df(h->z, h->x2, h->n_total, h->n_total, 1, nullptr, st);
}

// Enqueues ||b - A x||^2 (FP64 matvec) into dots[0]; the caller syncs and divides by dots[3].
fdst_status member_residual(fdst_ctx *h, cudaStream_t st) {
  const int64_t m = h->n_total;
  TRY(run_matvec(h, h->hx, h->Az, 1, nullptr, st, true));
  launch_axpby(h->hb, h->Az, 1.0, -1.0, m, m, 1, st);
  launch_dot(h->Az, h->Az, m, m, 1, h->partials, h->counters, h->dots, nullptr, st);
  return FDST_OK;
}

fdst_status batch_step(fdst_batch b, int maxit, cudaStream_t st) { return batch_iterate(b, maxit, st); }

fdst_status batch_new(const std::vector<fdst_ctx *> &hs, int ring, int threads, fdst_batch *out) {
  *out = nullptr;
  fdst_batch b = new fdst_batch_ctx();
  b->n = (int)hs.size();
  b->hs = hs;
  b->tc = hs[0]->desc.fd_precision != FDST_FD_F64;
  b->df = hs[0]->desc.matvec_precision == FDST_MV_DF64;
  b->use_graph = false;
  b->ring = ring;
  b->threads = threads;
  fdst_status st = build_batch(b);
  if (st != FDST_OK) {
    for (void *p : b->allocs) cudaFree(p);
    if (b->h_n_stopped) cudaFreeHost(b->h_n_stopped);
    delete b;
    return st;
  }
  for (auto &S : b->steps) S.ring = ring;
  *out = b;
  return FDST_OK;
}

int *batch_stop_counter(fdst_batch b) { return b->n_stopped; }

}  // namespace fdst

extern "C" {

fdst_status fdst_batch_destroy(fdst_batch b) {
  if (!b) return FDST_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->allocs) cudaFree(p);
  if (b->h_n_stopped) cudaFreeHost(b->h_n_stopped);
  if (b->bs) cudaStreamDestroy(b->bs);
  delete b;
  return FDST_OK;
}

fdst_status fdst_batch_create(const fdst_handle *handles, int n, int autotune, fdst_batch *out) {
  if (!out || !handles || n < 1) {
    set_error("fdst_batch_create: NULL argument or n < 1");
    return FDST_INVALID_ARGUMENT;
  }
  *out = nullptr;
  fdst_batch b = new fdst_batch_ctx();
  b->n = n;
  for (int i = 0; i < n; ++i) {
    fdst_ctx *h = handles[i];
    if (!h) { fdst_batch_destroy(b); set_error("fdst_batch_create: NULL handle"); return FDST_INVALID_ARGUMENT; }
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) {
        fdst_batch_destroy(b);
        set_error("fdst_batch_create: a handle appears twice");
        return FDST_INVALID_ARGUMENT;
      }
    const bool tc = h->desc.fd_precision != FDST_FD_F64, df = h->desc.matvec_precision == FDST_MV_DF64;
    if (h->mapped) { fdst_batch_destroy(b); set_error("fdst_batch_create: identity-geometry handles only"); return FDST_NOT_SUPPORTED; }
    if (i == 0) { b->tc = tc; b->df = df; }
    if (tc != b->tc || df != b->df || h->desc.fd_precision != handles[0]->desc.fd_precision) {
      fdst_batch_destroy(b);
      set_error("fdst_batch_create: all handles must share the FD and matvec precision");
      return FDST_INVALID_ARGUMENT;
    }
    b->hs.push_back(h);
  }
  if (cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess) {
    fdst_batch_destroy(b);
    set_error("fdst_batch_create: stream creation failed");
    return FDST_CUDA_ERROR;
  }
  fdst_status st = build_batch(b);
  if (st == FDST_OK && autotune) st = batch_autotune(b);
  if (st != FDST_OK) { fdst_batch_destroy(b); return st; }
  *out = b;
  return FDST_OK;
}

fdst_status fdst_batch_info(fdst_batch b, int *ring, int *threads, double *ms_apply, double *ms_matvec) {
  if (!b) { set_error("NULL batch"); return FDST_INVALID_ARGUMENT; }
  if (ring) *ring = b->ring;
  if (threads) *threads = b->threads;
  if (ms_apply) *ms_apply = b->ms_apply;
  if (ms_matvec) *ms_matvec = b->ms_matvec;
  return FDST_OK;
}

fdst_status fdst_batch_tuning(fdst_batch b, int cap, int *nsteps, int *modes, int *rings) {
  if (!b || !nsteps) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (cap < 0 || (cap > 0 && (!modes || !rings))) { set_error("cap must be >= 0 with modes and rings given"); return FDST_INVALID_ARGUMENT; }
  *nsteps = (int)b->steps.size();
  for (int i = 0; i < *nsteps && i < cap; ++i) {
    modes[i] = b->tc ? b->steps[i].mode : 0;
    rings[i] = b->tc ? b->steps[i].ring : 0;
  }
  return FDST_OK;
}

fdst_status fdst_batch_set_tuning(fdst_batch b, int n, const int *modes, const int *rings) {
  if (!b || !modes || !rings) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (!b->tc) { set_error("fdst_batch_set_tuning: FP64 batches have no tensor-core launches"); return FDST_NOT_SUPPORTED; }
  if (n != (int)b->steps.size()) { set_error("fdst_batch_set_tuning: n must equal the number of steps"); return FDST_INVALID_ARGUMENT; }
  for (int i = 0; i < n; ++i) {
    if (modes[i] < 1 || modes[i] > 3 || rings[i] < 0) {
      set_error("fdst_batch_set_tuning: modes in {1, 2, 3}, rings >= 0");
      return FDST_INVALID_ARGUMENT;
    }
    const auto &S = b->steps[i];
    if (S.count > 0) TRY(tc_mode_fits(step_group(b, S, modes[i]), rings[i]));
  }
  for (int i = 0; i < n; ++i) {
    b->steps[i].mode = modes[i];
    b->steps[i].ring = rings[i];
  }
  if (b->graph) {   // the captured iteration holds the old launches
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_maxit = -1;
  }
  return FDST_OK;
}

fdst_status fdst_batch_solve(fdst_batch b, const double *const *d_b, double *const *d_x, double tol, int maxit,
                             fdst_solve_info *info, fdst_stream stream) {
  if (!b || !d_b || !d_x || !info) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (!(tol >= 0.0) || maxit < 1) { set_error("tol must be >= 0 and maxit >= 1"); return FDST_INVALID_ARGUMENT; }
  cudaStream_t us = (cudaStream_t)stream, st = b->bs;
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, us));
  CK(cudaStreamWaitEvent(st, ev, 0));
  const int n = b->n;
  // ---- per-problem start: v = b - A x0, z = P^{-1} v, gamma_1, |b|^2 (x0 = 0, found on
  // the device in one pass over all members, spares the FP64 matvec)
  CK(cudaMemsetAsync(b->n_stopped, 0, sizeof(int), st));
  std::vector<int> nz(n, 1);
  for (int i = 0; i < n; ++i) {
    fdst_ctx *h = b->hs[i];
    const int64_t m = h->n_total;
    CK(cudaMemcpyAsync(h->hb, d_b[i], sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->hx, d_x[i], sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    launch_any_nonzero(h->hx, m, h->n_stopped, st);
    CK(cudaMemcpyAsync(&nz[i], h->n_stopped, sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) TRY(member_init(b->hs[i], b->n_stopped, tol, st, nz[i] == 0));
  std::vector<double> bb(n), true_rel(n, -1.0);
  for (int i = 0; i < n; ++i) CK(cudaMemcpyAsync(&bb[i], b->hs[i]->dots + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  auto true_residuals = [&]() -> fdst_status {
    std::vector<double> rr(n);
    for (int i = 0; i < n; ++i) {
      TRY(member_residual(b->hs[i], st));
      CK(cudaMemcpyAsync(&rr[i], b->hs[i]->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) true_rel[i] = bb[i] > 0 ? std::sqrt(rr[i] / bb[i]) : std::sqrt(rr[i]);
    return FDST_OK;
  };
  if (b->graph && b->graph_maxit != maxit) {   // maxit is baked into the captured iteration
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  std::vector<MinresState> hs(n);
  std::vector<double> prev_true(n, -1.0);
  std::vector<int> restarts(n, 0), est_iters(n, -1);
  int it = 0;
  bool residuals_current = false;
  const int check_every = 4;
  while (it < maxit) {
    residuals_current = false;
    if (b->use_graph && b->graph && it > 0) {
      CK(cudaGraphLaunch(b->graph, st));
    } else {
      TRY(batch_iterate(b, maxit, st));
      if (b->use_graph && !b->graph && it == 0) {
        // capture one iteration (all launches; pointers are fixed) for the following ones
        cudaGraph_t gph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        fdst_status cs = batch_iterate(b, maxit, st);
        cudaError_t ce = cudaStreamEndCapture(st, &gph);
        if (cs != FDST_OK || ce != cudaSuccess) { set_error("batch: graph capture failed"); return FDST_CUDA_ERROR; }
        CK(cudaGraphInstantiate(&b->graph, gph, 0));
        cudaGraphDestroy(gph);
        b->graph_maxit = maxit;
      }
    }
    ++it;
    if (it % check_every == 0 || it == maxit) {
      CK(cudaMemcpyAsync(b->h_n_stopped, b->n_stopped, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*b->h_n_stopped >= n) {
        TRY(true_residuals());
        residuals_current = true;
        int running = 0;
        for (int i = 0; i < n; ++i) {
          fdst_ctx *h = b->hs[i];
          CK(cudaMemcpy(&hs[i], h->state, sizeof(MinresState), cudaMemcpyDeviceToHost));
          if (est_iters[i] < 0) est_iters[i] = hs[i].iters;
          const int a = resume_action(hs[i], true_rel[i], prev_true[i], restarts[i], tol, maxit);
          if (a == kKeepStopped) continue;
          prev_true[i] = true_rel[i];
          std::vector<MinresState> one{hs[i]};
          if (a == kStagnated) {
            one[0].status = FDST_STAGNATION;
            CK(cudaMemcpy(h->state, one.data(), sizeof(MinresState), cudaMemcpyHostToDevice));
          } else if (a == kRestart) {
            ++restarts[i];
            TRY(minres_restart(h, h->hb, h->hx, 1, {0}, {true_rel[i]}, tol, one, st));
            member_split_z(h, st);
            if (!one[0].stop && one[0].status == 0) ++running;
          } else {
            one[0].tau = 0.5 * one[0].tau * tol / true_rel[i];
            one[0].stop = 0;
            const int zero = 0;
            CK(cudaMemcpy(h->state, one.data(), sizeof(MinresState), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->done, &zero, sizeof(int), cudaMemcpyHostToDevice));
            ++running;
          }
        }
        if (running == 0) break;
        const int ns = n - running;
        CK(cudaMemcpy(b->n_stopped, &ns, sizeof(int), cudaMemcpyHostToDevice));
      }
    }
  }
  CK(cudaGetLastError());
  if (!residuals_current) TRY(true_residuals());
  fdst_status ret = FDST_OK;
  for (int i = 0; i < n; ++i) {
    fdst_ctx *h = b->hs[i];
    CK(cudaMemcpyAsync(d_x[i], h->hx, sizeof(double) * h->n_total, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy(&hs[i], h->state, sizeof(MinresState), cudaMemcpyDeviceToHost));
    info[i].iterations = hs[i].iters;
    info[i].status = hs[i].stop || hs[i].status ? hs[i].status : FDST_MAXIT;
    if (hs[i].eta0 == 0.0 && hs[i].status == 0) info[i].status = FDST_OK;
    info[i].eta_rel = hs[i].eta0 > 0 ? std::fabs(hs[i].eta) / hs[i].eta0 : 0.0;
    info[i].true_rel_res = true_rel[i];
    info[i].iterations_estimate = est_iters[i] >= 0 ? est_iters[i] : hs[i].iters;
    if (ret == FDST_OK && info[i].status != FDST_OK) ret = (fdst_status)info[i].status;
  }
  CK(cudaEventRecord(ev, st));
  CK(cudaStreamWaitEvent(us, ev, 0));
  CK(cudaStreamSynchronize(st));
  cudaEventDestroy(ev);
  return ret;
}

}  // extern "C"

// Continuous-batching request server for FD-preconditioned MINRES solves.
//
// Requests (a problem description and a host right-hand side) queue on
// submission. Every fdst_server_step: (1) active problems whose recurrence
// stopped get their FP64 true residual checked; finished ones copy their
// solution to host memory and free their slot (the device handle goes to an
// idle cache keyed by problem shape, so U_d, Lambda_d, banded factors and
// workspaces stay resident for the next request of the same shape), the
// others continue with a tighter threshold; (2) device handles for queued
// requests are set up on host threads while the GPU iterates (within the HBM
// budget, evicting idle handles least-recently-used first), and queued
// requests whose handle is ready are admitted in arrival order while
// active slots are free; (3) the active set, if it changed, is
// re-tabled as one batch, and (4) a few MINRES iterations advance every
// active problem together with grouped launches. Requests that arrive while
// others are on the GPU join between steps; their work overlaps on the device.
#include <cuda_runtime.h>

#include <cmath>
#include <deque>
#include <future>
#include <list>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "batch.h"
#include "ctx.h"
#include "kernels_tc.h"

using namespace fdst;

namespace {

struct Req {
  int64_t id = 0;
  fdst_desc desc{};
  std::vector<double> knots[3];
  std::vector<double> b, x;
  double t_arrival = 0.0, t_admit = -1.0, t_done = -1.0;
  fdst_ctx *h = nullptr;
  int state = 0;   // 0 queued, 1 active, 2 finished
  fdst_solve_info info{};
  std::string key;
  double bb = 0.0;
  std::shared_future<fdst_ctx *> prep;   // handle being set up in the background
  bool preparing = false;
  fdst_status prep_status = FDST_OK;
  double prev_true = -1.0;   // true residual at the previous check of a stopped recurrence
  int restarts = 0;
  int est_iters = -1;        // iteration at which the estimate first met tol
  bool cancel_pending = false;   // active and cancelled: retired at the next step
};

std::string problem_key(const fdst_desc &d, const std::vector<double> *knots) {
  std::ostringstream o;
  o.precision(17);
  o << d.dim << "|" << d.discretization << "|" << d.degree << "|" << d.viscosity << "|" << d.fd_precision << "|"
    << d.matvec_precision << "|" << d.cpen << "|" << d.geometry << "|" << d.variant << "|" << d.geometry_amplitude
    << "|" << d.viscosity_contrast << "|" << d.matvec_form;
  for (int e = 0; e < d.dim; ++e) {
    o << "#";
    for (double v : knots[e]) o << v << ",";
  }
  return o.str();
}

// Block-vector length from the pressure knot vectors (TH: interior velocity of
// degree p+1 with one more copy of every breakpoint; RT: see Sec. 2.2.2).
int64_t problem_size(const fdst_desc &d, const std::vector<double> *knots) {
  const int p = d.degree;
  int64_t nq = 1, total = 0;
  std::vector<int> mq(d.dim), nbr(d.dim);
  for (int e = 0; e < d.dim; ++e) {
    mq[e] = (int)knots[e].size() - p - 1;
    int nb = 0;
    for (size_t i = 0; i < knots[e].size(); ++i)
      if (i == 0 || knots[e][i] != knots[e][i - 1]) ++nb;
    nbr[e] = nb;
    nq *= mq[e];
  }
  for (int k = 0; k < d.dim; ++k) {
    int64_t nv = 1;
    for (int e = 0; e < d.dim; ++e) {
      if (d.discretization == FDST_TH) nv *= ((int)knots[e].size() + nbr[e]) - (p + 2) - 2;
      else nv *= (e == k) ? (mq[e] + 1 - 2) : mq[e];
    }
    total += nv;
  }
  return total + nq;
}

}  // namespace

struct fdst_server_ctx {
  fdst_server_opts o{};
  std::map<int64_t, Req> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;
  std::list<std::pair<std::string, fdst_ctx *>> idle;   // front = most recently used
  int64_t bytes_held = 0, next_id = 1;
  double bytes_per_dof[4] = {0, 0, 0, 0};
  fdst_batch batch = nullptr;
  bool dirty = true;
  cudaStream_t st = nullptr;
  int *dev_counter = nullptr;
  int64_t created = 0, reused = 0, finished = 0, evicted = 0;
  int max_active_seen = 0;
  int device = 0, preparing = 0;
  std::vector<int64_t> orphans;   // cancelled while their handle was being set up
  double last_now = 0.0;
  int tc_err = 0;                 // expired tensor-core waits seen so far
  static constexpr int kMaxPrepare = 8;   // handles set up concurrently on host threads
};

namespace {

void release(fdst_server s, Req &r) {
  s->idle.emplace_front(r.key, r.h);
  r.h = nullptr;
}

void evict_one(fdst_server s) {
  auto &e = s->idle.back();
  s->bytes_held -= e.second->device_bytes;
  fdst_destroy(e.second);
  s->idle.pop_back();
  ++s->evicted;
}

// Retires an active request without a solution (cancelled, or its step's
// tensor-core work gave up on an expired wait).
void retire(fdst_server s, Req &r, int status, double now) {
  r.info = fdst_solve_info{};
  r.info.status = status;
  r.info.true_rel_res = -1.0;
  r.t_done = now;
  r.state = 2;
  ++s->finished;
  release(s, r);
}

fdst_status finish(fdst_server s, Req &r, const MinresState &S, double true_rel, double now) {
  r.x.resize(r.h->n_total);
  CK(cudaMemcpy(r.x.data(), r.h->hx, sizeof(double) * r.h->n_total, cudaMemcpyDeviceToHost));
  r.info.iterations = S.iters;
  r.info.status = S.stop || S.status ? S.status : FDST_MAXIT;
  if (S.eta0 == 0.0 && S.status == 0) r.info.status = FDST_OK;
  r.info.eta_rel = S.eta0 > 0 ? std::fabs(S.eta) / S.eta0 : 0.0;
  r.info.true_rel_res = true_rel;
  r.info.iterations_estimate = r.est_iters >= 0 ? r.est_iters : S.iters;
  r.t_done = now;
  r.state = 2;
  ++s->finished;
  release(s, r);
  return FDST_OK;
}

}  // namespace

extern "C" {

fdst_status fdst_server_create(const fdst_server_opts *o, fdst_server *out) {
  if (!o || !out) { set_error("fdst_server_create: NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (o->max_active < 1 || o->iters_per_step < 1 || o->maxit < 1 || !(o->tol >= 0.0)) {
    set_error("fdst_server_create: max_active, iters_per_step, maxit must be >= 1 and tol >= 0");
    return FDST_INVALID_ARGUMENT;
  }
  fdst_server s = new fdst_server_ctx();
  s->o = *o;
  cudaGetDevice(&s->device);
  if (tc_error_count(&s->tc_err) != FDST_OK) {
    delete s;
    return FDST_CUDA_ERROR;
  }
  if (s->o.hbm_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->o.hbm_budget_bytes = (int64_t)(0.9 * (double)fr);
  }
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&s->dev_counter, sizeof(int)) != cudaSuccess) {
    delete s;
    set_error("fdst_server_create: stream / counter allocation failed");
    return FDST_CUDA_ERROR;
  }
  *out = s;
  return FDST_OK;
}

fdst_status fdst_server_destroy(fdst_server s) {
  if (!s) return FDST_OK;
  for (auto &kv : s->reqs)
    if (kv.second.preparing) {
      fdst_ctx *h = kv.second.prep.get();
      if (h) fdst_destroy(h);
      kv.second.preparing = false;
    }
  if (s->batch) fdst_batch_destroy(s->batch);
  for (auto &kv : s->reqs)
    if (kv.second.h) fdst_destroy(kv.second.h);
  for (auto &e : s->idle) fdst_destroy(e.second);
  if (s->dev_counter) cudaFree(s->dev_counter);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
  return FDST_OK;
}

fdst_status fdst_server_submit(fdst_server s, const fdst_desc *problem, const double *h_b, double t_arrival,
                               int64_t *id) {
  if (!s || !problem || !h_b || !id) { set_error("fdst_server_submit: NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (problem->dim != 2 && problem->dim != 3) { set_error("fdst_server_submit: dim must be 2 or 3"); return FDST_INVALID_ARGUMENT; }
  Req r;
  r.id = s->next_id++;
  r.desc = *problem;
  r.desc.max_rhs = 1;
  r.desc.fd_precision = s->o.fd_precision;
  r.desc.matvec_precision = s->o.matvec_precision;
  for (int e = 0; e < problem->dim; ++e) {
    if (!problem->h_knots[e] || problem->nknots[e] <= 0) { set_error("fdst_server_submit: missing knots"); return FDST_INVALID_ARGUMENT; }
    r.knots[e].assign(problem->h_knots[e], problem->h_knots[e] + problem->nknots[e]);
    std::string msg = validate_knots(r.knots[e], problem->degree);
    if (!msg.empty()) { set_error("fdst_server_submit: " + msg); return FDST_INVALID_ARGUMENT; }
  }
  for (int e = 0; e < 3; ++e) r.desc.h_knots[e] = nullptr;
  const int64_t n = problem_size(r.desc, r.knots);
  r.b.assign(h_b, h_b + n);
  r.key = problem_key(r.desc, r.knots);
  r.t_arrival = t_arrival;
  *id = r.id;
  s->queue.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  return FDST_OK;
}

fdst_status fdst_server_step(fdst_server s, double now, int *n_active, int *n_queued, int64_t *n_finished) {
  if (!s) { set_error("NULL server"); return FDST_INVALID_ARGUMENT; }
  cudaStream_t st = s->st;
  s->last_now = now;
  // ---- (0a) requests cancelled while their handle was being set up: the handle joins the idle cache
  for (auto it = s->orphans.begin(); it != s->orphans.end();) {
    Req &r = s->reqs[*it];
    if (r.prep.wait_for(std::chrono::seconds(0)) != std::future_status::ready) { ++it; continue; }
    fdst_ctx *h = r.prep.get();
    r.preparing = false;
    --s->preparing;
    s->bytes_held -= (int64_t)r.bb;
    if (h) {
      s->bytes_held += h->device_bytes;
      ++s->created;
      s->idle.emplace_front(r.key, h);
    }
    it = s->orphans.erase(it);
  }
  // ---- (0b) active requests cancelled since the last step retire (their device work is ordered on st)
  {
    std::vector<int64_t> keep;
    for (int64_t id : s->active) {
      Req &r = s->reqs[id];
      if (r.cancel_pending) retire(s, r, FDST_CANCELLED, now);
      else keep.push_back(id);
    }
    if (keep.size() != s->active.size()) {
      s->active.swap(keep);
      s->dirty = true;
    }
  }
  // ---- (1) stopped recurrences: true residual, finish or continue
  if (!s->active.empty()) {
    CK(cudaStreamSynchronize(st));
    int err = 0;
    TRY(tc_error_count(&err));
    if (err != s->tc_err) {
      // a tensor-core wait expired in the last step: none of its results can be trusted
      s->tc_err = err;
      for (int64_t id : s->active) retire(s, s->reqs[id], FDST_TIMEOUT, now);
      s->active.clear();
      s->dirty = true;
      set_error("fdst_server_step: a bounded device-side wait expired; the active requests finished with FDST_TIMEOUT");
    }
  }
  if (!s->active.empty()) {
    const size_t na = s->active.size();
    std::vector<MinresState> S(na);
    std::vector<int> done(na);
    for (size_t i = 0; i < na; ++i) {
      Req &r = s->reqs[s->active[i]];
      CK(cudaMemcpyAsync(&S[i], r.h->state, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&done[i], r.h->done, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    std::vector<size_t> stopped;
    for (size_t i = 0; i < na; ++i)
      if (done[i]) stopped.push_back(i);
    if (!stopped.empty()) {
      std::vector<double> rr(stopped.size());
      for (size_t k = 0; k < stopped.size(); ++k) {
        Req &r = s->reqs[s->active[stopped[k]]];
        TRY(member_residual(r.h, st));
        CK(cudaMemcpyAsync(&rr[k], r.h->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
      }
      CK(cudaStreamSynchronize(st));
      std::vector<int64_t> keep;
      std::vector<bool> gone(na, false);
      for (size_t k = 0; k < stopped.size(); ++k) {
        const size_t i = stopped[k];
        Req &r = s->reqs[s->active[i]];
        const double tr = r.bb > 0 ? std::sqrt(rr[k] / r.bb) : std::sqrt(rr[k]);
        if (r.est_iters < 0) r.est_iters = S[i].iters;
        const int a = resume_action(S[i], tr, r.prev_true, r.restarts, s->o.tol, s->o.maxit);
        if (a != kKeepStopped) r.prev_true = tr;
        std::vector<MinresState> one{S[i]};
        bool cont = false;
        if (a == kResume) {
          one[0].tau = 0.5 * one[0].tau * s->o.tol / tr;
          one[0].stop = 0;
          const int zero = 0;
          CK(cudaMemcpyAsync(r.h->state, one.data(), sizeof(MinresState), cudaMemcpyHostToDevice, st));
          CK(cudaMemcpyAsync(r.h->done, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
          CK(cudaStreamSynchronize(st));
          cont = true;
        } else if (a == kRestart) {
          ++r.restarts;
          TRY(minres_restart(r.h, r.h->hb, r.h->hx, 1, {0}, {tr}, s->o.tol, one, st));
          member_split_z(r.h, st);
          cont = !one[0].stop && one[0].status == 0;
        } else if (a == kStagnated) {
          one[0].status = FDST_STAGNATION;
        }
        if (!cont) {
          TRY(finish(s, r, one[0], tr, now));
          gone[i] = true;
        }
      }
      for (size_t i = 0; i < na; ++i)
        if (!gone[i]) keep.push_back(s->active[i]);
      if (keep.size() != na) s->dirty = true;
      s->active.swap(keep);
    }
  }
  // ---- (2a) set up handles for queued requests in the background (host threads)
  for (int64_t id : s->queue) {
    if (s->preparing >= fdst_server_ctx::kMaxPrepare) break;
    Req &r = s->reqs[id];
    if (r.preparing || r.h) continue;
    bool cached = false;
    for (auto &e : s->idle)
      if (e.first == r.key) { cached = true; break; }
    if (cached) continue;
    const int64_t ndof = problem_size(r.desc, r.knots);
    const double bpd = s->bytes_per_dof[r.desc.dim] > 0 ? s->bytes_per_dof[r.desc.dim] : 600.0;
    const int64_t est = (int64_t)(bpd * ndof);
    while (s->bytes_held + est > s->o.hbm_budget_bytes && !s->idle.empty()) evict_one(s);
    if (s->bytes_held + est > s->o.hbm_budget_bytes && !(s->active.empty() && s->preparing == 0)) break;
    s->bytes_held += est;   // reserved until the handle reports its real size
    fdst_desc d = r.desc;
    Req *rp = &r;
    const int dev = s->device;
    r.prep = std::async(std::launch::async, [d, rp, dev]() -> fdst_ctx * {
               cudaSetDevice(dev);
               fdst_desc dd = d;
               for (int e = 0; e < dd.dim; ++e) {
                 dd.h_knots[e] = rp->knots[e].data();
                 dd.nknots[e] = (int)rp->knots[e].size();
               }
               fdst_ctx *h = nullptr;
               rp->prep_status = fdst_setup(&dd, &h);
               if (h && !h->hb) {
                 if (dalloc(h, &h->hb, (size_t)h->n_total) != FDST_OK ||
                     dalloc(h, &h->hx, (size_t)h->n_total) != FDST_OK) {
                   fdst_destroy(h);
                   rp->prep_status = FDST_OUT_OF_MEMORY;
                   return nullptr;
                 }
               }
               return h;
             }).share();
    r.preparing = true;
    r.bb = (double)est;   // remembered reservation until admission
    ++s->preparing;
  }
  // ---- (2b) admission in arrival order among the requests whose handle is ready
  // (with nothing on the GPU, wait for the earliest handle being set up)
  if (s->active.empty())
    for (int64_t id : s->queue) {
      Req &r = s->reqs[id];
      if (r.preparing) {
        r.prep.wait();
        break;
      }
    }
  for (auto qit = s->queue.begin(); qit != s->queue.end() && (int)s->active.size() < s->o.max_active;) {
    Req &r = s->reqs[*qit];
    fdst_ctx *h = nullptr;
    for (auto it = s->idle.begin(); it != s->idle.end(); ++it)
      if (it->first == r.key) {
        h = it->second;
        s->idle.erase(it);
        ++s->reused;
        break;
      }
    if (!h && r.preparing) {
      if (r.prep.wait_for(std::chrono::seconds(0)) != std::future_status::ready) { ++qit; continue; }
      h = r.prep.get();
      r.preparing = false;
      --s->preparing;
      s->bytes_held -= (int64_t)r.bb;
      if (!h) {
        r.info.status = r.prep_status;
        r.state = 2;
        r.t_done = now;
        ++s->finished;
        qit = s->queue.erase(qit);
        continue;
      }
      s->bytes_per_dof[r.desc.dim] = (double)h->device_bytes / (double)h->n_total;
      if (h->device_bytes > s->o.hbm_budget_bytes) {
        // this problem alone needs more than the whole budget: it can never be admitted
        fdst_destroy(h);
        r.info.status = FDST_ADMISSION_REJECTED;
        r.state = 2;
        r.t_done = now;
        ++s->finished;
        qit = s->queue.erase(qit);
        continue;
      }
      s->bytes_held += h->device_bytes;
      ++s->created;
    }
    if (!h) { ++qit; continue; }
    r.h = h;
    if ((int64_t)r.b.size() != h->n_total) {
      set_error("fdst_server_step: right-hand side length does not match the problem");
      return FDST_INVALID_ARGUMENT;
    }
    CK(cudaMemcpyAsync(h->hb, r.b.data(), sizeof(double) * h->n_total, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->hx, 0, sizeof(double) * h->n_total, st));
    TRY(member_init(h, s->dev_counter, s->o.tol, st, true));   // hx was just cleared
    CK(cudaMemcpyAsync(&r.bb, h->dots + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    r.t_admit = now;
    r.state = 1;
    s->active.push_back(r.id);
    qit = s->queue.erase(qit);
    s->dirty = true;
  }
  if ((int)s->active.size() > s->max_active_seen) s->max_active_seen = (int)s->active.size();
  // ---- (3) re-table the active set, (4) advance it
  if (s->dirty) {
    if (s->batch) fdst_batch_destroy(s->batch);
    s->batch = nullptr;
    if (!s->active.empty()) {
      std::vector<fdst_ctx *> hs;
      for (int64_t id : s->active) hs.push_back(s->reqs[id].h);
      TRY(batch_new(hs, 0, 256, &s->batch));
    }
    s->dirty = false;
  }
  if (s->batch)
    for (int k = 0; k < s->o.iters_per_step; ++k) TRY(batch_step(s->batch, s->o.maxit, st));
  CK(cudaGetLastError());
  if (n_active) *n_active = (int)s->active.size();
  if (n_queued) *n_queued = (int)s->queue.size();
  if (n_finished) *n_finished = s->finished;
  return FDST_OK;
}

fdst_status fdst_server_result(fdst_server s, int64_t id, int *finished, double *h_x, fdst_solve_info *info,
                               double *t_arrival, double *t_admit, double *t_done) {
  if (!s || !finished) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) { set_error("fdst_server_result: unknown request id"); return FDST_INVALID_ARGUMENT; }
  Req &r = it->second;
  *finished = r.state == 2;
  if (t_arrival) *t_arrival = r.t_arrival;
  if (t_admit) *t_admit = r.t_admit;
  if (t_done) *t_done = r.t_done;
  if (r.state == 2) {
    if (info) *info = r.info;
    if (h_x && !r.x.empty()) std::copy(r.x.begin(), r.x.end(), h_x);
  }
  return FDST_OK;
}

fdst_status fdst_server_cancel(fdst_server s, int64_t id) {
  if (!s) { set_error("NULL server"); return FDST_INVALID_ARGUMENT; }
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) { set_error("fdst_server_cancel: unknown request id"); return FDST_INVALID_ARGUMENT; }
  Req &r = it->second;
  if (r.state == 2) return FDST_OK;
  if (r.state == 1) {
    r.cancel_pending = true;
    return FDST_OK;
  }
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == id) {
      s->queue.erase(q);
      break;
    }
  if (r.preparing) s->orphans.push_back(id);
  r.info = fdst_solve_info{};
  r.info.status = FDST_CANCELLED;
  r.info.true_rel_res = -1.0;
  r.t_done = s->last_now > r.t_arrival ? s->last_now : r.t_arrival;
  r.state = 2;
  ++s->finished;
  return FDST_OK;
}

fdst_status fdst_server_stats(fdst_server s, int64_t *handles_created, int64_t *handles_reused,
                              int64_t *handles_evicted, int64_t *bytes_held, int *max_active_seen) {
  if (!s) { set_error("NULL server"); return FDST_INVALID_ARGUMENT; }
  if (handles_created) *handles_created = s->created;
  if (handles_reused) *handles_reused = s->reused;
  if (handles_evicted) *handles_evicted = s->evicted;
  if (bytes_held) *bytes_held = s->bytes_held;
  if (max_active_seen) *max_active_seen = s->max_active_seen;
  return FDST_OK;
}

}  // extern "C"

// C ABI implementation: setup of the spaces, univariate matrices and FD
// factors (paper Sec. 2.2, Sec. 5, Algorithm 1 step 1), the preconditioner
// apply as a chain of rotation GEMMs (Algorithm 1 steps 2-4), the
// matrix-free Kronecker Stokes matvec (Sec. 3 blocks on the identity map)
// and the multi-right-hand-side MINRES driver (Sec. 4, Sec. 7).
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <tuple>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ctx.h"
#include "mapped.h"

namespace fdst {

static thread_local std::string g_err;
void set_error(const std::string &s) { g_err = s; }

static std::string space_key(const Space1D &s) {
  std::ostringstream o;
  o.precision(17);
  o << s.degree << "|" << s.first << "|" << s.n << "|" << s.nitsche << "|" << s.cpen << "|" << s.h << "|";
  for (double k : s.knots) o << k << ",";
  return o.str();
}

// ------------------------------------------------------------------ setup: spaces

static fdst_status build_spaces(fdst_ctx *h) {
  const fdst_desc &d = h->desc;
  const int dim = h->dim, p = h->p;
  h->pres.resize(dim);
  h->vel.assign(dim, std::vector<Space1D>(dim));
  for (int e = 0; e < dim; ++e) {
    Space1D s;
    s.knots = h->knots[e];
    s.degree = p;
    s.first = 0;
    s.n = s.m();
    h->pres[e] = s;
  }
  for (int k = 0; k < dim; ++k)
    for (int e = 0; e < dim; ++e) {
      Space1D s;
      if (d.discretization == FDST_TH) {
        s.knots = elevate(h->knots[e]);
        s.degree = p + 1;
        s.first = 1;
        s.n = s.m() - 2;
      } else {
        if (e == k) {
          s.knots = h->knots[e];
          s.knots.insert(s.knots.begin(), 0.0);
          s.knots.push_back(1.0);
          s.degree = p + 1;
          s.first = 1;
          s.n = s.m() - 2;
        } else {
          s.knots = h->knots[e];
          s.degree = p;
          s.first = 0;
          s.n = s.m();
          s.nitsche = true;
          double hmax = 0.0;
          for (size_t i = 1; i < s.knots.size(); ++i) hmax = std::max(hmax, s.knots[i] - s.knots[i - 1]);
          s.h = hmax;
          int alpha = p - inner_multiplicity(s.knots);
          s.cpen = d.cpen > 0.0 ? d.cpen : 5.0 * (alpha + 1);
        }
      }
      if (s.n < 1) {
        set_error("velocity space has no interior functions (too few elements)");
        return FDST_INVALID_ARGUMENT;
      }
      h->vel[k][e] = s;
    }
  h->nblocks = dim + 1;
  int64_t o = 0;
  for (int b = 0; b <= dim; ++b) {
    for (int e = 0; e < 3; ++e) h->shape[b][e] = 1;
    for (int e = 0; e < dim; ++e) h->shape[b][e] = b < dim ? h->vel[b][e].n : h->pres[e].n;
    h->off[b] = o;
    o += (int64_t)h->shape[b][0] * h->shape[b][1] * h->shape[b][2];
  }
  h->off[dim + 1] = o;
  h->n_total = o;
  return FDST_OK;
}

// ------------------------------------------------------------------ setup: FD chains

static fdst_status build_fd(fdst_ctx *h) {
  const int dim = h->dim, p = h->p;
  const int npts = p + 2;
  // process-wide cache of eigen-factors of identical univariate pencils (handles of
  // problems that share a direction's space skip the Jacobi solve)
  static std::mutex cache_mutex;
  static std::map<std::string, std::pair<std::vector<double>, Mat>> eig_cache;  // key -> (lam, U)
  std::map<std::string, const double *> dev_cache;
  auto dev_mat = [&](const std::string &key, const Mat &A, const double **out) -> fdst_status {
    auto it = dev_cache.find(key);
    if (it != dev_cache.end()) { *out = it->second; return FDST_OK; }
    double *d = nullptr;
    TRY(upload(h, &d, A.a));
    dev_cache[key] = d;
    *out = d;
    return FDST_OK;
  };
  auto transpose = [](const Mat &A) {
    Mat T(A.cols, A.rows);
    for (int i = 0; i < A.rows; ++i)
      for (int j = 0; j < A.cols; ++j) T(j, i) = A(i, j);
    return T;
  };
  h->chains.clear();
  for (int k = 0; k < dim; ++k) {
    FdChain c;
    c.off = h->off[k];
    c.size = h->off[k + 1] - h->off[k];
    std::vector<double> lam[3];
    const double *Uf[3], *Ub[3];
    std::vector<double> Ufh[3], Ubh[3];
    for (int e = 0; e < dim; ++e) {
      const Space1D &s = h->vel[k][e];
      std::string key = space_key(s);
      const bool geo = h->desc.variant == FDST_VARIANT_PD_GEO;
      if (geo) key = "geo" + std::to_string(k) + "_" + std::to_string(e) + "_" + key;
      // lookups and inserts under the lock; the Jacobi solve itself runs outside it
      std::pair<std::vector<double>, Mat> fac;
      bool found = false;
      if (!geo) {
        std::lock_guard<std::mutex> lock(cache_mutex);
        auto it = eig_cache.find(key);
        if (it != eig_cache.end()) { fac = it->second; found = true; }
      }
      if (!found) {
        Mat K = geo ? h->geo_K[k][e] : stiffness_matrix(s, npts);
        Mat M = geo ? h->geo_M[k][e] : mixed_matrix(s, 0, s, 0, npts);
        if (!gen_eig(K, M, fac.first, fac.second)) {
          set_error("univariate velocity mass matrix is not SPD");
          return FDST_NOT_SPD;
        }
        if (!geo) {
          std::lock_guard<std::mutex> lock(cache_mutex);
          if (eig_cache.size() > 4096) eig_cache.clear();
          eig_cache.emplace(key, fac);
        }
      }
      lam[e] = fac.first;
      Mat Ut = transpose(fac.second);
      TRY(dev_mat("U" + key, fac.second, &Uf[e]));
      TRY(dev_mat("Ut" + key, Ut, &Ub[e]));
      Ufh[e] = fac.second.a;
      Ubh[e] = Ut.a;
    }
    const int n1 = h->shape[k][0], n2 = h->shape[k][1], n3 = h->shape[k][2];
    // c_{k,d} = 2 for d = k in P_{V,k} (eq. prec3D_TH); the weighted pencils of P~_V carry
    // that factor inside C_k (Appendix), so their coefficients are all 1
    double cf[3];
    for (int e = 0; e < 3; ++e) cf[e] = (e == k && h->desc.variant != FDST_VARIANT_PD_GEO) ? 2.0 : 1.0;
    std::vector<double> lr, lc;
    if (dim == 3) {
      c.nsteps = 6;
      int Rs[6] = {n2 * n3, n1 * n3, n1 * n2, n2 * n3, n1 * n3, n1 * n2};
      int Ns[6] = {n1, n2, n3, n1, n2, n3};
      for (int j = 0; j < 6; ++j) {
        c.R[j] = Rs[j];
        c.K[j] = c.N[j] = Ns[j];
        c.B[j] = j < 3 ? Uf[j] : Ub[j - 3];
        c.Bh[j] = j < 3 ? Ufh[j] : Ubh[j - 3];
      }
      c.div_step = 2;
      lr.resize((size_t)n1 * n2);
      for (int b = 0; b < n2; ++b)
        for (int a = 0; a < n1; ++a) lr[(size_t)b * n1 + a] = cf[0] * lam[0][a] + cf[1] * lam[1][b];
      lc.resize(n3);
      for (int cc = 0; cc < n3; ++cc) lc[cc] = cf[2] * lam[2][cc];
    } else {
      c.nsteps = 4;
      int Rs[4] = {n2, n1, n2, n1};
      int Ns[4] = {n1, n2, n1, n2};
      for (int j = 0; j < 4; ++j) {
        c.R[j] = Rs[j];
        c.K[j] = c.N[j] = Ns[j];
        c.B[j] = j < 2 ? Uf[j] : Ub[j - 2];
        c.Bh[j] = j < 2 ? Ufh[j] : Ubh[j - 2];
      }
      c.div_step = 1;
      lr.resize(n1);
      for (int a = 0; a < n1; ++a) lr[a] = cf[0] * lam[0][a];
      lc.resize(n2);
      for (int b = 0; b < n2; ++b) lc[b] = cf[1] * lam[1][b];
    }
    TRY(upload(h, &c.lam_row, lr));
    TRY(upload(h, &c.lam_col, lc));
    std::vector<float> lrf(lr.begin(), lr.end()), lcf(lc.begin(), lc.end());
    TRY(upload(h, &c.lam_row_f, lrf));
    TRY(upload(h, &c.lam_col_f, lcf));
    h->chains.push_back(c);
  }
  // pressure: P_Q^{-1} = W3 x W2 x W1 with W_d = M_d^{-1} (eq. precQ, eq. kroninv)
  {
    FdChain c;
    c.off = h->off[dim];
    c.size = h->off[dim + 1] - h->off[dim];
    const double *W[3];
    std::vector<double> Wh[3];
    for (int e = 0; e < dim; ++e) {
      Mat M = mixed_matrix(h->pres[e], 0, h->pres[e], 0, npts), Mi;
      if (!spd_inverse(M, Mi)) {
        set_error("univariate pressure mass matrix is not SPD");
        return FDST_NOT_SPD;
      }
      TRY(dev_mat("W" + space_key(h->pres[e]), Mi, &W[e]));
      Wh[e] = Mi.a;
    }
    const int n1 = h->shape[dim][0], n2 = h->shape[dim][1], n3 = h->shape[dim][2];
    if (dim == 3) {
      c.nsteps = 3;
      int Rs[3] = {n2 * n3, n1 * n3, n1 * n2};
      int Ns[3] = {n1, n2, n3};
      for (int j = 0; j < 3; ++j) { c.R[j] = Rs[j]; c.K[j] = c.N[j] = Ns[j]; c.B[j] = W[j]; c.Bh[j] = Wh[j]; }
    } else {
      c.nsteps = 2;
      int Rs[2] = {n2, n1};
      int Ns[2] = {n1, n2};
      for (int j = 0; j < 2; ++j) { c.R[j] = Rs[j]; c.K[j] = c.N[j] = Ns[j]; c.B[j] = W[j]; c.Bh[j] = Wh[j]; }
    }
    h->chains.push_back(c);
  }
  return FDST_OK;
}

// ------------------------------------------------------------------ setup: matvec plan

// The common-subexpression plan of a set of Kronecker terms: stage 1 = distinct
// (src, f0); stage 2 (3D) = each term into the accumulator G(dst, f2); stage 3 =
// dst += G x_3 f2. In 2D stage 2 writes dst. Also its double-float form
// (coefficients folded into the band values; in 3D T1 held with its slow
// coordinates swapped). T1/G buffer sizes per right-hand side are appended.
static fdst_status build_plan(fdst_ctx *h, const std::vector<Term> &terms, std::vector<PlanOp> &plan,
                              std::vector<PlanOp> &plan_df, std::vector<int64_t> &t1_size,
                              std::vector<int64_t> &g_size, const std::vector<std::array<int, 3>> *shapes = nullptr,
                              int ndst = 0) {
  const int dim = h->dim;
  plan.clear();
  plan_df.clear();
  t1_size.clear();
  g_size.clear();
  std::map<std::pair<int, int>, int> t1_ids;
  std::map<std::pair<int, int>, int> g_ids;
  std::vector<PlanOp> st1, st2, st3;
  std::vector<int> g_first;            // whether the G buffer was written yet
  std::vector<int> dst_written(std::max(dim + 1, ndst), 0);
  // source block shapes: the solution blocks, or the given ones (quadrature-point fields)
  auto srcdims = [&](int b, int out[3]) {
    for (int e = 0; e < 3; ++e) out[e] = shapes ? (*shapes)[b][e] : h->shape[b][e];
  };
  for (const Term &t : terms) {
    auto k1 = std::make_pair(t.src, t.f[0]);
    int t1;
    auto it = t1_ids.find(k1);
    if (it == t1_ids.end()) {
      t1 = (int)t1_size.size();
      t1_ids[k1] = t1;
      PlanOp op{};
      op.stage = 1;
      op.in_kind = 0; op.in_id = t.src;
      op.out_kind = 1; op.out_id = t1;
      op.band = t.f[0]; op.mode = 0;
      srcdims(t.src, op.dims);
      op.coef = 1.0; op.accumulate = 0;
      st1.push_back(op);
      int64_t sz = (int64_t)h->bands[t.f[0]].rows * op.dims[1] * op.dims[2];
      t1_size.push_back(sz);
    } else t1 = it->second;
    int d1[3];
    srcdims(t.src, d1);
    d1[0] = h->bands[t.f[0]].rows;
    if (dim == 2) {
      PlanOp op{};
      op.stage = 2;
      op.in_kind = 1; op.in_id = t1;
      op.out_kind = 3; op.out_id = t.dst;
      op.band = t.f[1]; op.mode = 1;
      for (int e = 0; e < 3; ++e) op.dims[e] = d1[e];
      op.coef = t.coef;
      op.accumulate = dst_written[t.dst];
      dst_written[t.dst] = 1;
      st2.push_back(op);
    } else {
      auto kg = std::make_pair(t.dst, t.f[2]);
      int gid;
      auto ig = g_ids.find(kg);
      if (ig == g_ids.end()) {
        gid = (int)g_size.size();
        g_ids[kg] = gid;
        g_size.push_back((int64_t)d1[0] * h->bands[t.f[1]].rows * d1[2]);
        g_first.push_back(0);
        PlanOp op3{};
        op3.stage = 3;
        op3.in_kind = 2; op3.in_id = gid;
        op3.out_kind = 3; op3.out_id = t.dst;
        op3.band = t.f[2]; op3.mode = 2;
        op3.dims[0] = d1[0]; op3.dims[1] = h->bands[t.f[1]].rows; op3.dims[2] = d1[2];
        op3.coef = 1.0;
        op3.accumulate = dst_written[t.dst];
        dst_written[t.dst] = 1;
        st3.push_back(op3);
      } else gid = ig->second;
      PlanOp op{};
      op.stage = 2;
      op.in_kind = 1; op.in_id = t1;
      op.out_kind = 2; op.out_id = gid;
      op.band = t.f[1]; op.mode = 1;
      for (int e = 0; e < 3; ++e) op.dims[e] = d1[e];
      op.coef = t.coef;
      op.accumulate = g_first[gid];
      g_first[gid] = 1;
      st2.push_back(op);
    }
  }
  plan.clear();
  plan.insert(plan.end(), st1.begin(), st1.end());
  plan.insert(plan.end(), st2.begin(), st2.end());
  plan.insert(plan.end(), st3.begin(), st3.end());
  // double-float band values with the op's coefficient folded in (the products are
  // then summed without a final scaling); one copy per distinct (band, coefficient)
  std::map<std::pair<int, double>, const float2 *> scaled;
  for (auto &op : plan) {
    const auto key = std::make_pair(op.band, op.coef);
    auto it = scaled.find(key);
    if (it == scaled.end()) {
      const BandDev &bd = h->bands[op.band];
      std::vector<float2> v(bd.hvals.size());
      for (size_t k = 0; k < v.size(); ++k) {
        const double a = op.coef * bd.hvals[k];
        const float hi = (float)a;
        v[k] = make_float2(hi, (float)(a - (double)hi));
      }
      float2 *d = nullptr;
      TRY(upload(h, &d, v));
      it = scaled.emplace(key, d).first;
    }
    op.vals_df = it->second;
  }
  // double-float plan: stage 1 writes T1 as (l1, l2, i0) (slow coordinates swapped),
  // stage 2 then contracts l1 as the slowest index (mode 2 over (i0, l2, l1)) and
  // writes G in its usual (i0, i1, l2) order by swapping back
  plan_df = plan;
  // ops of a stage ordered by band width (stable), so that a launch groups ops of one
  // width (the banded kernel then unrolls its band loop fully); the accumulate flags
  // follow the new order (the first op into each output of the stage stores)
  std::stable_sort(plan_df.begin(), plan_df.end(), [&](const PlanOp &a, const PlanOp &b) {
    if (a.stage != b.stage) return a.stage < b.stage;
    return h->bands[a.band].w < h->bands[b.band].w;
  });
  {
    std::map<std::tuple<int, int, int>, int> written;
    for (auto &op : plan_df) {
      int &wr = written[std::make_tuple(op.stage, op.out_kind, op.out_id)];
      op.accumulate = wr;
      wr = 1;
    }
  }
  if (dim == 3)
    for (auto &op : plan_df) {
      if (op.stage == 1) {
        op.swap = 1;
      } else if (op.stage == 2) {
        op.mode = 2;
        std::swap(op.dims[1], op.dims[2]);
        op.swap = 1;
      }
    }
  return FDST_OK;
}

static fdst_status alloc_plan_buffers(fdst_ctx *h, const std::vector<int64_t> &t1_size,
                                      const std::vector<int64_t> &g_size, std::vector<double *> &t1,
                                      std::vector<double *> &g) {
  for (int64_t sz : t1_size) {
    double *b = nullptr;
    TRY(dalloc(h, &b, (size_t)sz * h->max_rhs));
    t1.push_back(b);
  }
  for (int64_t sz : g_size) {
    double *b = nullptr;
    TRY(dalloc(h, &b, (size_t)sz * h->max_rhs));
    g.push_back(b);
  }
  return FDST_OK;
}

// Banded device form of a matrix (rows x w values, first column per row; FP64
// and FP32 pairs), appended to h->bands.
static fdst_status band_from_mat(fdst_ctx *h, const Mat &A, int *id) {
  int w = 0;
  std::vector<int> first(A.rows, 0), last(A.rows, -1);
  for (int i = 0; i < A.rows; ++i) {
    for (int j = 0; j < A.cols; ++j)
      if (A(i, j) != 0.0) { if (last[i] < 0) first[i] = j; last[i] = j; }
    if (last[i] >= 0) w = std::max(w, last[i] - first[i] + 1);
  }
  if (w == 0) w = 1;
  std::vector<int> lo(A.rows);
  std::vector<double> vals((size_t)A.rows * w, 0.0);
  for (int i = 0; i < A.rows; ++i) {
    int l = last[i] < 0 ? 0 : first[i];
    if (l + w > A.cols) l = A.cols - w;
    lo[i] = l;
    for (int j = 0; j < w; ++j) vals[(size_t)i * w + j] = A(i, l + j);
  }
  BandDev b{A.rows, A.cols, w, nullptr, nullptr, nullptr};
  TRY(upload(h, &b.vals, vals));
  TRY(upload(h, &b.lo, lo));
  std::vector<float2> vdf(vals.size());
  for (size_t i = 0; i < vals.size(); ++i) {
    const float hi = (float)vals[i];
    vdf[i] = make_float2(hi, (float)(vals[i] - (double)hi));
  }
  TRY(upload(h, &b.vals_df, vdf));
  b.hvals = vals;
  for (int i = 0; i < std::min(A.rows, A.cols); ++i) b.hdiag.push_back(A(i, i));
  *id = (int)h->bands.size();
  h->bands.push_back(b);
  return FDST_OK;
}

static fdst_status build_matvec(fdst_ctx *h) {
  const int dim = h->dim, p = h->p, npts = p + 2;
  // The one-coordinate viscosity family on the identity map: nu(eta_1) multiplies every
  // integrand of a (and sigma), so each A-block term's direction-1 factor is weighted by
  // nu at the quadrature points, and its Nitsche boundary values by nu(0), nu(1).
  const bool nu_field = h->desc.geometry == FDST_GEOM_IDENTITY && h->desc.viscosity_contrast >= 1.0;
  const double nu = nu_field ? 1.0 : (h->desc.viscosity > 0.0 ? h->desc.viscosity : 1.0);
  std::vector<double> nu_w;
  double nu0 = 1.0, nu1 = 1.0;
  if (nu_field) {
    std::vector<double> x, w;
    span_rule(h->pres[0].knots, npts, x, w);
    for (double e : x) nu_w.push_back(contrast_viscosity(e, h->desc.viscosity_contrast));
    nu0 = contrast_viscosity(0.0, h->desc.viscosity_contrast);
    nu1 = contrast_viscosity(1.0, h->desc.viscosity_contrast);
  }
  std::map<std::string, int> band_ids;
  // factor key -> band id; builds int_0^1 [nu] b_a^(da) b_b^(db) (stiffness with Nitsche when both
  // da=db=1 and same space); weighted: the nu(eta_1) weight of direction 1
  auto band_of = [&](const Space1D &sa, int da, const Space1D &sb, int db, bool weighted, int *id) -> fdst_status {
    std::string key = space_key(sa) + "#" + std::to_string(da) + "#" + space_key(sb) + "#" + std::to_string(db) +
                      (weighted ? "#nu" : "");
    auto it = band_ids.find(key);
    if (it != band_ids.end()) { *id = it->second; return FDST_OK; }
    static const std::vector<double> none;
    const std::vector<double> &wt = weighted ? nu_w : none;
    Mat A = (da == 1 && db == 1 && space_key(sa) == space_key(sb))
                ? stiffness_matrix(sa, npts, wt, weighted ? nu0 : 1.0, weighted ? nu1 : 1.0)
                : mixed_matrix(sa, da, sb, db, npts, wt);
    TRY(band_from_mat(h, A, id));
    band_ids[key] = *id;
    return FDST_OK;
  };
  std::vector<Term> terms;
  for (int r = 0; r < dim; ++r) {
    for (int s = 0; s < dim; ++s) {
      if (r == s) {
        for (int d = 0; d < dim; ++d) {
          Term t{r, s, nu * (d == r ? 2.0 : 1.0), {-1, -1, -1}};
          for (int e = 0; e < dim; ++e) {
            const Space1D &sp = h->vel[r][e];
            TRY(band_of(sp, e == d, sp, e == d, nu_field && e == 0, &t.f[e]));
          }
          terms.push_back(t);
        }
      } else {
        // [A_rs]_{ij} = nu int d_s B_i d_r B_j: direction s: (b_i)' b_j, direction r: b_i (b_j)'
        Term t{r, s, nu, {-1, -1, -1}};
        for (int e = 0; e < dim; ++e)
          TRY(band_of(h->vel[r][e], e == s, h->vel[s][e], e == r, nu_field && e == 0, &t.f[e]));
        terms.push_back(t);
      }
    }
    // B_r^T p: direction r: (b^v)' b^p, others b^v b^p ; coefficient -1
    Term t{r, dim, -1.0, {-1, -1, -1}};
    for (int e = 0; e < dim; ++e) TRY(band_of(h->vel[r][e], e == r, h->pres[e], 0, false, &t.f[e]));
    terms.push_back(t);
  }
  for (int r = 0; r < dim; ++r) {
    Term t{dim, r, -1.0, {-1, -1, -1}};
    for (int e = 0; e < dim; ++e) TRY(band_of(h->pres[e], 0, h->vel[r][e], e == r, false, &t.f[e]));
    terms.push_back(t);
  }
  h->terms = terms;
  TRY(build_plan(h, terms, h->plan, h->plan_df, h->t1_size, h->g_size));
  TRY(alloc_plan_buffers(h, h->t1_size, h->g_size, h->t1, h->g));
  if (h->desc.matvec_precision == FDST_MV_DF64) {
    TRY(dalloc(h, &h->x2, (size_t)h->n_total * h->max_rhs));
    TRY(dalloc(h, &h->y2, (size_t)h->n_total * h->max_rhs));
  }
  return FDST_OK;
}

// ------------------------------------------------------------------ setup: matrix-free mapped operator

// Sum factorization of the mapped operator (Sec. 3 forms on the mapped domain,
// the quadrature of the assembly): per direction d the values Bv_d and
// derivatives Dv_d of the velocity basis and the values Bp_d of the pressure
// basis at the quadrature points (banded: a point sees p + 2 functions), and
// their transposes. Forward plan: G[r][a] = (x)_e (e == a ? Dv_e : Bv_e) u_r,
// P = (x)_e Bp_e p; backward plan: y_r = sum_a (x)_e (e == a ? Dv_e : Bv_e)^T F[r][a],
// y_p = (x)_e Bp_e^T E, with the point stage (launch_mf_points_*) in between.
static fdst_status build_matrix_free(fdst_ctx *h) {
  const GeoPoints &gp = h->gp;
  int bv[3], dv[3], bp[3], bvt[3], dvt[3], bpt[3];
  for (int d = 0; d < 3; ++d) {
    std::vector<double> x, w;
    span_rule(h->pres[d].knots, h->p + 2, x, w);
    if ((int)x.size() != gp.nq[d]) { set_error("quadrature grid mismatch"); return FDST_CUDA_ERROR; }
    const Space1D &sv = h->vel[0][d], &sp = h->pres[d];
    Mat Bv((int)x.size(), sv.n), Dv((int)x.size(), sv.n), Bp((int)x.size(), sp.n);
    double N[32], dN[32];
    for (size_t q = 0; q < x.size(); ++q) {
      int s_ = eval_nonzero(sv.knots, sv.degree, x[q], N, dN);
      for (int i = 0; i <= sv.degree; ++i) {
        const int gi = s_ - sv.degree + i - sv.first;
        if (gi < 0 || gi >= sv.n) continue;
        Bv((int)q, gi) = N[i];
        Dv((int)q, gi) = dN[i];
      }
      s_ = eval_nonzero(sp.knots, sp.degree, x[q], N, dN);
      for (int i = 0; i <= sp.degree; ++i) {
        const int gi = s_ - sp.degree + i - sp.first;
        if (gi < 0 || gi >= sp.n) continue;
        Bp((int)q, gi) = N[i];
      }
    }
    auto tr = [](const Mat &A) {
      Mat T(A.cols, A.rows);
      for (int i = 0; i < A.rows; ++i)
        for (int j = 0; j < A.cols; ++j) T(j, i) = A(i, j);
      return T;
    };
    TRY(band_from_mat(h, Bv, &bv[d]));
    TRY(band_from_mat(h, Dv, &dv[d]));
    TRY(band_from_mat(h, Bp, &bp[d]));
    TRY(band_from_mat(h, tr(Bv), &bvt[d]));
    TRY(band_from_mat(h, tr(Dv), &dvt[d]));
    TRY(band_from_mat(h, tr(Bp), &bpt[d]));
  }
  std::vector<Term> fwd, bwd;
  for (int r = 0; r < 3; ++r)
    for (int a = 0; a < 3; ++a) {
      Term t{3 * r + a, r, 1.0, {-1, -1, -1}};
      for (int e = 0; e < 3; ++e) t.f[e] = e == a ? dv[e] : bv[e];
      fwd.push_back(t);
      Term u{r, 3 * r + a, 1.0, {-1, -1, -1}};
      for (int e = 0; e < 3; ++e) u.f[e] = e == a ? dvt[e] : bvt[e];
      bwd.push_back(u);
    }
  fwd.push_back(Term{9, 3, 1.0, {bp[0], bp[1], bp[2]}});
  bwd.push_back(Term{3, 9, 1.0, {bpt[0], bpt[1], bpt[2]}});
  h->mf_fwd_terms = fwd;
  h->mf_bwd_terms = bwd;
  const std::array<int, 3> pts{gp.nq[0], gp.nq[1], gp.nq[2]};
  std::vector<std::array<int, 3>> shapes(10, pts);
  TRY(build_plan(h, fwd, h->mf_fwd, h->mf_fwd_df, h->mf_fwd_t1s, h->mf_fwd_gs, nullptr, 10));
  TRY(build_plan(h, bwd, h->mf_bwd, h->mf_bwd_df, h->mf_bwd_t1s, h->mf_bwd_gs, &shapes, 4));
  TRY(alloc_plan_buffers(h, h->mf_fwd_t1s, h->mf_fwd_gs, h->mf_fwd_t1, h->mf_fwd_g));
  TRY(alloc_plan_buffers(h, h->mf_bwd_t1s, h->mf_bwd_gs, h->mf_bwd_t1, h->mf_bwd_g));
  h->mf_Q = gp.Q;
  for (int f = 0; f < 10; ++f) h->mf_foff[f] = f * gp.Q;
  const size_t nf = (size_t)10 * gp.Q * h->max_rhs;
  TRY(dalloc(h, &h->mf_F, nf));            // FP64 fields (true residuals; FP64 iterations)
  if (h->desc.matvec_precision == FDST_MV_DF64) {
    TRY(dalloc(h, &h->mf_Fw, nf));
    TRY(dalloc(h, &h->mf_jd, (size_t)9 * gp.Q));
    TRY(dalloc(h, &h->mf_wd, (size_t)gp.Q));
    TRY(dalloc(h, &h->mf_nu, (size_t)gp.Q));
    if (!h->y2) TRY(dalloc(h, &h->y2, (size_t)h->n_total * h->max_rhs));
    launch_mf_geo_df(gp, h->mf_jd, h->mf_wd, h->mf_nu, 0);
  }
  h->mf = true;
  for (int d = 0; d < 3; ++d) {
    h->mf_bv[d] = bv[d];
    h->mf_dv[d] = dv[d];
  }
  return FDST_OK;
}

// ------------------------------------------------------------------ split-TF32 operands

// Packs every FD step's factor into the tensor-core operand image (TF32
// hi/lo or three bf16 pieces, swizzled per stage) and allocates the FP32
// intermediates.
static fdst_status tc_prepare(fdst_ctx *h) {
  const int split = h->desc.fd_precision == FDST_FD_BF16X6 ? 1 : 0;
  std::map<const double *, const uint8_t *> cache;
  for (auto &c : h->chains)
    for (int j = 0; j < c.nsteps; ++j) {
      auto it = cache.find(c.B[j]);
      if (it != cache.end()) { c.Bt[j] = it->second; continue; }
      std::vector<uint8_t> packed;
      tc_pack(c.Bh[j].data(), c.K[j], c.N[j], split, packed);
      uint8_t *d = nullptr;
      TRY(upload(h, &d, packed));
      c.Bt[j] = d;
      cache[c.B[j]] = d;
    }
  // padded FP32 operands (TcLayout): step j reads R[j] rows at pitch lda (K[j]
  // rounded up to 8: 32-byte TMA pitch); step 0's operand is the FP32 image
  // of the FP64 input, later ones the previous step's output
  h->f_off.clear();
  h->f_total = 0;
  int maxsteps = 0;
  for (auto &c : h->chains) {
    int64_t fsize = 0;
    for (int j = 0; j < c.nsteps; ++j) fsize = std::max(fsize, (int64_t)c.R[j] * tc_round(c.K[j], 8));
    h->f_off.push_back(h->f_total);
    h->f_total += (fsize + 63) & ~(int64_t)63;
    maxsteps = std::max(maxsteps, c.nsteps);
  }
  const size_t nv = (size_t)h->f_total * h->max_rhs;
  TRY(dalloc(h, &h->work_f[0], nv));
  TRY(dalloc(h, &h->work_f[1], nv));
  // one TMA descriptor per (chain, step): step j reads work_f[(j + 1) % 2]
  h->tmap_steps = maxsteps;
  std::vector<uint8_t> maps((size_t)128 * h->chains.size() * maxsteps, 0);
  for (size_t ci = 0; ci < h->chains.size(); ++ci) {
    const FdChain &c = h->chains[ci];
    for (int j = 0; j < c.nsteps; ++j)
      TRY(tc_encode_map(maps.data() + 128 * (ci * maxsteps + j), h->work_f[(j + 1) % 2] + h->f_off[ci], c.K[j],
                        c.R[j], tc_round(c.K[j], 8), h->f_total, h->max_rhs));
  }
  TRY(upload(h, &h->tmaps, maps));
  return FDST_OK;
}

// ------------------------------------------------------------------ execution

// The block of the block vector a chain applies to (velocity components 0..dim-1, pressure dim).
static int chain_block(const fdst_ctx *h, const FdChain &c) {
  for (int b = 0; b <= h->dim; ++b)
    if (h->off[b] == c.off) return b;
  return -1;
}

fdst_status run_apply(fdst_ctx *h, const double *r, double *s, int nrhs, const int *done, cudaStream_t st,
                      unsigned block_mask) {
  auto in_mask = [&](const FdChain &c) { return ((block_mask >> chain_block(h, c)) & 1u) != 0; };
  int maxsteps = 0;
  for (auto &c : h->chains)
    if (in_mask(c)) maxsteps = std::max(maxsteps, c.nsteps);
  const bool tc = h->desc.fd_precision != FDST_FD_F64;
  for (int j = 0; j < maxsteps; ++j) {
    if (tc) {
      TcGroup g;
      g.split = h->desc.fd_precision == FDST_FD_BF16X6 ? 1 : 0;
      for (size_t ci = 0; ci < h->chains.size(); ++ci) {
        const FdChain &c = h->chains[ci];
        if (j >= c.nsteps || !in_mask(c)) continue;
        TcProb &P = g.p[g.nprob++];
        const bool first = j == 0, last = j == c.nsteps - 1;
        if (first) {
          P.A64 = r + c.off;
          P.a64_rhs_stride = h->n_total;
          g.convert = 1;
        }
        const TcLayout L = tc_layout(c.R[j], c.K[j], c.K[(j + 1) % c.nsteps], last);
        P.A32 = h->work_f[(j + 1) % 2] + h->f_off[ci];
        P.a_rhs_stride = h->f_total;
        P.lda = L.lda;
        P.tmap = h->tmaps + 128 * (ci * h->tmap_steps + j);
        P.out_nv = c.K[(j + 1) % c.nsteps];
        P.ldv = L.ldv;
        P.c_cs = L.c_cs;
        if (last) {
          P.C64 = s + c.off;
          P.c_rhs_stride = h->n_total;
        } else {
          P.C32 = h->work_f[j % 2] + h->f_off[ci];
          P.c_rhs_stride = h->f_total;
        }
        P.Bt = c.Bt[j];
        P.R = c.R[j]; P.K = c.K[j]; P.N = c.N[j];
        if (j == c.div_step) { P.lam_row = c.lam_row_f; P.lam_col = c.lam_col_f; }
        P.scale_in = first ? c.scale : nullptr;
        P.scale_out = last ? c.scale : nullptr;
      }
      if (g.nprob) TRY(launch_gemm_tc(g, nrhs, done, st));
    } else {
      GemmGroup g;
      for (auto &c : h->chains) {
        if (j >= c.nsteps || !in_mask(c)) continue;
        GemmProb &P = g.p[g.nprob++];
        P.A = j == 0 ? r + c.off : h->work[(j - 1) % 2] + c.off;
        P.C = j == c.nsteps - 1 ? s + c.off : h->work[j % 2] + c.off;
        P.B = c.B[j];
        P.a_rhs_stride = P.c_rhs_stride = h->n_total;
        P.R = c.R[j]; P.K = c.K[j]; P.N = c.N[j];
        if (j == c.div_step) { P.lam_row = c.lam_row; P.lam_col = c.lam_col; }
        P.scale_in = j == 0 ? c.scale : nullptr;
        P.scale_out = j == c.nsteps - 1 ? c.scale : nullptr;
      }
      if (g.nprob) launch_gemm_f64(g, nrhs, done, st);
    }
  }
  CK(cudaGetLastError());
  return FDST_OK;
}

// Timing of the matvec's compute launches alone: an event before the first and
// after the last launch, kept in h->kev (only when timing is on).
static cudaEvent_t kernel_mark(fdst_ctx *h, cudaStream_t st) {
  if (!h->timing) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, st);
  return e;
}

static void kernel_span(fdst_ctx *h, cudaEvent_t a, int64_t launches, cudaStream_t st) {
  if (!a) return;
  cudaEvent_t b = kernel_mark(h, st);
  if (!b) { cudaEventDestroy(a); return; }
  h->kev.emplace_back(a, b);
  h->n_kernel += launches;
}

// A plan's ops over the buffers of that plan (the full operator, or its B or B^T part).
// Source blocks (in_kind 0) at x + in_off[id] and result blocks (out_kind 3) at
// y + out_off[id], right-hand sides in_stride / out_stride apart; xw, yw the
// double-float images of x and y (same offsets and strides).
struct PlanView {
  const std::vector<PlanOp> *ops;
  const std::vector<double *> *t1, *g;
  const std::vector<int64_t> *t1_size, *g_size;
  const int64_t *in_off, *out_off;
  int64_t in_stride, out_stride;
  float2 *xw, *yw;
};

static PlanView full_view(fdst_ctx *h, bool df) {
  return PlanView{df ? &h->plan_df : &h->plan, &h->t1, &h->g, &h->t1_size, &h->g_size,
                  h->off, h->off, h->n_total, h->n_total, h->x2, h->y2};
}

// Adds the durations of the recorded compute-launch spans to ms_kernel (the stream
// has been synchronized) and releases their events.
static void resolve_kernel_events(fdst_ctx *h) {
  for (auto &k : h->kev) {
    float ms = 0.f;
    if (h->timing) cudaEventElapsedTime(&ms, k.first, k.second);
    h->ms_kernel += ms;
    cudaEventDestroy(k.first);
    cudaEventDestroy(k.second);
  }
  h->kev.clear();
}

static fdst_status run_plan_f64(fdst_ctx *h, const PlanView &V, const double *x, double *y, int nrhs,
                                const int *done, cudaStream_t st, bool timed) {
  // pack consecutive ops of a stage into launches with pairwise distinct outputs
  cudaEvent_t k0 = timed ? kernel_mark(h, st) : nullptr;
  int64_t nl = 0;
  size_t i = 0;
  const auto &P = *V.ops;
  while (i < P.size()) {
    BandGroup g;
    std::vector<std::pair<int, int>> outs;
    int stage = P[i].stage;
    while (i < P.size() && P[i].stage == stage && g.nop < kMaxGroup) {
      auto o = std::make_pair(P[i].out_kind, P[i].out_id);
      if (std::find(outs.begin(), outs.end(), o) != outs.end()) break;
      outs.push_back(o);
      const PlanOp &op = P[i];
      BandOp &b = g.op[g.nop++];
      const BandDev &bd = h->bands[op.band];
      b.vals = bd.vals; b.lo = bd.lo; b.w = bd.w; b.rows = bd.rows;
      b.d0 = op.dims[0]; b.d1 = op.dims[1]; b.d2 = op.dims[2]; b.mode = op.mode;
      b.coef = op.coef; b.accumulate = op.accumulate;
      if (op.in_kind == 0) { b.X = x + V.in_off[op.in_id]; b.x_rhs_stride = V.in_stride; }
      else if (op.in_kind == 1) { b.X = (*V.t1)[op.in_id]; b.x_rhs_stride = (*V.t1_size)[op.in_id]; }
      else { b.X = (*V.g)[op.in_id]; b.x_rhs_stride = (*V.g_size)[op.in_id]; }
      if (op.out_kind == 3) { b.Y = y + V.out_off[op.out_id]; b.y_rhs_stride = V.out_stride; }
      else if (op.out_kind == 1) { b.Y = (*V.t1)[op.out_id]; b.y_rhs_stride = (*V.t1_size)[op.out_id]; }
      else { b.Y = (*V.g)[op.out_id]; b.y_rhs_stride = (*V.g_size)[op.out_id]; }
      ++i;
    }
    launch_band(g, nrhs, done, st);
    ++nl;
  }
  kernel_span(h, k0, nl, st);
  CK(cudaGetLastError());
  return FDST_OK;
}

// Same plan in double-float arithmetic: the entries [in_lo, in_hi) of x split once
// into FP32 pairs, every banded mode product on the FP32 units, the entries
// [out_lo, out_hi) of the result joined back to FP64.
static fdst_status run_plan_df(fdst_ctx *h, const PlanView &V, const double *x, double *y, int nrhs,
                               const int *done, cudaStream_t st, int64_t in_lo, int64_t in_hi, int64_t out_lo,
                               int64_t out_hi, bool timed) {
  if (x) launch_split_df(x + in_lo, V.xw + in_lo, in_hi - in_lo, V.in_stride, nrhs, done, st);
  cudaEvent_t k0 = timed ? kernel_mark(h, st) : nullptr;
  int64_t nl = 0;
  size_t i = 0;
  const auto &P = *V.ops;
  // With an FP64 result requested, the last product into each result block writes
  // the joined FP64 value itself, so no separate join pass reads the pairs back.
  std::vector<int> last_writer(P.size(), 0);
  bool all_joined = y != nullptr;
  if (y) {
    std::map<int, size_t> last;
    for (size_t k = 0; k < P.size(); ++k)
      if (P[k].out_kind == 3) last[P[k].out_id] = k;
    for (auto &kv : last) last_writer[kv.second] = 1;
    for (int64_t b = 0; b < (int64_t)h->dim + 1 && all_joined; ++b)
      if (V.out_off[b] >= out_lo && V.out_off[b] < out_hi && !last.count((int)b)) all_joined = false;
  }
  while (i < P.size()) {
    BandGroupDF g;
    std::vector<std::pair<int, int>> outs;
    int stage = P[i].stage;
    const int width = h->bands[P[i].band].w;
    while (i < P.size() && P[i].stage == stage && g.nop < kMaxGroup && h->bands[P[i].band].w == width) {
      auto o = std::make_pair(P[i].out_kind, P[i].out_id);
      if (std::find(outs.begin(), outs.end(), o) != outs.end()) break;
      outs.push_back(o);
      const PlanOp &op = P[i];
      BandOpDF &b = g.op[g.nop++];
      const BandDev &bd = h->bands[op.band];
      b.vals = op.vals_df; b.lo = bd.lo; b.w = bd.w; b.rows = bd.rows;
      b.d0 = op.dims[0]; b.d1 = op.dims[1]; b.d2 = op.dims[2]; b.mode = op.mode;
      b.accumulate = op.accumulate;
      b.swap = op.swap;
      if (op.in_kind == 0) { b.X = V.xw + V.in_off[op.in_id]; b.x_rhs_stride = V.in_stride; }
      else if (op.in_kind == 1) { b.X = reinterpret_cast<const float2 *>((*V.t1)[op.in_id]); b.x_rhs_stride = (*V.t1_size)[op.in_id]; }
      else { b.X = reinterpret_cast<const float2 *>((*V.g)[op.in_id]); b.x_rhs_stride = (*V.g_size)[op.in_id]; }
      if (op.out_kind == 3) {
        b.Y = V.yw + V.out_off[op.out_id];
        b.y_rhs_stride = V.out_stride;
        if (all_joined && last_writer[i]) b.Y64 = y + V.out_off[op.out_id];
      }
      else if (op.out_kind == 1) { b.Y = reinterpret_cast<float2 *>((*V.t1)[op.out_id]); b.y_rhs_stride = (*V.t1_size)[op.out_id]; }
      else { b.Y = reinterpret_cast<float2 *>((*V.g)[op.out_id]); b.y_rhs_stride = (*V.g_size)[op.out_id]; }
      ++i;
    }
    launch_band_df(g, nrhs, done, st);
    ++nl;
  }
  kernel_span(h, k0, nl, st);
  if (y && !all_joined) launch_join_df(V.yw + out_lo, y + out_lo, out_hi - out_lo, V.out_stride, nrhs, done, st);
  CK(cudaGetLastError());
  return FDST_OK;
}

// The B^T and B parts of the sum-factorized operator (built on first use):
// B^T: pressure -> P -> fluxes of sigma = -P I -> velocity; B: velocity -> G -> E -> pressure.
static fdst_status mf_build_parts(fdst_ctx *h) {
  if (h->mf_parts) return FDST_OK;
  const GeoPoints &gp = h->gp;
  const std::array<int, 3> pts{gp.nq[0], gp.nq[1], gp.nq[2]};
  std::vector<std::array<int, 3>> shapes(10, pts);
  for (int part = 0; part < 2; ++part) {
    auto &P = part == 0 ? h->mf_bt : h->mf_b;
    std::vector<Term> f, b;
    for (const Term &t : h->mf_fwd_terms)
      if ((part == 0) == (t.src == 3)) f.push_back(t);
    for (const Term &t : h->mf_bwd_terms)
      if ((part == 0) == (t.dst < 3)) b.push_back(t);
    TRY(build_plan(h, f, P.fwd, P.fwd_df, P.fwd_t1s, P.fwd_gs, nullptr, 10));
    TRY(build_plan(h, b, P.bwd, P.bwd_df, P.bwd_t1s, P.bwd_gs, &shapes, 4));
    TRY(alloc_plan_buffers(h, P.fwd_t1s, P.fwd_gs, P.fwd_t1, P.fwd_g));
    TRY(alloc_plan_buffers(h, P.bwd_t1s, P.bwd_gs, P.bwd_t1, P.bwd_g));
  }
  h->mf_parts = true;
  return FDST_OK;
}

// y = A x (which = 0), y_u = B^T x_p (1) or y_p = B x_u (2) by sum factorization, in
// double-float (fields kept as FP32 pairs between the stages) or FP64.
static fdst_status run_matvec_mf(fdst_ctx *h, const double *x, double *y, int nrhs, const int *done,
                                 cudaStream_t st, bool df, int which = 0) {
  const int64_t fs = 10 * h->mf_Q, n = h->n_total, nv = h->off[3];
  if (which) TRY(mf_build_parts(h));
  const auto *P = which == 1 ? &h->mf_bt : which == 2 ? &h->mf_b : nullptr;
  const auto &fo = P ? (df ? P->fwd_df : P->fwd) : (df ? h->mf_fwd_df : h->mf_fwd);
  const auto &bo = P ? (df ? P->bwd_df : P->bwd) : (df ? h->mf_bwd_df : h->mf_bwd);
  const auto &ft1 = P ? P->fwd_t1 : h->mf_fwd_t1, &fg = P ? P->fwd_g : h->mf_fwd_g;
  const auto &bt1 = P ? P->bwd_t1 : h->mf_bwd_t1, &bg = P ? P->bwd_g : h->mf_bwd_g;
  const auto &ft1s = P ? P->fwd_t1s : h->mf_fwd_t1s, &fgs = P ? P->fwd_gs : h->mf_fwd_gs;
  const auto &bt1s = P ? P->bwd_t1s : h->mf_bwd_t1s, &bgs = P ? P->bwd_gs : h->mf_bwd_gs;
  // entries read and written: all (operator), pressure -> velocity (B^T), velocity -> pressure (B)
  const int64_t in_lo = which == 1 ? nv : 0, in_hi = which == 2 ? nv : n;
  const int64_t out_lo = which == 2 ? nv : 0, out_hi = which == 1 ? nv : n;
  const bool timed = which == 0;
  if (df) {
    const PlanView Vf{&fo, &ft1, &fg, &ft1s, &fgs, h->off, h->mf_foff, n, fs, h->x2, h->mf_Fw};
    const PlanView Vb{&bo, &bt1, &bg, &bt1s, &bgs, h->mf_foff, h->off, fs, n, h->mf_Fw, h->y2};
    TRY(run_plan_df(h, Vf, x, nullptr, nrhs, done, st, in_lo, in_hi, 0, 0, timed));
    launch_mf_points_df(h->mf_Fw, h->mf_Q, fs, nrhs, h->mf_jd, h->mf_wd, h->mf_nu, done, which, st);
    TRY(run_plan_df(h, Vb, nullptr, y, nrhs, done, st, 0, 0, out_lo, out_hi, timed));
  } else {
    const PlanView Vf{&fo, &ft1, &fg, &ft1s, &fgs, h->off, h->mf_foff, n, fs, nullptr, nullptr};
    const PlanView Vb{&bo, &bt1, &bg, &bt1s, &bgs, h->mf_foff, h->off, fs, n, nullptr, nullptr};
    TRY(run_plan_f64(h, Vf, x, h->mf_F, nrhs, done, st, timed));
    launch_mf_points_f64(h->mf_F, h->mf_Q, fs, nrhs, h->gp, done, which, st);
    TRY(run_plan_f64(h, Vb, h->mf_F, y, nrhs, done, st, timed));
  }
  CK(cudaGetLastError());
  return FDST_OK;
}

int resume_action(const MinresState &S, double true_rel, double prev_true, int restarts, double tol, int maxit) {
  if (!(S.status == 0 && S.stop && S.gamma > 0.0 && true_rel > tol && S.iters < maxit)) return kKeepStopped;
  if (prev_true < 0.0 && 0.5 * S.tau * tol / true_rel >= kTauFloor) return kResume;
  return restarts < kMaxRestarts ? kRestart : kStagnated;
}

fdst_status minres_restart(fdst_ctx *h, const double *b, double *x, int nrhs, const std::vector<int> &which,
                           const std::vector<double> &true_rel, double tol, std::vector<MinresState> &hs,
                           cudaStream_t st, double *const *vecs) {
  const int64_t n = h->n_total;
  double *v = vecs ? vecs[0] : h->v, *v_old = vecs ? vecs[1] : h->v_old;
  double *w = vecs ? vecs[2] : h->w, *w_old = vecs ? vecs[3] : h->w_old;
  std::vector<int> mask(nrhs, 1);
  for (int j : which) mask[j] = 0;
  CK(cudaMemcpyAsync(h->done, mask.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  TRY(run_matvec(h, x, h->Az, nrhs, h->done, st, true));
  launch_restart_vectors(b, h->Az, v, v_old, w, w_old, n, n, nrhs, h->done, st);
  TRY(run_apply(h, v, h->z, nrhs, h->done, st));
  launch_dot(v, h->z, n, n, nrhs, h->partials, h->counters, h->dots, h->done, st);
  std::vector<double> g(nrhs);
  CK(cudaMemcpyAsync(g.data(), h->dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int j : which) {
    MinresState &S = hs[j];
    if (!(g[j] > 0.0) || std::isinf(g[j])) {
      S.status = std::isnan(g[j]) || std::isinf(g[j]) ? FDST_NAN_DETECTED : FDST_BREAKDOWN;
      S.stop = 1;
      mask[j] = 1;
      continue;
    }
    const double gamma = std::sqrt(g[j]);
    S.gamma = gamma;
    S.gamma_old = 1.0;
    S.c = S.c_old = 1.0;
    S.s = S.s_old = 0.0;
    S.eta = gamma;
    S.inv_gamma_new = 1.0 / gamma;
    S.tau = std::max(kTauFloor, 0.5 * (S.eta0 > 0.0 ? gamma / S.eta0 : 1.0) * tol / true_rel[j]);
    S.stop = 0;
    S.status = 0;
  }
  CK(cudaMemcpyAsync(h->state, hs.data(), sizeof(MinresState) * nrhs, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->done, mask.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  launch_scale_by_inv_gamma(h->z, h->state, n, n, nrhs, h->done, st);
  CK(cudaStreamSynchronize(st));
  return FDST_OK;
}

// exact = true forces the FP64 (DFMA) evaluation (true-residual checks).
fdst_status run_matvec(fdst_ctx *h, const double *x, double *y, int nrhs, const int *done, cudaStream_t st,
                       bool exact) {
  if (h->mapped && h->mf)
    return run_matvec_mf(h, x, y, nrhs, done, st, !exact && h->desc.matvec_precision == FDST_MV_DF64);
  if (h->mapped) {
    if (!exact && h->csr.val_df) {
      launch_split_df(x, h->x2, h->n_total, h->n_total, nrhs, done, st);
      cudaEvent_t k0 = kernel_mark(h, st);
      launch_spmv_df(h->csr, h->x2, y, h->n_total, nrhs, done, st);
      kernel_span(h, k0, 1, st);
    } else {
      cudaEvent_t k0 = exact ? nullptr : kernel_mark(h, st);
      launch_spmv(h->csr, x, y, h->n_total, nrhs, done, st);
      kernel_span(h, k0, 1, st);
    }
    CK(cudaGetLastError());
    return FDST_OK;
  }
  if (!exact && h->desc.matvec_precision == FDST_MV_DF64)
    return run_plan_df(h, full_view(h, true), x, y, nrhs, done, st, 0, h->n_total, 0, h->n_total, true);
  return run_plan_f64(h, full_view(h, false), x, y, nrhs, done, st, !exact);
}

// ------------------------------------------------------------------ P_T, P_C and GMRES workspace

// The B and B^T parts of the operator as plans of their own (built on first use),
// the GMRES work vectors and a Krylov basis of cap + 1 block vectors.
static void release(fdst_ctx *h, double *&p, size_t count) {
  if (!p) return;
  cudaFree(p);
  h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), (void *)p));
  h->device_bytes -= (int64_t)(count * sizeof(double));
  p = nullptr;
}

static fdst_status ensure_gmres(fdst_ctx *h, int cap, bool flexible) {
  if (!h->gm_w && h->mapped && !h->mf) TRY(build_coupling_csr(h));
  if (!h->gm_w && !h->mapped) {
    std::vector<Term> tb, tbt;
    for (const Term &t : h->terms) {
      if (t.dst == h->dim) tb.push_back(t);
      else if (t.src == h->dim) tbt.push_back(t);
    }
    auto &B = h->plan_b, &Bt = h->plan_bt;
    TRY(build_plan(h, tb, B.ops, B.ops_df, B.t1_size, B.g_size));
    TRY(alloc_plan_buffers(h, B.t1_size, B.g_size, B.t1, B.g));
    TRY(build_plan(h, tbt, Bt.ops, Bt.ops_df, Bt.t1_size, Bt.g_size));
    TRY(alloc_plan_buffers(h, Bt.t1_size, Bt.g_size, Bt.t1, Bt.g));
  }
  if (!h->gm_w) {
    const size_t nv = (size_t)h->n_total * h->max_rhs;
    TRY(dalloc(h, &h->gm_t, nv));
    TRY(dalloc(h, &h->gm_u, nv));
    TRY(dalloc(h, &h->gm_part, (size_t)8 * 304 * h->max_rhs));
    TRY(dalloc(h, &h->gm_scal, (size_t)4 * h->max_rhs));
    TRY(dalloc(h, &h->gm_mask, (size_t)h->max_rhs));
    TRY(dalloc(h, &h->gm_w, nv));
  }
  const size_t nv = (size_t)h->n_total * h->max_rhs;
  if (cap > h->gm_cap) {
    release(h, h->gm_V, (size_t)(h->gm_cap + 1) * nv);
    release(h, h->gm_coef, (size_t)3 * (h->gm_cap + 1) * h->max_rhs);
    h->gm_cap = 0;
    TRY(dalloc(h, &h->gm_V, (size_t)(cap + 1) * nv));
    TRY(dalloc(h, &h->gm_coef, (size_t)3 * (cap + 1) * h->max_rhs));
    h->gm_cap = cap;
  }
  if (flexible && cap > h->gm_zcap) {
    release(h, h->gm_Z, (size_t)h->gm_zcap * nv);
    h->gm_zcap = 0;
    TRY(dalloc(h, &h->gm_Z, (size_t)cap * nv));
    h->gm_zcap = cap;
  }
  return FDST_OK;
}

// y[velocity blocks] = B^T x[pressure block]; y[pressure block] = B x[velocity blocks]
// (the iterations' matvec arithmetic).
static fdst_status apply_coupling(fdst_ctx *h, bool transpose, const double *x, double *y, int nrhs,
                                  const int *done, cudaStream_t st) {
  const bool df = h->desc.matvec_precision == FDST_MV_DF64;
  if (h->mapped && h->mf) return run_matvec_mf(h, x, y, nrhs, done, st, df, transpose ? 1 : 2);
  if (h->mapped) {
    const CsrDev &C = transpose ? h->csr_bt : h->csr_b;
    const int64_t nv = h->off[h->dim], n = h->n_total;
    const int64_t in_lo = transpose ? nv : 0, in_hi = transpose ? n : nv, out_lo = transpose ? 0 : nv;
    if (df && C.val_df) {
      launch_split_df(x + in_lo, h->x2 + in_lo, in_hi - in_lo, n, nrhs, done, st);
      launch_spmv_df(C, h->x2, y + out_lo, n, nrhs, done, st);
    } else {
      launch_spmv(C, x, y + out_lo, n, nrhs, done, st);
    }
    CK(cudaGetLastError());
    return FDST_OK;
  }
  const auto &S = transpose ? h->plan_bt : h->plan_b;
  const PlanView V{df ? &S.ops_df : &S.ops, &S.t1, &S.g, &S.t1_size, &S.g_size, h->off, h->off, h->n_total,
                   h->n_total, h->x2, h->y2};
  const int64_t nv = h->off[h->dim], n = h->n_total;
  if (df)
    return transpose ? run_plan_df(h, V, x, y, nrhs, done, st, nv, n, 0, nv, false)
                     : run_plan_df(h, V, x, y, nrhs, done, st, 0, nv, nv, n, false);
  return run_plan_f64(h, V, x, y, nrhs, done, st, false);
}

// s = P^{-1} r for the block triangular P_T = [[P_V, B^T], [0, -P_Q]] (back
// substitution) or the constraint P_C = [[P_V, B^T], [B, B P_V^{-1} B^T - P_Q]]
// (the paper's product form of P_C^{-1}); P_V^{-1}, P_Q^{-1} are the FD applies.
static fdst_status apply_block_prec(fdst_ctx *h, int kind, const double *r, double *s, int nrhs, const int *done,
                                    cudaStream_t st) {
  const int dim = h->dim;
  const int64_t n = h->n_total, nv = h->off[dim], nq = n - nv;
  const unsigned vel = (1u << dim) - 1u, pres = 1u << dim;
  double *t = h->gm_t, *u = h->gm_u;
  if (kind == FDST_PREC_PT) {
    TRY(run_apply(h, r, s, nrhs, done, st, pres));             // s_q = P_Q^{-1} r_q (q = -s_q)
    TRY(apply_coupling(h, true, s, t, nrhs, done, st));        // t_u = B^T s_q
    launch_axpby(r, t, 1.0, 1.0, nv, n, nrhs, st);             // t_u = r_u - B^T q
    TRY(run_apply(h, t, s, nrhs, done, st, vel));              // s_u = P_V^{-1} t_u
  } else {
    TRY(run_apply(h, r, s, nrhs, done, st, vel));              // z = P_V^{-1} r_u in s_u
    TRY(apply_coupling(h, false, s, t, nrhs, done, st));       // t_q = B z
    launch_axpby(r + nv, t + nv, 1.0, -1.0, nq, n, nrhs, st);  // t_q = r_q - B z
    TRY(run_apply(h, t, s, nrhs, done, st, pres));             // s_q = P_Q^{-1} t_q (q = -s_q)
    TRY(apply_coupling(h, true, s, u, nrhs, done, st));        // u_u = B^T s_q = -B^T q
    TRY(run_apply(h, u, t, nrhs, done, st, vel));              // t_u = P_V^{-1} u_u
    launch_axpby(t, s, 1.0, 1.0, nv, n, nrhs, st);             // s_u = z - P_V^{-1} B^T q
  }
  launch_axpby(s + nv, s + nv, 0.0, -1.0, nq, n, nrhs, st);    // q = -s_q
  CK(cudaGetLastError());
  return FDST_OK;
}

// D_V of P_D^G for a matrix-free handle: diag(A) by sum factorization (the squared
// point-basis bands tested against the 18 coefficient fields of launch_mf_diag_coef).
static fdst_status mf_velocity_scaling(fdst_ctx *h) {
  const GeoPoints &gp = h->gp;
  const std::array<int, 3> pts{gp.nq[0], gp.nq[1], gp.nq[2]};
  // diag(A) by sum factorization: the squared point-basis bands tested against the
  // 18 coefficient fields of launch_mf_diag_coef, for D_V of P_D^G
  int sq[3][3];   // [d][0: B.B, 1: B.D, 2: D.D], transposed (functions x points)
  for (int d = 0; d < 3; ++d) {
    const BandDev &B = h->bands[h->mf_bv[d]], &D = h->bands[h->mf_dv[d]];
    const int nr = B.rows, nc = B.cols;
    Mat bb(nc, nr), bd(nc, nr), dd(nc, nr);
    std::vector<double> Bd((size_t)nr * nc, 0.0), Dd((size_t)nr * nc, 0.0);
    std::vector<int> blo(nr), dlo(nr);
    CK(cudaMemcpy(blo.data(), B.lo, sizeof(int) * nr, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(dlo.data(), D.lo, sizeof(int) * nr, cudaMemcpyDeviceToHost));
    for (int i = 0; i < nr; ++i) {
      for (int j = 0; j < B.w; ++j) Bd[(size_t)i * nc + blo[i] + j] = B.hvals[(size_t)i * B.w + j];
      for (int j = 0; j < D.w; ++j) Dd[(size_t)i * nc + dlo[i] + j] = D.hvals[(size_t)i * D.w + j];
    }
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nc; ++j) {
        const double b = Bd[(size_t)i * nc + j], e = Dd[(size_t)i * nc + j];
        bb(j, i) = b * b;
        bd(j, i) = b * e;
        dd(j, i) = e * e;
      }
    TRY(band_from_mat(h, bb, &sq[d][0]));
    TRY(band_from_mat(h, bd, &sq[d][1]));
    TRY(band_from_mat(h, dd, &sq[d][2]));
  }
  std::vector<Term> dterms;
  for (int r = 0; r < 3; ++r) {
    int pi = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b, ++pi) {
        Term t{r, 6 * r + pi, 1.0, {-1, -1, -1}};
        for (int d = 0; d < 3; ++d) t.f[d] = sq[d][(d == a) + (d == b)];
        dterms.push_back(t);
      }
  }
  std::vector<std::array<int, 3>> dshapes(18, pts);
  std::vector<PlanOp> dops, dops_df;
  std::vector<int64_t> dt1s, dgs;
  std::vector<double *> dt1, dg;
  TRY(build_plan(h, dterms, dops, dops_df, dt1s, dgs, &dshapes, 4));
  TRY(alloc_plan_buffers(h, dt1s, dgs, dt1, dg));
  double *C = nullptr, *dA = nullptr;
  TRY(dalloc(h, &C, (size_t)18 * gp.Q));
  TRY(dalloc(h, &dA, (size_t)h->n_total));
  launch_mf_diag_coef(C, gp, 0);
  int64_t coff[18];
  for (int f = 0; f < 18; ++f) coff[f] = f * gp.Q;
  const PlanView V{&dops, &dt1, &dg, &dt1s, &dgs, coff, h->off, 18 * gp.Q, h->n_total, nullptr, nullptr};
  TRY(run_plan_f64(h, V, C, dA, 1, nullptr, 0, false));
  std::vector<double> diagA((size_t)h->n_total);
  CK(cudaMemcpy(diagA.data(), dA, sizeof(double) * h->off[3], cudaMemcpyDeviceToHost));
  set_velocity_scaling(h, diagA);
  // the coefficient fields and the diagonal plan's buffers are not needed again
  release(h, C, (size_t)18 * gp.Q);
  release(h, dA, (size_t)h->n_total);
  for (size_t k = 0; k < dt1.size(); ++k) release(h, dt1[k], (size_t)dt1s[k] * h->max_rhs);
  for (size_t k = 0; k < dg.size(); ++k) release(h, dg[k], (size_t)dgs[k] * h->max_rhs);
  return FDST_OK;
}

}  // namespace fdst

using namespace fdst;

extern "C" {

const char *fdst_last_error(void) { return g_err.c_str(); }

int64_t fdst_kernel_launches(void) { return (int64_t)launch_count(); }

fdst_status fdst_convert(int kind, const void *d_in, void *d_out, int64_t n, fdst_stream stream) {
  if (kind < 0 || kind > 3 || n < 0 || (n > 0 && (!d_in || !d_out))) {
    set_error("fdst_convert: kind in 0..3, n >= 0 and device buffers required");
    return FDST_INVALID_ARGUMENT;
  }
  if (n == 0) return FDST_OK;
  launch_convert(kind, d_in, d_out, n, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return FDST_OK;
}

fdst_status fdst_check_bounded_wait(int *gave_up, double *seconds) {
  if (!gave_up || !seconds) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  TRY(tc_wait_selftest(gave_up, seconds));
  if (*gave_up) {
    set_error("bounded device-side wait expired (self-test: expected)");
    return FDST_TIMEOUT;
  }
  return FDST_OK;
}

}  // extern "C"

namespace fdst {
static std::atomic<int64_t> g_alloc_countdown{0};
static std::atomic<int> g_alloc_status{FDST_OUT_OF_MEMORY};

fdst_status injected_alloc_failure() {
  int64_t c = g_alloc_countdown.load();
  while (c > 0)
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1 ? (fdst_status)g_alloc_status.load() : FDST_OK;
  return FDST_OK;
}
}  // namespace fdst

extern "C" {

fdst_status fdst_inject_alloc_failure(int64_t nth, int status) {
  if (status != FDST_OUT_OF_MEMORY && status != FDST_CUDA_ERROR) {
    set_error("fdst_inject_alloc_failure: status must be FDST_OUT_OF_MEMORY or FDST_CUDA_ERROR");
    return FDST_INVALID_ARGUMENT;
  }
  fdst::g_alloc_status.store(status);
  fdst::g_alloc_countdown.store(nth > 0 ? nth : 0);
  return FDST_OK;
}

fdst_status fdst_device_error(int *flag) {
  if (!flag) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  return tc_error_flag(flag);
}

fdst_status fdst_destroy(fdst_handle h) {
  if (!h) return FDST_OK;
  for (auto &k : h->kev) {
    cudaEventDestroy(k.first);
    cudaEventDestroy(k.second);
  }
  for (void *p : h->allocs) cudaFree(p);
  if (h->h_n_stopped) cudaFreeHost(h->h_n_stopped);
  if (h->h_dots) cudaFreeHost(h->h_dots);
  delete h;
  return FDST_OK;
}

fdst_status fdst_setup(const fdst_desc *desc, fdst_handle *out) {
  if (!out) { set_error("out is NULL"); return FDST_INVALID_ARGUMENT; }
  *out = nullptr;
  if (!desc) { set_error("desc is NULL"); return FDST_INVALID_ARGUMENT; }
  if (desc->dim != 2 && desc->dim != 3) { set_error("dim must be 2 or 3"); return FDST_INVALID_ARGUMENT; }
  if (desc->discretization != FDST_TH && desc->discretization != FDST_RT) {
    set_error("unknown discretization");
    return FDST_INVALID_ARGUMENT;
  }
  if (desc->degree < 1 || desc->degree > 12) { set_error("degree must be in [1, 12]"); return FDST_INVALID_ARGUMENT; }
  if (desc->max_rhs < 1) { set_error("max_rhs must be >= 1"); return FDST_INVALID_ARGUMENT; }
  if (desc->geometry != FDST_GEOM_IDENTITY && desc->geometry != FDST_GEOM_SINE_BUMP &&
      desc->geometry != FDST_GEOM_ANNULUS) {
    set_error("unknown geometry");
    return FDST_INVALID_ARGUMENT;
  }
  if (desc->variant != FDST_VARIANT_PD && desc->variant != FDST_VARIANT_PD_GEO) {
    set_error("unknown preconditioner variant");
    return FDST_INVALID_ARGUMENT;
  }
  if (desc->geometry == FDST_GEOM_IDENTITY && desc->viscosity_contrast > 0.0) {
    if (desc->viscosity_contrast < 1.0) {
      set_error("viscosity_contrast must be >= 1 (or <= 0 for a constant viscosity)");
      return FDST_INVALID_ARGUMENT;
    }
    if (desc->dim != 3) {
      set_error("the viscosity family on the identity map is built in 3D");
      return FDST_NOT_SUPPORTED;
    }
  }
  if (desc->variant == FDST_VARIANT_PD_GEO && desc->geometry == FDST_GEOM_IDENTITY &&
      !(desc->viscosity_contrast >= 1.0)) {
    set_error("P_D^G on the identity map needs the viscosity family (viscosity_contrast >= 1); "
              "with a constant viscosity it equals P_D");
    return FDST_NOT_SUPPORTED;
  }
  if (desc->matvec_form != FDST_MATVEC_ASSEMBLED && desc->matvec_form != FDST_MATVEC_MATRIX_FREE) {
    set_error("unknown matvec form");
    return FDST_INVALID_ARGUMENT;
  }
  if (desc->matvec_precision != FDST_MV_F64 && desc->matvec_precision != FDST_MV_DF64) {
    set_error("unknown matvec precision");
    return FDST_INVALID_ARGUMENT;
  }
  if (desc->fd_precision != FDST_FD_F64 && desc->fd_precision != FDST_FD_TF32X3 &&
      desc->fd_precision != FDST_FD_BF16X6) {
    set_error("unknown FD precision");
    return FDST_INVALID_ARGUMENT;
  }
  std::unique_ptr<fdst_ctx> h(new fdst_ctx());
  h->desc = *desc;
  h->dim = desc->dim;
  h->p = desc->degree;
  h->max_rhs = desc->max_rhs;
  for (int e = 0; e < h->dim; ++e) {
    if (!desc->h_knots[e] || desc->nknots[e] <= 0) { set_error("missing knot vector"); return FDST_INVALID_ARGUMENT; }
    std::vector<double> t(desc->h_knots[e], desc->h_knots[e] + desc->nknots[e]);
    std::string msg = validate_knots(t, h->p);
    if (!msg.empty()) { set_error("direction " + std::to_string(e + 1) + ": " + msg); return FDST_INVALID_ARGUMENT; }
    h->knots.push_back(t);
  }
  for (int e = h->dim; e < 3; ++e) h->desc.h_knots[e] = nullptr;
  for (int e = 0; e < 3; ++e) h->desc.h_knots[e] = nullptr;   // not kept: the caller owns them
  fdst_ctx *hp = h.get();
  fdst_status st;
  auto fail = [&](fdst_status s) { fdst_destroy(h.release()); return s; };
  if ((st = build_spaces(hp)) != FDST_OK) return fail(st);
  if (desc->geometry != FDST_GEOM_IDENTITY && (st = build_mapped_pre(hp)) != FDST_OK) return fail(st);
  if (!hp->mapped && (st = build_matvec(hp)) != FDST_OK) return fail(st);
  if (desc->geometry == FDST_GEOM_IDENTITY && desc->variant == FDST_VARIANT_PD_GEO &&
      (st = build_identity_geo(hp)) != FDST_OK)
    return fail(st);
  if (hp->mapped && desc->matvec_form == FDST_MATVEC_MATRIX_FREE) {
    if ((st = build_matrix_free(hp)) != FDST_OK) return fail(st);
    if (desc->variant == FDST_VARIANT_PD_GEO && (st = mf_velocity_scaling(hp)) != FDST_OK) return fail(st);
  }
  if ((st = build_fd(hp)) != FDST_OK) return fail(st);
  if ((hp->mapped || desc->variant == FDST_VARIANT_PD_GEO) && (st = build_mapped_post(hp)) != FDST_OK)
    return fail(st);
  if (desc->fd_precision != FDST_FD_F64) {
    if ((st = tc_prepare(hp)) != FDST_OK) return fail(st);
  }
  const size_t nv = (size_t)hp->n_total * hp->max_rhs;
  if ((st = dalloc(hp, &hp->work[0], nv)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->work[1], nv)) != FDST_OK) return fail(st);
  double **vecs[] = {&hp->v, &hp->v_old, &hp->z, &hp->z_new, &hp->Az, &hp->w, &hp->w_old};
  for (double **pv : vecs)
    if ((st = dalloc(hp, pv, nv)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->partials, (size_t)304 * hp->max_rhs)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->dots, (size_t)4 * hp->max_rhs)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->counters, (size_t)hp->max_rhs)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->state, (size_t)hp->max_rhs)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->done, (size_t)hp->max_rhs)) != FDST_OK) return fail(st);
  if ((st = dalloc(hp, &hp->n_stopped, 1)) != FDST_OK) return fail(st);
  if (cudaMemset(hp->counters, 0, sizeof(unsigned) * hp->max_rhs) != cudaSuccess ||
      cudaMallocHost((void **)&hp->h_n_stopped, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void **)&hp->h_dots, sizeof(double) * 4 * hp->max_rhs) != cudaSuccess) {
    set_error("pinned host allocation failed");
    return fail(FDST_CUDA_ERROR);
  }
  // Setup work runs on the legacy default stream only; waiting on it (not on
  // the whole device) lets a handle be set up while other streams compute.
  if (cudaStreamSynchronize(0) != cudaSuccess) {
    set_error(std::string("setup: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(FDST_CUDA_ERROR);
  }
  *out = h.release();
  return FDST_OK;
}

fdst_status fdst_get_sizes(fdst_handle h, fdst_sizes *out) {
  if (!h || !out) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  std::memset(out, 0, sizeof(*out));
  out->dim = h->dim;
  out->n_total = h->n_total;
  out->nblocks = h->nblocks;
  for (int b = 0; b < h->nblocks; ++b) {
    out->block_offset[b] = h->off[b];
    for (int e = 0; e < 3; ++e) out->block_shape[b][e] = h->shape[b][e];
  }
  out->device_bytes = h->device_bytes;
  double fa = 0.0;
  for (auto &c : h->chains) {
    double sum_n = 0.0;
    for (int j = 0; j < c.nsteps; ++j) sum_n += c.N[j];
    fa += 2.0 * (double)c.size * sum_n;   // each step: 2 K N R flops with K = N = n_d, R N = size
  }
  out->flops_apply = fa;
  // matvec flops: 2 x nonzeros of the CSR, or 2 x (band entries used) over the banded
  // products of the Kronecker plan or of the matrix-free plans (their point stage not counted)
  double fm = h->mapped && !h->mf ? 2.0 * (double)h->csr.nnz : 0.0;
  auto add_plan = [&](const std::vector<PlanOp> &P) {
    for (auto &op : P) {
      int od[3] = {op.dims[0], op.dims[1], op.dims[2]};
      od[op.mode] = h->bands[op.band].rows;
      fm += 2.0 * h->bands[op.band].w * (double)od[0] * od[1] * od[2];
    }
  };
  add_plan(h->plan);
  add_plan(h->mf_fwd);
  add_plan(h->mf_bwd);
  out->flops_matvec = fm;
  return FDST_OK;
}

fdst_status fdst_apply_prec(fdst_handle h, const double *d_r, double *d_s, int nrhs, fdst_stream stream) {
  if (!h || !d_r || !d_s) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  if (d_r == d_s) { set_error("r and s alias"); return FDST_INVALID_ARGUMENT; }
  return run_apply(h, d_r, d_s, nrhs, nullptr, (cudaStream_t)stream);
}

fdst_status fdst_matvec(fdst_handle h, const double *d_x, double *d_y, int nrhs, fdst_stream stream) {
  if (!h || !d_x || !d_y) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  if (d_x == d_y) { set_error("x and y alias"); return FDST_INVALID_ARGUMENT; }
  return run_matvec(h, d_x, d_y, nrhs, nullptr, (cudaStream_t)stream, false);
}

fdst_status fdst_set_timing(fdst_handle h, int on) {
  if (!h) { set_error("NULL handle"); return FDST_INVALID_ARGUMENT; }
  h->timing = on;
  h->ms_matvec = h->ms_prec = h->ms_vector = 0;
  h->n_matvec = h->n_prec = 0;
  h->ms_kernel = 0;
  h->n_kernel = 0;
  return FDST_OK;
}

fdst_status fdst_get_kernel_timing(fdst_handle h, double *ms, int64_t *launches) {
  if (!h) { set_error("NULL handle"); return FDST_INVALID_ARGUMENT; }
  if (ms) *ms = h->ms_kernel;
  if (launches) *launches = h->n_kernel;
  return FDST_OK;
}

fdst_status fdst_get_timing(fdst_handle h, double *ms_matvec, double *ms_prec, double *ms_vector, int64_t *n_matvec,
                            int64_t *n_prec) {
  if (!h) { set_error("NULL handle"); return FDST_INVALID_ARGUMENT; }
  if (ms_matvec) *ms_matvec = h->ms_matvec;
  if (ms_prec) *ms_prec = h->ms_prec;
  if (ms_vector) *ms_vector = h->ms_vector;
  if (n_matvec) *n_matvec = h->n_matvec;
  if (n_prec) *n_prec = h->n_prec;
  return FDST_OK;
}

fdst_status fdst_apply_block_prec(fdst_handle h, int prec, const double *d_r, double *d_s, int nrhs,
                                  fdst_stream stream) {
  if (!h || !d_r || !d_s) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (d_r == d_s) { set_error("r and s must not alias"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  if (prec != FDST_PREC_PT && prec != FDST_PREC_PC) { set_error("prec must be FDST_PREC_PT or FDST_PREC_PC");
    return FDST_INVALID_ARGUMENT; }
  TRY(ensure_gmres(h, 1, false));
  return apply_block_prec(h, prec, d_r, d_s, nrhs, nullptr, (cudaStream_t)stream);
}

// A bounded wait inside a tensor-core contraction that expired during a solve
// (the kernel then skipped its output) makes every right-hand side of the solve
// FDST_TIMEOUT: its iterates are not trustworthy.
static fdst_status timeout_check(int err0, fdst_solve_info *info, int nrhs, fdst_status ret) {
  int err1 = err0;
  TRY(tc_error_count(&err1));
  if (err1 == err0) return ret;
  for (int j = 0; j < nrhs; ++j) info[j].status = FDST_TIMEOUT;
  set_error("a bounded device-side wait in the tensor-core FD contraction expired during the solve");
  return FDST_TIMEOUT;
}

fdst_status fdst_solve_gmres(fdst_handle h, int prec, int form, const double *d_b, double *d_x, int nrhs,
                             double tol, int maxit, int restart, fdst_solve_info *info, fdst_stream stream) {
  if (!h || !d_b || !d_x || !info) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  if (!(tol >= 0.0) || maxit < 1) { set_error("tol must be >= 0 and maxit >= 1"); return FDST_INVALID_ARGUMENT; }
  if (prec != FDST_PREC_PT && prec != FDST_PREC_PC) { set_error("prec must be FDST_PREC_PT or FDST_PREC_PC");
    return FDST_INVALID_ARGUMENT; }
  if (restart < 1 || restart > 255) { set_error("restart must be in [1, 255]"); return FDST_INVALID_ARGUMENT; }
  if (form != FDST_GMRES_LEFT && form != FDST_GMRES_FLEXIBLE && form != FDST_GMRES_AUTO) {
    set_error("form must be FDST_GMRES_LEFT, FDST_GMRES_FLEXIBLE or FDST_GMRES_AUTO");
    return FDST_INVALID_ARGUMENT;
  }
  const bool flex = form == FDST_GMRES_FLEXIBLE || (form == FDST_GMRES_AUTO && h->desc.fd_precision != FDST_FD_F64);
  TRY(ensure_gmres(h, restart, flex));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->n_total;
  const int m = restart, ld = m + 1;
  const int64_t vstride = n * h->max_rhs;    // basis vector k at V + k * vstride, right-hand side r at + r * n
  double *V = h->gm_V, *Z = h->gm_Z, *w = h->gm_w, *u = h->gm_u;
  double *X = flex ? Z : V;   // the basis the iterate is formed from
  double *c1 = h->gm_coef, *c2 = h->gm_coef + (size_t)ld * h->max_rhs, *cy = h->gm_coef + (size_t)2 * ld * h->max_rhs;
  std::vector<double> H((size_t)nrhs * ld * m, 0.0), cs((size_t)nrhs * m), sn((size_t)nrhs * m), g((size_t)nrhs * ld);
  std::vector<double> bn(nrhs), bref(nrhs), tau(nrhs, tol), est(nrhs, 1.0), true_rel(nrhs, -1.0);
  std::vector<double> hc1((size_t)nrhs * ld), hc2((size_t)nrhs * ld), hy((size_t)nrhs * ld), hs(nrhs);
  std::vector<int> iters(nrhs, 0), done(nrhs, 0), status(nrhs, FDST_MAXIT), est_it(nrhs, -1);
  auto sync_done = [&](const std::vector<int> &mask, int *dst) -> fdst_status {
    CK(cudaMemcpyAsync(dst, mask.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    return FDST_OK;
  };
  auto norms2 = [&](const double *a, const int *skip) -> fdst_status {   // hs[r] = <a_r, a_r>
    launch_dot(a, a, n, n, nrhs, h->partials, h->counters, h->dots, skip, st);
    CK(cudaMemcpyAsync(hs.data(), h->dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return FDST_OK;
  };
  // ||b|| and the estimate's reference: ||P^{-1} b|| (left) or ||b|| (flexible)
  TRY(norms2(d_b, nullptr));
  for (int r = 0; r < nrhs; ++r) bn[r] = std::sqrt(hs[r]);
  if (!flex) {
    TRY(apply_block_prec(h, prec, d_b, w, nrhs, nullptr, st));
    TRY(norms2(w, nullptr));
  }
  for (int r = 0; r < nrhs; ++r) {
    bref[r] = std::sqrt(hs[r]);
    if (bn[r] == 0.0 || bref[r] == 0.0) { done[r] = 1; status[r] = FDST_OK; est[r] = 0.0; true_rel[r] = 0.0; }
  }
  for (int r = 0; r < nrhs; ++r)
    if (bn[r] == 0.0) CK(cudaMemsetAsync(d_x + (size_t)r * n, 0, sizeof(double) * n, st));
  TRY(sync_done(done, h->done));
  // x0 = 0 (the paper's start) is detected on the device: the first cycle's residual
  // is then b itself and spares a matvec
  launch_any_nonzero(d_x, n * nrhs, h->n_stopped, st);
  CK(cudaMemcpyAsync(h->h_n_stopped, h->n_stopped, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  bool x_zero = *h->h_n_stopped == 0;
  CK(cudaMemsetAsync(h->n_stopped, 0, sizeof(int), st));
  auto active = [&]() { for (int r = 0; r < nrhs; ++r) if (!done[r]) return true; return false; };
  // x_try_r = x_r + V_{0..j-1} y_r for the right-hand sides with mask[r] == 0 (into u)
  auto form_x = [&](int j, const std::vector<int> &mask) -> fdst_status {
    for (int r = 0; r < nrhs; ++r) {
      double *yr = &hy[(size_t)r * ld];
      std::fill(yr, yr + ld, 0.0);
      if (mask[r]) continue;
      const double *Hr = &H[(size_t)r * ld * m];
      const double *gr = &g[(size_t)r * ld];
      for (int i = j - 1; i >= 0; --i) {
        double a = gr[i];
        for (int k = i + 1; k < j; ++k) a -= Hr[(size_t)i * m + k] * yr[k];
        yr[i] = Hr[(size_t)i * m + i] != 0.0 ? a / Hr[(size_t)i * m + i] : 0.0;
      }
    }
    CK(cudaMemcpyAsync(cy, hy.data(), sizeof(double) * nrhs * ld, cudaMemcpyHostToDevice, st));
    TRY(sync_done(mask, h->gm_mask));
    launch_axpby(d_x, u, 1.0, 0.0, n, n, nrhs, st);
    launch_basis_axpy(X, vstride, j, cy, ld, 1.0, u, n, n, nrhs, h->gm_mask, st);
    return FDST_OK;
  };
  int it = 0;
  while (active() && it < maxit) {
    // r0 = P^{-1}(b - A x) (left) or b - A x (flexible), V_0 = r0 / ||r0||
    if (x_zero) {
      launch_axpby(d_b, h->Az, 1.0, 0.0, n, n, nrhs, st);
      x_zero = false;
    } else {
      TRY(run_matvec(h, d_x, h->Az, nrhs, h->done, st, false));
      launch_axpby(d_b, h->Az, 1.0, -1.0, n, n, nrhs, st);
    }
    if (flex) launch_axpby(h->Az, w, 1.0, 0.0, n, n, nrhs, st);
    else TRY(apply_block_prec(h, prec, h->Az, w, nrhs, h->done, st));
    TRY(norms2(w, h->done));
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) continue;
      g[(size_t)r * ld] = std::sqrt(hs[r]);
      for (int i = 1; i < ld; ++i) g[(size_t)r * ld + i] = 0.0;
    }
    launch_scale_by_norm(w, V, h->dots, n, n, nrhs, h->done, st);
    int j = 0;
    while (j < m && it < maxit && active()) {
      // w = P^{-1} A V_j (left) or A Z_j with Z_j = P^{-1} V_j (flexible), then classical
      // Gram-Schmidt twice against V_0..V_j
      if (flex) {
        TRY(apply_block_prec(h, prec, V + (size_t)j * vstride, Z + (size_t)j * vstride, nrhs, h->done, st));
        TRY(run_matvec(h, Z + (size_t)j * vstride, w, nrhs, h->done, st, false));
      } else {
        TRY(run_matvec(h, V + (size_t)j * vstride, h->Az, nrhs, h->done, st, false));
        TRY(apply_block_prec(h, prec, h->Az, w, nrhs, h->done, st));
      }
      h->n_matvec += 1;
      h->n_prec += 1;
      launch_basis_dots(V, vstride, 0, j + 1, w, n, n, nrhs, h->gm_part, c1, ld, h->done, st);
      launch_basis_axpy(V, vstride, j + 1, c1, ld, -1.0, w, n, n, nrhs, h->done, st);
      launch_basis_dots(V, vstride, 0, j + 1, w, n, n, nrhs, h->gm_part, c2, ld, h->done, st);
      launch_basis_axpy(V, vstride, j + 1, c2, ld, -1.0, w, n, n, nrhs, h->done, st);
      launch_dot(w, w, n, n, nrhs, h->partials, h->counters, h->dots, h->done, st);
      launch_scale_by_norm(w, V + (size_t)(j + 1) * vstride, h->dots, n, n, nrhs, h->done, st);
      CK(cudaMemcpyAsync(hc1.data(), c1, sizeof(double) * nrhs * ld, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hc2.data(), c2, sizeof(double) * nrhs * ld, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hs.data(), h->dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      std::vector<int> cand(nrhs, 1);   // 0: estimate below its threshold (true residual to check)
      bool any = false;
      for (int r = 0; r < nrhs; ++r) {
        if (done[r]) continue;
        double *Hr = &H[(size_t)r * ld * m];
        double *gr = &g[(size_t)r * ld];
        double *csr = &cs[(size_t)r * m], *snr = &sn[(size_t)r * m];
        for (int i = 0; i <= j; ++i) Hr[(size_t)i * m + j] = hc1[(size_t)r * ld + i] + hc2[(size_t)r * ld + i];
        double hn = std::sqrt(std::max(hs[r], 0.0));
        for (int i = 0; i < j; ++i) {   // earlier rotations on the new column
          const double a = Hr[(size_t)i * m + j], b = Hr[(size_t)(i + 1) * m + j];
          Hr[(size_t)i * m + j] = csr[i] * a + snr[i] * b;
          Hr[(size_t)(i + 1) * m + j] = -snr[i] * a + csr[i] * b;
        }
        const double a = Hr[(size_t)j * m + j];
        const double den = std::hypot(a, hn);
        csr[j] = den == 0.0 ? 1.0 : a / den;
        snr[j] = den == 0.0 ? 0.0 : hn / den;
        Hr[(size_t)j * m + j] = csr[j] * a + snr[j] * hn;
        gr[j + 1] = -snr[j] * gr[j];
        gr[j] = csr[j] * gr[j];
        iters[r] += 1;
        est[r] = std::fabs(gr[j + 1]) / bref[r];
        if (est[r] <= tol && est_it[r] < 0) est_it[r] = iters[r];
        if (!(std::isfinite(est[r]))) { status[r] = FDST_NAN_DETECTED; done[r] = 1; continue; }
        if (est[r] <= tau[r]) { cand[r] = 0; any = true; }
      }
      ++j;
      ++it;
      if (any) {
        // true residual of x + V y for the candidates (FP64 matvec)
        TRY(form_x(j, cand));
        TRY(run_matvec(h, u, h->Az, nrhs, h->gm_mask, st, true));
        launch_axpby(d_b, h->Az, 1.0, -1.0, n, n, nrhs, st);
        TRY(norms2(h->Az, h->gm_mask));
        for (int r = 0; r < nrhs; ++r) {
          if (cand[r]) continue;
          const double tr = std::sqrt(hs[r]) / bn[r];
          true_rel[r] = tr;
          if (tr <= tol) {
            CK(cudaMemcpyAsync(d_x + (size_t)r * n, u + (size_t)r * n, sizeof(double) * n,
                               cudaMemcpyDeviceToDevice, st));
            status[r] = FDST_OK;
            done[r] = 1;
          } else {
            tau[r] = 0.5 * tau[r] * tol / tr;
          }
        }
      }
      TRY(sync_done(done, h->done));
    }
    if (active()) {
      // basis full (or maxit): x <- x + V y for the right-hand sides still running
      TRY(form_x(j, done));
      for (int r = 0; r < nrhs; ++r)
        if (!done[r])
          CK(cudaMemcpyAsync(d_x + (size_t)r * n, u + (size_t)r * n, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                             st));
    }
  }
  // FP64 true residuals of the returned iterates
  std::vector<int> none(nrhs, 0);
  TRY(sync_done(none, h->gm_mask));
  TRY(run_matvec(h, d_x, h->Az, nrhs, h->gm_mask, st, true));
  launch_axpby(d_b, h->Az, 1.0, -1.0, n, n, nrhs, st);
  TRY(norms2(h->Az, h->gm_mask));
  fdst_status ret = FDST_OK;
  for (int r = 0; r < nrhs; ++r) {
    true_rel[r] = bn[r] > 0.0 ? std::sqrt(hs[r]) / bn[r] : 0.0;
    if (status[r] == FDST_MAXIT && true_rel[r] <= tol) status[r] = FDST_OK;
    info[r].iterations = iters[r];
    info[r].status = status[r];
    info[r].eta_rel = est[r];
    info[r].true_rel_res = true_rel[r];
    info[r].iterations_estimate = est_it[r] >= 0 ? est_it[r] : iters[r];
    if (ret == FDST_OK && status[r] != FDST_OK) ret = (fdst_status)status[r];
  }
  TRY(sync_done(none, h->done));
  CK(cudaStreamSynchronize(st));
  resolve_kernel_events(h);
  return ret;
}

fdst_status fdst_solve(fdst_handle h, const double *d_b, double *d_x, int nrhs, double tol, int maxit,
                       fdst_solve_info *info, fdst_stream stream) {
  if (!h || !d_b || !d_x || !info) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  if (!(tol >= 0.0) || maxit < 1) { set_error("tol must be >= 0 and maxit >= 1"); return FDST_INVALID_ARGUMENT; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->n_total;
  int tc_err0 = 0;
  TRY(tc_error_count(&tc_err0));
  // timing events: (matvec, prec, vector) per phase
  std::vector<cudaEvent_t> ev;
  auto mark = [&](void) -> cudaEvent_t {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back(e);
    return e;
  };
  struct Span { int kind; size_t a, b; };
  std::vector<Span> spans;
  // ---- init: v = b - A x0 ; v_old = w = w_old = 0 ; z = P^{-1} v ; gamma_1 = sqrt(<v, z>)
  // (x0 = 0, the paper's start, is detected on the device and spares the FP64 matvec)
  CK(cudaMemsetAsync(h->done, 0, sizeof(int) * nrhs, st));
  launch_any_nonzero(d_x, n * nrhs, h->n_stopped, st);
  CK(cudaMemcpyAsync(h->h_n_stopped, h->n_stopped, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const bool x0_zero = *h->h_n_stopped == 0;
  CK(cudaMemsetAsync(h->n_stopped, 0, sizeof(int), st));
  launch_axpby(d_b, h->v, 1.0, 0.0, n, n, nrhs, st);
  if (!x0_zero) {
    TRY(run_matvec(h, d_x, h->Az, nrhs, nullptr, st, true));
    launch_axpby(h->Az, h->v, -1.0, 1.0, n, n, nrhs, st);
  }
  CK(cudaMemsetAsync(h->v_old, 0, sizeof(double) * n * nrhs, st));
  CK(cudaMemsetAsync(h->w, 0, sizeof(double) * n * nrhs, st));
  CK(cudaMemsetAsync(h->w_old, 0, sizeof(double) * n * nrhs, st));
  TRY(run_apply(h, h->v, h->z, nrhs, nullptr, st));
  launch_dot(h->v, h->z, n, n, nrhs, h->partials, h->counters, h->dots, nullptr, st);
  launch_minres_init(h->state, h->dots, h->done, nrhs, h->n_stopped, tol, st);
  launch_scale_by_inv_gamma(h->z, h->state, n, n, nrhs, h->done, st);
  double *v = h->v, *v_old = h->v_old, *w = h->w, *w_old = h->w_old;
  double *delta = h->dots + nrhs, *g2 = h->dots + 2 * nrhs;
  // ||b||_2^2 once (dots[3 nrhs ..])
  launch_dot(d_b, d_b, n, n, nrhs, h->partials, h->counters, h->dots + 3 * nrhs, nullptr, st);
  std::vector<double> bb(nrhs), true_rel(nrhs, -1.0);
  CK(cudaMemcpyAsync(h->h_dots, h->dots + 3 * nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int j = 0; j < nrhs; ++j) bb[j] = h->h_dots[j];
  // true relative residual ||b - A x||_2 / ||b||_2 in FP64 (Az is free between iterations)
  auto true_residuals = [&]() -> fdst_status {
    TRY(run_matvec(h, d_x, h->Az, nrhs, nullptr, st, true));
    launch_axpby(d_b, h->Az, 1.0, -1.0, n, n, nrhs, st);
    launch_dot(h->Az, h->Az, n, n, nrhs, h->partials, h->counters, h->dots, nullptr, st);
    CK(cudaMemcpyAsync(h->h_dots, h->dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < nrhs; ++j) true_rel[j] = bb[j] > 0 ? std::sqrt(h->h_dots[j] / bb[j]) : std::sqrt(h->h_dots[j]);
    return FDST_OK;
  };
  std::vector<MinresState> hs(nrhs);
  std::vector<double> prev_true(nrhs, -1.0);
  std::vector<int> restarts(nrhs, 0), est_iters(nrhs, -1);
  // The Lanczos and update passes write the new vector over the old one and the
  // roles of (v, v_old) and (w, w_old) are exchanged by pointer after every
  // iteration, for every right-hand side at once. A right-hand side that sits
  // stopped for an odd number of iterations therefore has its pairs in the
  // opposite roles; before it resumes, its slices are exchanged back.
  std::vector<int> sync_it(nrhs, 0), sync_iters(nrhs, 0);
  const int check_every = 4;
  int it = 0;
  bool residuals_current = false;
  // Double-float banded matvec on the identity map: the update writes the FP32 pairs of
  // the next z alongside z, so no separate split pass runs per iteration. (The matvec's
  // result is joined to FP64 for the dot and the Lanczos step: folding the join into them
  // moves FP64 work onto GB300's slow FP64 pipe and measured slower.)
  const bool dfp = !h->mapped && h->desc.matvec_precision == FDST_MV_DF64;
  bool z_pairs = false;   // h->x2 holds the pairs of the current z
  while (it < maxit) {
    residuals_current = false;
    size_t e0 = 0;
    if (h->timing) { mark(); e0 = ev.size() - 1; }
    if (dfp)
      TRY(run_plan_df(h, full_view(h, true), z_pairs ? nullptr : h->z, h->Az, nrhs, h->done, st, 0, n, 0, n,
                      true));
    else
      TRY(run_matvec(h, h->z, h->Az, nrhs, h->done, st, false));
    size_t e1 = 0;
    if (h->timing) { mark(); e1 = ev.size() - 1; spans.push_back({0, e0, e1}); }
    launch_dot(h->Az, h->z, n, n, nrhs, h->partials, h->counters, delta, h->done, st);
    launch_minres_lanczos(h->Az, v, v_old, h->state, delta, n, n, nrhs, h->done, st, true);
    std::swap(v, v_old);
    size_t e2 = 0;
    if (h->timing) { mark(); e2 = ev.size() - 1; spans.push_back({2, e1, e2}); }
    TRY(run_apply(h, v, h->z_new, nrhs, h->done, st));
    size_t e3 = 0;
    if (h->timing) { mark(); e3 = ev.size() - 1; spans.push_back({1, e2, e3}); }
    launch_dot(v, h->z_new, n, n, nrhs, h->partials, h->counters, g2, h->done, st);
    launch_minres_scalars(h->state, delta, g2, nrhs, maxit, h->done, h->n_stopped, st);
    launch_minres_update(w_old, w, d_x, h->z, h->z_new, h->state, n, n, nrhs, h->done, st, dfp ? h->x2 : nullptr,
                         true);
    std::swap(w, w_old);
    z_pairs = dfp;
    launch_minres_commit(h->state, h->done, nrhs, st);
    if (h->timing) { mark(); spans.push_back({2, e3, ev.size() - 1}); }
    ++it;
    h->n_matvec += 1;
    h->n_prec += 1;
    if (it % check_every == 0 || it == maxit) {
      CK(cudaMemcpyAsync(h->h_n_stopped, h->n_stopped, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*h->h_n_stopped >= nrhs) {
        // every right-hand side met its estimate threshold: check the true residual and
        // resume the ones above tol with a tighter threshold (recurrences intact); the
        // check is FP64: a double-float residual has a floor near 1e-14 |A||x| / |b|, which
        // on high-degree instances reaches the tolerance and reads as stagnation
        TRY(true_residuals());
        residuals_current = true;
        CK(cudaMemcpy(hs.data(), h->state, sizeof(MinresState) * nrhs, cudaMemcpyDeviceToHost));
        for (int j = 0; j < nrhs; ++j)
          if (est_iters[j] < 0) est_iters[j] = hs[j].iters;
        std::vector<int> resume, restart;
        for (int j = 0; j < nrhs; ++j) {
          const int a = resume_action(hs[j], true_rel[j], prev_true[j], restarts[j], tol, maxit);
          if (a == kKeepStopped) continue;
          if (a == kStagnated) hs[j].status = FDST_STAGNATION;
          else (a == kResume ? resume : restart).push_back(j);
          prev_true[j] = true_rel[j];
        }
        if (resume.empty() && restart.empty()) {
          CK(cudaMemcpy(h->state, hs.data(), sizeof(MinresState) * nrhs, cudaMemcpyHostToDevice));
          break;
        }
        for (int j : resume) {
          hs[j].tau = 0.5 * hs[j].tau * tol / true_rel[j];
          hs[j].stop = 0;
          const int idle = (it - sync_it[j]) - (hs[j].iters - sync_iters[j]);   // iterations spent stopped
          if (idle & 1) {
            launch_swap(v + (size_t)j * n, v_old + (size_t)j * n, n, st);
            launch_swap(w + (size_t)j * n, w_old + (size_t)j * n, n, st);
          }
        }
        if (!restart.empty()) {
          for (int j : restart) ++restarts[j];
          double *const vecs[4] = {v, v_old, w, w_old};
          TRY(minres_restart(h, d_b, d_x, nrhs, restart, true_rel, tol, hs, st, vecs));
          z_pairs = false;   // the restarted right-hand sides have a new z
        }
        for (int j = 0; j < nrhs; ++j) {
          sync_it[j] = it;
          sync_iters[j] = hs[j].iters;
        }
        std::vector<int> hd(nrhs, 1);
        for (int j : resume) hd[j] = 0;
        for (int j : restart)
          if (!hs[j].stop && hs[j].status == 0) hd[j] = 0;
        int ns = 0;
        for (int j = 0; j < nrhs; ++j) ns += hd[j];
        CK(cudaMemcpy(h->state, hs.data(), sizeof(MinresState) * nrhs, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->done, hd.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->n_stopped, &ns, sizeof(int), cudaMemcpyHostToDevice));
      }
    }
  }
  CK(cudaGetLastError());
  if (!residuals_current) TRY(true_residuals());
  CK(cudaMemcpyAsync(hs.data(), h->state, sizeof(MinresState) * nrhs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h->timing) {
    for (auto &sp : spans) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[sp.a], ev[sp.b]);
      (sp.kind == 0 ? h->ms_matvec : sp.kind == 1 ? h->ms_prec : h->ms_vector) += ms;
    }
    for (auto e : ev) cudaEventDestroy(e);
  }
  resolve_kernel_events(h);
  fdst_status ret = FDST_OK;
  for (int j = 0; j < nrhs; ++j) {
    info[j].iterations = hs[j].iters;
    info[j].status = hs[j].stop || hs[j].status ? hs[j].status : FDST_MAXIT;
    if (hs[j].eta0 == 0.0 && hs[j].status == 0) info[j].status = FDST_OK;
    info[j].eta_rel = hs[j].eta0 > 0 ? std::fabs(hs[j].eta) / hs[j].eta0 : 0.0;
    info[j].true_rel_res = true_rel[j];
    info[j].iterations_estimate = est_iters[j] >= 0 ? est_iters[j] : hs[j].iters;
    if (ret == FDST_OK && info[j].status != FDST_OK) ret = (fdst_status)info[j].status;
  }
  return timeout_check(tc_err0, info, nrhs, ret);
}

static fdst_status ensure_host_buffers(fdst_handle h) {
  if (h->hb) return FDST_OK;
  const size_t nv = (size_t)h->n_total * h->max_rhs;
  TRY(dalloc(h, &h->hb, nv));
  TRY(dalloc(h, &h->hx, nv));
  return FDST_OK;
}

fdst_status fdst_solve_host(fdst_handle h, const double *h_b, double *h_x, int nrhs, double tol, int maxit,
                            fdst_solve_info *info, fdst_stream stream) {
  if (!h || !h_b || !h_x || !info) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  TRY(ensure_host_buffers(h));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * h->n_total * nrhs;
  CK(cudaMemcpyAsync(h->hb, h_b, bytes, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->hx, h_x, bytes, cudaMemcpyHostToDevice, st));
  fdst_status s = fdst_solve(h, h->hb, h->hx, nrhs, tol, maxit, info, stream);
  CK(cudaMemcpyAsync(h_x, h->hx, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

fdst_status fdst_solve_host_zero(fdst_handle h, const double *h_b, double *h_x, int nrhs, double tol, int maxit,
                                 fdst_solve_info *info, fdst_stream stream) {
  if (!h || !h_b || !h_x || !info) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  TRY(ensure_host_buffers(h));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * h->n_total * nrhs;
  CK(cudaMemcpyAsync(h->hb, h_b, bytes, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h->hx, 0, bytes, st));
  fdst_status s = fdst_solve(h, h->hb, h->hx, nrhs, tol, maxit, info, stream);
  CK(cudaMemcpyAsync(h_x, h->hx, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

fdst_status fdst_apply_prec_host(fdst_handle h, const double *h_r, double *h_s, int nrhs, fdst_stream stream) {
  if (!h || !h_r || !h_s) { set_error("NULL argument"); return FDST_INVALID_ARGUMENT; }
  if (nrhs < 1 || nrhs > h->max_rhs) { set_error("nrhs out of range [1, max_rhs]"); return FDST_INVALID_ARGUMENT; }
  TRY(ensure_host_buffers(h));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * h->n_total * nrhs;
  CK(cudaMemcpyAsync(h->hb, h_r, bytes, cudaMemcpyHostToDevice, st));
  TRY(run_apply(h, h->hb, h->hx, nrhs, nullptr, st));
  CK(cudaMemcpyAsync(h_s, h->hx, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FDST_OK;
}

}  // extern "C"

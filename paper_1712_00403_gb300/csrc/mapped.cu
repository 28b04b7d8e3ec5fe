// Setup of the mapped-geometry case (3D, Taylor-Hood): geometry at the
// quadrature points, separable approximation of diag(C_k) (Appendix) and the
// weighted pencils of P~_V, the assembled FP64 CSR operator (Sec. 3 forms on
// the mapped domain) and the diagonal scalings D_V, D_Q of P_D^G (Sec. 6).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.h"
#include "mapped.h"

namespace fdst {

namespace {
constexpr double kAmp = 0.1;     // sine-bump amplitude of the map
constexpr int kSweeps = 12;      // Diliberto-Straus sweeps

// element ranges [lo, hi] of every function of a space with the given knot vector / degree
void element_ranges(const std::vector<double> &t, int deg, int ne, const std::vector<int> &first_of_elem,
                    std::vector<int> &elo, std::vector<int> &ehi) {
  const int m = (int)t.size() - deg - 1;
  elo.assign(m, ne);
  ehi.assign(m, -1);
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j <= deg; ++j) {
      const int g = first_of_elem[e] + j;
      elo[g] = std::min(elo[g], e);
      ehi[g] = std::max(ehi[g], e);
    }
}

// column range (in the index space of "cols", restricted to [c0, c0 + nc)) of functions
// whose element ranges intersect that of each row function
void overlap_ranges(const std::vector<int> &relo, const std::vector<int> &rehi, int r0, int nr,
                    const std::vector<int> &celo, const std::vector<int> &cehi, int c0, int nc, std::vector<int> &lo,
                    std::vector<int> &w) {
  lo.assign(nr, 0);
  w.assign(nr, 0);
  for (int i = 0; i < nr; ++i) {
    int a = -1, b = -2;
    for (int j = 0; j < nc; ++j) {
      const bool ov = celo[c0 + j] <= rehi[r0 + i] && relo[r0 + i] <= cehi[c0 + j];
      if (ov) {
        if (a < 0) a = j;
        b = j;
      }
    }
    lo[i] = a < 0 ? 0 : a;
    w[i] = a < 0 ? 0 : b - a + 1;
  }
}
}  // namespace

// Separable fit of the nine diagonal coefficients c^k_jj of C_k at the
// quadrature points gp (Appendix: log c ~ f_1 + f_2 + f_3 by Diliberto-Straus
// midrange sweeps), normalized so that each fit's two non-own factors have
// zero mean log; tau^k_d = exp(f^{k,d}_d), mu^k_d = exp(mean over j != d of
// f^{k,j}_d). Fills geo_K, geo_M with the weighted pencils. For a Nitsche
// (RT tangential) factor the K~ boundary terms take tau^k_d at eta_d = 0 and 1:
// the fit's own direction-d update evaluated on those faces (the midrange over
// the face points of log c^k_dd minus the other two factors), which leaves the
// fit at the quadrature points unchanged.
fdst_status fit_pencils(fdst_ctx *h, const GeoPoints &gp, int kind, double amp, double contrast, cudaStream_t st) {
  const int nq = h->p + 2;
  const int fstride = std::max(gp.nq[0], std::max(gp.nq[1], gp.nq[2]));
  double *L = nullptr, *f = nullptr;
  CK(cudaMalloc(&L, sizeof(double) * 9 * gp.Q));
  if (cudaMalloc(&f, sizeof(double) * 27 * fstride) != cudaSuccess) {
    cudaFree(L);
    set_error("cudaMalloc failed for the separable fit");
    return FDST_OUT_OF_MEMORY;
  }
  cudaMemset(f, 0, sizeof(double) * 27 * fstride);
  launch_logc(gp, L, st);
  for (int sw = 0; sw < kSweeps; ++sw)
    for (int d = 0; d < 3; ++d) launch_fit_sweep(L, f, d, gp, fstride, st);
  std::vector<double> fh((size_t)27 * fstride);
  cudaError_t e1 = cudaMemcpy(fh.data(), f, sizeof(double) * fh.size(), cudaMemcpyDeviceToHost);
  cudaFree(L);
  cudaFree(f);
  if (e1 != cudaSuccess) {
    set_error(std::string("separable fit: ") + cudaGetErrorString(e1));
    return FDST_CUDA_ERROR;
  }
  auto F = [&](int k, int j, int d) -> double * { return fh.data() + (size_t)((3 * k + j) * 3 + d) * fstride; };
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) {
        if (d == j) continue;
        double m = 0.0;
        for (int t = 0; t < gp.nq[d]; ++t) m += F(k, j, d)[t];
        m /= gp.nq[d];
        for (int t = 0; t < gp.nq[d]; ++t) F(k, j, d)[t] -= m;
        for (int t = 0; t < gp.nq[j]; ++t) F(k, j, j)[t] += m;
      }
  // tau^k_d on the faces eta_d = 0 and 1 (needed by Nitsche factors only)
  double tau_end[3][3][2];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) tau_end[k][d][0] = tau_end[k][d][1] = 1.0;
  bool any_nitsche = false;
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) any_nitsche = any_nitsche || h->vel[k][d].nitsche;
  for (int d = 0; d < 3 && any_nitsche; ++d)
    for (int side = 0; side < 2; ++side) {
      GeoPoints fp;
      for (int e = 0; e < 3; ++e) {
        fp.nq[e] = e == d ? 1 : gp.nq[e];
        fp.pts[e] = gp.pts[e];
        fp.wts[e] = gp.wts[e];
      }
      const double t = side;
      double *tp = nullptr, *buf = nullptr;
      fp.Q = (int64_t)fp.nq[0] * fp.nq[1] * fp.nq[2];
      CK(cudaMalloc(&tp, sizeof(double)));
      if (cudaMalloc(&buf, sizeof(double) * 20 * fp.Q) != cudaSuccess) {
        cudaFree(tp);
        set_error("cudaMalloc failed for the face points of the separable fit");
        return FDST_OUT_OF_MEMORY;
      }
      cudaMemcpy(tp, &t, sizeof(double), cudaMemcpyHostToDevice);
      fp.pts[d] = tp;
      fp.jinv = buf;
      fp.det = buf + 9 * fp.Q;
      fp.nu = buf + 10 * fp.Q;
      double *Lf = buf + 11 * fp.Q;
      launch_geo_points(fp, kind, amp, contrast, st);
      launch_logc(fp, Lf, st);
      std::vector<double> lh((size_t)9 * fp.Q);
      cudaError_t e2 = cudaMemcpy(lh.data(), Lf, sizeof(double) * lh.size(), cudaMemcpyDeviceToHost);
      cudaFree(tp);
      cudaFree(buf);
      if (e2 != cudaSuccess) {
        set_error(std::string("separable fit (faces): ") + cudaGetErrorString(e2));
        return FDST_CUDA_ERROR;
      }
      const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
      for (int k = 0; k < 3; ++k) {
        const double *Lk = lh.data() + (size_t)(3 * k + d) * fp.Q;
        double mx = -INFINITY, mn = INFINITY;
        for (int64_t q = 0; q < fp.Q; ++q) {
          int qq[3];
          qq[0] = (int)(q % fp.nq[0]);
          qq[1] = (int)((q / fp.nq[0]) % fp.nq[1]);
          qq[2] = (int)(q / ((int64_t)fp.nq[0] * fp.nq[1]));
          const double r = Lk[q] - F(k, d, da)[qq[da]] - F(k, d, db)[qq[db]];
          mx = std::max(mx, r);
          mn = std::min(mn, r);
        }
        tau_end[k][d][side] = std::exp(0.5 * (mx + mn));
      }
    }
  h->geo_K.assign(3, std::vector<Mat>(3));
  h->geo_M.assign(3, std::vector<Mat>(3));
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) {
      std::vector<double> tau(gp.nq[d]), mu(gp.nq[d]);
      for (int t = 0; t < gp.nq[d]; ++t) {
        tau[t] = std::exp(F(k, d, d)[t]);
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
          if (j != d) s += F(k, j, d)[t];
        mu[t] = std::exp(0.5 * s);
      }
      h->geo_K[k][d] = stiffness_matrix(h->vel[k][d], nq, tau, tau_end[k][d][0], tau_end[k][d][1]);
      h->geo_M[k][d] = mixed_matrix(h->vel[k][d], 0, h->vel[k][d], 0, nq, mu);
    }
  return FDST_OK;
}

// D_V^{-1/2} of P_D^G from diag(A) (the velocity entries of the block vector):
// [D_V]_ii = A_ii / (P~_V)_ii with diag(P~_V) the Kronecker sum of the pencils' diagonals.
void set_velocity_scaling(fdst_ctx *h, const std::vector<double> &diagA) {
  for (int k = 0; k < 3; ++k) {
    const int n1 = h->shape[k][0], n2 = h->shape[k][1], n3 = h->shape[k][2];
    std::vector<double> &sc = h->geo_scale[k];
    sc.resize((size_t)n1 * n2 * n3);
    const Mat *Kf = h->geo_K[k].data(), *Mf = h->geo_M[k].data();
    for (int i3 = 0; i3 < n3; ++i3)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1) {
          const double dp = Kf[2](i3, i3) * Mf[1](i2, i2) * Mf[0](i1, i1) + Mf[2](i3, i3) * Kf[1](i2, i2) * Mf[0](i1, i1) +
                            Mf[2](i3, i3) * Mf[1](i2, i2) * Kf[0](i1, i1);
          const size_t li = ((size_t)i3 * n2 + i2) * n1 + i1;
          sc[li] = 1.0 / std::sqrt(diagA[h->off[k] + li] / dp);
        }
  }
}

fdst_status build_mapped_pre(fdst_ctx *h) {
  if (h->dim != 3 || h->desc.discretization != FDST_TH) {
    set_error("the mapped geometry is built for the 3D Taylor-Hood discretization");
    return FDST_NOT_SUPPORTED;
  }
  if (h->p > 3 && h->desc.matvec_form != FDST_MATVEC_MATRIX_FREE) {
    set_error("mapped-geometry assembly supports pressure degree p <= 3 (element matrices in shared memory); "
              "the matrix-free operator takes p <= 8");
    return FDST_NOT_SUPPORTED;
  }
  if (h->p > 8) {
    set_error("mapped geometry supports pressure degree p <= 8");
    return FDST_NOT_SUPPORTED;
  }
  h->mapped = true;
  const int p = h->p, q = p + 1, nq = p + 2;
  cudaStream_t st = 0;
  // ---- quadrature grid and geometry at the points
  GeoPoints gp;
  std::vector<std::vector<double>> px(3), pw(3);
  for (int d = 0; d < 3; ++d) {
    span_rule(h->pres[d].knots, nq, px[d], pw[d]);
    gp.nq[d] = (int)px[d].size();
    double *dp = nullptr, *dw = nullptr;
    TRY(upload(h, &dp, px[d]));
    TRY(upload(h, &dw, pw[d]));
    gp.pts[d] = dp;
    gp.wts[d] = dw;
  }
  gp.Q = (int64_t)gp.nq[0] * gp.nq[1] * gp.nq[2];
  TRY(dalloc(h, &gp.jinv, (size_t)9 * gp.Q));
  TRY(dalloc(h, &gp.det, (size_t)gp.Q));
  TRY(dalloc(h, &gp.nu, (size_t)gp.Q));
  const double amp = h->desc.geometry_amplitude > 0.0 ? h->desc.geometry_amplitude : kAmp;
  if (h->desc.geometry == FDST_GEOM_SINE_BUMP && amp > 0.25) {
    set_error("geometry_amplitude must be at most 0.25 (det J stays positive)");
    return FDST_INVALID_ARGUMENT;
  }
  if (h->desc.viscosity_contrast > 0.0 && h->desc.viscosity_contrast < 1.0) {
    set_error("viscosity_contrast must be >= 1 (or <= 0 for the default field)");
    return FDST_INVALID_ARGUMENT;
  }
  launch_geo_points(gp, h->desc.geometry == FDST_GEOM_ANNULUS ? kGeoAnnulus : kGeoSineBump, amp,
                    h->desc.viscosity_contrast, st);
  h->gp = gp;
  TRY(fit_pencils(h, gp, h->desc.geometry == FDST_GEOM_ANNULUS ? kGeoAnnulus : kGeoSineBump, amp,
                  h->desc.viscosity_contrast, st));
  // ---- element tables per direction
  MeshTables mt;
  mt.nq = nq;
  mt.p = p;
  std::vector<std::vector<int>> vfirst(3), pfirst(3), velo(3), vehi(3), pelo(3), pehi(3);
  for (int d = 0; d < 3; ++d) {
    const Space1D &sv = h->vel[0][d], &sp = h->pres[d];
    const int ne = gp.nq[d] / nq;
    mt.ne[d] = ne;
    mt.np[d] = sp.n;
    std::vector<double> vt((size_t)ne * (q + 1) * nq * 2), pt((size_t)ne * (p + 1) * nq);
    vfirst[d].resize(ne);
    pfirst[d].resize(ne);
    double N[32], dN[32];
    for (int e = 0; e < ne; ++e)
      for (int a = 0; a < nq; ++a) {
        const double x = px[d][(size_t)e * nq + a];
        int s = eval_nonzero(sv.knots, q, x, N, dN);
        vfirst[d][e] = s - q;
        for (int i = 0; i <= q; ++i) {
          vt[(((size_t)e * (q + 1) + i) * nq + a) * 2 + 0] = N[i];
          vt[(((size_t)e * (q + 1) + i) * nq + a) * 2 + 1] = dN[i];
        }
        s = eval_nonzero(sp.knots, p, x, N, dN);
        pfirst[d][e] = s - p;
        for (int l = 0; l <= p; ++l) pt[((size_t)e * (p + 1) + l) * nq + a] = N[l];
      }
    element_ranges(sv.knots, q, ne, vfirst[d], velo[d], vehi[d]);
    element_ranges(sp.knots, p, ne, pfirst[d], pelo[d], pehi[d]);
    double *dvt = nullptr, *dpt = nullptr;
    int *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *a4 = nullptr;
    TRY(upload(h, &dvt, vt));
    TRY(upload(h, &dpt, pt));
    TRY(upload(h, &a1, vfirst[d]));
    TRY(upload(h, &a2, pfirst[d]));
    TRY(upload(h, &a3, pelo[d]));
    TRY(upload(h, &a4, pehi[d]));
    mt.vtab[d] = dvt;
    mt.ptab[d] = dpt;
    mt.v_first[d] = a1;
    mt.p_first[d] = a2;
    mt.p_elo[d] = a3;
    mt.p_ehi[d] = a4;
  }
  // ---- CSR (not built for a matrix-free handle: its operator, diag(A), B and B^T are
  // evaluated by sum factorization)
  const bool mf_only = h->desc.matvec_form == FDST_MATVEC_MATRIX_FREE;
  const int64_t nrows = h->n_total;
  if (!mf_only) {
    // ---- CSR layout
    CsrTables ct;
    for (int b = 0; b < 5; ++b) ct.off[b] = h->off[b];
    std::vector<std::vector<int>> vvlo(3), vvw(3), vplo(3), vpw(3), pvlo(3), pvw(3);
    for (int d = 0; d < 3; ++d) {
      const int nv = h->vel[0][d].n, np = h->pres[d].n;
      ct.nv[d] = nv;
      ct.np[d] = np;
      overlap_ranges(velo[d], vehi[d], 1, nv, velo[d], vehi[d], 1, nv, vvlo[d], vvw[d]);
      overlap_ranges(velo[d], vehi[d], 1, nv, pelo[d], pehi[d], 0, np, vplo[d], vpw[d]);
      overlap_ranges(pelo[d], pehi[d], 0, np, velo[d], vehi[d], 1, nv, pvlo[d], pvw[d]);
      int *t[6];
      TRY(upload(h, &t[0], vvlo[d]));
      TRY(upload(h, &t[1], vvw[d]));
      TRY(upload(h, &t[2], vplo[d]));
      TRY(upload(h, &t[3], vpw[d]));
      TRY(upload(h, &t[4], pvlo[d]));
      TRY(upload(h, &t[5], pvw[d]));
      ct.vv_lo[d] = t[0]; ct.vv_w[d] = t[1];
      ct.vp_lo[d] = t[2]; ct.vp_w[d] = t[3];
      ct.pv_lo[d] = t[4]; ct.pv_w[d] = t[5];
    }
    std::vector<int64_t> rp(nrows + 1, 0);
    for (int r = 0; r < 3; ++r)
      for (int i3 = 0; i3 < ct.nv[2]; ++i3)
        for (int i2 = 0; i2 < ct.nv[1]; ++i2)
          for (int i1 = 0; i1 < ct.nv[0]; ++i1) {
            const int64_t row = h->off[r] + ((int64_t)i3 * ct.nv[1] + i2) * ct.nv[0] + i1;
            rp[row + 1] = 3LL * vvw[0][i1] * vvw[1][i2] * vvw[2][i3] + (int64_t)vpw[0][i1] * vpw[1][i2] * vpw[2][i3];
          }
    for (int l3 = 0; l3 < ct.np[2]; ++l3)
      for (int l2 = 0; l2 < ct.np[1]; ++l2)
        for (int l1 = 0; l1 < ct.np[0]; ++l1) {
          const int64_t row = h->off[3] + ((int64_t)l3 * ct.np[1] + l2) * ct.np[0] + l1;
          rp[row + 1] = 3LL * pvw[0][l1] * pvw[1][l2] * pvw[2][l3];
        }
    for (int64_t r = 0; r < nrows; ++r) rp[r + 1] += rp[r];
    const int64_t nnz = rp[nrows];
    int64_t *drp = nullptr;
    int *dcol = nullptr;
    double *dval = nullptr;
    TRY(upload(h, &drp, rp));
    TRY(dalloc(h, &dcol, (size_t)nnz));
    TRY(dalloc(h, &dval, (size_t)nnz));
    ct.row_ptr = drp;
    CK(cudaMemsetAsync(dval, 0, sizeof(double) * nnz, st));
    launch_csr_cols(ct, dcol, st);
    TRY(launch_assemble(gp, mt, ct, dval, st));
    h->csr.row_ptr = drp;
    h->csr.col = dcol;
    h->csr.val = dval;
    h->csr.nrows = nrows;
    h->csr.nnz = nnz;
    if (h->desc.matvec_precision == FDST_MV_DF64) {
      // FP32-pair copy of the values and a split right-hand-side buffer for the
      // double-float SpMV inside the iterations (true residuals use FP64)
      float2 *vdf = nullptr;
      TRY(dalloc(h, &vdf, (size_t)nnz));
      launch_split_df(dval, vdf, nnz, nnz, 1, nullptr, st);
      h->csr.val_df = vdf;
      TRY(dalloc(h, &h->x2, (size_t)h->n_total * h->max_rhs));
    }
  }
  if (h->desc.matvec_precision == FDST_MV_DF64 && !h->x2)
    TRY(dalloc(h, &h->x2, (size_t)h->n_total * h->max_rhs));
  // ---- diagonal scalings of P_D^G: D_V = diag(A) / diag(P~_V), D_Q = diag(Q) / diag(P_Q)
  h->geo_scale.assign(4, std::vector<double>());
  if (h->desc.variant == FDST_VARIANT_PD_GEO) {
    double *dQ = nullptr;
    TRY(dalloc(h, &dQ, (size_t)(h->off[4] - h->off[3])));
    launch_diag_q(gp, mt, dQ, st);
    std::vector<double> diagQ(h->off[4] - h->off[3]);
    CK(cudaMemcpy(diagQ.data(), dQ, sizeof(double) * diagQ.size(), cudaMemcpyDeviceToHost));
    if (!mf_only) {
      double *dA = nullptr;
      TRY(dalloc(h, &dA, (size_t)nrows));
      launch_csr_diag(h->csr, dA, st);
      std::vector<double> diagA(nrows);
      CK(cudaMemcpy(diagA.data(), dA, sizeof(double) * nrows, cudaMemcpyDeviceToHost));
      set_velocity_scaling(h, diagA);
    }
    {
      const int n1 = h->shape[3][0], n2 = h->shape[3][1], n3 = h->shape[3][2];
      std::vector<Mat> Mp(3);
      for (int d = 0; d < 3; ++d) Mp[d] = mixed_matrix(h->pres[d], 0, h->pres[d], 0, nq);
      std::vector<double> &sc = h->geo_scale[3];
      sc.resize((size_t)n1 * n2 * n3);
      for (int i3 = 0; i3 < n3; ++i3)
        for (int i2 = 0; i2 < n2; ++i2)
          for (int i1 = 0; i1 < n1; ++i1) {
            const size_t li = ((size_t)i3 * n2 + i2) * n1 + i1;
            const double dp = Mp[2](i3, i3) * Mp[1](i2, i2) * Mp[0](i1, i1);
            sc[li] = 1.0 / std::sqrt(diagQ[li] / dp);
          }
    }
  }
  CK(cudaStreamSynchronize(st));
  return FDST_OK;
}

double contrast_viscosity(double eta1, double k) {
  const double pi = 3.14159265358979323846;
  return 1.0 + (k - 1.0) * (1.0 - std::cos(2.0 * pi * eta1)) * 0.5;
}

// P_D^G on the identity map with the one-coordinate viscosity family (3D, TH or
// RT): the fit of diag(C_k) at the quadrature points (C_k^RT = C_k^TH = nu (I +
// e_k e_k^T) on this map, eq. Q_TH / Q_RT), the weighted pencils, and the
// scalings D_V = diag(A) / diag(P~_V) (diag(A) from the operator's Kronecker
// terms, the Nitsche terms included) and D_Q = diag(Q) / diag(P_Q), Q the
// 1/nu-weighted pressure mass (Sec. 6). Needs the operator's terms (build_matvec).
fdst_status build_identity_geo(fdst_ctx *h) {
  const int nq = h->p + 2;
  const double contrast = h->desc.viscosity_contrast;
  cudaStream_t st = 0;
  GeoPoints gp;
  std::vector<std::vector<double>> px(3), pw(3);
  std::vector<double *> owned;
  auto release = [&]() {
    for (double *q : owned) cudaFree(q);
    owned.clear();
  };
  for (int d = 0; d < 3; ++d) {
    span_rule(h->pres[d].knots, nq, px[d], pw[d]);
    gp.nq[d] = (int)px[d].size();
    double *dp = nullptr;
    if (cudaMalloc(&dp, sizeof(double) * 2 * px[d].size()) != cudaSuccess) {
      release();
      set_error("cudaMalloc failed for the quadrature points");
      return FDST_OUT_OF_MEMORY;
    }
    owned.push_back(dp);
    cudaMemcpy(dp, px[d].data(), sizeof(double) * px[d].size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dp + px[d].size(), pw[d].data(), sizeof(double) * px[d].size(), cudaMemcpyHostToDevice);
    gp.pts[d] = dp;
    gp.wts[d] = dp + px[d].size();
  }
  gp.Q = (int64_t)gp.nq[0] * gp.nq[1] * gp.nq[2];
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * 11 * gp.Q) != cudaSuccess) {
    release();
    set_error("cudaMalloc failed for the geometry at the quadrature points");
    return FDST_OUT_OF_MEMORY;
  }
  owned.push_back(buf);
  gp.jinv = buf;
  gp.det = buf + 9 * gp.Q;
  gp.nu = buf + 10 * gp.Q;
  // the sine bump with amplitude 0 is the identity map (J = I, det J = 1)
  launch_geo_points(gp, kGeoSineBump, 0.0, contrast, st);
  fdst_status s = fit_pencils(h, gp, kGeoSineBump, 0.0, contrast, st);
  release();
  TRY(s);
  // diag(A) of the velocity blocks from the Kronecker terms dst = src = k
  std::vector<double> diagA(h->n_total, 0.0);
  for (const Term &t : h->terms) {
    if (t.dst != t.src || t.dst >= 3) continue;
    const int k = t.dst;
    const int n1 = h->shape[k][0], n2 = h->shape[k][1], n3 = h->shape[k][2];
    const std::vector<double> &d0 = h->bands[t.f[0]].hdiag, &d1 = h->bands[t.f[1]].hdiag, &d2 = h->bands[t.f[2]].hdiag;
    for (int i3 = 0; i3 < n3; ++i3)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1)
          diagA[h->off[k] + ((size_t)i3 * n2 + i2) * n1 + i1] += t.coef * d0[i1] * d1[i2] * d2[i3];
  }
  h->geo_scale.assign(4, std::vector<double>());
  set_velocity_scaling(h, diagA);
  // D_Q: Q = M_1^{1/nu} (x) M_2 (x) M_3 on this map, P_Q = M_1 (x) M_2 (x) M_3
  std::vector<double> x1, w1, inv_nu;
  span_rule(h->pres[0].knots, nq, x1, w1);
  for (double e : x1) inv_nu.push_back(1.0 / contrast_viscosity(e, contrast));
  const Mat Mq = mixed_matrix(h->pres[0], 0, h->pres[0], 0, nq, inv_nu);
  const Mat M0 = mixed_matrix(h->pres[0], 0, h->pres[0], 0, nq);
  const int n1 = h->shape[3][0], n2 = h->shape[3][1], n3 = h->shape[3][2];
  std::vector<double> &sc = h->geo_scale[3];
  sc.resize((size_t)n1 * n2 * n3);
  for (size_t li = 0; li < sc.size(); ++li) {
    const int i1 = (int)(li % n1);
    sc[li] = 1.0 / std::sqrt(Mq(i1, i1) / M0(i1, i1));
  }
  return FDST_OK;
}

// Attach the D^{-1/2} scalings of P_D^G to the FD chains (after build_fd).
fdst_status build_mapped_post(fdst_ctx *h) {
  if (h->desc.variant != FDST_VARIANT_PD_GEO) return FDST_OK;
  for (size_t c = 0; c < h->chains.size() && c < h->geo_scale.size(); ++c) {
    double *d = nullptr;
    TRY(upload(h, &d, h->geo_scale[c]));
    h->chains[c].scale = d;
  }
  return FDST_OK;
}

// The B and B^T blocks of the assembled operator as CSR matrices of their own
// (rows of the pressure block with the velocity columns; rows of the velocity
// blocks with the pressure columns), for the block preconditioners P_T^G, P_C^G.
fdst_status build_coupling_csr(fdst_ctx *h) {
  const int64_t nv = h->off[h->dim], n = h->n_total;
  auto extract = [&](int64_t r0, int64_t nr, int c_lo, int c_hi, CsrDev &out) -> fdst_status {
    int64_t *dcnt = nullptr;
    TRY(dalloc(h, &dcnt, (size_t)nr));
    launch_csr_count_range(h->csr, r0, nr, c_lo, c_hi, dcnt, 0);
    std::vector<int64_t> cnt((size_t)nr), rp((size_t)nr + 1, 0);
    CK(cudaMemcpy(cnt.data(), dcnt, sizeof(int64_t) * nr, cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < nr; ++q) rp[q + 1] = rp[q] + cnt[q];
    const int64_t nnz = rp[nr];
    int64_t *drp = nullptr;
    int *dcol = nullptr;
    double *dval = nullptr;
    float2 *ddf = nullptr;
    TRY(upload(h, &drp, rp));
    TRY(dalloc(h, &dcol, (size_t)nnz));
    TRY(dalloc(h, &dval, (size_t)nnz));
    if (h->csr.val_df) TRY(dalloc(h, &ddf, (size_t)nnz));
    launch_csr_copy_range(h->csr, r0, nr, c_lo, c_hi, drp, dcol, dval, ddf, 0);
    CK(cudaStreamSynchronize(0));
    out.row_ptr = drp;
    out.col = dcol;
    out.val = dval;
    out.val_df = ddf;
    out.nrows = nr;
    out.nnz = nnz;
    return FDST_OK;
  };
  TRY(extract(nv, n - nv, 0, (int)nv, h->csr_b));          // B: pressure rows, velocity columns
  TRY(extract(0, nv, (int)nv, (int)n, h->csr_bt));         // B^T: velocity rows, pressure columns
  return FDST_OK;
}

}  // namespace fdst

// Mapped geometry (analytic sine-bump map, variable viscosity): geometry at
// the quadrature points, the separable approximation of diag(C_k)
// (Appendix), the weighted pressure-mass diagonal (Sec. 6), and the
// assembled FP64 CSR Stokes operator with its SpMV (Sec. 3 forms pushed
// forward with grad_x = J^{-T} grad_eta).
#include <cuda_runtime.h>

#include <cmath>

#include "df_arith.cuh"
#include "fp_bits.cuh"
#include "geometry.h"
#include "kernels.h"

namespace fdst {

// ------------------------------------------------------------------ points

// Sine bump: x = eta + a s(eta) 1, s = sin(pi e1) sin(pi e2) sin(pi e3); J = I + 1 g^T
// with g = a grad s; det J = 1 + 1.g; J^{-1} = I - 1 g^T / det (Sherman-Morrison);
// nu(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2).
// Annulus (eighth of a thick annulus, Sec. 7): r = 1 + e1, t = pi e2 / 4,
// x = (r cos t, r sin t, e3); the columns of J are (cos t, sin t, 0), (pi r / 4)
// (-sin t, cos t, 0) and e3, so det J = pi r / 4 and the rows of J^{-1} are
// (cos t, sin t, 0), (-sin t, cos t, 0) / (pi r / 4) and e3; nu = 1.
// Either map with a contrast k >= 1: nu(x) = 1 + (k - 1)(1 - cos(2 pi x1)) / 2.
__global__ void k_geo_points(GeoPoints gp, int kind, double amp, double contrast) {
  const int64_t Q = gp.Q;
  const double pi = 3.14159265358979323846;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    const int q1 = (int)(q % gp.nq[0]);
    const int64_t t = q / gp.nq[0];
    const int q2 = (int)(t % gp.nq[1]), q3 = (int)(t / gp.nq[1]);
    const double e1 = gp.pts[0][q1], e2 = gp.pts[1][q2], e3 = gp.pts[2][q3];
    if (kind == kGeoAnnulus) {
      const double r = 1.0 + e1, t = 0.25 * pi * e2, c = cos(t), s = sin(t), dt = 0.25 * pi * r;
      const double Ji[9] = {c, s, 0.0, -s / dt, c / dt, 0.0, 0.0, 0.0, 1.0};
      for (int i = 0; i < 9; ++i) gp.jinv[(int64_t)i * Q + q] = Ji[i];
      gp.det[q] = dt;
      gp.nu[q] = contrast > 0.0 ? 1.0 + (contrast - 1.0) * (1.0 - cos(2.0 * pi * r * c)) * 0.5 : 1.0;
      continue;
    }
    const double s1 = sin(pi * e1), s2 = sin(pi * e2), s3 = sin(pi * e3);
    const double c1 = cos(pi * e1), c2 = cos(pi * e2), c3 = cos(pi * e3);
    const double s = amp * s1 * s2 * s3;
    const double g[3] = {amp * pi * c1 * s2 * s3, amp * pi * s1 * c2 * s3, amp * pi * s1 * s2 * c3};
    const double det = 1.0 + g[0] + g[1] + g[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gp.jinv[(int64_t)(i * 3 + j) * Q + q] = (i == j ? 1.0 : 0.0) - g[j] / det;
    gp.det[q] = det;
    const double x1 = e1 + s, x2 = e2 + s;
    gp.nu[q] = contrast > 0.0 ? 1.0 + (contrast - 1.0) * (1.0 - cos(2.0 * pi * x1)) * 0.5
                              : 1.0 + 0.5 * sin(2.0 * pi * x1) * cos(2.0 * pi * x2);
  }
}

void launch_geo_points(const GeoPoints &gp, int kind, double amp, double contrast, cudaStream_t s) {
  int64_t blocks = (gp.Q + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  count_launch(1);
  k_geo_points<<<(unsigned)blocks, 256, 0, s>>>(gp, kind, amp, contrast);
}

// ------------------------------------------------------------------ separable fit

// L[f][q] = log c^k_jj(q), f = 3k + j, c^k_jj = nu |det| ((J^-1 J^-T)_jj + (J^-1)_jk^2).
__global__ void k_logc(GeoPoints gp, double *L) {
  const int64_t Q = gp.Q;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    double Ji[9];
    for (int i = 0; i < 9; ++i) Ji[i] = gp.jinv[(int64_t)i * Q + q];
    const double w = gp.nu[q] * fabs(gp.det[q]);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) {
        const double jj = Ji[j * 3 + 0] * Ji[j * 3 + 0] + Ji[j * 3 + 1] * Ji[j * 3 + 1] + Ji[j * 3 + 2] * Ji[j * 3 + 2];
        L[(int64_t)(3 * k + j) * Q + q] = log(w * (jj + Ji[j * 3 + k] * Ji[j * 3 + k]));
      }
  }
}

void launch_logc(const GeoPoints &gp, double *L, cudaStream_t s) {
  int64_t blocks = (gp.Q + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  count_launch(1);
  k_logc<<<(unsigned)blocks, 256, 0, s>>>(gp, L);
}

// One Diliberto-Straus update of direction d for all 9 fits: for every index t
// along d, f_d[t] = (max + min)/2 of L - sum_{e != d} f_e over the other two
// directions (block = (t, fit)). max/min are exact, so the result depends on
// the order of nothing.
__global__ void k_fit_sweep(const double *L, double *f, int d, int64_t Q, int n1, int n2, int n3, int fstride) {
  const int t = blockIdx.x, fit = blockIdx.y;
  const int n[3] = {n1, n2, n3};
  const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;       // the two other directions
  const double *Lf = L + (int64_t)fit * Q;
  const double *f0 = f + (int64_t)(fit * 3 + 0) * fstride, *f1 = f + (int64_t)(fit * 3 + 1) * fstride,
               *f2 = f + (int64_t)(fit * 3 + 2) * fstride;
  const double *fs[3] = {f0, f1, f2};
  double mx = -INFINITY, mn = INFINITY;
  const int m = n[da] * n[db];
  for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
    int qq[3];
    qq[d] = t;
    qq[da] = idx % n[da];
    qq[db] = idx / n[da];
    const int64_t q = ((int64_t)qq[2] * n2 + qq[1]) * n1 + qq[0];
    const double r = Lf[q] - fs[da][qq[da]] - fs[db][qq[db]];
    mx = fmax(mx, r);
    mn = fmin(mn, r);
  }
  __shared__ double smx[256], smn[256];
  smx[threadIdx.x] = mx;
  smn[threadIdx.x] = mn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) f[(int64_t)(fit * 3 + d) * fstride + t] = 0.5 * (smx[0] + smn[0]);
}

void launch_fit_sweep(const double *L, double *f, int d, const GeoPoints &gp, int fstride, cudaStream_t s) {
  count_launch(1);
  k_fit_sweep<<<dim3(gp.nq[d], 9), 256, 0, s>>>(L, f, d, gp.Q, gp.nq[0], gp.nq[1], gp.nq[2], fstride);
}

// ------------------------------------------------------------------ weighted pressure mass diagonal

// Q_ll = sum over the support of rho_l of w |det| / nu rho_l^2 (eq. weighted-pressure-mass).
__global__ void k_diag_q(GeoPoints gp, MeshTables mt, double *dq) {
  const int np1 = mt.np[0], np2 = mt.np[1], np3 = mt.np[2];
  const int64_t N = (int64_t)np1 * np2 * np3;
  const int nq = mt.nq, p = mt.p;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
    const int l1 = (int)(l % np1);
    const int64_t t = l / np1;
    const int l2 = (int)(t % np2), l3 = (int)(t / np2);
    const int ll[3] = {l1, l2, l3};
    double acc = 0.0;
    int elo[3], ehi[3];
    for (int d = 0; d < 3; ++d) {
      elo[d] = mt.p_elo[d][ll[d]];
      ehi[d] = mt.p_ehi[d][ll[d]];
    }
    for (int e3 = elo[2]; e3 <= ehi[2]; ++e3)
      for (int e2 = elo[1]; e2 <= ehi[1]; ++e2)
        for (int e1 = elo[0]; e1 <= ehi[0]; ++e1) {
          const int k1 = ll[0] - mt.p_first[0][e1], k2 = ll[1] - mt.p_first[1][e2], k3 = ll[2] - mt.p_first[2][e3];
          for (int a3 = 0; a3 < nq; ++a3) {
            const double v3 = mt.ptab[2][((int64_t)e3 * (p + 1) + k3) * nq + a3];
            const int64_t q3 = (int64_t)e3 * nq + a3;
            for (int a2 = 0; a2 < nq; ++a2) {
              const double v23 = v3 * mt.ptab[1][((int64_t)e2 * (p + 1) + k2) * nq + a2];
              const int64_t q2 = (int64_t)e2 * nq + a2;
              for (int a1 = 0; a1 < nq; ++a1) {
                const double v = v23 * mt.ptab[0][((int64_t)e1 * (p + 1) + k1) * nq + a1];
                const int64_t q1 = (int64_t)e1 * nq + a1;
                const int64_t q = (q3 * gp.nq[1] + q2) * gp.nq[0] + q1;
                const double w = gp.wts[0][q1] * gp.wts[1][q2] * gp.wts[2][q3];
                acc += w * fabs(gp.det[q]) / gp.nu[q] * v * v;
              }
            }
          }
        }
    dq[l] = acc;
  }
}

void launch_diag_q(const GeoPoints &gp, const MeshTables &mt, double *dq, cudaStream_t s) {
  const int64_t N = (int64_t)mt.np[0] * mt.np[1] * mt.np[2];
  int64_t blocks = (N + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  k_diag_q<<<(unsigned)blocks, 128, 0, s>>>(gp, mt, dq);
}

// ------------------------------------------------------------------ CSR structure

__device__ __forceinline__ void unflat(int64_t i, const int n[3], int o[3]) {
  o[0] = (int)(i % n[0]);
  const int64_t t = i / n[0];
  o[1] = (int)(t % n[1]);
  o[2] = (int)(t / n[1]);
}

// Column indices of every row: velocity row (r, i): [3 velocity boxes][pressure box];
// pressure row l: [3 velocity boxes]. Boxes enumerate j1 fastest.
__global__ void k_csr_cols(CsrTables ct, int *col) {
  const int64_t nrows = ct.off[4];
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    int64_t pos = ct.row_ptr[row];
    if (row < ct.off[3]) {
      const int r = row < ct.off[1] ? 0 : (row < ct.off[2] ? 1 : 2);
      int i[3];
      unflat(row - ct.off[r], ct.nv, i);
      const int lo[3] = {ct.vv_lo[0][i[0]], ct.vv_lo[1][i[1]], ct.vv_lo[2][i[2]]};
      const int w[3] = {ct.vv_w[0][i[0]], ct.vv_w[1][i[1]], ct.vv_w[2][i[2]]};
      const int box = w[0] * w[1] * w[2];
      for (int s = 0; s < 3; ++s)
        for (int k = threadIdx.x; k < box; k += blockDim.x) {
          const int j1 = k % w[0], j2 = (k / w[0]) % w[1], j3 = k / (w[0] * w[1]);
          col[pos + (int64_t)s * box + k] =
              (int)(ct.off[s] + ((int64_t)(lo[2] + j3) * ct.nv[1] + (lo[1] + j2)) * ct.nv[0] + (lo[0] + j1));
        }
      pos += 3 * (int64_t)box;
      const int plo[3] = {ct.vp_lo[0][i[0]], ct.vp_lo[1][i[1]], ct.vp_lo[2][i[2]]};
      const int pw[3] = {ct.vp_w[0][i[0]], ct.vp_w[1][i[1]], ct.vp_w[2][i[2]]};
      const int pbox = pw[0] * pw[1] * pw[2];
      for (int k = threadIdx.x; k < pbox; k += blockDim.x) {
        const int j1 = k % pw[0], j2 = (k / pw[0]) % pw[1], j3 = k / (pw[0] * pw[1]);
        col[pos + k] = (int)(ct.off[3] + ((int64_t)(plo[2] + j3) * ct.np[1] + (plo[1] + j2)) * ct.np[0] + (plo[0] + j1));
      }
    } else {
      int l[3];
      unflat(row - ct.off[3], ct.np, l);
      const int lo[3] = {ct.pv_lo[0][l[0]], ct.pv_lo[1][l[1]], ct.pv_lo[2][l[2]]};
      const int w[3] = {ct.pv_w[0][l[0]], ct.pv_w[1][l[1]], ct.pv_w[2][l[2]]};
      const int box = w[0] * w[1] * w[2];
      for (int s = 0; s < 3; ++s)
        for (int k = threadIdx.x; k < box; k += blockDim.x) {
          const int j1 = k % w[0], j2 = (k / w[0]) % w[1], j3 = k / (w[0] * w[1]);
          col[pos + (int64_t)s * box + k] =
              (int)(ct.off[s] + ((int64_t)(lo[2] + j3) * ct.nv[1] + (lo[1] + j2)) * ct.nv[0] + (lo[0] + j1));
        }
    }
  }
}

void launch_csr_cols(const CsrTables &ct, int *col, cudaStream_t s) {
  count_launch(1);
  k_csr_cols<<<8192, 128, 0, s>>>(ct, col);
}

// position of the entry (velocity row (r, i), velocity column (s, j)) / (velocity row, pressure column l)
__device__ __forceinline__ int64_t pos_vv(const CsrTables &ct, int r, const int i[3], int s, const int j[3]) {
  const int64_t row = ct.off[r] + ((int64_t)i[2] * ct.nv[1] + i[1]) * ct.nv[0] + i[0];
  const int w0 = ct.vv_w[0][i[0]], w1 = ct.vv_w[1][i[1]], w2 = ct.vv_w[2][i[2]];
  return ct.row_ptr[row] + (int64_t)s * w0 * w1 * w2 +
         ((int64_t)(j[2] - ct.vv_lo[2][i[2]]) * w1 + (j[1] - ct.vv_lo[1][i[1]])) * w0 + (j[0] - ct.vv_lo[0][i[0]]);
}

__device__ __forceinline__ int64_t pos_vp(const CsrTables &ct, int r, const int i[3], const int l[3]) {
  const int64_t row = ct.off[r] + ((int64_t)i[2] * ct.nv[1] + i[1]) * ct.nv[0] + i[0];
  const int64_t box = (int64_t)ct.vv_w[0][i[0]] * ct.vv_w[1][i[1]] * ct.vv_w[2][i[2]];
  const int w0 = ct.vp_w[0][i[0]], w1 = ct.vp_w[1][i[1]];
  return ct.row_ptr[row] + 3 * box +
         ((int64_t)(l[2] - ct.vp_lo[2][i[2]]) * w1 + (l[1] - ct.vp_lo[1][i[1]])) * w0 + (l[0] - ct.vp_lo[0][i[0]]);
}

__device__ __forceinline__ int64_t pos_pv(const CsrTables &ct, const int l[3], int r, const int j[3]) {
  const int64_t row = ct.off[3] + ((int64_t)l[2] * ct.np[1] + l[1]) * ct.np[0] + l[0];
  const int w0 = ct.pv_w[0][l[0]], w1 = ct.pv_w[1][l[1]], w2 = ct.pv_w[2][l[2]];
  return ct.row_ptr[row] + (int64_t)r * w0 * w1 * w2 +
         ((int64_t)(j[2] - ct.pv_lo[2][l[2]]) * w1 + (j[1] - ct.pv_lo[1][l[1]])) * w0 + (j[0] - ct.pv_lo[0][l[0]]);
}

// ------------------------------------------------------------------ element assembly

// Sum-factorized E[i][j] += sum_q F[q] prod_d L_d[i_d][q_d] R_d[j_d][q_d] over the
// element's nq^3 points (F indexed q1 fastest; E indexed i = (i3 nl + i2) nl + i1,
// j likewise with nr). T1: nl nr nq nq, T2: nl nr nl nr nq doubles.
__device__ void sumfact_acc(const double *F, const double *L[3], const double *R[3], int nl, int nr, int nq,
                            double *T1, double *T2, double *E) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n1 = nl * nr * nq * nq;
  for (int x = tid; x < n1; x += nt) {   // T1[i1][j1][q2][q3]
    const int q3 = x % nq, q2 = (x / nq) % nq, j1 = (x / (nq * nq)) % nr, i1 = x / (nq * nq * nr);
    double acc = 0.0;
    for (int q1 = 0; q1 < nq; ++q1) acc += F[(q3 * nq + q2) * nq + q1] * L[0][i1 * nq + q1] * R[0][j1 * nq + q1];
    T1[x] = acc;
  }
  __syncthreads();
  const int n2 = nl * nr * nl * nr * nq;
  for (int x = tid; x < n2; x += nt) {   // T2[i1][j1][i2][j2][q3]
    const int q3 = x % nq, j2 = (x / nq) % nr, i2 = (x / (nq * nr)) % nl, j1 = (x / (nq * nr * nl)) % nr,
              i1 = x / (nq * nr * nl * nr);
    double acc = 0.0;
    for (int q2 = 0; q2 < nq; ++q2)
      acc += T1[((i1 * nr + j1) * nq + q2) * nq + q3] * L[1][i2 * nq + q2] * R[1][j2 * nq + q2];
    T2[x] = acc;
  }
  __syncthreads();
  const int nli = nl * nl * nl, nrj = nr * nr * nr;
  for (int x = tid; x < nli * nrj; x += nt) {
    const int i = x / nrj, j = x % nrj;
    const int i1 = i % nl, i2 = (i / nl) % nl, i3 = i / (nl * nl);
    const int j1 = j % nr, j2 = (j / nr) % nr, j3 = j / (nr * nr);
    const double *t2 = T2 + (((i1 * nr + j1) * nl + i2) * nr + j2) * nq;
    double acc = 0.0;
    for (int q3 = 0; q3 < nq; ++q3) acc += t2[q3] * L[2][i3 * nq + q3] * R[2][j3 * nq + q3];
    E[x] += acc;
  }
  __syncthreads();
}

// One CTA per element: velocity blocks A_rs (C^rs_ab = nu |J| (delta_rs (J^-1 J^-T)_ab
// + (J^-1)_as (J^-1)_br)) and pressure blocks B_r (F = -w |J| (J^-1)_br), scattered
// with FP64 atomics into the CSR values.
__global__ void __launch_bounds__(256) k_assemble(GeoPoints gp, MeshTables mt, CsrTables ct, double *val) {
  extern __shared__ double sm[];
  const int nq = mt.nq, q = mt.p + 1, p = mt.p;
  const int nvl = q + 1, npl = p + 1;          // local velocity / pressure functions per direction
  const int e[3] = {(int)(blockIdx.x % mt.ne[0]), (int)((blockIdx.x / mt.ne[0]) % mt.ne[1]),
                    (int)(blockIdx.x / (mt.ne[0] * mt.ne[1]))};
  const int nq3 = nq * nq * nq;
  double *Ji = sm;                    // 9 * nq3
  double *wd = Ji + 9 * nq3;          // nq3: w |det|
  double *nuw = wd + nq3;             // nq3: nu w |det|
  double *F = nuw + nq3;              // nq3
  double *VT = F + nq3;               // [d][der][i][q]: 3 * 2 * nvl * nq
  double *PT = VT + 6 * nvl * nq;     // [d][l][q]: 3 * npl * nq
  double *T1 = PT + 3 * npl * nq;     // nvl^2 nq^2
  double *T2 = T1 + nvl * nvl * nq * nq;   // nvl^4 nq
  double *E = T2 + nvl * nvl * nvl * nvl * nq;   // nvl^6
  const int tid = threadIdx.x;
  for (int x = tid; x < nq3; x += blockDim.x) {
    const int a1 = x % nq, a2 = (x / nq) % nq, a3 = x / (nq * nq);
    const int64_t q1 = (int64_t)e[0] * nq + a1, q2 = (int64_t)e[1] * nq + a2, q3 = (int64_t)e[2] * nq + a3;
    const int64_t qq = (q3 * gp.nq[1] + q2) * gp.nq[0] + q1;
    for (int c = 0; c < 9; ++c) Ji[c * nq3 + x] = gp.jinv[(int64_t)c * gp.Q + qq];
    const double w = gp.wts[0][q1] * gp.wts[1][q2] * gp.wts[2][q3] * fabs(gp.det[qq]);
    wd[x] = w;
    nuw[x] = w * gp.nu[qq];
  }
  for (int x = tid; x < 6 * nvl * nq; x += blockDim.x) {
    const int d = x / (2 * nvl * nq), der = (x / (nvl * nq)) % 2, rest = x % (nvl * nq);
    const int i = rest / nq, a = rest % nq;
    VT[x] = mt.vtab[d][(((int64_t)e[d] * nvl + i) * nq + a) * 2 + der];
  }
  for (int x = tid; x < 3 * npl * nq; x += blockDim.x) {
    const int d = x / (npl * nq), rest = x % (npl * nq);
    const int l = rest / nq, a = rest % nq;
    PT[x] = mt.ptab[d][((int64_t)e[d] * npl + l) * nq + a];
  }
  __syncthreads();
  const int nE = nvl * nvl * nvl;
  // ---- velocity blocks
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      for (int x = tid; x < nE * nE; x += blockDim.x) E[x] = 0.0;
      __syncthreads();
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          for (int x = tid; x < nq3; x += blockDim.x) {
            double JJ = 0.0;
            if (r == s)
              for (int c = 0; c < 3; ++c) JJ += Ji[(a * 3 + c) * nq3 + x] * Ji[(b * 3 + c) * nq3 + x];
            F[x] = nuw[x] * (JJ + Ji[(a * 3 + s) * nq3 + x] * Ji[(b * 3 + r) * nq3 + x]);
          }
          __syncthreads();
          const double *Lt[3], *Rt[3];
          for (int d = 0; d < 3; ++d) {
            Lt[d] = VT + ((d * 2 + (d == a ? 1 : 0)) * nvl) * nq;
            Rt[d] = VT + ((d * 2 + (d == b ? 1 : 0)) * nvl) * nq;
          }
          sumfact_acc(F, Lt, Rt, nvl, nvl, nq, T1, T2, E);
        }
      for (int x = tid; x < nE * nE; x += blockDim.x) {
        const int il = x / nE, jl = x % nE;
        int i[3] = {il % nvl, (il / nvl) % nvl, il / (nvl * nvl)};
        int j[3] = {jl % nvl, (jl / nvl) % nvl, jl / (nvl * nvl)};
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          i[d] = mt.v_first[d][e[d]] + i[d] - 1;   // global -> interior index
          j[d] = mt.v_first[d][e[d]] + j[d] - 1;
          ok = ok && i[d] >= 0 && i[d] < ct.nv[d] && j[d] >= 0 && j[d] < ct.nv[d];
        }
        if (ok && E[x] != 0.0) atomicAdd(&val[pos_vv(ct, r, i, s, j)], E[x]);
      }
      __syncthreads();
    }
  // ---- pressure blocks: E[l][j] = sum_b int F_b rho_l d_b B_j, F_b = -w |J| (J^-1)_{b r}
  const int nP = npl * npl * npl;
  for (int r = 0; r < 3; ++r) {
    for (int x = tid; x < nP * nE; x += blockDim.x) E[x] = 0.0;
    __syncthreads();
    for (int b = 0; b < 3; ++b) {
      for (int x = tid; x < nq3; x += blockDim.x) F[x] = -wd[x] * Ji[(b * 3 + r) * nq3 + x];
      __syncthreads();
      const double *Lt[3], *Rt[3];
      for (int d = 0; d < 3; ++d) {
        Lt[d] = PT + d * npl * nq;
        Rt[d] = VT + ((d * 2 + (d == b ? 1 : 0)) * nvl) * nq;
      }
      sumfact_acc(F, Lt, Rt, npl, nvl, nq, T1, T2, E);
    }
    for (int x = tid; x < nP * nE; x += blockDim.x) {
      const int ll = x / nE, jl = x % nE;
      int l[3] = {ll % npl, (ll / npl) % npl, ll / (npl * npl)};
      int j[3] = {jl % nvl, (jl / nvl) % nvl, jl / (nvl * nvl)};
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        l[d] = mt.p_first[d][e[d]] + l[d];
        j[d] = mt.v_first[d][e[d]] + j[d] - 1;
        ok = ok && j[d] >= 0 && j[d] < ct.nv[d];
      }
      if (ok && E[x] != 0.0) {
        atomicAdd(&val[pos_pv(ct, l, r, j)], E[x]);
        atomicAdd(&val[pos_vp(ct, r, j, l)], E[x]);
      }
    }
    __syncthreads();
  }
}

size_t assemble_smem_bytes(int p) {
  const int nq = p + 2, nvl = p + 2, npl = p + 1;
  const size_t nq3 = (size_t)nq * nq * nq;
  size_t d = 12 * nq3 + 6 * nvl * nq + 3 * npl * nq + (size_t)nvl * nvl * nq * nq +
             (size_t)nvl * nvl * nvl * nvl * nq + (size_t)nvl * nvl * nvl * nvl * nvl * nvl;
  return d * sizeof(double);
}

fdst_status launch_assemble(const GeoPoints &gp, const MeshTables &mt, const CsrTables &ct, double *val,
                            cudaStream_t s) {
  const size_t smem = assemble_smem_bytes(mt.p);
  if (cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FDST_CUDA_ERROR;
  const int nel = mt.ne[0] * mt.ne[1] * mt.ne[2];
  count_launch(1);
  k_assemble<<<nel, 256, smem, s>>>(gp, mt, ct, val);
  return cudaGetLastError() == cudaSuccess ? FDST_OK : FDST_CUDA_ERROR;
}

// ------------------------------------------------------------------ SpMV and diagonal

// y_j = A x_j, one warp per row, up to 4 right-hand sides per pass over the row.
__global__ void k_spmv(const int64_t *row_ptr, const int *col, const double *val, int64_t nrows, const double *x,
                       double *y, int64_t stride, int nrhs, const int *done) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const int64_t a = row_ptr[row], b = row_ptr[row + 1];
    for (int j0 = 0; j0 < nrhs; j0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      const int nj = nrhs - j0 < 4 ? nrhs - j0 : 4;
      for (int64_t k = a + lane; k < b; k += 32) {
        const double v = val[k];
        const int c = col[k];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (jj < nj && !(done && done[j0 + jj])) acc[jj] = fma(v, x[(int64_t)(j0 + jj) * stride + c], acc[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        double t = acc[jj];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0 && jj < nj && !(done && done[j0 + jj])) y[(int64_t)(j0 + jj) * stride + row] = t;
      }
    }
  }
}

void launch_spmv(const CsrDev &A, const double *x, double *y, int64_t stride, int nrhs, const int *done,
                 cudaStream_t s) {
  count_launch(1);
  k_spmv<<<152 * 16, 256, 0, s>>>(A.row_ptr, A.col, A.val, A.nrows, x, y, stride, nrhs, done);
}

// Double-float SpMV: the same row-per-warp pass over 4 right-hand sides with
// every multiply-add on the FP32 units (12 operations instead of one FP64
// FMA at 1/64 of the rate); lanes' partial pairs are combined by shuffles.
__global__ void k_spmv_df(const int64_t *row_ptr, const int *col, const float2 *val, int64_t nrows, const float2 *x,
                          double *y, int64_t stride, int nrhs, const int *done) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const int64_t a = row_ptr[row], b = row_ptr[row + 1];
    for (int j0 = 0; j0 < nrhs; j0 += 4) {
      float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
      const int nj = nrhs - j0 < 4 ? nrhs - j0 : 4;
      bool act[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) act[jj] = jj < nj && !(done && done[j0 + jj]);
      // four nonzeros per lane per pass, 32 apart (consecutive lanes read consecutive
      // nonzeros, so the gathers of x stay coalesced); their loads are in flight together
      int64_t k = a + lane;
      for (; k + 96 < b; k += 128) {
        float2 v[4];
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = val[k + 32 * u];
          c[u] = col[k + 32 * u];
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (act[jj]) {
            const float2 *xr = x + (int64_t)(j0 + jj) * stride;
            float2 xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = xr[c[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) df_fma_acc(v[u], xv[u], sh[jj], sl[jj]);
          }
      }
      for (; k < b; k += 32) {
        const float2 vv = val[k];
        const int cc = col[k];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (act[jj]) df_fma_acc(vv, x[(int64_t)(j0 + jj) * stride + cc], sh[jj], sl[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        float h = sh[jj], l = sl[jj];
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
          df_add(h, l, oh, ol);
        }
        if (lane == 0 && act[jj]) y[(int64_t)(j0 + jj) * stride + row] = (double)h + (double)l;
      }
    }
  }
}

void launch_spmv_df(const CsrDev &A, const float2 *x2, double *y, int64_t stride, int nrhs, const int *done,
                    cudaStream_t s) {
  count_launch(1);
  k_spmv_df<<<152 * 16, 256, 0, s>>>(A.row_ptr, A.col, A.val_df, A.nrows, x2, y, stride, nrhs, done);
}

__global__ void k_csr_diag(const int64_t *row_ptr, const int *col, const double *val, int64_t nrows, double *d) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrows;
       row += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t k = row_ptr[row]; k < row_ptr[row + 1]; ++k)
      if (col[k] == row) { v = val[k]; break; }
    d[row] = v;
  }
}

void launch_csr_diag(const CsrDev &A, double *d, cudaStream_t s) {
  count_launch(1);
  k_csr_diag<<<2048, 256, 0, s>>>(A.row_ptr, A.col, A.val, A.nrows, d);
}

// ------------------------------------------------------------------ CSR blocks
// Rows [r0, r0 + nr) of a CSR matrix restricted to the columns [c_lo, c_hi): a warp
// per row, entries kept in their order (ballot prefix within each 32-entry chunk).

__global__ void k_csr_count_range(const int64_t *row_ptr, const int *col, int64_t r0, int64_t nr, int c_lo,
                                  int c_hi, int64_t *cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nr; q += nwarps) {
    const int64_t a = row_ptr[r0 + q], b = row_ptr[r0 + q + 1];
    int64_t c = 0;
    for (int64_t k0 = a; k0 < b; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool in = k < b && col[k] >= c_lo && col[k] < c_hi;
      c += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) cnt[q] = c;
  }
}

__global__ void k_csr_copy_range(const int64_t *row_ptr, const int *col, const double *val, const float2 *val_df,
                                 int64_t r0, int64_t nr, int c_lo, int c_hi, const int64_t *out_ptr, int *ocol,
                                 double *oval, float2 *oval_df) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nr; q += nwarps) {
    const int64_t a = row_ptr[r0 + q], b = row_ptr[r0 + q + 1];
    int64_t pos = out_ptr[q];
    for (int64_t k0 = a; k0 < b; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool in = k < b && col[k] >= c_lo && col[k] < c_hi;
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int64_t o = pos + __popc(m & ((1u << lane) - 1u));
        ocol[o] = col[k];
        oval[o] = val[k];
        if (oval_df) oval_df[o] = val_df[k];
      }
      pos += __popc(m);
    }
  }
}

void launch_csr_count_range(const CsrDev &A, int64_t r0, int64_t nr, int c_lo, int c_hi, int64_t *cnt,
                            cudaStream_t s) {
  count_launch(1);
  k_csr_count_range<<<152 * 16, 256, 0, s>>>(A.row_ptr, A.col, r0, nr, c_lo, c_hi, cnt);
}

void launch_csr_copy_range(const CsrDev &A, int64_t r0, int64_t nr, int c_lo, int c_hi, const int64_t *out_ptr,
                           int *ocol, double *oval, float2 *oval_df, cudaStream_t s) {
  count_launch(1);
  k_csr_copy_range<<<152 * 16, 256, 0, s>>>(A.row_ptr, A.col, A.val, A.val_df, r0, nr, c_lo, c_hi, out_ptr, ocol,
                                            oval, oval_df);
}

// ------------------------------------------------------------------ matrix-free mapped operator: the points
// At each quadrature point q (q0 fastest) and right-hand side, from the fields
// G[r][a] = d u_r / d eta_a (r, a < 3) and P = p(q) (field 3 r + a and 9, Q apart):
//   gx[r][c] = sum_a G[r][a] (J^{-1})_{ac},  sigma = nu (gx + gx^T) - P I,
//   F[r][a]  = wd sum_c sigma[r][c] (J^{-1})_{ac},  E = -wd (gx[0][0] + gx[1][1] + gx[2][2]),
// wd = w0 w1 w2 det J; F and E overwrite G and P (Sec. 3 forms a, b on the mapped domain).

__global__ void k_mf_points_f64(double *Fd, int64_t Q, int64_t fstride, const double *jinv, const double *det,
                                const double *nu, const double *w0, const double *w1, const double *w2, int q0,
                                int q1, const int *done, int mode) {
  const int rhs = blockIdx.y;
  if (done && done[rhs]) return;
  double *F = Fd + rhs * fstride;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(q % q0);
    const int64_t t = q / q0;
    const int i1 = (int)(t % q1), i2 = (int)(t / q1);
    const double wd = w0[i0] * w1[i1] * w2[i2] * det[q];
    double Ji[3][3], G[3][3], gx[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Ji[a][c] = jinv[(3 * a + c) * Q + q];
        G[a][c] = mode == 1 ? 0.0 : F[(3 * a + c) * Q + q];
      }
    const double P = mode == 2 ? 0.0 : F[9 * Q + q], nq = nu[q];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) gx[r][c] = G[r][0] * Ji[0][c] + G[r][1] * Ji[1][c] + G[r][2] * Ji[2][c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double sg[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) sg[c] = nq * (gx[r][c] + gx[c][r]) - (r == c ? P : 0.0);
      if (mode != 2)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          F[(3 * r + a) * Q + q] = wd * (sg[0] * Ji[a][0] + sg[1] * Ji[a][1] + sg[2] * Ji[a][2]);
    }
    if (mode != 1) F[9 * Q + q] = -wd * (gx[0][0] + gx[1][1] + gx[2][2]);
  }
}

__device__ __forceinline__ float2 dfx_mul(float2 a, float2 b) {
  float sh = 0.f, sl = 0.f;
  df_fma_acc(a, b, sh, sl);
  return df_norm(sh, sl);
}

__device__ __forceinline__ float2 dfx_add(float2 a, float2 b) {
  float sh = a.x, sl = a.y;
  df_add(sh, sl, b.x, b.y);
  return df_norm(sh, sl);
}

__device__ __forceinline__ float2 dfx_dot3(float2 a0, float2 b0, float2 a1, float2 b1, float2 a2, float2 b2) {
  float sh = 0.f, sl = 0.f;
  df_fma_acc(a0, b0, sh, sl);
  df_fma_acc(a1, b1, sh, sl);
  df_fma_acc(a2, b2, sh, sl);
  return df_norm(sh, sl);
}

// The same in double-float arithmetic on FP32 pairs (geometry: J^{-1}, wd and nu as pairs).
__global__ void k_mf_points_df(float2 *Fd, int64_t Q, int64_t fstride, int nrhs, const float2 *jinv,
                               const float2 *wd2, const float2 *nu2, const int *done, int mode) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    // the geometry of the point once, then every right-hand side
    float2 Ji[3][3], gx[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) Ji[a][c] = jinv[(3 * a + c) * Q + q];
    const float2 nq = nu2[q], wd = wd2[q];
    for (int rhs = 0; rhs < nrhs; ++rhs) {
    if (done && done[rhs]) continue;
    float2 *F = Fd + rhs * fstride;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 z = make_float2(0.f, 0.f);
      const float2 g0 = mode == 1 ? z : F[(3 * r) * Q + q], g1 = mode == 1 ? z : F[(3 * r + 1) * Q + q],
                   g2 = mode == 1 ? z : F[(3 * r + 2) * Q + q];
#pragma unroll
      for (int c = 0; c < 3; ++c) gx[r][c] = dfx_dot3(g0, Ji[0][c], g1, Ji[1][c], g2, Ji[2][c]);
    }
    const float2 P = mode == 2 ? make_float2(0.f, 0.f) : F[9 * Q + q];
    const float2 mP = make_float2(-P.x, -P.y);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float2 sg[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sg[c] = dfx_mul(nq, dfx_add(gx[r][c], gx[c][r]));
        if (r == c) sg[c] = dfx_add(sg[c], mP);
      }
      if (mode != 2)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          F[(3 * r + a) * Q + q] = dfx_mul(wd, dfx_dot3(sg[0], Ji[a][0], sg[1], Ji[a][1], sg[2], Ji[a][2]));
    }
    if (mode != 1) {
      const float2 dv = dfx_add(dfx_add(gx[0][0], gx[1][1]), gx[2][2]);
      const float2 e = dfx_mul(wd, dv);
      F[9 * Q + q] = make_float2(-e.x, -e.y);
    }
    }
  }
}

// Geometry as FP32 pairs: J^{-1} (9 x Q), wd = w0 w1 w2 det J, nu.
__global__ void k_mf_geo_df(const double *jinv, const double *det, const double *nu, const double *w0,
                            const double *w1, const double *w2, int q0, int q1, int64_t Q, float2 *jd, float2 *wdd,
                            float2 *nud) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(q % q0);
    const int64_t t = q / q0;
    const int i1 = (int)(t % q1), i2 = (int)(t / q1);
    for (int k = 0; k < 9; ++k) jd[k * Q + q] = f64_split(jinv[k * Q + q]);
    wdd[q] = f64_split(w0[i0] * w1[i1] * w2[i2] * det[q]);
    nud[q] = f64_split(nu[q]);
  }
}

// Coefficient fields of diag(A) at the points: for velocity component r and the
// direction pair (a, b), a <= b, C = m wd nu (sum_c Ji[a][c] Ji[b][c] + Ji[a][r] Ji[b][r])
// with m = 2 for a < b, so that A_ii = sum_pairs sum_q C (d_a phi_i)(d_b phi_i)
// (the symmetric-gradient form a(e_r phi, e_r phi)); field 6 r + pair, Q apart.
__global__ void k_mf_diag_coef(double *C, int64_t Q, const double *jinv, const double *det, const double *nu,
                               const double *w0, const double *w1, const double *w2, int q0, int q1) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(q % q0);
    const int64_t t = q / q0;
    const int i1 = (int)(t % q1), i2 = (int)(t / q1);
    const double wn = w0[i0] * w1[i1] * w2[i2] * det[q] * nu[q];
    double Ji[3][3];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) Ji[a][c] = jinv[(3 * a + c) * Q + q];
    for (int r = 0; r < 3; ++r) {
      int pi = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++pi) {
          const double g = Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2] + Ji[a][r] * Ji[b][r];
          C[(6 * r + pi) * Q + q] = (a == b ? 1.0 : 2.0) * wn * g;
        }
    }
  }
}

void launch_mf_diag_coef(double *C, const GeoPoints &gp, cudaStream_t s) {
  int64_t blocks = (gp.Q + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  k_mf_diag_coef<<<(unsigned)blocks, 256, 0, s>>>(C, gp.Q, gp.jinv, gp.det, gp.nu, gp.wts[0], gp.wts[1], gp.wts[2],
                                                  gp.nq[0], gp.nq[1]);
}

void launch_mf_points_f64(double *F, int64_t Q, int64_t fstride, int nrhs, const GeoPoints &gp, const int *done,
                          int mode, cudaStream_t s) {
  int64_t blocks = (Q + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  k_mf_points_f64<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(F, Q, fstride, gp.jinv, gp.det, gp.nu, gp.wts[0],
                                                                gp.wts[1], gp.wts[2], gp.nq[0], gp.nq[1], done, mode);
}

void launch_mf_points_df(float2 *F, int64_t Q, int64_t fstride, int nrhs, const float2 *jd, const float2 *wdd,
                         const float2 *nud, const int *done, int mode, cudaStream_t s) {
  int64_t blocks = (Q + 127) / 128;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launch(1);
  k_mf_points_df<<<(unsigned)blocks, 128, 0, s>>>(F, Q, fstride, nrhs, jd, wdd, nud, done, mode);
}

void launch_mf_geo_df(const GeoPoints &gp, float2 *jd, float2 *wdd, float2 *nud, cudaStream_t s) {
  int64_t blocks = (gp.Q + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  k_mf_geo_df<<<(unsigned)blocks, 256, 0, s>>>(gp.jinv, gp.det, gp.nu, gp.wts[0], gp.wts[1], gp.wts[2], gp.nq[0],
                                               gp.nq[1], gp.Q, jd, wdd, nud);
}

}  // namespace fdst

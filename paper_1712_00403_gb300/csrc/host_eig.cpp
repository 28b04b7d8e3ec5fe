// Host FP64 dense linear algebra for the setup: Cholesky, SPD inverse and the
// generalized symmetric eigenproblem K U = M U Lambda with U^T M U = I
// (paper eq. eig_dec; Algorithm 1 step 1). Reduction to a standard problem
// C = L^{-1} K L^{-T}, then for n <= 48 cyclic Jacobi rotations (Jacobi 1846;
// Rutishauser's stable rotation formulas) and for larger n Householder
// reduction to tridiagonal form followed by the implicit QL iteration with
// Wilkinson shifts (Bowdler, Martin, Reinsch and Wilkinson 1968), both
// accumulating the orthogonal V; U = L^{-T} V.
#include <cmath>
#include <vector>

#include "internal.h"

namespace fdst {

bool cholesky(Mat &M) {
  const int n = M.rows;
  for (int j = 0; j < n; ++j) {
    double d = M(j, j);
    for (int k = 0; k < j; ++k) d -= M(j, k) * M(j, k);
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    M(j, j) = d;
    for (int i = j + 1; i < n; ++i) {
      double s = M(i, j);
      for (int k = 0; k < j; ++k) s -= M(i, k) * M(j, k);
      M(i, j) = s / d;
    }
    for (int i = 0; i < j; ++i) M(i, j) = 0.0;
  }
  return true;
}

// X <- L^{-1} X (forward substitution, row by row: contiguous row updates), L lower triangular.
static void lower_solve(const Mat &L, Mat &X) {
  const int n = L.rows, m = X.cols;
  for (int i = 0; i < n; ++i) {
    double *xi = &X.a[(size_t)i * m];
    for (int k = 0; k < i; ++k) {
      const double l = L(i, k);
      if (l == 0.0) continue;
      const double *xk = &X.a[(size_t)k * m];
      for (int c = 0; c < m; ++c) xi[c] -= l * xk[c];
    }
    const double inv = 1.0 / L(i, i);
    for (int c = 0; c < m; ++c) xi[c] *= inv;
  }
}

// X <- L^{-T} X (back substitution with L^T, row by row).
static void upper_t_solve(const Mat &L, Mat &X) {
  const int n = L.rows, m = X.cols;
  for (int i = n - 1; i >= 0; --i) {
    double *xi = &X.a[(size_t)i * m];
    for (int k = i + 1; k < n; ++k) {
      const double l = L(k, i);
      if (l == 0.0) continue;
      const double *xk = &X.a[(size_t)k * m];
      for (int c = 0; c < m; ++c) xi[c] -= l * xk[c];
    }
    const double inv = 1.0 / L(i, i);
    for (int c = 0; c < m; ++c) xi[c] *= inv;
  }
}

static Mat transpose(const Mat &A) {
  Mat T(A.cols, A.rows);
  for (int i = 0; i < A.rows; ++i)
    for (int j = 0; j < A.cols; ++j) T(j, i) = A(i, j);
  return T;
}

// Cyclic Jacobi on a symmetric matrix A (destroyed): A = V diag(lam) V^T.
static void jacobi(Mat &A, std::vector<double> &lam, Mat &V) {
  const int n = A.rows;
  V = Mat(n, n);
  for (int i = 0; i < n; ++i) V(i, i) = 1.0;
  // A rotation is skipped when |a_pq| is below 1e-15 sqrt(a_pp a_qq) (the
  // relative rounding level); the sweeps stop when every pair is skipped.
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A(p, q);
        double app = A(p, p), aqq = A(q, q);
        if (std::fabs(apq) <= 1e-15 * std::sqrt(std::fabs(app * aqq)) || std::fabs(apq) < 1e-300) continue;
        rotated = true;
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c, tau = s / (1.0 + c);
        A(p, p) = app - t * apq;
        A(q, q) = aqq + t * apq;
        A(p, q) = A(q, p) = 0.0;
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          double arp = A(r, p), arq = A(r, q);
          double nrp = arp - s * (arq + tau * arp);
          double nrq = arq + s * (arp - tau * arq);
          A(r, p) = A(p, r) = nrp;
          A(r, q) = A(q, r) = nrq;
        }
        for (int r = 0; r < n; ++r) {
          double vrp = V(r, p), vrq = V(r, q);
          V(r, p) = vrp - s * (vrq + tau * vrp);
          V(r, q) = vrq + s * (vrp - tau * vrq);
        }
      }
    if (!rotated) break;
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A(i, i);
}

// Householder reduction of the symmetric matrix A (destroyed) to tridiagonal
// form A = Q T Q^T (diagonal d, subdiagonal e[1..n-1]), Q accumulated.
static void tridiagonalize(Mat &A, std::vector<double> &d, std::vector<double> &e, Mat &Q) {
  const int n = A.rows;
  d.assign(n, 0.0);
  e.assign(n, 0.0);
  Q = Mat(n, n);
  for (int i = 0; i < n; ++i) Q(i, i) = 1.0;
  std::vector<double> v(n), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    // reflector H = I - beta v v^T mapping A[k+1:, k] onto a multiple of e_{k+1}
    double norm = 0.0;
    for (int i = k + 1; i < n; ++i) norm += A(i, k) * A(i, k);
    norm = std::sqrt(norm);
    if (norm == 0.0) continue;
    const double x0 = A(k + 1, k);
    const double alpha = x0 >= 0 ? -norm : norm;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = A(i, k);
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // A <- H A H on the trailing block: p = beta A v, w = p - (beta/2)(v.p) v, A -= v w^T + w v^T
    for (int i = k; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += A(i, j) * v[j];
      p[i] = beta * s;
    }
    double vp = 0.0;
    for (int i = k + 1; i < n; ++i) vp += v[i] * p[i];
    const double kk = 0.5 * beta * vp;
    for (int i = k; i < n; ++i) w[i] = p[i] - kk * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j) A(i, j) -= v[i] * w[j] + w[i] * v[j];
    // Q <- Q H
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += Q(i, j) * v[j];
      s *= beta;
      for (int j = k + 1; j < n; ++j) Q(i, j) -= s * v[j];
    }
  }
  for (int i = 0; i < n; ++i) d[i] = A(i, i);
  for (int i = 1; i < n; ++i) e[i] = A(i, i - 1);
}

// Implicit QL iteration with Wilkinson shifts on the tridiagonal (d, e),
// rotations accumulated into the rows of Zt (the transposed eigenvector
// matrix, so that each rotation updates two contiguous rows; eigenvalues in d).
static bool tridiag_ql(std::vector<double> &d, std::vector<double> &e, Mat &Zt) {
  const int n = (int)d.size();
  for (int i = 1; i < n; ++i) e[i - 1] = e[i];
  if (n > 0) e[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-16 * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        double *zi = &Zt.a[(size_t)i * Zt.cols], *zj = &Zt.a[(size_t)(i + 1) * Zt.cols];
        for (int k = 0; k < Zt.cols; ++k) {
          const double zf = zj[k];
          zj[k] = s * zi[k] + c * zf;
          zi[k] = c * zi[k] - s * zf;
        }
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

bool gen_eig(const Mat &K, const Mat &M, std::vector<double> &lam, Mat &U) {
  Mat L = M;
  if (!cholesky(L)) return false;
  // C = L^{-1} K L^{-T}
  Mat C = K;
  lower_solve(L, C);          // L^{-1} K
  Mat Ct = transpose(C);      // (L^{-1} K)^T = K L^{-T} since K is symmetric
  lower_solve(L, Ct);         // L^{-1} K L^{-T}, symmetric up to rounding
  for (int i = 0; i < C.rows; ++i)
    for (int j = i + 1; j < C.cols; ++j) {
      double v = 0.5 * (Ct(i, j) + Ct(j, i));
      Ct(i, j) = Ct(j, i) = v;
    }
  Mat V;
  if (Ct.rows <= 48) {
    jacobi(Ct, lam, V);
  } else {
    // larger pencils: Householder tridiagonalization + implicit QL (about 4 n^3 flops
    // instead of about 20 n^3 for the Jacobi sweeps)
    std::vector<double> d, e;
    Mat Q;
    tridiagonalize(Ct, d, e, Q);
    Mat Vt = transpose(Q);
    if (!tridiag_ql(d, e, Vt)) return false;
    V = transpose(Vt);
    lam = d;
  }
  U = V;
  upper_t_solve(L, U);        // U = L^{-T} V
  return true;
}

bool spd_inverse(const Mat &M, Mat &Minv) {
  Mat L = M;
  if (!cholesky(L)) return false;
  Minv = Mat(M.rows, M.cols);
  for (int i = 0; i < M.rows; ++i) Minv(i, i) = 1.0;
  lower_solve(L, Minv);
  upper_t_solve(L, Minv);
  for (int i = 0; i < M.rows; ++i)
    for (int j = i + 1; j < M.cols; ++j) {
      double v = 0.5 * (Minv(i, j) + Minv(j, i));
      Minv(i, j) = Minv(j, i) = v;
    }
  return true;
}

}  // namespace fdst

// Host FP64 dense linear algebra for the setup: Cholesky, SPD inverse and the
// generalized symmetric eigenproblem K U = M U Lambda with U^T M U = I
// (paper eq. eig_dec; Algorithm 1 step 1). Reduction to a standard problem
// C = L^{-1} K L^{-T} and cyclic Jacobi rotations (Jacobi 1846; Rutishauser's
// stable rotation formulas), U = L^{-T} V.
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

// X <- L^{-1} X (forward substitution on every column), L lower triangular.
static void lower_solve(const Mat &L, Mat &X) {
  const int n = L.rows;
  for (int c = 0; c < X.cols; ++c)
    for (int i = 0; i < n; ++i) {
      double s = X(i, c);
      for (int k = 0; k < i; ++k) s -= L(i, k) * X(k, c);
      X(i, c) = s / L(i, i);
    }
}

// X <- L^{-T} X (back substitution with L^T).
static void upper_t_solve(const Mat &L, Mat &X) {
  const int n = L.rows;
  for (int c = 0; c < X.cols; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = X(i, c);
      for (int k = i + 1; k < n; ++k) s -= L(k, i) * X(k, c);
      X(i, c) = s / L(i, i);
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
  jacobi(Ct, lam, V);
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

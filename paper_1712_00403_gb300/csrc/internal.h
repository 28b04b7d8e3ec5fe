// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fdst.h"

namespace fdst {

// ----------------------------------------------------------------- host setup

// One univariate spline space restricted to a contiguous index range
// [first, first + n) of its m B-splines (Sec. 2.1; Dirichlet removal drops
// the first and last function, Sec. 2.2).
struct Space1D {
  std::vector<double> knots;
  int degree = 0;
  int first = 0;       // first kept index (0-based)
  int n = 0;           // number of kept functions
  bool nitsche = false;
  double cpen = 0.0, h = 1.0;
  int m() const { return (int)knots.size() - degree - 1; }
};

// Dense row-major matrix.
struct Mat {
  int rows = 0, cols = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int r, int c) : rows(r), cols(c), a((size_t)r * c, 0.0) {}
  double &operator()(int i, int j) { return a[(size_t)i * cols + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * cols + j]; }
};

// Validates an open knot vector on [0,1] of degree p (nondecreasing, p+1
// equal end knots, interior multiplicity in [1, p]). Returns "" when valid.
std::string validate_knots(const std::vector<double> &t, int p);

// Knot vector of degree p+1 with the same regularity (each breakpoint one more copy).
std::vector<double> elevate(const std::vector<double> &t);

// Interior multiplicity of the first interior breakpoint (1 if none).
int inner_multiplicity(const std::vector<double> &t);

// Nonzero B-splines of degree p at x (and derivatives): returns the span s;
// N[j], dN[j] belong to function s - p + j, j = 0..p.
int eval_nonzero(const std::vector<double> &t, int p, double x, double *N, double *dN);

// Gauss-Legendre rule with n points on [-1,1] (Newton on P_n).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);

// Quadrature on all nonzero spans of the breakpoints of t, npts per span.
void span_rule(const std::vector<double> &t, int npts, std::vector<double> &x, std::vector<double> &w);

// int_0^1 wt(x) b_{a,i}^(da) b_{b,j}^(db) over kept indices. wt may be empty (= 1);
// otherwise it holds the weight at every point of span_rule(knots of a, npts).
Mat mixed_matrix(const Space1D &sa, int da, const Space1D &sb, int db, int npts,
                 const std::vector<double> &wt = {});
// Stiffness with the Nitsche boundary terms when s.nitsche (tau0/tau1 scale them).
Mat stiffness_matrix(const Space1D &s, int npts, const std::vector<double> &wt = {}, double tau0 = 1.0,
                     double tau1 = 1.0);

// Cholesky M = L L^T in place (lower). Returns false when M is not SPD.
bool cholesky(Mat &M);
// Generalized symmetric eigenproblem K U = M U diag(lam), U^T M U = I (eq. eig_dec),
// by Cholesky reduction, then cyclic Jacobi (n <= 48) or Householder
// tridiagonalization + implicit QL (larger n). Returns false when M is not SPD.
bool gen_eig(const Mat &K, const Mat &M, std::vector<double> &lam, Mat &U);
// Inverse of an SPD matrix via Cholesky. Returns false when not SPD.
bool spd_inverse(const Mat &M, Mat &Minv);

// ----------------------------------------------------------------- device side

struct Band {               // banded (possibly rectangular) matrix, row i: cols [lo[i], lo[i]+w)
  int rows = 0, cols = 0, w = 0;
  double *vals = nullptr;   // device rows*w
  int *lo = nullptr;        // device rows
};

void set_error(const std::string &s);

}  // namespace fdst

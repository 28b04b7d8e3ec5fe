// Test-only C entry points onto the library's host setup code (knot checks,
// degree elevation, Gauss-Legendre, B-spline evaluation, univariate Galerkin
// matrices, the generalized eigensolver), compiled with g++ by
// tests/test_host_setup.py so that these steps of the path are checked on a
// machine without a GPU. Spaces are passed as (knots, degree, first kept
// index, kept count); matrices come back row-major.
#include <cstring>
#include <string>
#include <vector>

#include "../paper_1712_00403_gb300/csrc/internal.h"

using fdst::Mat;
using fdst::Space1D;

static Space1D space(const double *t, int nt, int p, int first, int n) {
  Space1D s;
  s.knots.assign(t, t + nt);
  s.degree = p;
  s.first = first;
  s.n = n;
  return s;
}

static void put(const Mat &A, double *out) { std::memcpy(out, A.a.data(), sizeof(double) * A.a.size()); }

extern "C" {

int shim_validate(const double *t, int nt, int p) {
  return fdst::validate_knots(std::vector<double>(t, t + nt), p).empty() ? 1 : 0;
}

// out must hold 2 nt entries; returns the length of the elevated vector.
int shim_elevate(const double *t, int nt, double *out) {
  std::vector<double> e = fdst::elevate(std::vector<double>(t, t + nt));
  std::memcpy(out, e.data(), sizeof(double) * e.size());
  return (int)e.size();
}

void shim_gauss(int n, double *x, double *w) {
  std::vector<double> gx, gw;
  fdst::gauss_legendre(n, gx, gw);
  std::memcpy(x, gx.data(), sizeof(double) * n);
  std::memcpy(w, gw.data(), sizeof(double) * n);
}

// Returns the span s; N[j], dN[j] (j = 0..p) belong to function s - p + j.
int shim_eval(const double *t, int nt, int p, double x, double *N, double *dN) {
  return fdst::eval_nonzero(std::vector<double>(t, t + nt), p, x, N, dN);
}

void shim_mixed(const double *ta, int nta, int pa, int fa, int na, int da, const double *tb, int ntb, int pb, int fb,
                int nb, int db, int npts, double *out) {
  put(fdst::mixed_matrix(space(ta, nta, pa, fa, na), da, space(tb, ntb, pb, fb, nb), db, npts), out);
}

void shim_stiffness(const double *t, int nt, int p, int first, int n, int nitsche, double cpen, double h, int npts,
                    double *out) {
  Space1D s = space(t, nt, p, first, n);
  s.nitsche = nitsche != 0;
  s.cpen = cpen;
  s.h = h;
  put(fdst::stiffness_matrix(s, npts), out);
}

// K U = M U diag(lam), U^T M U = I. Returns 1 on success, 0 when M is not SPD.
int shim_gen_eig(const double *K, const double *M, int n, double *lam, double *U) {
  Mat k(n, n), m(n, n), u;
  std::memcpy(k.a.data(), K, sizeof(double) * n * n);
  std::memcpy(m.a.data(), M, sizeof(double) * n * n);
  std::vector<double> l;
  if (!fdst::gen_eig(k, m, l, u)) return 0;
  std::memcpy(lam, l.data(), sizeof(double) * n);
  put(u, U);
  return 1;
}

}  // extern "C"

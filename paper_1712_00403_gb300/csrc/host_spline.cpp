// Host setup: knot vectors, Gauss-Legendre quadrature, B-spline evaluation
// and univariate Galerkin matrices (paper Sec. 2.1, Sec. 5 univariate factors,
// Appendix weighted factors). Runs once per handle; not on the hot path.
#include <algorithm>
#include <cmath>
#include <sstream>

#include "internal.h"

namespace fdst {

std::string validate_knots(const std::vector<double> &t, int p) {
  std::ostringstream e;
  if (p < 1) return "degree must be >= 1";
  if ((int)t.size() < 2 * (p + 1)) return "knot vector shorter than 2(p+1)";
  for (size_t i = 1; i < t.size(); ++i)
    if (!(t[i] >= t[i - 1])) return "knot vector is not nondecreasing";
  for (int i = 0; i <= p; ++i) {
    if (t[i] != 0.0) return "knot vector is not open at 0 (needs p+1 zeros)";
    if (t[t.size() - 1 - i] != 1.0) return "knot vector is not open at 1 (needs p+1 ones)";
  }
  if (t[p + 1] == 0.0 || t[t.size() - p - 2] == 1.0) return "end knot multiplicity exceeds p+1";
  size_t i = p + 1;
  while (i < t.size() - p - 1) {
    size_t j = i;
    while (j < t.size() - p - 1 && t[j] == t[i]) ++j;
    if ((int)(j - i) > p) {
      e << "interior knot " << t[i] << " has multiplicity " << (j - i) << " > p = " << p;
      return e.str();
    }
    i = j;
  }
  return "";
}

std::vector<double> elevate(const std::vector<double> &t) {
  std::vector<double> out;
  for (size_t i = 0; i < t.size(); ++i) {
    out.push_back(t[i]);
    if (i + 1 == t.size() || t[i + 1] != t[i]) out.push_back(t[i]);
  }
  return out;
}

int inner_multiplicity(const std::vector<double> &t) {
  double z1 = -1.0;
  for (double v : t)
    if (v > 0.0 && v < 1.0) { z1 = v; break; }
  if (z1 < 0) return 1;
  return (int)std::count(t.begin(), t.end(), z1);
}

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      // three-term recurrence (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1}
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1.0; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static std::vector<double> breaks(const std::vector<double> &t) {
  std::vector<double> z;
  for (double v : t)
    if (z.empty() || v != z.back()) z.push_back(v);
  return z;
}

void span_rule(const std::vector<double> &t, int npts, std::vector<double> &x, std::vector<double> &w) {
  std::vector<double> gx, gw;
  gauss_legendre(npts, gx, gw);
  std::vector<double> z = breaks(t);
  x.clear();
  w.clear();
  for (size_t e = 0; e + 1 < z.size(); ++e) {
    double a = z[e], b = z[e + 1];
    for (int q = 0; q < npts; ++q) {
      x.push_back(0.5 * (b - a) * gx[q] + 0.5 * (a + b));
      w.push_back(0.5 * (b - a) * gw[q]);
    }
  }
}

// Nonzero B-splines of degree p at x and their first derivatives: returns the
// span s (t[s] <= x < t[s+1], last nonzero span closed at 1); N[j], dN[j] are
// the values of b_{s-p+j}, j = 0..p. Triangular Cox-de Boor scheme with the
// degree p-1 values kept for the derivative formula.
int eval_nonzero(const std::vector<double> &t, int p, double x, double *N, double *dN) {
  int m = (int)t.size() - p - 1;
  int s;
  if (x >= t[m]) {
    s = m - 1;
    while (s > p && t[s] == t[s + 1]) --s;
  } else {
    s = (int)(std::upper_bound(t.begin(), t.end(), x) - t.begin()) - 1;
    if (s < p) s = p;
  }
  double left[32], right[32], Nd[32];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - t[s + 1 - j];
    right[j] = t[s + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double tmp = den != 0.0 ? N[r] / den : 0.0;
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
    if (j == p - 1)
      for (int r = 0; r <= j; ++r) Nd[r] = N[r];
  }
  if (p == 0) {
    dN[0] = 0.0;
    return s;
  }
  if (p == 1) { Nd[0] = 1.0; }
  // b_i^p' = p b_i^{p-1}/(t_{i+p}-t_i) - p b_{i+1}^{p-1}/(t_{i+p+1}-t_{i+1}); nonzero
  // degree p-1 functions at x are b_{s-p+1..s}^{p-1} = Nd[0..p-1].
  for (int j = 0; j <= p; ++j) {
    int i = s - p + j;
    double v = 0.0;
    if (j >= 1) {  // b_i^{p-1} = Nd[j-1]
      double d1 = t[i + p] - t[i];
      if (d1 > 0) v += p * Nd[j - 1] / d1;
    }
    if (j <= p - 1) {  // b_{i+1}^{p-1} = Nd[j]
      double d2 = t[i + p + 1] - t[i + 1];
      if (d2 > 0) v -= p * Nd[j] / d2;
    }
    dN[j] = v;
  }
  return s;
}

Mat mixed_matrix(const Space1D &sa, int da, const Space1D &sb, int db, int npts, const std::vector<double> &wt) {
  std::vector<double> x, w;
  span_rule(sa.knots, npts, x, w);
  Mat out(sa.n, sb.n);
  double Na[32], dNa[32], Nb[32], dNb[32];
  for (size_t q = 0; q < x.size(); ++q) {
    double wq = w[q] * (wt.empty() ? 1.0 : wt[q]);
    int s_a = eval_nonzero(sa.knots, sa.degree, x[q], Na, dNa);
    int s_b = eval_nonzero(sb.knots, sb.degree, x[q], Nb, dNb);
    const double *fa = da ? dNa : Na;
    const double *fb = db ? dNb : Nb;
    for (int i = 0; i <= sa.degree; ++i) {
      int gi = s_a - sa.degree + i - sa.first;
      if (gi < 0 || gi >= sa.n) continue;
      for (int j = 0; j <= sb.degree; ++j) {
        int gj = s_b - sb.degree + j - sb.first;
        if (gj < 0 || gj >= sb.n) continue;
        out(gi, gj) += wq * fa[i] * fb[j];
      }
    }
  }
  return out;
}

Mat stiffness_matrix(const Space1D &s, int npts, const std::vector<double> &wt, double tau0, double tau1) {
  Mat K = mixed_matrix(s, 1, s, 1, npts, wt);
  if (s.nitsche) {
    // Nitsche terms of the tangential RT factor (Sec. 5): K~ = int b'b' - [b_l'(1) b_s(1)
    // - b_l'(0) b_s(0) + b_s'(1) b_l(1) - b_s'(0) b_l(0) - 2 C_pen/h (b_l(1) b_s(1) + b_l(0) b_s(0))]
    std::vector<double> b0(s.n, 0.0), d0(s.n, 0.0), b1(s.n, 0.0), d1(s.n, 0.0);
    double N[32], dN[32];
    int sp = eval_nonzero(s.knots, s.degree, 0.0, N, dN);
    for (int j = 0; j <= s.degree; ++j) {
      int g = sp - s.degree + j - s.first;
      if (g >= 0 && g < s.n) { b0[g] = N[j]; d0[g] = dN[j]; }
    }
    sp = eval_nonzero(s.knots, s.degree, 1.0, N, dN);
    for (int j = 0; j <= s.degree; ++j) {
      int g = sp - s.degree + j - s.first;
      if (g >= 0 && g < s.n) { b1[g] = N[j]; d1[g] = dN[j]; }
    }
    double pen = 2.0 * s.cpen / s.h;
    for (int l = 0; l < s.n; ++l)
      for (int k = 0; k < s.n; ++k)
        K(l, k) -= tau1 * d1[l] * b1[k] - tau0 * d0[l] * b0[k] + tau1 * d1[k] * b1[l] - tau0 * d0[k] * b0[l] -
                   pen * (tau1 * b1[l] * b1[k] + tau0 * b0[l] * b0[k]);
  }
  return K;
}

}  // namespace fdst

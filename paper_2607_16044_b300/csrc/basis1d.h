// 1D nodal basis on the (p+1) Gauss-Legendre points, evaluated at compile time.
//
// Nodes: Newton's method on P_n from the guess -cos(pi (j + 3/4) / (n + 1/2))
// (three-term recurrence for P_n and P_n'); weights 2 / ((1 - x^2) P_n'(x)^2);
// Lagrange derivative matrix D[i][j] = l_j'(x_i) from barycentric weights,
// diagonal = -(sum of the row's off-diagonal entries); end values l_j(-1),
// l_j(+1) as products.  Derived tables: Dh = W^{-1} D^T W (the weak-form
// divergence), L(+-1) = l(+-1) / w (the lift).
//
// Everything is constexpr, so kernels declare `constexpr Tab1<S> tb =
// make_tab1<S>(P)` and, inside fully unrolled loops, every table entry is a
// compile-time constant (an instruction operand, no memory load).  The host
// runtime uses the same functions, so host and device tables are identical.
#pragma once

namespace dgx {

constexpr int MAXN = 8;  // p <= 7 (degrees 6 and 7 serve only as the point operator of over-integration)

struct Basis1 {
  int n;
  double x[MAXN], w[MAXN], D[MAXN][MAXN], lm[MAXN], lp[MAXN], dlm[MAXN], dlp[MAXN];
};

// dlm / dlp: l_j'(-1), l_j'(+1); dLm / dLp: the same divided by w_j (the
// normal derivative of a test function at a face, as the interior-penalty
// adjoint-consistency term lifts it).
template <typename S>
struct Tab1 {
  S D[MAXN][MAXN], Dh[MAXN][MAXN], lm[MAXN], lp[MAXN], Lm[MAXN], Lp[MAXN], dlm[MAXN], dlp[MAXN], dLm[MAXN],
      dLp[MAXN];
};

// cos(t) for t in [0, pi] by its Taylor series (36 terms: remainder < 1e-30)
constexpr double cos_series(double t) {
  double term = 1.0, s = 1.0;
  for (int k = 1; k < 36; ++k) {
    term *= -t * t / ((2.0 * k - 1.0) * (2.0 * k));
    s += term;
  }
  return s;
}

constexpr double abs_c(double x) { return x < 0 ? -x : x; }

// P_n(x) and P_n'(x)
constexpr void legendre_c(int n, double x, double& p, double& dp) {
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (p0 - x * p1) / (1.0 - x * x);
}

constexpr Basis1 make_basis1(int p) {
  constexpr double pi = 3.14159265358979323846;
  Basis1 B{};
  const int n = p + 1;
  B.n = n;
  for (int j = 0; j < n; ++j) {
    double x = -cos_series(pi * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P = 0, dP = 0;
      legendre_c(n, x, P, dP);
      const double dx = P / dP;
      x -= dx;
      if (abs_c(dx) < 1e-16) break;
    }
    double P = 0, dP = 0;
    legendre_c(n, x, P, dP);
    B.x[j] = x;
    B.w[j] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
  double bw[MAXN] = {};
  for (int j = 0; j < n; ++j) {
    bw[j] = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) bw[j] /= (B.x[j] - B.x[k]);
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j)
      if (i != j) {
        B.D[i][j] = (bw[j] / bw[i]) / (B.x[i] - B.x[j]);
        diag -= B.D[i][j];
      }
    B.D[i][i] = diag;
  }
  for (int j = 0; j < n; ++j) {
    B.lm[j] = 1.0;
    B.lp[j] = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) {
        B.lm[j] *= (-1.0 - B.x[k]) / (B.x[j] - B.x[k]);
        B.lp[j] *= (1.0 - B.x[k]) / (B.x[j] - B.x[k]);
      }
  }
  // l_j'(e) = l_j(e) sum_{k != j} 1 / (e - x_k) at the ends e = -1, +1 (not nodes)
  for (int j = 0; j < n; ++j) {
    double sm = 0.0, sp = 0.0;
    for (int k = 0; k < n; ++k)
      if (k != j) {
        sm += 1.0 / (-1.0 - B.x[k]);
        sp += 1.0 / (1.0 - B.x[k]);
      }
    B.dlm[j] = B.lm[j] * sm;
    B.dlp[j] = B.lp[j] * sp;
  }
  return B;
}

template <typename S>
constexpr Tab1<S> make_tab1(int p) {
  const Basis1 B = make_basis1(p);
  Tab1<S> t{};
  const int n = B.n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      t.D[i][j] = (S)B.D[i][j];
      t.Dh[i][j] = (S)(B.w[j] * B.D[j][i] / B.w[i]);
    }
  for (int j = 0; j < n; ++j) {
    t.lm[j] = (S)B.lm[j];
    t.lp[j] = (S)B.lp[j];
    t.Lm[j] = (S)(B.lm[j] / B.w[j]);
    t.Lp[j] = (S)(B.lp[j] / B.w[j]);
    t.dlm[j] = (S)B.dlm[j];
    t.dlp[j] = (S)B.dlp[j];
    t.dLm[j] = (S)(B.dlm[j] / B.w[j]);
    t.dLp[j] = (S)(B.dlp[j] / B.w[j]);
  }
  return t;
}

}  // namespace dgx

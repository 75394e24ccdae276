// Reconstruction coefficients of the tendency kernel, derived at compile time.
//
// Finite-volume reconstruction (Appendix B.2): a polynomial P(x) = sum_p a_p x^p
// whose averages over the stencil cells [n, n+1] equal the cell values q_n is
// found by solving the moment system A a = q with A[n][p] = int_n^{n+1} x^p dx.
// The interface value is P(0) = a_0, i.e. the first row of A^{-1}.  The
// Jiang-Shu smoothness indicator of a substencil is
//   beta = sum_{l=1}^{r-1} int_{-1}^{0} (d^l P/dx^l)^2 dx = a^T M a,
// a quadratic form in q through a = A^{-1} q.  Linear weights solve
// sum_s d_s c^(s) = c^(2r-1) (the full upwind stencil) in the least-squares
// sense (the system is consistent).
//
// Index space: cell n covers [n, n+1], the interface is x = 0, the upwind cell
// for flow in +x is n = -1; substencil s of WENO(2r-1) covers cells
// -r+s .. s-1; centered order 2p covers -p .. p-1.
//
// Everything here is constexpr, so the FP32 kernels see each coefficient as a
// compile-time constant: an immediate operand rather than a load from constant
// memory.  The elimination runs in double, which leaves relative errors up to
// about 1e-12 in the WENO9 entries (the moment matrices are ill conditioned) but
// rounds to the same FP32 values as the long-double derivation of coeffs.cpp for
// all 1590 entries; the FP64 kernels keep the long-double tables (uploaded to
// constant memory).
#pragma once

#include "ocn_internal.cuh"

namespace ocn {
namespace wc {

constexpr int kMaxN = 2 * kMaxR;

struct Mat {
  double m[kMaxN][kMaxN];
};

constexpr double cabs(double x) { return x < 0.0 ? -x : x; }
constexpr double cpow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// Inverse of the leading n x n block (Gauss-Jordan, partial pivoting).
constexpr Mat invert(Mat a, int n) {
  Mat inv{};
  for (int i = 0; i < n; ++i) inv.m[i][i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (cabs(a.m[r][c]) > cabs(a.m[piv][c])) piv = r;
    for (int j = 0; j < n; ++j) {
      double t = a.m[c][j]; a.m[c][j] = a.m[piv][j]; a.m[piv][j] = t;
      t = inv.m[c][j]; inv.m[c][j] = inv.m[piv][j]; inv.m[piv][j] = t;
    }
    const double d = a.m[c][c];
    for (int j = 0; j < n; ++j) { a.m[c][j] /= d; inv.m[c][j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a.m[r][c];
      for (int j = 0; j < n; ++j) { a.m[r][j] -= f * a.m[c][j]; inv.m[r][j] -= f * inv.m[c][j]; }
    }
  }
  return inv;
}

// Inverse moment matrix of cells n0 .. n0+s-1: Ainv[p][cell].
constexpr Mat moment_inverse(int n0, int s) {
  Mat A{};
  for (int c = 0; c < s; ++c) {
    const double lo = (double)(n0 + c), hi = lo + 1.0;
    for (int p = 0; p < s; ++p) A.m[c][p] = (cpow(hi, p + 1) - cpow(lo, p + 1)) / (double)(p + 1);
  }
  return invert(A, s);
}

constexpr double falling(int p, int l) {  // p (p-1) ... (p-l+1)
  double f = 1.0;
  for (int t = 0; t < l; ++t) f *= (double)(p - t);
  return f;
}

constexpr WenoTables<double> derive() {
  WenoTables<double> out{};
  for (int p = 1; p <= kMaxR; ++p) {
    const Mat Ai = moment_inverse(-p, 2 * p);
    for (int n = 0; n < 2 * p; ++n) out.cen[p][n] = Ai.m[0][n];
  }
  for (int r = 1; r <= kMaxR; ++r) {
    double sub[kMaxR][kMaxR] = {};
    for (int s = 0; s < r; ++s) {
      const Mat Ai = moment_inverse(-r + s, r);
      for (int n = 0; n < r; ++n) { sub[s][n] = Ai.m[0][n]; out.sub[r][s][n] = Ai.m[0][n]; }
      // smoothness form: beta = a^T M a, a = Ainv q
      double M[kMaxR][kMaxR] = {};
      for (int p = 0; p < r; ++p)
        for (int pp = 0; pp < r; ++pp) {
          double acc = 0.0;
          for (int l = 1; l < r; ++l) {
            if (p < l || pp < l) continue;
            const int e = p + pp - 2 * l;
            // int_{-1}^{0} x^e dx = (0 - (-1)^{e+1}) / (e+1)
            const double integral = ((e % 2) == 0 ? 1.0 : -1.0) / (double)(e + 1);
            acc += falling(p, l) * falling(pp, l) * integral;
          }
          M[p][pp] = acc;
        }
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
          double acc = 0.0;
          for (int p = 0; p < r; ++p)
            for (int pp = 0; pp < r; ++pp) acc += Ai.m[p][a] * M[p][pp] * Ai.m[pp][b];
          out.beta[r][s][a][b] = acc;
        }
    }
    // Difference form.  With d_m = t_{m+1} - t_m, t_j - t_{r-1} is a signed sum of the d between
    // r-1 and j, so q_s - t_{r-1} is linear in the r-1 differences inside substencil s; and since
    // beta_s is shift invariant (its form annihilates constants), beta_s = d^T (L^T B L) d with
    // t_local = t_local[0] + L d_local, L[n][a] = 1 for a < n.
    for (int s = 0; s < r; ++s) {
      for (int n = 0; n < r; ++n) {
        const int j = s + n;              // cell index in the upwind frame (0 .. 2r-2)
        const double c = sub[s][n];
        if (j > r - 1) for (int m = r - 1; m < j; ++m) out.gq[r][s][m - s] += c;
        if (j < r - 1) for (int m = j; m < r - 1; ++m) out.gq[r][s][m - s] -= c;
      }
      for (int a = 0; a < r - 1; ++a)
        for (int b = 0; b < r - 1; ++b) {
          double acc = 0.0;
          for (int n = 0; n < r; ++n)
            for (int n2 = 0; n2 < r; ++n2)
              if (a < n && b < n2) acc += out.beta[r][s][n][n2];
          out.dbeta[r][s][a][b] = acc;
        }
    }
    // linear weights: normal equations of the (2r-1) x r system
    const Mat Af = moment_inverse(-r, 2 * r - 1);
    double B[kMaxN][kMaxR] = {};   // B[cell][s]
    for (int c = 0; c < 2 * r - 1; ++c)
      for (int s = 0; s < r; ++s) {
        const int off = c - s;     // cell -r+c sits at position off of substencil s (covers -r+s .. s-1)
        B[c][s] = (off >= 0 && off < r) ? sub[s][off] : 0.0;
      }
    Mat N{};
    double rhs[kMaxR] = {};
    for (int s = 0; s < r; ++s) {
      for (int c = 0; c < 2 * r - 1; ++c) rhs[s] += B[c][s] * Af.m[0][c];
      for (int t = 0; t < r; ++t)
        for (int c = 0; c < 2 * r - 1; ++c) N.m[s][t] += B[c][s] * B[c][t];
    }
    const Mat Ni = invert(N, r);
    for (int s = 0; s < r; ++s) {
      double acc = 0.0;
      for (int t = 0; t < r; ++t) acc += Ni.m[s][t] * rhs[t];
      out.d[r][s] = acc;
    }
  }
  // the kernels evaluate each quadratic form over its upper triangle: off-diagonal terms doubled
  for (int r = 1; r <= kMaxR; ++r)
    for (int s = 0; s < r; ++s)
      for (int a = 0; a < r - 1; ++a)
        for (int b = 0; b < r - 1; ++b) {
          if (b > a) out.dbeta[r][s][a][b] *= 2.0;
          else if (b < a) out.dbeta[r][s][a][b] = 0.0;
        }
  return out;
}

constexpr WenoTables<double> kTables = derive();

}  // namespace wc

// Compile-time coefficients in the kernel's precision (scalar constants usable in device code).
template <typename T, int r, int s, int a>
struct WenoGq {
  static constexpr T value = (T)wc::kTables.gq[r][s][a];
};
// substencil coefficients times the substencil's linear weight d_s (the weighted sum of the
// substencil values then needs no separate multiplication by d_s)
template <typename T, int r, int s, int a>
struct WenoGqD {
  static constexpr T value = (T)(wc::kTables.gq[r][s][a] * wc::kTables.d[r][s]);
};
template <typename T, int r, int s, int a, int b>
struct WenoDb {
  static constexpr T value = (T)wc::kTables.dbeta[r][s][a][b];
};
template <typename T, int r, int s>
struct WenoD {
  static constexpr T value = (T)wc::kTables.d[r][s];
};
template <typename T, int p, int n>
struct WenoCen {
  static constexpr T value = (T)wc::kTables.cen[p][n];
};

}  // namespace ocn

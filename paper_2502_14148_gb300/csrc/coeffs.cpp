// Host derivation of the reconstruction tables used by the tendency kernel.
//
// Finite-volume reconstruction (Appendix B.2): a polynomial P(x) = sum_p a_p x^p
// whose averages over the stencil cells [n, n+1] equal the cell values q_n is
// found by solving the moment system A a = q with A[n][p] = int_n^{n+1} x^p dx.
// The interface value is P(0) = a_0, i.e. the first row of A^{-1}.  The
// Jiang-Shu smoothness indicator of a substencil is
//   beta = sum_{l=1}^{r-1} int_{-1}^{0} (d^l P/dx^l)^2 dx = a^T M a,
// a quadratic form in q through a = A^{-1} q.  Linear weights solve
// sum_s d_s c^(s) = c^(2r-1) (the full upwind stencil) in the least-squares
// sense (the system is consistent).  All in long double, then rounded.
//
// Index space: cell n covers [n, n+1], the interface is x = 0, the upwind cell
// for flow in +x is n = -1; substencil s of WENO(2r-1) covers cells
// -r+s .. s-1; centered order 2p covers -p .. p-1.
#include <math.h>
#include <string.h>

#include "ocn_internal.cuh"

namespace ocn {
namespace {

typedef long double ld;
constexpr int kMaxN = 2 * kMaxR;

// Invert an n x n matrix in place (Gauss-Jordan, partial pivoting).
void invert(ld a[kMaxN][kMaxN], int n) {
  ld inv[kMaxN][kMaxN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i][j] = (i == j) ? 1.0L : 0.0L;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(a[r][c]) > fabsl(a[piv][c])) piv = r;
    for (int j = 0; j < n; ++j) {
      ld t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
      t = inv[c][j]; inv[c][j] = inv[piv][j]; inv[piv][j] = t;
    }
    ld d = a[c][c];
    for (int j = 0; j < n; ++j) { a[c][j] /= d; inv[c][j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = a[r][c];
      for (int j = 0; j < n; ++j) { a[r][j] -= f * a[c][j]; inv[r][j] -= f * inv[c][j]; }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) a[i][j] = inv[i][j];
}

// Moment matrix of cells n0 .. n0+s-1 and its inverse: Ainv[p][cell].
void moment_inverse(int n0, int s, ld Ainv[kMaxN][kMaxN]) {
  for (int c = 0; c < s; ++c) {
    ld lo = (ld)(n0 + c), hi = lo + 1.0L;
    for (int p = 0; p < s; ++p) Ainv[c][p] = (powl(hi, p + 1) - powl(lo, p + 1)) / (ld)(p + 1);
  }
  invert(Ainv, s);
}

void reconstruction(int n0, int s, ld* w) {
  ld Ainv[kMaxN][kMaxN];
  moment_inverse(n0, s, Ainv);
  for (int c = 0; c < s; ++c) w[c] = Ainv[0][c];
}

ld falling(int p, int l) {  // p (p-1) ... (p-l+1)
  ld f = 1.0L;
  for (int t = 0; t < l; ++t) f *= (ld)(p - t);
  return f;
}

}  // namespace

void derive_weno_tables(WenoTables<double>* out) {
  memset(out, 0, sizeof(*out));
  for (int p = 1; p <= kMaxR; ++p) {
    ld w[kMaxN];
    reconstruction(-p, 2 * p, w);
    for (int n = 0; n < 2 * p; ++n) out->cen[p][n] = (double)w[n];
  }
  for (int r = 1; r <= kMaxR; ++r) {
    ld sub[kMaxR][kMaxR];
    for (int s = 0; s < r; ++s) {
      ld w[kMaxN];
      reconstruction(-r + s, r, w);
      for (int n = 0; n < r; ++n) { sub[s][n] = w[n]; out->sub[r][s][n] = (double)w[n]; }
      // smoothness form: beta = a^T M a, a = Ainv q
      ld Ainv[kMaxN][kMaxN];
      moment_inverse(-r + s, r, Ainv);
      ld M[kMaxN][kMaxN];
      for (int p = 0; p < r; ++p)
        for (int pp = 0; pp < r; ++pp) {
          ld acc = 0.0L;
          for (int l = 1; l < r; ++l) {
            if (p < l || pp < l) continue;
            int e = p + pp - 2 * l;
            // int_{-1}^{0} x^e dx = (0 - (-1)^{e+1}) / (e+1)
            ld integral = ((e % 2) == 0 ? 1.0L : -1.0L) / (ld)(e + 1);
            acc += falling(p, l) * falling(pp, l) * integral;
          }
          M[p][pp] = acc;
        }
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
          ld acc = 0.0L;
          for (int p = 0; p < r; ++p)
            for (int pp = 0; pp < r; ++pp) acc += Ainv[p][a] * M[p][pp] * Ainv[pp][b];
          out->beta[r][s][a][b] = (double)acc;
        }
    }
    // Difference form.  With d_m = t_{m+1} - t_m, t_j - t_{r-1} is a signed sum of the d between
    // r-1 and j, so q_s - t_{r-1} is linear in the r-1 differences inside substencil s; and since
    // beta_s is shift invariant (its form annihilates constants), beta_s = d^T (L^T B L) d with
    // t_local = t_local[0] + L d_local, L[n][a] = 1 for a < n.
    for (int s = 0; s < r; ++s) {
      for (int a = 0; a < r - 1; ++a) out->gq[r][s][a] = 0.0;
      for (int n = 0; n < r; ++n) {
        const int j = s + n;              // cell index in the upwind frame (0 .. 2r-2)
        const ld c = sub[s][n];
        if (j > r - 1) for (int m = r - 1; m < j; ++m) out->gq[r][s][m - s] += (double)c;
        if (j < r - 1) for (int m = j; m < r - 1; ++m) out->gq[r][s][m - s] -= (double)c;
      }
      for (int a = 0; a < r - 1; ++a)
        for (int b = 0; b < r - 1; ++b) {
          ld acc = 0.0L;
          for (int n = 0; n < r; ++n)
            for (int n2 = 0; n2 < r; ++n2)
              if (a < n && b < n2) acc += (ld)out->beta[r][s][n][n2];
          out->dbeta[r][s][a][b] = (double)acc;
        }
    }
    // linear weights: normal equations of the (2r-1) x r system
    ld full[kMaxN];
    reconstruction(-r, 2 * r - 1, full);
    ld B[kMaxN][kMaxN];   // (2r-1) x r: B[cell][s]
    for (int c = 0; c < 2 * r - 1; ++c)
      for (int s = 0; s < r; ++s) {
        int off = c - s;  // cell -r+c sits at position off of substencil s (covers -r+s .. s-1)
        B[c][s] = (off >= 0 && off < r) ? sub[s][off] : 0.0L;
      }
    ld N[kMaxN][kMaxN], rhs[kMaxN];
    for (int s = 0; s < r; ++s) {
      rhs[s] = 0.0L;
      for (int c = 0; c < 2 * r - 1; ++c) rhs[s] += B[c][s] * full[c];
      for (int t = 0; t < r; ++t) {
        N[s][t] = 0.0L;
        for (int c = 0; c < 2 * r - 1; ++c) N[s][t] += B[c][s] * B[c][t];
      }
    }
    invert(N, r);
    for (int s = 0; s < r; ++s) {
      ld acc = 0.0L;
      for (int t = 0; t < r; ++t) acc += N[s][t] * rhs[t];
      out->d[r][s] = (double)acc;
    }
  }
}

}  // namespace ocn

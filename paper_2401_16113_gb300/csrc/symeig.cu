// Dense symmetric eigendecomposition on the host, FP64: the setup of the spectral step (b) for a
// symmetric spatial operator (Riesz without drift), where (mu_k I - tau Abar)^{-1} =
// Q diag(1 / (mu_k - lambda_j)) Q^T for every frequency k once tau Abar = Q diag(lambda) Q^T.
//
// Two classical stages (Golub and Van Loan, Matrix Computations, Sec. 8.3):
//  1. Householder reduction to tridiagonal form, T = Q1^T A Q1, Q1 = H_0 H_1 ... H_{n-3}, each
//     H_k = I - 2 v v^T / (v^T v) zeroing column k below its subdiagonal;
//  2. the implicit-shift QL iteration on T (shift from the leading 2 x 2 block of the unreduced
//     part), the plane rotations accumulated into the rows of Q^T.
#include <math.h>

#include <vector>

#include "aao_internal.cuh"

namespace aao {

bool sym_eig(int n, double* A, double* w) {
  if (n <= 0) return true;
  const size_t N = (size_t)n;
  std::vector<double> d(N), e(N, 0.0);
  std::vector<std::vector<double>> refl;  // Householder vectors v_k (length n - k - 1)
  std::vector<double> beta;               // 2 / (v^T v), 0 for an identity step
  std::vector<double> p(N), q(N);
  // 1. tridiagonalisation, trailing block updated by the symmetric rank-2 form
  //    H B H = B - v q^T - q v^T, p = beta B v, q = p - (beta/2)(v^T p) v
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the part below the diagonal
    double* col = A + (size_t)(k + 1) * N + k;  // A[k+1+i][k] at col[i * n]
    double s2 = 0.0;
    for (int i = 0; i < m; ++i) s2 += col[(size_t)i * N] * col[(size_t)i * N];
    std::vector<double> v(m);
    double bk = 0.0;
    double alpha = col[0];
    if (s2 > 0.0) {
      const double x0 = col[0];
      alpha = x0 >= 0.0 ? -sqrt(s2) : sqrt(s2);
      for (int i = 0; i < m; ++i) v[i] = col[(size_t)i * N];
      v[0] = x0 - alpha;
      double vn = 0.0;
      for (int i = 0; i < m; ++i) vn += v[i] * v[i];
      bk = vn > 0.0 ? 2.0 / vn : 0.0;
    }
    if (bk != 0.0) {
      double* B = A + (size_t)(k + 1) * N + (k + 1);  // B[i][j] at B[i n + j]
      for (int i = 0; i < m; ++i) {
        const double* Bi = B + (size_t)i * N;
        double acc = 0.0;
        for (int j = 0; j < m; ++j) acc += Bi[j] * v[j];
        p[i] = bk * acc;
      }
      double vp = 0.0;
      for (int i = 0; i < m; ++i) vp += v[i] * p[i];
      const double kq = 0.5 * bk * vp;
      for (int i = 0; i < m; ++i) q[i] = p[i] - kq * v[i];
      for (int i = 0; i < m; ++i) {
        double* Bi = B + (size_t)i * N;
        const double vi = v[i], qi = q[i];
        for (int j = 0; j < m; ++j) Bi[j] -= vi * q[j] + qi * v[j];
      }
    }
    d[k] = A[(size_t)k * N + k];
    e[k] = alpha;  // T[k+1][k]
    refl.push_back(std::move(v));
    beta.push_back(bk);
  }
  if (n >= 2) {
    d[n - 2] = A[(size_t)(n - 2) * N + (n - 2)];
    e[n - 2] = A[(size_t)(n - 1) * N + (n - 2)];
  }
  d[n - 1] = A[(size_t)(n - 1) * N + (n - 1)];

  // Q1 accumulated into A as Q1^T (row r of A = column r of Q1): Q1 = H_0 (H_1 (... H_{n-3})),
  // applied innermost first; H_k touches indices >= k + 1 only. Row-wise: Q1^T <- Q1^T H_k is
  // the same update on columns k+1.. of every row.
  for (size_t i = 0; i < N * N; ++i) A[i] = 0.0;
  for (int i = 0; i < n; ++i) A[(size_t)i * N + i] = 1.0;
  for (int k = (int)refl.size() - 1; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    const std::vector<double>& v = refl[k];
    const int m = (int)v.size(), o = k + 1;
    // Q1 <- H_k Q1 on rows/cols >= o; in the transposed storage Qt = Q1^T: Qt <- Qt H_k,
    // rows r >= o of Qt carry the non-identity part (Qt is identity on indices <= k)
    for (int r = o; r < n; ++r) {
      double* Qr = A + (size_t)r * N + o;
      double dot = 0.0;
      for (int j = 0; j < m; ++j) dot += Qr[j] * v[j];
      const double f = beta[k] * dot;
      for (int j = 0; j < m; ++j) Qr[j] -= f * v[j];
    }
  }
  // (A now holds Q1^T: column j of Q1 is row j of A.)

  // 2. implicit-shift QL on (d, e), e[i] = T[i+1][i]; rotations of columns (i, i+1) of the
  //    eigenvector matrix Q = Q1 G_1 G_2 ... act on rows (i, i+1) of Q^T = A
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 64) return false;
      // Wilkinson-type shift from the 2 x 2 block at l
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      bool deflated = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // underflow: the block splits at i
          d[i + 1] -= pp;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        double* Qi = A + (size_t)i * N;
        double* Qj = A + (size_t)(i + 1) * N;
        for (int k = 0; k < n; ++k) {
          const double qa = Qi[k], qb = Qj[k];
          Qj[k] = s * qa + c * qb;
          Qi[k] = c * qa - s * qb;
        }
      }
      if (deflated) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  for (int j = 0; j < n; ++j) w[j] = d[j];
  return true;
}

}  // namespace aao

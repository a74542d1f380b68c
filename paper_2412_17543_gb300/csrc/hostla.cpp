// Dense FP64 linear algebra for the one-time setup (host). Plain loops ordered so
// that the inner loop is a contiguous dot product or axpy (auto-vectorised).
#include "hostla.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace dd {
namespace la {

bool cholesky(int n, double* A) {
  // left-looking, row oriented: row j of L from rows 0..j-1
  for (int j = 0; j < n; ++j) {
    double* Aj = A + (size_t)j * n;
    for (int i = 0; i < j; ++i) {
      const double* Li = A + (size_t)i * n;
      double s = Aj[i];
      for (int k = 0; k < i; ++k) s -= Aj[k] * Li[k];
      Aj[i] = s / Li[i];
    }
    double d = Aj[j];
    for (int k = 0; k < j; ++k) d -= Aj[k] * Aj[k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    Aj[j] = std::sqrt(d);
    for (int k = j + 1; k < n; ++k) Aj[k] = 0.0;
  }
  return true;
}

void tri_inv_lower(int n, const double* L, double* X) {
  // solve L X = I column block by row: X row i from rows < i
  std::fill(X, X + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double* Xi = X + (size_t)i * n;
    const double* Li = L + (size_t)i * n;
    // X[i][j] = (delta_ij - sum_{k<i} L[i][k] X[k][j]) / L[i][i], for j <= i
    for (int k = 0; k < i; ++k) {
      double lik = Li[k];
      if (lik == 0.0) continue;
      const double* Xk = X + (size_t)k * n;
      for (int j = 0; j <= k; ++j) Xi[j] -= lik * Xk[j];
    }
    Xi[i] += 1.0;
    double inv = 1.0 / Li[i];
    for (int j = 0; j <= i; ++j) Xi[j] *= inv;
  }
}

bool spd_inverse(int n, const double* A, double* Ainv) {
  std::vector<double> L(A, A + (size_t)n * n), Li((size_t)n * n);
  if (!cholesky(n, L.data())) return false;
  tri_inv_lower(n, L.data(), Li.data());
  // A^{-1} = Li^T Li : entry (i,j) = sum_k Li[k][i] Li[k][j], k >= max(i,j)
  // transpose so the sums become row dot products: T = Li^T (upper), A^{-1}[i][j] = T[i].T[j]
  std::vector<double> T((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) T[(size_t)i * n + k] = Li[(size_t)k * n + i];
  for (int i = 0; i < n; ++i) {
    const double* Ti = T.data() + (size_t)i * n;
    for (int j = 0; j <= i; ++j) {
      const double* Tj = T.data() + (size_t)j * n;
      double s = 0.0;
      for (int k = i; k < n; ++k) s += Ti[k] * Tj[k];
      Ainv[(size_t)i * n + j] = s;
      Ainv[(size_t)j * n + i] = s;
    }
  }
  return true;
}

void gemm_nt(int n, int m, int k, double alpha, const double* A, const double* B, double beta, double* C) {
  const int BS = 32;
  for (int i0 = 0; i0 < n; i0 += BS)
    for (int j0 = 0; j0 < m; j0 += BS)
      for (int i = i0; i < std::min(n, i0 + BS); ++i) {
        const double* Ai = A + (size_t)i * k;
        for (int j = j0; j < std::min(m, j0 + BS); ++j) {
          const double* Bj = B + (size_t)j * k;
          double s = 0.0;
          for (int t = 0; t < k; ++t) s += Ai[t] * Bj[t];
          double& c = C[(size_t)i * m + j];
          c = alpha * s + (beta == 0.0 ? 0.0 : beta * c);
        }
      }
}

void gemm_nn(int n, int m, int k, const double* A, const double* B, double* C) {
  std::fill(C, C + (size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i) {
    double* Ci = C + (size_t)i * m;
    const double* Ai = A + (size_t)i * k;
    for (int t = 0; t < k; ++t) {
      double a = Ai[t];
      if (a == 0.0) continue;
      const double* Bt = B + (size_t)t * m;
      for (int j = 0; j < m; ++j) Ci[j] += a * Bt[j];
    }
  }
}

void trmm_lower(int n, int m, const double* L, const double* X, double* Y) {
  std::fill(Y, Y + (size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i) {
    double* Yi = Y + (size_t)i * m;
    const double* Li = L + (size_t)i * n;
    for (int t = 0; t <= i; ++t) {
      double a = Li[t];
      if (a == 0.0) continue;
      const double* Xt = X + (size_t)t * m;
      for (int j = 0; j < m; ++j) Yi[j] += a * Xt[j];
    }
  }
}

void sym_eig(int n, double* A, double* w, double* V) {
  // 1) Householder reduction A = Q T Q^T (T tridiagonal), Q accumulated (Golub & Van Loan Sect. 8.3.1).
  //    Q is kept transposed (row r of Qt = column r of Q), so that the reflections and the
  //    rotations of step 2 update contiguous rows.
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  std::vector<double> Qt((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Qt[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), q(n), dots(n);
  for (int k = 0; k + 2 < n; ++k) {
    int m = n - k - 1;  // trailing size
    double alpha = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = a(k + 1 + i, k);
      alpha += v[i] * v[i];
    }
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (v[0] > 0) alpha = -alpha;
    v[0] -= alpha;
    double vn2 = 0.0;
    for (int i = 0; i < m; ++i) vn2 += v[i] * v[i];
    if (vn2 == 0.0) continue;
    double beta = 2.0 / vn2;
    for (int i = 0; i < m; ++i) {  // p = beta B v
      const double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      double sacc = 0.0;
      for (int j = 0; j < m; ++j) sacc += row[j] * v[j];
      p[i] = beta * sacc;
    }
    double K = 0.0;
    for (int i = 0; i < m; ++i) K += v[i] * p[i];
    K *= 0.5 * beta;
    for (int i = 0; i < m; ++i) q[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i) {  // B -= v q^T + q v^T
      double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      const double vi = v[i], qi = q[i];
      for (int j = 0; j < m; ++j) row[j] -= vi * q[j] + qi * v[j];
    }
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    for (int i = 1; i < m; ++i) a(k + 1 + i, k) = a(k, k + 1 + i) = 0.0;
    // Q = Q H, i.e. Qt = H Qt on rows k+1 .. n-1: Qt_rows -= beta v (v^T Qt_rows)
    std::fill(dots.begin(), dots.end(), 0.0);
    for (int i = 0; i < m; ++i) {
      const double* row = Qt.data() + (size_t)(k + 1 + i) * n;
      const double vi = v[i];
      for (int c = 0; c < n; ++c) dots[c] += vi * row[c];
    }
    for (int i = 0; i < m; ++i) {
      double* row = Qt.data() + (size_t)(k + 1 + i) * n;
      const double f = beta * v[i];
      for (int c = 0; c < n; ++c) row[c] -= f * dots[c];
    }
  }
  // 2) implicit symmetric QR steps with Wilkinson shifts on the tridiagonal (d, e), bulge
  //    chased by Givens rotations (Golub & Van Loan Alg. 8.3.2), rotations accumulated in Qt
  std::vector<double> d(n), e(n, 0.0);  // e[i] = T(i, i-1)
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 1; i < n; ++i) e[i] = a(i, i - 1);
  const double eps = 2.220446049250313e-16;
  // an off-diagonal entry is negligible relative to its diagonal neighbours or to the norm of T
  // (the latter deflates blocks of numerically zero eigenvalues, whose neighbours are ~0 too)
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    double rs = std::fabs(d[i]) + (i > 0 ? std::fabs(e[i]) : 0.0) + (i + 1 < n ? std::fabs(e[i + 1]) : 0.0);
    tnorm = std::max(tnorm, rs);
  }
  auto small = [&](int i) {  // entry (i, i-1)
    double ei = std::fabs(e[i]);
    return ei <= eps * (std::fabs(d[i]) + std::fabs(d[i - 1])) || ei <= 4 * eps * tnorm;
  };
  int hi = n - 1, iter = 0;
  while (hi > 0 && iter < 100 * n) {
    if (small(hi)) {
      e[hi] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !small(lo)) --lo;
    if (lo > 0) e[lo] = 0.0;
    double dd = 0.5 * (d[hi - 1] - d[hi]), eh = e[hi];
    double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::sqrt(dd * dd + eh * eh);
    double mu = d[hi] - (den != 0.0 ? eh * eh / den : 0.0);
    double x = d[lo] - mu, z = e[lo + 1];
    double bulge = 0.0;  // T(k+2, k) while chasing
    for (int k = lo; k < hi; ++k) {
      double r = std::hypot(x, z);
      double c = r > 0 ? x / r : 1.0, sn = r > 0 ? z / r : 0.0;
      // similarity with the rotation G(k, k+1) on the 4 x 4 band window rows/columns k-1 .. k+2
      if (k > lo) e[k] = r;  // the rotated (k, k-1) entry; the bulge (k+1, k-1) becomes 0
      const double dk = d[k], dk1 = d[k + 1], ek1 = e[k + 1];
      d[k] = c * c * dk + 2 * c * sn * ek1 + sn * sn * dk1;
      d[k + 1] = sn * sn * dk - 2 * c * sn * ek1 + c * c * dk1;
      e[k + 1] = c * sn * (dk1 - dk) + (c * c - sn * sn) * ek1;
      if (k + 1 < hi) {
        const double ek2 = e[k + 2];
        bulge = sn * ek2;
        e[k + 2] = c * ek2;
        x = e[k + 1];
        z = bulge;
      }
      double* r0 = Qt.data() + (size_t)k * n;
      double* r1 = r0 + n;
      for (int t = 0; t < n; ++t) {
        const double xx = r0[t], yy = r1[t];
        r0[t] = c * xx + sn * yy;
        r1[t] = -sn * xx + c * yy;
      }
    }
    ++iter;
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] < d[j]; });
  for (int c = 0; c < n; ++c) {
    w[c] = d[idx[c]];
    const double* row = Qt.data() + (size_t)idx[c] * n;
    for (int k = 0; k < n; ++k) V[(size_t)k * n + c] = row[k];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) a(i, j) = i == j ? d[i] : (std::abs(i - j) == 1 ? e[std::max(i, j)] : 0.0);
}

}  // namespace la
}  // namespace dd

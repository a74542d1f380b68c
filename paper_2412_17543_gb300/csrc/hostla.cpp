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
  // cyclic Jacobi rotations (Golub & Van Loan, Alg. 8.5.3); converges quadratically
  std::fill(V, V + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  double fro = 0.0;
  for (size_t t = 0; t < (size_t)n * n; ++t) fro += A[t] * A[t];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    if (off <= 1e-30 * fro || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return a(i, i) < a(j, j); });
  std::vector<double> Vs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    w[c] = a(idx[c], idx[c]);
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + c] = V[(size_t)k * n + idx[c]];
  }
  std::copy(Vs.begin(), Vs.end(), V);
}

}  // namespace la
}  // namespace dd

// Dense FP64 linear algebra for the one-time setup (host, row-major storage).
#pragma once
#include <vector>

namespace dd {
namespace la {

using Mat = std::vector<double>;  // row-major n x m

// A (n x n SPD) -> lower Cholesky factor in place (upper part zeroed). Returns false on a
// non-positive pivot.
bool cholesky(int n, double* A);
// Inverse of a lower-triangular L (n x n) -> lower-triangular Linv (separate buffer).
void tri_inv_lower(int n, const double* L, double* Linv);
// Inverse of an SPD matrix (n x n) via Cholesky; returns false if not SPD.
bool spd_inverse(int n, const double* A, double* Ainv);
// C (n x m) = alpha * A (n x k) * B(m x k)^T + beta * C  (dot products of rows)
void gemm_nt(int n, int m, int k, double alpha, const double* A, const double* B, double beta, double* C);
// C (n x m) = A (n x k) * B (k x m)
void gemm_nn(int n, int m, int k, const double* A, const double* B, double* C);
// Y (n x m) = L (n x n lower) * X (n x m)
void trmm_lower(int n, int m, const double* L, const double* X, double* Y);
// Symmetric eigen-decomposition (Householder tridiagonalization, implicit shifted QR):
// A (n x n, destroyed) -> eigenvalues w
// (ascending) and eigenvectors as columns of V (n x n row-major).
void sym_eig(int n, double* A, double* w, double* V);

}  // namespace la
}  // namespace dd

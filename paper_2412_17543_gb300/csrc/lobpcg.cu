// Batched block LOBPCG for the adaptive face eigenproblems (Sect. 3.3, eq. 10): for every
// face shared by two subdomains s, t, the k largest eigenpairs of
//   Lhs w = lambda Rhs w,  Lhs = Pi (I-E)^T A (I-E) Pi,  Rhs = Pi A Pi,  A = diag(A_s, A_t),
// on the 2m unknowns of the face's common interface (both copies). The paper solves these by
// LOBPCG with at most 15 steps and 10 vectors per face. Here each face is a CTA of a
// persistent kernel; Lhs and Rhs are applied matrix-free from the two m x m Schur
// complements, the weights of E and an orthonormal basis Q of the jumps that Pi removes.
//
// The steps, in this order (the oracle's lobpcg_largest with its face projector):
//   X = proj(unit vectors at the k largest diag((I-E)^T A (I-E)) / diag(A));
//   Rayleigh-Ritz on X; then `iters` times: W = proj(Lhs X - Rhs X theta), Rayleigh-Ritz on
//   S = [X, W] (first step) or [X, W, P], X <- S Y, P <- S Y with the X rows of Y zeroed.
// Rayleigh-Ritz: columns scaled to unit Rhs-norm (columns below 1e-14 of the largest are
// dropped), an in-order Cholesky of the scaled S^T Rhs S dropping pivots below 1e-8, the
// eigen-decomposition of L^{-1} (S^T Lhs S) L^{-T} by cyclic Jacobi (parallel ordering), the
// k largest pairs. proj: remove the span of Q and, when both subdomains float (A_s 1 = A_t 1
// = 0), the common constant.
// FP64 throughout (one-time setup work).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.h"
#include "lobpcg.h"

namespace dd {

namespace {

constexpr int LT = 256;       // threads per CTA
constexpr int LW = LT / 32;   // warps
constexpr int MAXQ = 3 * LOBPCG_MAXK;

struct FaceView {
  int m, n, nq, floating;
  const double* As;  // m x m row-major
  const double* At;
  const double* ws;  // m
  const double* wt;
  const double* Q;   // nq columns of n
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// V[:, c] (c < kc, column stride ld) <- proj(V[:, c])
__device__ void proj_cols(const FaceView& f, double* V, int ld, int kc, double* coef) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < f.nq * kc; p += LW) {
    const int a = p % f.nq, c = p / f.nq;
    double sacc = 0.0;
    for (int i = lane; i < f.n; i += 32) sacc += f.Q[(size_t)a * f.n + i] * V[(size_t)c * ld + i];
    sacc = warp_sum_d(sacc);
    if (lane == 0) coef[c * LOBPCG_MAXNQ + a] = sacc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < f.n * kc; e += LT) {
    const int i = e % f.n, c = e / f.n;
    double v = V[(size_t)c * ld + i];
    for (int a = 0; a < f.nq; ++a) v -= coef[c * LOBPCG_MAXNQ + a] * f.Q[(size_t)a * f.n + i];
    V[(size_t)c * ld + i] = v;
  }
  __syncthreads();
  if (!f.floating) return;
  const double isq = 1.0 / sqrt((double)f.n);
  for (int c = warp; c < kc; c += LW) {
    double sacc = 0.0;
    for (int i = lane; i < f.n; i += 32) sacc += V[(size_t)c * ld + i];
    sacc = warp_sum_d(sacc);
    if (lane == 0) coef[c * LOBPCG_MAXNQ] = sacc * isq;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < f.n * kc; e += LT) {
    const int i = e % f.n, c = e / f.n;
    V[(size_t)c * ld + i] -= coef[c * LOBPCG_MAXNQ] * isq;
  }
  __syncthreads();
}

// Out[:, c] = diag(A_s, A_t) In[:, c]: a warp per output row, lanes along the row
__device__ void block_a(const FaceView& f, const double* In, double* Out, int ld, int kc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < f.n; r += LW) {
    const bool second = r >= f.m;
    const double* row = (second ? f.At : f.As) + (size_t)(second ? r - f.m : r) * f.m;
    const int off = second ? f.m : 0;
    double acc[LOBPCG_MAXK];
#pragma unroll
    for (int c = 0; c < LOBPCG_MAXK; ++c) acc[c] = 0.0;
    for (int j = lane; j < f.m; j += 32) {
      const double a = row[j];
#pragma unroll
      for (int c = 0; c < LOBPCG_MAXK; ++c)
        if (c < kc) acc[c] += a * In[(size_t)c * ld + off + j];
    }
#pragma unroll
    for (int c = 0; c < LOBPCG_MAXK; ++c)
      if (c < kc) {
        const double v = warp_sum_d(acc[c]);
        if (lane == 0) Out[(size_t)c * ld + r] = v;
      }
  }
  __syncthreads();
}

// AW = Lhs W, BW = Rhs W for the kc columns of W (U, T: work blocks of kc columns)
__device__ void apply_pencil(const FaceView& f, const double* W, double* AW, double* BW, double* U, double* T,
                             int ld, int kc, double* coef) {
  for (int e = threadIdx.x; e < f.n * kc; e += LT) U[(size_t)(e / f.n) * ld + e % f.n] = W[(size_t)(e / f.n) * ld + e % f.n];
  __syncthreads();
  proj_cols(f, U, ld, kc, coef);  // U = Pi W
  block_a(f, U, T, ld, kc);
  for (int e = threadIdx.x; e < f.n * kc; e += LT) BW[(size_t)(e / f.n) * ld + e % f.n] = T[(size_t)(e / f.n) * ld + e % f.n];
  __syncthreads();
  proj_cols(f, BW, ld, kc, coef);  // Rhs W = Pi A Pi W
  for (int e = threadIdx.x; e < f.m * kc; e += LT) {  // U <- (I - E) U
    const int i = e % f.m, c = e / f.m;
    double* u = U + (size_t)c * ld;
    const double ev = f.ws[i] * u[i] + f.wt[i] * u[f.m + i];
    u[i] -= ev;
    u[f.m + i] -= ev;
  }
  __syncthreads();
  block_a(f, U, T, ld, kc);
  for (int e = threadIdx.x; e < f.m * kc; e += LT) {  // T <- (I - E)^T T
    const int i = e % f.m, c = e / f.m;
    double* t = T + (size_t)c * ld;
    const double sv = t[i] + t[f.m + i];
    t[i] -= f.ws[i] * sv;
    t[f.m + i] -= f.wt[i] * sv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < f.n * kc; e += LT) AW[(size_t)(e / f.n) * ld + e % f.n] = T[(size_t)(e / f.n) * ld + e % f.n];
  __syncthreads();
  proj_cols(f, AW, ld, kc, coef);  // Lhs W = Pi (I-E)^T A (I-E) Pi W
}

struct RRShared {
  double GA[MAXQ * MAXQ], GB[MAXQ * MAXQ], L[MAXQ * MAXQ], Li[MAXQ * MAXQ], C[MAXQ * MAXQ], V[MAXQ * MAXQ];
  double d[MAXQ], th[MAXQ], cs[MAXQ / 2], sn[MAXQ / 2];
  int keep[MAXQ], ord[MAXQ], pp[MAXQ / 2], qq[MAXQ / 2];
  int r, msel;
  double off;
  double Y[MAXQ * LOBPCG_MAXK];  // q x msel
};

// Rayleigh-Ritz on the q columns S[:, col(c)] (col: slot of RR column c); fills sh.Y, sh.th
// (descending, msel of them) and returns msel
__device__ int rayleigh_ritz(const double* S, const double* AS, const double* BS, const int* col, int q, int k, int ld,
                             int n, RRShared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < q * q; p += LW) {
    const int a = p / q, b = p % q;
    const double* sa = S + (size_t)col[a] * ld;
    const double* ab = AS + (size_t)col[b] * ld;
    const double* bb = BS + (size_t)col[b] * ld;
    double ga = 0.0, gb = 0.0;
    for (int i = lane; i < n; i += 32) {
      ga += sa[i] * ab[i];
      gb += sa[i] * bb[i];
    }
    ga = warp_sum_d(ga);
    gb = warp_sum_d(gb);
    if (lane == 0) {
      sh.GA[a * MAXQ + b] = ga;
      sh.GB[a * MAXQ + b] = gb;
    }
  }
  __syncthreads();
  // symmetrize, scale the columns to unit B-norm (dropping B-null columns)
  if (threadIdx.x == 0) {
    double gmax = 0.0;
    for (int j = 0; j < q; ++j) gmax = fmax(gmax, 0.5 * (sh.GB[j * MAXQ + j] + sh.GB[j * MAXQ + j]));
    for (int j = 0; j < q; ++j) {
      const double g = sh.GB[j * MAXQ + j];
      sh.d[j] = g > 1e-14 * gmax ? 1.0 / sqrt(g) : 0.0;
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < q * q; p += LT) {
    const int a = p / q, b = p % q;
    if (a < b) continue;
    const double ga = 0.5 * (sh.GA[a * MAXQ + b] + sh.GA[b * MAXQ + a]) * sh.d[a] * sh.d[b];
    const double gb = 0.5 * (sh.GB[a * MAXQ + b] + sh.GB[b * MAXQ + a]) * sh.d[a] * sh.d[b];
    sh.C[a * MAXQ + b] = ga;  // scaled GA (lower half, C used as a staging buffer)
    sh.C[b * MAXQ + a] = ga;
    sh.V[a * MAXQ + b] = gb;  // scaled GB
    sh.V[b * MAXQ + a] = gb;
  }
  __syncthreads();
  // in-order Cholesky of the scaled GB, dropping pivots below 1e-8 of the largest diagonal
  if (threadIdx.x == 0) {
    double scale = 0.0;
    for (int j = 0; j < q; ++j) scale = fmax(scale, sh.V[j * MAXQ + j]);
    int r = 0;
    double row[MAXQ];
    for (int j = 0; j < q; ++j) {
      for (int a = 0; a < r; ++a) {
        double v = sh.V[j * MAXQ + sh.keep[a]];
        for (int b = 0; b < a; ++b) v -= sh.L[a * MAXQ + b] * row[b];
        row[a] = v / sh.L[a * MAXQ + a];
      }
      double piv = sh.V[j * MAXQ + j];
      for (int a = 0; a < r; ++a) piv -= row[a] * row[a];
      if (piv > 1e-8 * scale) {
        for (int a = 0; a < r; ++a) sh.L[r * MAXQ + a] = row[a];
        sh.L[r * MAXQ + r] = sqrt(piv);
        sh.keep[r] = j;
        ++r;
      }
    }
    sh.r = r;
  }
  __syncthreads();
  const int r = sh.r;
  // Li = L^{-1}: column c by forward substitution (a thread per column)
  if (threadIdx.x < r) {
    const int c = threadIdx.x;
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int b = c; b < i; ++b) v -= sh.L[i * MAXQ + b] * sh.Li[b * MAXQ + c];
      sh.Li[i * MAXQ + c] = i >= c ? v / sh.L[i * MAXQ + i] : 0.0;
    }
  }
  __syncthreads();
  // C = Li GA_kk Li^T (GA_kk: the kept rows/columns of the scaled GA, staged in C): via GB buffer
  for (int p = threadIdx.x; p < r * r; p += LT) {  // GB <- GA_kk Li^T
    const int i = p / r, j = p % r;
    double v = 0.0;
    for (int b = 0; b <= j; ++b) v += sh.C[sh.keep[i] * MAXQ + sh.keep[b]] * sh.Li[j * MAXQ + b];
    sh.GB[i * MAXQ + j] = v;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < r * r; p += LT) {  // GA <- Li GB
    const int i = p / r, j = p % r;
    double v = 0.0;
    for (int b = 0; b <= i; ++b) v += sh.Li[i * MAXQ + b] * sh.GB[b * MAXQ + j];
    sh.GA[i * MAXQ + j] = v;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < r * r; p += LT) {
    const int i = p / r, j = p % r;
    sh.C[i * MAXQ + j] = 0.5 * (sh.GA[i * MAXQ + j] + sh.GA[j * MAXQ + i]);
    sh.V[i * MAXQ + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  // cyclic Jacobi with the round-robin ordering: each step rotates r'/2 disjoint pairs
  const int re = (r + 1) / 2 * 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
          const double v = sh.C[i * MAXQ + j] * sh.C[i * MAXQ + j];
          tot += v;
          if (i != j) off += v;
        }
      sh.off = off <= 1e-30 * tot ? 0.0 : off;
    }
    __syncthreads();
    if (sh.off == 0.0) break;
    for (int step = 0; step < re - 1; ++step) {
      if (threadIdx.x < re / 2) {
        const int t = threadIdx.x;
        // round-robin: player re-1 fixed, the others rotate
        int a = t == 0 ? re - 1 : (step + t) % (re - 1);
        int b = (step + re - 1 - t) % (re - 1);
        if (t == 0) b = step % (re - 1);
        if (a > b) {
          const int x = a;
          a = b;
          b = x;
        }
        sh.pp[t] = a;
        sh.qq[t] = b;
        double c = 1.0, sv = 0.0;
        if (b < r) {
          const double apq = sh.C[a * MAXQ + b];
          if (apq != 0.0) {
            const double tau = (sh.C[b * MAXQ + b] - sh.C[a * MAXQ + a]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            sv = tt * c;
          }
        }
        sh.cs[t] = c;
        sh.sn[t] = sv;
      }
      __syncthreads();
      // rows p, q of C <- J^T C
      for (int e = threadIdx.x; e < (re / 2) * r; e += LT) {
        const int t = e / r, x = e % r;
        const int a = sh.pp[t], b = sh.qq[t];
        if (b >= r) continue;
        const double c = sh.cs[t], sv = sh.sn[t];
        const double ca = sh.C[a * MAXQ + x], cb = sh.C[b * MAXQ + x];
        sh.C[a * MAXQ + x] = c * ca - sv * cb;
        sh.C[b * MAXQ + x] = sv * ca + c * cb;
      }
      __syncthreads();
      // columns p, q of C <- C J, and of V <- V J
      for (int e = threadIdx.x; e < (re / 2) * r; e += LT) {
        const int t = e / r, x = e % r;
        const int a = sh.pp[t], b = sh.qq[t];
        if (b >= r) continue;
        const double c = sh.cs[t], sv = sh.sn[t];
        const double ca = sh.C[x * MAXQ + a], cb = sh.C[x * MAXQ + b];
        sh.C[x * MAXQ + a] = c * ca - sv * cb;
        sh.C[x * MAXQ + b] = sv * ca + c * cb;
        const double va = sh.V[x * MAXQ + a], vb = sh.V[x * MAXQ + b];
        sh.V[x * MAXQ + a] = c * va - sv * vb;
        sh.V[x * MAXQ + b] = sv * va + c * vb;
      }
      __syncthreads();
    }
  }
  // the k largest eigenvalues, descending (ties: lower index first)
  if (threadIdx.x == 0) {
    for (int i = 0; i < r; ++i) {
      sh.th[i] = sh.C[i * MAXQ + i];
      sh.ord[i] = i;
    }
    for (int i = 1; i < r; ++i) {
      const int x = sh.ord[i];
      int j = i - 1;
      while (j >= 0 && sh.th[sh.ord[j]] < sh.th[x]) {
        sh.ord[j + 1] = sh.ord[j];
        --j;
      }
      sh.ord[j + 1] = x;
    }
    sh.msel = min(k, r);
  }
  __syncthreads();
  const int msel = sh.msel;
  // Y[c][j] = d_c (Li^T U)[.][ord_j] on the kept columns c, zero on the dropped ones
  for (int p = threadIdx.x; p < q * msel; p += LT) {
    const int c = p / msel, j = p % msel;
    sh.Y[c * LOBPCG_MAXK + j] = 0.0;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < r * msel; p += LT) {
    const int a = p / msel, j = p % msel;
    double v = 0.0;
    for (int b = a; b < r; ++b) v += sh.Li[b * MAXQ + a] * sh.V[b * MAXQ + sh.ord[j]];
    sh.Y[sh.keep[a] * LOBPCG_MAXK + j] = sh.d[sh.keep[a]] * v;
  }
  __syncthreads();
  return msel;
}

__global__ void __launch_bounds__(LT) k_face_lobpcg(FaceLobpcgIn in) {
  __shared__ RRShared sh;
  __shared__ double coef[LOBPCG_MAXK * LOBPCG_MAXNQ];
  __shared__ double theta[LOBPCG_MAXK];
  __shared__ int col[MAXQ];
  const int ld = in.max_n;
  const int K = in.k;
  // per-CTA scratch: S, AS, BS (3K columns each), new X/AX/BX and P/AP/BP (K each), U, T (K each)
  double* S = in.scratch + (size_t)blockIdx.x * LOBPCG_SCRATCH_COLS * K * ld;
  double* AS = S + (size_t)3 * K * ld;
  double* BS = AS + (size_t)3 * K * ld;
  double* NX = BS + (size_t)3 * K * ld;
  double* NAX = NX + (size_t)K * ld;
  double* NBX = NAX + (size_t)K * ld;
  double* NP = NBX + (size_t)K * ld;
  double* NAP = NP + (size_t)K * ld;
  double* NBP = NAP + (size_t)K * ld;
  double* U = NBP + (size_t)K * ld;
  double* Tm = U + (size_t)K * ld;
  for (int face = blockIdx.x; face < in.count; face += gridDim.x) {
    FaceView f;
    f.m = in.m[face];
    f.n = 2 * f.m;
    f.nq = in.nq[face];
    f.floating = in.floating[face];
    f.As = in.A + in.aoff[face];
    f.At = f.As + (size_t)f.m * f.m;
    f.ws = in.w + in.woff[face];
    f.wt = f.ws + f.m;
    f.Q = in.Q + in.qoff[face];
    const int n = f.n;
    const int k0 = min(K, n);
    // start block: unit vectors at the k0 largest diag((I-E)^T A (I-E)) / diag(A)
    if (threadIdx.x == 0) {
      double rv[2 * LOBPCG_MAXM];
      for (int i = 0; i < n; ++i) {
        const int j = i % f.m;
        const double as = f.As[(size_t)j * f.m + j], at = f.At[(size_t)j * f.m + j];
        const double w1 = f.ws[j], w2 = f.wt[j];
        const double num = i < f.m ? (1 - w1) * (1 - w1) * as + w1 * w1 * at : w2 * w2 * as + (1 - w2) * (1 - w2) * at;
        const double den = i < f.m ? as : at;
        rv[i] = den > 0.0 ? num / den : -INFINITY;
      }
      for (int c = 0; c < k0; ++c) {  // selection in order: largest ratio, lower index on ties
        int best = -1;
        for (int i = 0; i < n; ++i) {
          bool used = false;
          for (int cc = 0; cc < c; ++cc) used |= col[cc] == i;
          if (used) continue;
          if (best < 0 || rv[i] > rv[best]) best = i;
        }
        col[c] = best;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * k0; e += LT) {
      const int i = e % n, c = e / n;
      S[(size_t)c * ld + i] = (i == col[c]) ? 1.0 : 0.0;
    }
    __syncthreads();
    proj_cols(f, S, ld, k0, coef);
    apply_pencil(f, S, AS, BS, U, Tm, ld, k0, coef);
    // Rayleigh-Ritz on X
    for (int c = threadIdx.x; c < k0; c += LT) col[c] = c;
    __syncthreads();
    int q = k0;
    int kxo = k0;  // X columns of the basis the last Rayleigh-Ritz ran on
    int kx = rayleigh_ritz(S, AS, BS, col, q, K, ld, n, sh);
    bool hasP = false;
    for (int it = 0; ; ++it) {
      // X <- S Y, and (after the first step) P <- S Y with the X rows of Y zeroed
      const int kprev = kxo;
      for (int e = threadIdx.x; e < n * kx; e += LT) {
        const int i = e % n, j = e / n;
        double x = 0.0, ax = 0.0, bx = 0.0, pv = 0.0, ap = 0.0, bp = 0.0;
        for (int c = 0; c < q; ++c) {
          const double y = sh.Y[c * LOBPCG_MAXK + j];
          const double sv = S[(size_t)col[c] * ld + i], av = AS[(size_t)col[c] * ld + i],
                       bv = BS[(size_t)col[c] * ld + i];
          x += sv * y;
          ax += av * y;
          bx += bv * y;
          if (c >= kprev && it > 0) {
            pv += sv * y;
            ap += av * y;
            bp += bv * y;
          }
        }
        NX[(size_t)j * ld + i] = x;
        NAX[(size_t)j * ld + i] = ax;
        NBX[(size_t)j * ld + i] = bx;
        NP[(size_t)j * ld + i] = pv;
        NAP[(size_t)j * ld + i] = ap;
        NBP[(size_t)j * ld + i] = bp;
      }
      if (threadIdx.x < kx) theta[threadIdx.x] = sh.th[sh.ord[threadIdx.x]];
      __syncthreads();
      for (int e = threadIdx.x; e < n * kx; e += LT) {
        const int i = e % n, j = e / n;
        S[(size_t)j * ld + i] = NX[(size_t)j * ld + i];
        AS[(size_t)j * ld + i] = NAX[(size_t)j * ld + i];
        BS[(size_t)j * ld + i] = NBX[(size_t)j * ld + i];
        if (it > 0) {
          S[(size_t)(2 * K + j) * ld + i] = NP[(size_t)j * ld + i];
          AS[(size_t)(2 * K + j) * ld + i] = NAP[(size_t)j * ld + i];
          BS[(size_t)(2 * K + j) * ld + i] = NBP[(size_t)j * ld + i];
        }
      }
      hasP = it > 0;
      __syncthreads();
      if (it == in.iters) break;
      // W = proj(Lhs X - Rhs X theta) in the slots K .. K + kx - 1, then Lhs W and Rhs W
      for (int e = threadIdx.x; e < n * kx; e += LT) {
        const int i = e % n, j = e / n;
        S[(size_t)(K + j) * ld + i] = AS[(size_t)j * ld + i] - BS[(size_t)j * ld + i] * theta[j];
      }
      __syncthreads();
      proj_cols(f, S + (size_t)K * ld, ld, kx, coef);
      apply_pencil(f, S + (size_t)K * ld, AS + (size_t)K * ld, BS + (size_t)K * ld, U, Tm, ld, kx, coef);
      // Rayleigh-Ritz on [X, W] or [X, W, P]
      q = hasP ? 3 * kx : 2 * kx;
      for (int c = threadIdx.x; c < q; c += LT) col[c] = c < kx ? c : (c < 2 * kx ? K + (c - kx) : 2 * K + (c - 2 * kx));
      __syncthreads();
      kxo = kx;
      kx = rayleigh_ritz(S, AS, BS, col, q, K, ld, n, sh);
    }
    // outputs: theta (descending) and Lhs x_j
    for (int j = threadIdx.x; j < K; j += LT) in.theta[(size_t)face * K + j] = j < kx ? theta[j] : 0.0;
    for (int e = threadIdx.x; e < n * kx; e += LT) {
      const int i = e % n, j = e / n;
      in.LX[((size_t)face * K + j) * ld + i] = AS[(size_t)j * ld + i];
    }
    if (threadIdx.x == 0) in.nout[face] = kx;
    __syncthreads();
  }
}

}  // namespace

}  // namespace dd

namespace dd {

size_t face_lobpcg_scratch_doubles(int max_n, int k) { return (size_t)LOBPCG_SCRATCH_COLS * k * max_n; }

void face_lobpcg(const FaceLobpcgIn& in, int grid, cudaStream_t s) {
  k_face_lobpcg<<<grid, LT, 0, s>>>(in);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

namespace dd {

void face_lobpcg_batch(const std::vector<FaceProblem>& P, int k, int iters, std::vector<FaceResult>& R) {
  const int count = (int)P.size();
  R.assign(count, FaceResult());
  if (count == 0) return;
  if (k < 1 || k > LOBPCG_MAXK) throw Error(DD_INVALID_ARG, "face LOBPCG: 1 <= vectors per face <= 10");
  std::vector<int> m(count), nq(count), fl(count);
  std::vector<int64_t> aoff(count), woff(count), qoff(count);
  int64_t na = 0, nw = 0, nqa = 0;
  int max_n = 0;
  for (int f = 0; f < count; ++f) {
    const FaceProblem& p = P[f];
    if (p.m < 1 || p.m > LOBPCG_MAXM || p.nq > LOBPCG_MAXNQ)
      throw Error(DD_INVALID_ARG, "face LOBPCG: face problem beyond the kernel's limits");
    m[f] = p.m;
    nq[f] = p.nq;
    fl[f] = p.floating;
    aoff[f] = na;
    woff[f] = nw;
    qoff[f] = nqa;
    na += 2 * (int64_t)p.m * p.m;
    nw += 2 * (int64_t)p.m;
    nqa += (int64_t)p.nq * 2 * p.m;
    max_n = std::max(max_n, 2 * p.m);
  }
  std::vector<double> A((size_t)na), w((size_t)nw), Q((size_t)std::max<int64_t>(nqa, 1));
  for (int f = 0; f < count; ++f) {
    const FaceProblem& p = P[f];
    std::copy(p.As.begin(), p.As.end(), A.begin() + aoff[f]);
    std::copy(p.At.begin(), p.At.end(), A.begin() + aoff[f] + (int64_t)p.m * p.m);
    std::copy(p.ws.begin(), p.ws.end(), w.begin() + woff[f]);
    std::copy(p.wt.begin(), p.wt.end(), w.begin() + woff[f] + p.m);
    std::copy(p.Q.begin(), p.Q.end(), Q.begin() + qoff[f]);
  }
  int dev_sms = 152;
  {
    int dev = 0;
    DD_CUDA(cudaGetDevice(&dev));
    DD_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int grid = std::min(count, 2 * dev_sms);
  DeviceArena arena;
  FaceLobpcgIn in;
  in.count = count;
  in.k = k;
  in.iters = iters;
  in.max_n = max_n;
  cudaStream_t s = nullptr;
  in.m = arena.upload(m, s);
  in.nq = arena.upload(nq, s);
  in.floating = arena.upload(fl, s);
  in.aoff = arena.upload(aoff, s);
  in.woff = arena.upload(woff, s);
  in.qoff = arena.upload(qoff, s);
  in.A = arena.upload(A, s);
  in.w = arena.upload(w, s);
  in.Q = arena.upload(Q, s);
  in.theta = arena.alloc<double>((size_t)count * k);
  in.LX = arena.alloc<double>((size_t)count * k * max_n);
  in.nout = arena.alloc<int>(count);
  in.scratch = arena.alloc<double>(face_lobpcg_scratch_doubles(max_n, k) * grid);
  face_lobpcg(in, grid, s);
  std::vector<double> th((size_t)count * k), LX((size_t)count * k * max_n);
  std::vector<int> nout(count);
  DD_CUDA(cudaMemcpyAsync(th.data(), in.theta, th.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaMemcpyAsync(LX.data(), in.LX, LX.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaMemcpyAsync(nout.data(), in.nout, nout.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  for (int f = 0; f < count; ++f) {
    const int n = 2 * m[f];
    R[f].theta.assign(th.begin() + (size_t)f * k, th.begin() + (size_t)f * k + nout[f]);
    R[f].LX.resize((size_t)nout[f] * n);
    for (int j = 0; j < nout[f]; ++j)
      std::copy(LX.begin() + ((size_t)f * k + j) * max_n, LX.begin() + ((size_t)f * k + j) * max_n + n,
                R[f].LX.begin() + (size_t)j * n);
  }
}

}  // namespace dd

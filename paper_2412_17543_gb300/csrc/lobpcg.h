// Batched block LOBPCG of the adaptive face eigenproblems (lobpcg.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dd {

constexpr int LOBPCG_MAXK = 10;      // vectors per face (the paper's limit)
constexpr int LOBPCG_MAXNQ = 16;     // initial coarse dofs of one face's common interface
constexpr int LOBPCG_MAXM = 128;     // unknowns of one copy of a face's common interface
constexpr int LOBPCG_SCRATCH_COLS = 17;  // per-CTA scratch, in units of k columns

// Device inputs and outputs of a batch of faces. For face f: m[f] unknowns per copy
// (n = 2 m), A_s at A + aoff[f] and A_t right after it (m x m, row-major), the weights
// ws at w + woff[f] and wt right after (m each), nq[f] orthonormal jump columns of n
// entries at Q + qoff[f], floating[f] = 1 when both Schur complements annihilate the
// constants. Out: theta [count][k] (descending, nout[f] valid), LX [count][k][max_n]
// (Lhs x_j), nout [count]. scratch: face_lobpcg_scratch_doubles(max_n, k) per CTA.
struct FaceLobpcgIn {
  int count = 0, k = 0, iters = 0, max_n = 0;
  const int* m = nullptr;
  const int* nq = nullptr;
  const int* floating = nullptr;
  const int64_t* aoff = nullptr;
  const int64_t* woff = nullptr;
  const int64_t* qoff = nullptr;
  const double* A = nullptr;
  const double* w = nullptr;
  const double* Q = nullptr;
  double* theta = nullptr;
  double* LX = nullptr;
  int* nout = nullptr;
  double* scratch = nullptr;
};
size_t face_lobpcg_scratch_doubles(int max_n, int k);
void face_lobpcg(const FaceLobpcgIn& in, int grid, cudaStream_t s);

// Host side: one face problem and its result.
struct FaceProblem {
  int m = 0, nq = 0, floating = 0;
  std::vector<double> As, At, ws, wt, Q;  // Q: nq columns of 2m
};
struct FaceResult {
  std::vector<double> theta;  // descending
  std::vector<double> LX;     // [theta.size()][2m]: Lhs x_j
};
// Runs the batched LOBPCG on the current device (allocates, copies, frees; setup only).
void face_lobpcg_batch(const std::vector<FaceProblem>& P, int k, int iters, std::vector<FaceResult>& R);

}  // namespace dd

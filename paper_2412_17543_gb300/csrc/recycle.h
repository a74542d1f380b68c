// Tall-skinny products of the recycling update (recycle.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.h"

namespace dd {

constexpr int REC_MAXM = 128;     // columns of V = [W, P] handled by the Gram kernels
constexpr int REC_CHUNKS = 304;   // row chunks of the Gram kernels (2 per SM; fixed => deterministic sums)
constexpr int REC_BLOCKS = 528;   // upper 4 x 4 blocks of a 128 x 128 Gram matrix
constexpr int REC_PTRS = 8 * REC_MAXM;  // device pointer table: V, AV, MAV, W', AW', MAW', df64 W', df64 AW'

// Upper 4 x 4 output blocks (a <= b) of an m x m Gram matrix, leaving out the blocks
// whose rows and columns all lie below `skip` (a leading block known already).
std::vector<short2> gram_block_list(int m, int skip);
// out[q][16] = the 4 x 4 block blocks[q] of X^T Y (X, Y: m device column pointers of
// length n, a device array of pointers); df: df64 accumulation (FP64-accurate), else
// FP32 per 16-row stage with a compensated sum across stages. part: [REC_CHUNKS][nq][16].
void gram_blocks(int64_t n, int m, const double* const* X, const double* const* Y, const short2* blocks, int nq,
                 bool df, double* part, double* out, cudaStream_t s);
// out[c][i] = sum_a V[a][i] Yc[a][c] (Yc device row-major m x kc); outd (df only, nullable)
// receives the df64 copy of each result.
void lincomb_src(int64_t n, int m, int kc, const double* const* V, const double* Yc, double* const* out,
                 df64* const* outd, bool df, cudaStream_t s);
// MAP_j = (Z_j - Z_{j+1}) / alphas[j] for j < l; Z, MAP: columns of stride n; alphas device.
void zdiff_all(int64_t n, int l, const double* Z, const double* alphas, double* MAP, cudaStream_t s);

}  // namespace dd

// Tall-skinny products of the recycling update (Sect. 4.2): the Gram matrices of the
// harmonic Ritz pencil (eq. 15) and the new basis W = V Y with A W and M^{-1} A W.
//
// Every product here reduces over the n_gamma interface rows (661,500 at 128^3) with at
// most 128 columns on each side, so the work is FP32-pipe arithmetic on data that is
// read once: the rows are staged in shared memory once per stage and every thread
// accumulates a 4 x 4 block of the output in registers. FP64-accurate products use df64
// (float pairs with error-free transformations, about 2^-44 per product) because GB300
// issues FP64 at 1/64 of the FP32 rate; products of FP32-accurate data (the
// preconditioned vectors of an FP32 BDDC) accumulate in FP32 per stage of 16 rows and
// across stages with a compensated sum.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.h"
#include "recycle.h"

namespace dd {

namespace {

constexpr int GS_R = 16;     // rows per shared-memory stage
constexpr int GS_T = 256;    // threads per CTA = 4 x 4 output blocks per CTA
constexpr int GS_MAXM = REC_MAXM;

__device__ __forceinline__ df64 to_df(double d) { return df64_from_double_bits(d); }

// compensated accumulation of float terms (two-sum of Knuth)
struct f32_acc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float t = s + v;
    float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// Partial sums over this CTA's rows of C[a][b] = sum_i X_a[i] Y_b[i] for the 4 x 4 output
// blocks blocks[q] = (ga, gb), q in [blockIdx.y * GS_T, +GS_T): part[chunk][q][16].
template <bool DF>
__global__ void __launch_bounds__(GS_T) k_gram_blocks(int64_t n, int m, const double* const* __restrict__ X,
                                                      const double* const* __restrict__ Y,
                                                      const short2* __restrict__ blocks, int nq,
                                                      double* __restrict__ part) {
  using E = typename std::conditional<DF, df64, float>::type;
  __shared__ __align__(16) E xs[GS_R][GS_MAXM];
  __shared__ __align__(16) E ys[GS_R][GS_MAXM];
  __shared__ const double* xp[GS_MAXM];
  __shared__ const double* yp[GS_MAXM];
  for (int a = threadIdx.x; a < m; a += GS_T) {
    xp[a] = X[a];
    yp[a] = Y[a];
  }
  const int q = blockIdx.y * GS_T + threadIdx.x;
  const bool active = q < nq;
  short2 blk = active ? blocks[q] : make_short2(0, 0);
  const int a0 = 4 * blk.x, b0 = 4 * blk.y;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
  df64_acc dacc[4][4];
  f32_acc facc[4][4];
  __syncthreads();
  for (int64_t base = i0; base < i1; base += GS_R) {
    const int rows = (int)min((int64_t)GS_R, i1 - base);
    // stage GS_R rows of every column (16 consecutive doubles per column: 128-byte reads)
    for (int t = threadIdx.x; t < GS_R * m; t += GS_T) {
      const int r = t % GS_R, a = t / GS_R;
      const double xv = r < rows ? xp[a][base + r] : 0.0;
      const double yv = r < rows ? yp[a][base + r] : 0.0;
      if constexpr (DF) {
        xs[r][a] = to_df(xv);
        ys[r][a] = to_df(yv);
      } else {
        xs[r][a] = (float)xv;
        ys[r][a] = (float)yv;
      }
    }
    __syncthreads();
    if (active) {
      if constexpr (DF) {
#pragma unroll 2
        for (int r = 0; r < GS_R; ++r) {
          df64 xv[4], yv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            xv[u] = a0 + u < m ? xs[r][a0 + u] : df64{0.f, 0.f};
            yv[u] = b0 + u < m ? ys[r][b0 + u] : df64{0.f, 0.f};
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) dacc[u][v].fma(xv[u], yv[v]);
        }
      } else {
        float st[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) st[u][v] = 0.f;
#pragma unroll 4
        for (int r = 0; r < GS_R; ++r) {
          float xv[4], yv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            xv[u] = a0 + u < m ? xs[r][a0 + u] : 0.f;
            yv[u] = b0 + u < m ? ys[r][b0 + u] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) st[u][v] = fmaf(xv[u], yv[v], st[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) facc[u][v].add(st[u][v]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  double* out = part + ((int64_t)blockIdx.x * nq + q) * 16;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[4 * u + v] = DF ? df64_to_double(dacc[u][v].get()) : facc[u][v].get();
}

// out[e] = fixed-order sum over the chunks of part[chunk][e] (a warp per entry)
__global__ void __launch_bounds__(256) k_gram_blocks_reduce(int nch, int64_t ne, const double* __restrict__ part,
                                                            double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < ne;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double sum = 0.0;
    for (int c = lane; c < nch; c += 32) sum += part[(int64_t)c * ne + e];
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) out[e] = sum;
  }
}

// out_s[c][i] = sum_a V_s[a][i] Y[a][c] for the source s = blockIdx.y and the output columns
// [blockIdx.z * LC_CH, +LC_CH): one row per thread, Y in shared memory (broadcast reads).
// df64 sources also write the df64 copy of the result when outd[s] is given.
constexpr int LC_CH = 20;
template <bool DF>
__global__ void __launch_bounds__(256) k_lincomb_src(int64_t n, int m, int kc, const double* const* __restrict__ V,
                                                     const double* __restrict__ Yc,
                                                     double* const* __restrict__ out, df64* const* __restrict__ outd) {
  using E = typename std::conditional<DF, df64, float>::type;
  extern __shared__ __align__(16) unsigned char lc_smem[];
  E* ysm = reinterpret_cast<E*>(lc_smem);  // [m][LC_CH]
  const int c0 = blockIdx.z * LC_CH;
  const int nc = min(LC_CH, kc - c0);
  for (int t = threadIdx.x; t < m * LC_CH; t += blockDim.x) {
    const int a = t / LC_CH, c = t % LC_CH;
    const double y = c < nc ? Yc[(size_t)a * kc + c0 + c] : 0.0;
    if constexpr (DF)
      ysm[t] = to_df(y);
    else
      ysm[t] = (float)y;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (DF) {
      df64_acc acc[LC_CH];
      for (int a = 0; a < m; ++a) {
        const df64 v = to_df(V[a][i]);
#pragma unroll
        for (int c = 0; c < LC_CH; ++c) acc[c].fma(v, ysm[a * LC_CH + c]);
      }
#pragma unroll
      for (int c = 0; c < LC_CH; ++c)
        if (c < nc) {
          const double r = df64_to_double(acc[c].get());
          out[c0 + c][i] = r;
          if (outd) outd[c0 + c][i] = to_df(r);
        }
    } else {
      float acc[LC_CH];
#pragma unroll
      for (int c = 0; c < LC_CH; ++c) acc[c] = 0.f;
      for (int a = 0; a < m; ++a) {
        const float v = (float)V[a][i];
#pragma unroll
        for (int c = 0; c < LC_CH; ++c) acc[c] = fmaf(v, ysm[a * LC_CH + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < LC_CH; ++c)
        if (c < nc) out[c0 + c][i] = (double)acc[c];
    }
  }
}

// MAP_j = (Z_j - Z_{j+1}) / alpha_j for j < l (columns of stride n)
__global__ void k_zdiff_all(int64_t n, int l, const double* __restrict__ Z, const double* __restrict__ alphas,
                            double* __restrict__ MAP) {
  const int j = blockIdx.y;
  const double ia = 1.0 / alphas[j];
  const double* z0 = Z + (int64_t)j * n;
  const double* z1 = z0 + n;
  double* o = MAP + (int64_t)j * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (z0[i] - z1[i]) * ia;
}

}  // namespace

std::vector<short2> gram_block_list(int m, int skip) {
  std::vector<short2> q;
  const int g = (m + 3) / 4;
  for (int a = 0; a < g; ++a)
    for (int b = a; b < g; ++b) {
      if (4 * a + 3 < skip && 4 * b + 3 < skip) continue;  // wholly inside the block known already
      q.push_back(make_short2((short)a, (short)b));
    }
  return q;
}

void gram_blocks(int64_t n, int m, const double* const* X, const double* const* Y, const short2* blocks, int nq,
                 bool df, double* part, double* out, cudaStream_t s) {
  if (nq == 0) return;
  if (m > GS_MAXM) throw Error(DD_INVALID_ARG, "gram_blocks: more than 128 columns");
  dim3 grid(REC_CHUNKS, (nq + GS_T - 1) / GS_T);
  if (df)
    k_gram_blocks<true><<<grid, GS_T, 0, s>>>(n, m, X, Y, blocks, nq, part);
  else
    k_gram_blocks<false><<<grid, GS_T, 0, s>>>(n, m, X, Y, blocks, nq, part);
  DD_CHECK_LAUNCH();
  const int64_t ne = (int64_t)nq * 16;
  k_gram_blocks_reduce<<<(unsigned)std::min<int64_t>(152 * 8, (ne + 7) / 8), 256, 0, s>>>(REC_CHUNKS, ne, part, out);
  DD_CHECK_LAUNCH();
}

void lincomb_src(int64_t n, int m, int kc, const double* const* V, const double* Yc, double* const* out,
                 df64* const* outd, bool df, cudaStream_t s) {
  if (kc == 0 || m == 0) return;
  const int nz = (kc + LC_CH - 1) / LC_CH;
  const size_t smem = (size_t)m * LC_CH * (df ? sizeof(df64) : sizeof(float));
  const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 4);
  dim3 grid(gx, 1, nz);
  if (df) {
    max_smem(k_lincomb_src<true>, smem);
    k_lincomb_src<true><<<grid, 256, smem, s>>>(n, m, kc, V, Yc, out, outd);
  } else {
    max_smem(k_lincomb_src<false>, smem);
    k_lincomb_src<false><<<grid, 256, smem, s>>>(n, m, kc, V, Yc, out, nullptr);
  }
  DD_CHECK_LAUNCH();
}

void zdiff_all(int64_t n, int l, const double* Z, const double* alphas, double* MAP, cudaStream_t s) {
  if (l <= 0) return;
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 152), l);
  k_zdiff_all<<<grid, 256, 0, s>>>(n, l, Z, alphas, MAP);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

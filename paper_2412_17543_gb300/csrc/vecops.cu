// Krylov-vector kernels: deterministic dot products (fixed grid, fixed-order
// two-stage reduction, no floating-point atomics), fused PCG updates, the
// deflation projection (Algorithm 1: mu = (W^T A W)^{-1} (AW)^T z, p = z + beta p - W mu),
// and tall-skinny Gram / combination kernels for the recycling update
// (eq. 15).
#include <algorithm>

#include "vecops.h"

namespace dd {

constexpr int RB = 256;  // threads per reduction block

template <int ND>
__device__ __forceinline__ void block_reduce_store(double (&v)[ND], double* partials) {
  __shared__ double sh[ND][RB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double x = v[d];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[d][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < ND) {
    double s = 0.0;
    for (int w = 0; w < RB / 32; ++w) s += sh[threadIdx.x][w];
    partials[blockIdx.x * MAXDOT + threadIdx.x] = s;
  }
}

// single-block finalization: sums the partials in a fixed order (a warp per dot product,
// fixed lane assignment and shuffle tree) and updates the scalars. CG: the partials were
// written by other blocks of the same launch (read through L2).
template <bool CG>
__device__ __forceinline__ void finalize_block(int nblk, const double* partials, double* sc, int op, int flexible,
                                               const int* its) {
  __shared__ double tot[3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 3) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += CG ? __ldcg(&partials[b * MAXDOT + warp]) : partials[b * MAXDOT + warp];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tot[warp] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (op == FIN_RZL) op = *its == 0 ? FIN_RZ0 : FIN_RZ;  // device-resident loop: first iteration or not
  switch (op) {
    case FIN_PQ: {
      double pq = tot[0];
      sc[SC_PQ] = pq;
      if (!(pq > 0.0) || !isfinite(pq) || !isfinite(sc[SC_RZ])) {
        sc[SC_FLAG] = 1.0;
        sc[SC_ALPHA] = 0.0;
      } else {
        sc[SC_ALPHA] = sc[SC_RZ] / pq;
      }
      break;
    }
    case FIN_RR:
      sc[SC_RR] = tot[0];
      if (!isfinite(tot[0])) sc[SC_FLAG] = 1.0;
      break;
    case FIN_RZ0:
      sc[SC_RZ] = tot[0];
      if (!(tot[0] > 0.0) || !isfinite(tot[0])) sc[SC_FLAG] = 1.0;
      break;
    case FIN_RZ: {
      double rz_new = tot[0], rz_old_z = tot[1];
      double num = flexible ? (rz_new - rz_old_z) : rz_new;
      double rz = sc[SC_RZ];
      sc[SC_BETA] = (rz != 0.0) ? num / rz : 0.0;
      sc[SC_RZ] = rz_new;
      if (!(rz_new > 0.0) || !isfinite(rz_new)) sc[SC_FLAG] = 1.0;
      break;
    }
    case FIN_BB:
      sc[SC_BB] = tot[0];
      sc[SC_RR] = tot[1];
      break;
    default:
      break;
  }
}

__global__ void k_finalize(int nblk, const double* __restrict__ partials, double* sc, int op, int flexible,
                           const int* __restrict__ its) {
  finalize_block<false>(nblk, partials, sc, op, flexible, its);
}

// Finalization by the last block of a reduction launch (ticket counter, reset by that
// block): the same sums in the same order as k_finalize, without a second launch.
struct FinArgs {
  double* sc;
  int op, flexible;
  const int* its;
  unsigned* ticket;
};
__device__ __forceinline__ void finalize_last(const double* partials, const FinArgs& f) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(f.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) *f.ticket = 0u;
  finalize_block<true>((int)gridDim.x, partials, f.sc, f.op, f.flexible, f.its);
}

// partial dots: d0 = a0.b0, d1 = a1.b1, d2 = a2.b2 (null pairs skipped); FIN: the last
// block finalizes (FinArgs)
template <bool FIN>
__global__ void __launch_bounds__(RB) k_dots(int64_t n, const double* __restrict__ a0, const double* __restrict__ b0,
                                             const double* __restrict__ a1, const double* __restrict__ b1,
                                             const double* __restrict__ a2, const double* __restrict__ b2,
                                             double* partials, FinArgs fin) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    v[0] = fma(a0[i], b0[i], v[0]);
    if (a1) v[1] = fma(a1[i], b1[i], v[1]);
    if (a2) v[2] = fma(a2[i], b2[i], v[2]);
  }
  block_reduce_store<3>(v, partials);
  if (FIN) finalize_last(partials, fin);
}

// x += alpha p ; r -= alpha q ; partial ||r||^2 (FIN: the last block finalizes)
template <bool FIN>
__global__ void __launch_bounds__(RB) k_axpy2(int64_t n, const double* __restrict__ sc, double* __restrict__ x,
                                              const double* __restrict__ p, double* __restrict__ r,
                                              const double* __restrict__ q, double* partials, FinArgs fin) {
  const double alpha = sc[SC_ALPHA];
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
  }
  block_reduce_store<1>(v, partials);
  if (FIN) finalize_last(partials, fin);
}

void vec_dots(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1, const double* a2,
              const double* b2, double* partials, cudaStream_t s) {
  k_dots<false><<<NBLK, RB, 0, s>>>(n, a0, b0, a1, b1, a2, b2, partials, FinArgs{});
  DD_CHECK_LAUNCH();
}
void vec_dots_fin(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1,
                  double* partials, double* sc, int op, int flexible, unsigned* ticket, cudaStream_t s,
                  const int* its) {
  k_dots<true><<<NBLK, RB, 0, s>>>(n, a0, b0, a1, b1, nullptr, nullptr, partials,
                                   FinArgs{sc, op, flexible, its, ticket});
  DD_CHECK_LAUNCH();
}
void vec_finalize(const double* partials, double* sc, int op, int flexible, cudaStream_t s, const int* its) {
  k_finalize<<<1, 96, 0, s>>>(NBLK, partials, sc, op, flexible, its);
  DD_CHECK_LAUNCH();
}
void vec_axpy2(int64_t n, const double* sc, double* x, const double* p, double* r, const double* q, double* partials,
               cudaStream_t s) {
  k_axpy2<false><<<NBLK, RB, 0, s>>>(n, sc, x, p, r, q, partials, FinArgs{});
  DD_CHECK_LAUNCH();
}
void vec_axpy2_fin(int64_t n, double* sc, double* x, const double* p, double* r, const double* q, double* partials,
                   unsigned* ticket, cudaStream_t s) {
  k_axpy2<true><<<NBLK, RB, 0, s>>>(n, sc, x, p, r, q, partials, FinArgs{sc, FIN_RR, 0, nullptr, ticket});
  DD_CHECK_LAUNCH();
}

// y = a - b
__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] - b[i];
}
void vec_sub(int64_t n, const double* a, const double* b, double* y, cudaStream_t s) {
  k_sub<<<NBLK, RB, 0, s>>>(n, a, b, y);
  DD_CHECK_LAUNCH();
}

// out = in - mean(in) (the l2 projection onto the complement of the constants): block sums
// on the fixed reduction grid, then every block adds the partial sums in the same order, so
// all subtract the same value
__global__ void __launch_bounds__(RB) k_sum(int64_t n, const double* __restrict__ in, double* partials) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) v[0] += in[i];
  block_reduce_store<1>(v, partials);
}
__global__ void __launch_bounds__(RB) k_sub_mean(int64_t n, const double* in, double* out,
                                                 const double* __restrict__ partials, int nblk) {
  __shared__ double mean;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partials[b * MAXDOT];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) mean = s / (double)n;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) out[i] = in[i] - mean;
}
void vec_sub_mean(int64_t n, const double* in, double* out, double* partials, cudaStream_t s) {
  if (n == 0) return;
  k_sum<<<NBLK, RB, 0, s>>>(n, in, partials);
  DD_CHECK_LAUNCH();
  k_sub_mean<<<NBLK, RB, 0, s>>>(n, in, out, partials, NBLK);
  DD_CHECK_LAUNCH();
}


// ---------------------------------------------------------------------------
// deflation with the basis stored as df64 (float pairs): the k-column products run on
// the FP32 pipes with error-free transformations (about 2^-44 relative), FP64 only
// converts the vector entries and forms the final update
// ---------------------------------------------------------------------------
__device__ __forceinline__ df64 dbl_to_df(double d) { return df64_from_double_bits(d); }

__global__ void k_to_df64(int64_t n, const double* __restrict__ in, df64* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = dbl_to_df(in[i]);
}
void to_df64(int64_t n, const double* in, df64* out, cudaStream_t s) {
  if (n == 0) return;
  k_to_df64<<<NBLK * 2, RB, 0, s>>>(n, in, out);
  DD_CHECK_LAUNCH();
}

constexpr int PT = 4;  // rows per thread of the row-blocked deflation update

// mu = Ginv (V^T v) with the basis V as df64 (k columns of stride ld), in one launch.
// Block b owns a contiguous range of `rows` rows (a multiple of 32, fixed by n alone): v's
// entries there are staged in shared memory as df64, warp w walks the columns
// c = w, w + RB/32, ... over the block's rows (eight coalesced loads in flight per lane,
// two sums per lane) and needs one warp reduction per column; the block writes wpart[b][c].
// The partials are then reduced in two levels, each by the last block to arrive (ticket
// counters, reset by that block): the last block of each group of WD_GROUP blocks sums
// the group's partials, and the last group sums the groups' sums and applies Ginv. In
// both, thread (c, s) adds column c over a fixed segment s of its inputs with all loads
// in flight, and the segments are added in order, so the reduction order depends only on
// n and k, not on which blocks end last.
constexpr int WD_GRID = 6 * 152;   // blocks of the deflation dots: six per SM, one wave
constexpr int WD_MAXROWS = 4096;   // rows per block at most (32 KiB of staged df64)
constexpr int WD_GROUP = 32;       // blocks per first-level reduction group

static int64_t wd_rows(int64_t n, int nb) { return ((n + nb - 1) / nb + 31) / 32 * 32; }

int defl_df_blocks(int64_t n) {
  int64_t nb = std::min<int64_t>(WD_GRID, (n + 255) / 256);
  nb = std::max<int64_t>(nb, (n + WD_MAXROWS - 1) / WD_MAXROWS);
  return (int)std::max<int64_t>(nb, 1);
}
__host__ __device__ static int wd_groups(int nb) { return (nb + WD_GROUP - 1) / WD_GROUP; }
int defl_df_part_rows(int64_t n) {
  const int nb = defl_df_blocks(n);
  return nb + wd_groups(nb);
}
int defl_df_tickets(int64_t n) { return 1 + wd_groups(defl_df_blocks(n)); }

// sum over i in [i0, i1) of src[i * MAXK + c], sixteen loads in flight, added in index order
__device__ __forceinline__ double wd_segment_sum(const double* src, int c, int i0, int i1) {
  double sum = 0.0;
  for (int i = i0; i < i1; i += 16) {
    double e[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) e[u] = i + u < i1 ? __ldcg(&src[(int64_t)(i + u) * MAXK + c]) : 0.0;
#pragma unroll
    for (int u = 0; u < 16; ++u) sum += e[u];
  }
  return sum;
}

// d[c] = sum over i in [0, m) of src[i][c] for c < k by the whole block (see above)
__device__ __forceinline__ void wd_reduce(const double* src, int m, int k, double* part, double* d) {
  const int t = threadIdx.x;
  const int ns = max(1, min(8, RB / k));
  if (t < ns * k) {
    const int c = t % k, sg = t / k;
    part[t] = wd_segment_sum(src, c, sg * m / ns, (sg + 1) * m / ns);
  }
  __syncthreads();
  if (t < k) {
    double sum = 0.0;
    for (int sg = 0; sg < ns; ++sg) sum += part[sg * k + t];
    d[t] = sum;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RB) k_wdots8(int64_t n, int64_t rows, int k, const df64* __restrict__ V,
                                               int64_t ld, const double* __restrict__ v, double* wpart,
                                               unsigned* __restrict__ ticket, const double* __restrict__ Ginv,
                                               double* __restrict__ mu) {
  __shared__ df64 zs[WD_MAXROWS];
  __shared__ double part[RB];
  __shared__ double d[MAXK];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t left = n - r0 < rows ? n - r0 : rows;
  const int nr = left > 0 ? (int)left : 0;
  for (int t = threadIdx.x; t < nr; t += RB) zs[t] = dbl_to_df(v[r0 + t]);
  __syncthreads();
  for (int c = warp; c < k; c += RB / 32) {
    const df64* col = V + (int64_t)c * ld + r0;
    df64_acc a0, a1;
    int j = lane;
    for (; j + 7 * 32 < nr; j += 8 * 32) {
      df64 e[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) e[u] = col[j + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        a0.fma(e[u], zs[j + 32 * u]);
        a1.fma(e[u + 1], zs[j + 32 * (u + 1)]);
      }
    }
    for (; j < nr; j += 32) a0.fma(col[j], zs[j]);
    df64 x = df64_add(a0.get(), a1.get());
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const df64 y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
      x = df64_add(x, y);
    }
    if (lane == 0) wpart[(int64_t)blockIdx.x * MAXK + c] = df64_to_double_bits(x);
  }
  // first level: the last block of the group sums the group's partials
  const int nb = (int)gridDim.x, ng = wd_groups(nb);
  const int g = blockIdx.x / WD_GROUP, gb0 = g * WD_GROUP, gn = min(nb, gb0 + WD_GROUP) - gb0;
  double* gpart = wpart + (int64_t)nb * MAXK;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ticket[1 + g], 1u) == (unsigned)gn - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  wd_reduce(wpart + (int64_t)gb0 * MAXK, gn, k, part, d);
  for (int c = threadIdx.x; c < k; c += RB) gpart[(int64_t)g * MAXK + c] = d[c];
  if (threadIdx.x == 0) ticket[1 + g] = 0u;
  // second level: the last group sums the groups and applies Ginv
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ticket[0], 1u) == (unsigned)ng - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  wd_reduce(gpart, ng, k, part, d);
  const int t = threadIdx.x;
  const int ns = max(1, min(8, RB / k));
  if (t < ns * k) {
    // row a of Ginv over the c-segment sg, all loads in flight
    const int a = t % k, sg = t / k;
    const int c0 = sg * k / ns, c1 = (sg + 1) * k / ns;
    double sum = 0.0;
    for (int c = c0; c < c1; c += 16) {
      double e[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) e[u] = c + u < c1 ? Ginv[a * k + c + u] : 0.0;
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (c + u < c1) sum = fma(e[u], d[c + u], sum);
    }
    part[t] = sum;
  }
  __syncthreads();
  if (t < k) {
    double sum = 0.0;
    for (int sg = 0; sg < ns; ++sg) sum += part[sg * k + t];
    mu[t] = sum;
  }
  if (t == 0) ticket[0] = 0u;
}

void defl_mu_df(int64_t n, int k, const df64* V, int64_t ld, const double* v, const double* Ginv, double* wpart,
                double* mu, unsigned* ticket, cudaStream_t s) {
  if (k == 0) return;
  const int nb = defl_df_blocks(n);
  k_wdots8<<<nb, RB, 0, s>>>(n, wd_rows(n, nb), k, V, ld, v, wpart, ticket, Ginv, mu);
  DD_CHECK_LAUNCH();
}

// y = z + beta y + sign_w W mu over row chunks of PT * RB rows: a block walks the k
// columns, each a contiguous 16-KiB piece per chunk, and keeps its rows' sums in df64
__global__ void __launch_bounds__(RB) k_pupdate2(int64_t n, int k, const df64* __restrict__ W, int64_t ld,
                                                 const double* __restrict__ mu, const double* __restrict__ z,
                                                 double* __restrict__ y, const double* __restrict__ sc, int beta_idx,
                                                 double sign_w) {
  __shared__ df64 m[MAXK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) m[c] = dbl_to_df(sign_w * mu[c]);
  __syncthreads();
  const double beta = beta_idx >= 0 ? sc[beta_idx] : 0.0;
  const int64_t i0 = (int64_t)blockIdx.x * PT * RB + threadIdx.x;
  df64_acc acc[PT];
  int c = 0;
  for (; c + 1 < k; c += 2) {
    // both columns' entries are loaded before any product (more loads in flight)
    const df64* c0 = W + (int64_t)c * ld;
    const df64* c1 = c0 + ld;
    df64 v0[PT], v1[PT];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int64_t i = i0 + (int64_t)r * RB;
      v0[r] = i < n ? c0[i] : df64{0.f, 0.f};
      v1[r] = i < n ? c1[i] : df64{0.f, 0.f};
    }
    const df64 m0 = m[c], m1 = m[c + 1];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      acc[r].fma(v0[r], m0);
      acc[r].fma(v1[r], m1);
    }
  }
  if (c < k) {
    const df64* c0 = W + (int64_t)c * ld;
    const df64 m0 = m[c];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int64_t i = i0 + (int64_t)r * RB;
      if (i < n) acc[r].fma(c0[i], m0);
    }
  }
#pragma unroll
  for (int r = 0; r < PT; ++r) {
    const int64_t i = i0 + (int64_t)r * RB;
    if (i < n) {
      const double v = (z ? z[i] : 0.0) + (beta_idx >= 0 ? beta * y[i] : (z ? 0.0 : y[i]));
      y[i] = v + df64_to_double(acc[r].get());
    }
  }
}

void defl_update_df(int64_t n, int k, const df64* W, int64_t ld, const double* mu, const double* z, double* y,
                    const double* sc, int beta_idx, double sign_w, cudaStream_t s) {
  const int64_t blocks = (n + (int64_t)PT * RB - 1) / ((int64_t)PT * RB);
  k_pupdate2<<<(unsigned)std::max<int64_t>(blocks, 1), RB, 0, s>>>(n, k, W, ld, mu, z, y, sc, beta_idx, sign_w);
  DD_CHECK_LAUNCH();
}

// The same update with the basis stored as FP32 values (the basis is rounded to
// FP32-representable numbers when it is formed, so these are its exact entries): the
// products w * mu run as float x df64 in df64 accumulation.
__global__ void __launch_bounds__(RB) k_pupdate_f(int64_t n, int k, const float* __restrict__ W, int64_t ld,
                                                  const double* __restrict__ mu, const double* __restrict__ z,
                                                  double* __restrict__ y, const double* __restrict__ sc, int beta_idx,
                                                  double sign_w) {
  __shared__ df64 m[MAXK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) m[c] = dbl_to_df(sign_w * mu[c]);
  __syncthreads();
  const double beta = beta_idx >= 0 ? sc[beta_idx] : 0.0;
  const int64_t i0 = (int64_t)blockIdx.x * PT * RB + threadIdx.x;
  df64_acc acc[PT];
  int c = 0;
  for (; c + 3 < k; c += 4) {
    // the four columns' entries are loaded before any product
    float e[4][PT];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float* col = W + (int64_t)(c + q) * ld;
#pragma unroll
      for (int r = 0; r < PT; ++r) {
        const int64_t i = i0 + (int64_t)r * RB;
        e[q][r] = i < n ? col[i] : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const df64 mq = m[c + q];
#pragma unroll
      for (int r = 0; r < PT; ++r) acc[r].fma(df64{e[q][r], 0.f}, mq);
    }
  }
  for (; c < k; ++c) {
    const float* col = W + (int64_t)c * ld;
    const df64 mc = m[c];
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int64_t i = i0 + (int64_t)r * RB;
      if (i < n) acc[r].fma(df64{col[i], 0.f}, mc);
    }
  }
#pragma unroll
  for (int r = 0; r < PT; ++r) {
    const int64_t i = i0 + (int64_t)r * RB;
    if (i < n) {
      const double v = (z ? z[i] : 0.0) + (beta_idx >= 0 ? beta * y[i] : (z ? 0.0 : y[i]));
      y[i] = v + df64_to_double(acc[r].get());
    }
  }
}

void defl_update_f(int64_t n, int k, const float* W, int64_t ld, const double* mu, const double* z, double* y,
                   const double* sc, int beta_idx, double sign_w, cudaStream_t s) {
  const int64_t blocks = (n + (int64_t)PT * RB - 1) / ((int64_t)PT * RB);
  k_pupdate_f<<<(unsigned)std::max<int64_t>(blocks, 1), RB, 0, s>>>(n, k, W, ld, mu, z, y, sc, beta_idx, sign_w);
  DD_CHECK_LAUNCH();
}

// wf = w rounded to FP32; where that changes w, w takes the rounded value and *changed = 1
__global__ void k_round_f32(int64_t n, double* __restrict__ w, float* __restrict__ wf, int* __restrict__ changed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[i];
    const float f = (float)v;
    wf[i] = f;
    if ((double)f != v) {
      w[i] = (double)f;
      *changed = 1;
    }
  }
}
void round_to_f32(int64_t n, double* w, float* wf, int* changed, cudaStream_t s) {
  if (n == 0) return;
  k_round_f32<<<NBLK * 2, RB, 0, s>>>(n, w, wf, changed);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// tall-skinny products for the recycling update
// ---------------------------------------------------------------------------
// partial C[a][b] = sum_i X_a[i] Y_b[i] over this block's rows (na, nb <= 128). The
// staged rows are converted once to df64 and the products accumulate with error-free
// FP32 transformations (about 2^-44 relative per product): each staged value feeds up
// to 128 products, so the FP64 pipe only converts.
constexpr int GR = 16;  // rows per smem stage (2 x 16 x 129 float pairs of static shared memory)
__global__ void __launch_bounds__(256) k_gram(int64_t n, int na, const double* const* __restrict__ X, int nb,
                                              const double* const* __restrict__ Y, double* part) {
  __shared__ df64 xs[GR][129];
  __shared__ df64 ys[GR][129];
  const int npair = na * nb;
  df64_acc acc[16];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int64_t base = i0; base < i1; base += GR) {
    int rows = (int)min((int64_t)GR, i1 - base);
    for (int t = threadIdx.x; t < GR * na; t += blockDim.x) {
      int r = t % GR, a = t / GR;
      xs[r][a] = dbl_to_df(r < rows ? X[a][base + r] : 0.0);
    }
    for (int t = threadIdx.x; t < GR * nb; t += blockDim.x) {
      int r = t % GR, b = t / GR;
      ys[r][b] = dbl_to_df(r < rows ? Y[b][base + r] : 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      int pr = threadIdx.x + t * 256;
      if (pr < npair) {
        int a = pr / nb, b = pr % nb;
        for (int r = 0; r < GR; ++r) acc[t].fma(xs[r][a], ys[r][b]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    int pr = threadIdx.x + t * 256;
    if (pr < npair) part[(int64_t)blockIdx.x * npair + pr] = df64_to_double(acc[t].get());
  }
}

// C[pr] = fixed-order sum of the block partials: a warp per pair, lanes over the blocks
__global__ void __launch_bounds__(256) k_gram_reduce(int nblk, int npair, const double* __restrict__ part,
                                                     double* C) {
  const int lane = threadIdx.x & 31;
  for (int pr = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pr < npair; pr += (gridDim.x * blockDim.x) >> 5) {
    double sum = 0.0;
    for (int b = lane; b < nblk; b += 32) sum += part[(int64_t)b * npair + pr];
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) C[pr] = sum;
  }
}

void gram(int64_t n, int na, const double* const* X, int nb, const double* const* Y, double* part, double* C,
          cudaStream_t s) {
  if (na == 0 || nb == 0) return;
  if (na > 128 || nb > 128 || na * nb > 16 * 256) throw Error(DD_INVALID_ARG, "gram: too many columns");
  k_gram<<<NBLK, 256, 0, s>>>(n, na, X, nb, Y, part);
  DD_CHECK_LAUNCH();
  k_gram_reduce<<<std::min(152 * 8, (na * nb + 7) / 8), 256, 0, s>>>(NBLK, na * nb, part, C);
  DD_CHECK_LAUNCH();
}

// out_c[i] = sum_a V_a[i] Y[a][c]   (Y row-major m x kc); V entries converted once per
// row to df64, sums with error-free FP32 transformations
__global__ void k_lincomb(int64_t n, int m, const double* const* __restrict__ V, const double* __restrict__ Yc, int kc,
                          double* const* __restrict__ out) {
  extern __shared__ df64 ysm[];
  for (int t = threadIdx.x; t < m * kc; t += blockDim.x) ysm[t] = dbl_to_df(Yc[t]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int c0 = 0; c0 < kc; c0 += 8) {
      df64_acc acc[8];
      for (int a = 0; a < m; ++a) {
        const df64 v = dbl_to_df(V[a][i]);
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (c0 + t < kc) acc[t].fma(v, ysm[a * kc + c0 + t]);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (c0 + t < kc) out[c0 + t][i] = df64_to_double(acc[t].get());
    }
  }
}

void lincomb(int64_t n, int m, const double* const* V, const double* Yc, int kc, double* const* out, cudaStream_t s) {
  if (kc == 0) return;
  size_t smem = (size_t)m * kc * sizeof(df64);
  if (smem > 48 * 1024) max_smem(k_lincomb, smem);
  k_lincomb<<<NBLK, RB, smem, s>>>(n, m, V, Yc, kc, out);
  DD_CHECK_LAUNCH();
}

// MAP_j = (z_j - z_{j+1}) / alpha_j
__global__ void k_zdiff(int64_t n, const double* __restrict__ z0, const double* __restrict__ z1, double inv_alpha,
                        double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (z0[i] - z1[i]) * inv_alpha;
}
void zdiff(int64_t n, const double* z0, const double* z1, double inv_alpha, double* out, cudaStream_t s) {
  k_zdiff<<<NBLK, RB, 0, s>>>(n, z0, z1, inv_alpha, out);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

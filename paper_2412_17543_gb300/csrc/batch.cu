// Ensemble kernels (interleaved [rows][BW] vectors, lane = member): the Schur operator,
// the BDDC preconditioner and the Krylov-vector steps applied to BW right-hand sides at
// once. Every operator is read once per application for all members, which turns the
// batched GEMVs of the single-vector path into small GEMMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "batch.h"
#include "policy.cuh"
#include "vecops.h"

namespace dd {

static int grid_for_b(int64_t rows, int rows_per_block) {
  int64_t g = (rows + rows_per_block - 1) / rows_per_block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------------------
// layout conversion (32 x 32 tiles through shared memory, both sides coalesced)
// ---------------------------------------------------------------------------
__global__ void k_pack_in(int64_t n, int nrhs, const double* __restrict__ F, df64* __restrict__ out) {
  __shared__ double t[BW][BW + 1];
  const int64_t i0 = (int64_t)blockIdx.x * BW;
  for (int m = threadIdx.y; m < BW; m += blockDim.y) {
    const int64_t i = i0 + threadIdx.x;
    t[m][threadIdx.x] = (m < nrhs && i < n) ? F[(int64_t)m * n + i] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < BW; r += blockDim.y) {
    const int64_t i = i0 + r;
    if (i < n) out[i * BW + threadIdx.x] = df64_from_double_bits(t[threadIdx.x][r]);
  }
}

__global__ void k_pack_out(int64_t n, int nrhs, const df64* __restrict__ in, double* __restrict__ X) {
  __shared__ double t[BW][BW + 1];
  const int64_t i0 = (int64_t)blockIdx.x * BW;
  for (int r = threadIdx.y; r < BW; r += blockDim.y) {
    const int64_t i = i0 + r;
    t[r][threadIdx.x] = (i < n) ? df64_to_double_bits(in[i * BW + threadIdx.x]) : 0.0;
  }
  __syncthreads();
  for (int m = threadIdx.y; m < nrhs; m += blockDim.y) {
    const int64_t i = i0 + threadIdx.x;
    if (i < n) X[(int64_t)m * n + i] = t[threadIdx.x][m];
  }
}

void launch_pack_in(int64_t n, int nrhs, const double* F, df64* out, cudaStream_t s) {
  if (n == 0) return;
  k_pack_in<<<(unsigned)((n + BW - 1) / BW), dim3(BW, 8), 0, s>>>(n, nrhs, F, out);
  DD_CHECK_LAUNCH();
}
void launch_pack_out(int64_t n, int nrhs, const df64* in, double* X, cudaStream_t s) {
  if (n == 0) return;
  k_pack_out<<<(unsigned)((n + BW - 1) / BW), dim3(BW, 8), 0, s>>>(n, nrhs, in, X);
  DD_CHECK_LAUNCH();
}

__global__ void k_to_float(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
void launch_to_float(int64_t n, const double* in, float* out, cudaStream_t s) {
  if (n == 0) return;
  k_to_float<<<grid_for_b(n, 256), 256, 0, s>>>(n, in, out);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// element passes (work lists as in the single-vector kernels). A block takes one
// subdomain and a chunk of RC members; lane = (item within the warp) * RC + member.
// ---------------------------------------------------------------------------
template <class P, int S, int RC>
__device__ __forceinline__ void apply_item_b(const DevMesh& m, const int16_t* it, const typename P::V* xl,
                                             const typename P::V* kd, int mm, typename P::V& out) {
  const int sx = S ? S : m.sx, sy = S ? S : m.sy, sz = S ? S : m.sz;
  const int NE = sx * sy * sz;
  const int NLx = sx + 1, NLy = sy + 1;
  typename P::Acc acc[2];
  P::init(acc[0]);
  P::init(acc[1]);
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int v = it[1 + k];
    if (v < 0) break;
    const int el = v >> 3, p = v & 7;
    const int ea = el % sx, eb = (el / sx) % sy, ec = el / (sx * sy);
    const int base = ea + NLx * (eb + NLy * ec);
    const typename P::V* kp = kd + el;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int lq = base + (q & 1) + NLx * (((q >> 1) & 1) + NLy * (q >> 2));
      P::fma(acc[q & 1], kp[(p ^ q) * NE], xl[lq * RC + mm]);
    }
  }
  out = P::add(P::get(acc[0]), P::get(acc[1]));
}

// A block takes one subdomain: the element entries are formed once, then the members
// pass through in chunks of RC (their local values staged in shared memory).
template <class P, int S, int RC>
__global__ void __launch_bounds__(512) k_elem_interior_b(DevMesh m, int mode, const df64* __restrict__ xg,
                                                         const df64* __restrict__ f, df64* __restrict__ tI) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_b[];
  V* xl = reinterpret_cast<V*>(smem_b);  // [NL][RC]
  V* kd = xl + (size_t)m.NL * RC;
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  const int* to = m.type_off + 6 * m.sub_type[s];
  const int64_t io = m.ioff[s];
  // every interior output first gets its base value (0 or f_I), all members
  for (int t = threadIdx.x; t < m.NL * BW; t += blockDim.x) {
    const int l = t / BW, mm = t % BW;
    const int cd = code[l];
    if (cd >= 0) tI[(io + cd) * BW + mm] = (mode == ELEM_SCHUR) ? df64{0.f, 0.f} : f[free_index(m, s, l) * BW + mm];
  }
  if (mode == ELEM_CONDENSE) return;
  build_kd_list<P, S>(m, s, m.type_bl + to[4], to[5] - to[4], kd);
  constexpr int IPW = 32 / RC;  // items per warp pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int mm = lane % RC;
  for (int m0 = 0; m0 < BW; m0 += RC) {
    for (int t = threadIdx.x; t < m.NL * RC; t += blockDim.x) {
      const int l = t / RC, c = t % RC;
      const int cd = code[l];
      xl[t] = (cd < 0 && cd != INT16_MIN) ? P::from_v(xg[(int64_t)m.gmap[m.goff[s] + (-1 - cd)] * BW + m0 + c])
                                          : P::zero();
    }
    __syncthreads();
    for (int i = to[0] + warp * IPW + lane / RC; i < to[1]; i += nw * IPW) {
      const int16_t* it = m.type_items + 9 * (size_t)i;
      const int l = it[0];
      V v;
      apply_item_b<P, S, RC>(m, it, xl, kd, mm, v);
      const int64_t o = (io + code[l]) * BW + m0 + mm;
      if (mode == ELEM_SCHUR)
        tI[o] = P::to_v(v);
      else
        tI[o] = df64_add(f[free_index(m, s, l) * BW + m0 + mm], df64_neg(P::to_v(v)));
    }
    __syncthreads();
  }
}

template <class P, int S, int RC>
__global__ void __launch_bounds__(512) k_elem_interface_b(DevMesh m, int mode, const df64* __restrict__ xg,
                                                          const df64* __restrict__ sI,
                                                          df64* __restrict__ yloc) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_b[];
  V* xl = reinterpret_cast<V*>(smem_b);
  V* kd = xl + (size_t)m.NL * RC;
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  const int* to = m.type_off + 6 * m.sub_type[s];
  build_kd_list<P, S>(m, s, m.type_bl + to[4], to[5] - to[4], kd);
  constexpr int IPW = 32 / RC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int mm = lane % RC;
  for (int m0 = 0; m0 < BW; m0 += RC) {
    for (int t = threadIdx.x; t < m.NL * RC; t += blockDim.x) {
      const int l = t / RC, c = t % RC;
      const int cd = code[l];
      V v = P::zero();
      if (cd >= 0)
        v = P::from_v(df64_neg(sI[(m.ioff[s] + cd) * BW + m0 + c]));
      else if (cd != INT16_MIN && mode == ELEM_SCHUR)
        v = P::from_v(xg[(int64_t)m.gmap[m.goff[s] + (-1 - cd)] * BW + m0 + c]);
      xl[t] = v;
    }
    __syncthreads();
    for (int i = to[2] + warp * IPW + lane / RC; i < to[3]; i += nw * IPW) {
      const int16_t* it = m.type_items + 9 * (size_t)i;
      V v;
      apply_item_b<P, S, RC>(m, it, xl, kd, mm, v);
      yloc[(m.goff[s] + (-1 - code[it[0]])) * BW + m0 + mm] = P::to_v(v);
    }
    __syncthreads();
  }
}

constexpr int ELEM_THREADS = 512;

// members per pass (RC) of the element kernels: 4, 8 or 16 for the 8^3 subdomains of the
// production meshes (chosen by timing at the first ensemble call), 8 otherwise
template <class P, int S, int RC>
static void elem_b_go(const DevMesh& m, bool interior, int mode, const df64* xg, const df64* in, df64* out,
                      cudaStream_t s) {
  const int NE = m.sx * m.sy * m.sz;
  const size_t smem = ((size_t)m.NL * RC + (size_t)NE * 8) * sizeof(typename P::V);
  if (interior) {
    max_smem(k_elem_interior_b<P, S, RC>, smem);
    k_elem_interior_b<P, S, RC><<<m.S, ELEM_THREADS, smem, s>>>(m, mode, xg, in, out);
  } else {
    max_smem(k_elem_interface_b<P, S, RC>, smem);
    k_elem_interface_b<P, S, RC><<<m.S, ELEM_THREADS, smem, s>>>(m, mode, xg, in, out);
  }
}

template <class P>
static void elem_b_dispatch(const DevMesh& m, bool interior, int mode, const df64* xg, const df64* in,
                            df64* out, int rc, cudaStream_t s) {
  if (m.sx == 8 && m.sy == 8 && m.sz == 8) {
    if (rc == 4)
      elem_b_go<P, 8, 4>(m, interior, mode, xg, in, out, s);
    else if (rc == 16)
      elem_b_go<P, 8, 16>(m, interior, mode, xg, in, out, s);
    else
      elem_b_go<P, 8, 8>(m, interior, mode, xg, in, out, s);
  } else if (m.sx == 4 && m.sy == 4 && m.sz == 4) {
    elem_b_go<P, 4, 8>(m, interior, mode, xg, in, out, s);
  } else {
    elem_b_go<P, 0, 8>(m, interior, mode, xg, in, out, s);
  }
}

void launch_elem_interior_b(const DevMesh& m, int mode, const df64* xg, const df64* f, df64* tI, int rc,
                            cudaStream_t s) {
  if (m.schur_prec == DD_PREC_DF64)
    elem_b_dispatch<PolDF>(m, true, mode, xg, f, tI, rc, s);
  else
    elem_b_dispatch<PolF64>(m, true, mode, xg, f, tI, 8, s);
  DD_CHECK_LAUNCH();
}

void launch_elem_interface_b(const DevMesh& m, int mode, const df64* xg, const df64* sI, df64* yloc, int rc,
                             cudaStream_t s) {
  if (m.schur_prec == DD_PREC_DF64)
    elem_b_dispatch<PolDF>(m, false, mode, xg, sI, yloc, rc, s);
  else
    elem_b_dispatch<PolF64>(m, false, mode, xg, sI, yloc, 8, s);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// K_II^{-1} of the ensemble: fast diagonalization with RC members per block
// ---------------------------------------------------------------------------
// contraction along axis ax, one thread per line (the other two indices and a member):
// the line's values sit in registers and all its outputs are formed at once
// (out_j = sum_i A(i, j) in_i when trans, else sum_i A(j, i) in_i)
template <class P, int RC>
__device__ __forceinline__ void fdm_contract_b(const typename P::V* A, int ax, bool trans, const int* n,
                                               const typename P::V* in, typename P::V* out) {
  using V = typename P::V;
  const int na = n[ax];
  const int stride = ax == 0 ? 1 : (ax == 1 ? n[0] : n[0] * n[1]);
  const int o1 = ax == 0 ? n[1] : n[0];
  const int o2 = ax == 2 ? n[1] : n[2];
  const int nl = o1 * o2 * RC;
  for (int t = threadIdx.x; t < nl; t += blockDim.x) {
    const int mm = t % RC, lw = t / RC;
    const int u = lw % o1, w = lw / o1;
    const int base = ax == 0 ? n[0] * (u + n[1] * w) : (ax == 1 ? u + n[0] * n[1] * w : u + n[0] * w);
    V x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = i < na ? in[(base + i * stride) * RC + mm] : P::zero();
    // two outputs of the line at a time: independent accumulation chains overlap
    const int ajs = trans ? 1 : 9, ais = trans ? 9 : 1;  // A(j, i) at A[j * ajs + i * ais]
    for (int j = 0; j < na; j += 2) {
      const bool two = j + 1 < na;
      typename P::Acc a0, a1;
      P::init(a0);
      P::init(a1);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        if (i < na) {
          P::fma(a0, A[j * ajs + i * ais], x[i]);
          if (two) P::fma(a1, A[(j + 1) * ajs + i * ais], x[i]);
        }
      out[(base + j * stride) * RC + mm] = P::get(a0);
      if (two) out[(base + (j + 1) * stride) * RC + mm] = P::get(a1);
    }
  }
}

// 56 lines (7 x 8: the largest two-axis face of an 8^3 subdomain's interior block) of RC
// members per thread pass
template <int RC>
constexpr int fdm_threads() {
  return 56 * RC;
}

template <class P, int RC>
__global__ void __launch_bounds__(fdm_threads<RC>()) k_fdm_apply_b(DevMesh m, const df64* __restrict__ tI,
                                                              df64* __restrict__ sI) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_f[];
  V* b0 = reinterpret_cast<V*>(smem_f);  // [729][RC]
  V* b1 = b0 + 729 * RC;
  __shared__ V Vs[3][81];
  __shared__ int n[3];
  const int s = blockIdx.x, m0 = blockIdx.y * RC;
  if (threadIdx.x < 3) n[threadIdx.x] = m.fdm_n[3 * s + threadIdx.x];
  for (int t = threadIdx.x; t < 243; t += blockDim.x) Vs[t / 81][t % 81] = ld_fdm<P>(m.fdm_V, (int64_t)s * 243 + t);
  __syncthreads();
  const int N = n[0] * n[1] * n[2];
  const int64_t off = m.ioff[s];
  for (int t = threadIdx.x; t < N * RC; t += blockDim.x)
    b0[t] = P::from_v(tI[(off + t / RC) * BW + m0 + t % RC]);
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[0], 0, true, n, b0, b1);
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[1], 1, true, n, b1, b0);
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[2], 2, true, n, b0, b1);
  __syncthreads();
  for (int t = threadIdx.x; t < N * RC; t += blockDim.x) {
    typename P::Acc acc;
    P::init(acc);
    P::fma(acc, b1[t], ld_fdm<P>(m.fdm_Dinv, off + t / RC));
    b1[t] = P::get(acc);
  }
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[0], 0, false, n, b1, b0);
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[1], 1, false, n, b0, b1);
  __syncthreads();
  fdm_contract_b<P, RC>(Vs[2], 2, false, n, b1, b0);
  __syncthreads();
  for (int t = threadIdx.x; t < N * RC; t += blockDim.x) sI[(off + t / RC) * BW + m0 + t % RC] = P::to_v(b0[t]);
}

template <class P, int RC>
static void fdm_b_go(const DevMesh& m, const df64* tI, df64* sI, cudaStream_t s) {
  const size_t smem = (size_t)2 * 729 * RC * sizeof(typename P::V);
  max_smem(k_fdm_apply_b<P, RC>, smem);
  k_fdm_apply_b<P, RC><<<dim3(m.S, BW / RC), fdm_threads<RC>(), smem, s>>>(m, tI, sI);
}

__global__ void k_df_to_dbl(int64_t n, const df64* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df64_to_double_bits(in[i]);
}
__global__ void k_dbl_to_df(int64_t n, const double* __restrict__ in, df64* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df64_from_double_bits(in[i]);
}

void launch_kii_apply_b(const DevMesh& m, const df64* tI, df64* sI, double* tmp, int rc, cudaStream_t s) {
  if (m.local_solver == DD_LOCAL_FDM) {
    if (m.schur_prec == DD_PREC_DF64) {
      if (rc == 4)
        fdm_b_go<PolDF, 4>(m, tI, sI, s);
      else
        fdm_b_go<PolDF, 8>(m, tI, sI, s);
    } else {
      fdm_b_go<PolF64, 8>(m, tI, sI, s);
    }
    DD_CHECK_LAUNCH();
  } else {
    // dense K_II^{-1} (FP64 tiles; the caller rejects df64 dense ensembles): the tiles work
    // on doubles, so the block passes through tmp ([n_int][BW] doubles) both ways
    const int64_t nn = m.n_int * BW;
    k_df_to_dbl<<<grid_for_b(nn, 256), 256, 0, s>>>(nn, tI, tmp);
    DD_CHECK_LAUNCH();
    launch_symm_b(m.KIIinv, m.ioff, tmp, tmp, s);
    k_dbl_to_df<<<grid_for_b(nn, 256), 256, 0, s>>>(nn, tmp, sI);
    DD_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------------------
// gathers and scatters (warp = one row, lane = member)
// ---------------------------------------------------------------------------
__global__ void k_gather_b(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                           const df64* __restrict__ loc, const df64* __restrict__ base,
                           const int64_t* __restrict__ bmap, df64* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < n;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    // copies summed in df64 in the fixed copy order
    df64_acc sum;
    if (base) sum.add(base[(bmap ? bmap[g] : g) * BW + lane]);
    for (int k = ptr[g]; k < ptr[g + 1]; ++k) sum.add(loc[(int64_t)idx[k] * BW + lane]);
    y[g * BW + lane] = sum.get();
  }
}
void launch_gather_b(int64_t n, const int* ptr, const int* idx, const df64* loc, const df64* base,
                     const int64_t* bmap, df64* y, cudaStream_t s) {
  if (n == 0) return;
  k_gather_b<<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, loc, base, bmap, y);
  DD_CHECK_LAUNCH();
}

__global__ void k_scatter_recover_b(DevMesh m, const df64* __restrict__ xg, const df64* __restrict__ sI,
                                    df64* __restrict__ x) {
  const int s = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  for (int l = warp; l < m.NL; l += nw) {
    int cd = code[l];
    if (cd >= 0) x[free_index(m, s, l) * BW + lane] = sI[(m.ioff[s] + cd) * BW + lane];
  }
  for (int j = warp; j < (int)(m.goff[s + 1] - m.goff[s]); j += nw) {
    int64_t k = m.goff[s] + j;
    int g = m.gmap[k];
    if (m.gidx[m.gptr[g]] == (int)k) x[m.gamma_free[g] * BW + lane] = xg[(int64_t)g * BW + lane];
  }
}
void launch_scatter_recover_b(const DevMesh& m, const df64* xg, const df64* sI, df64* x, cudaStream_t s) {
  k_scatter_recover_b<<<m.S, 256, 0, s>>>(m, xg, sI, x);
  DD_CHECK_LAUNCH();
}

// rloc = D_k r with r in df64: the FP32 preconditioner takes the float weight times the
// float sum of the pair; the FP64 one widens both
template <class T>
__global__ void k_restrict_b(int64_t nflat, const int* __restrict__ gmap, const float* __restrict__ Df,
                             const double* __restrict__ D, const df64* __restrict__ r, T* __restrict__ rloc) {
  const int lane = threadIdx.x & 31;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < nflat;
       k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const df64 rv = r[(int64_t)gmap[k] * BW + lane];
    if (sizeof(T) == 4)
      rloc[k * BW + lane] = (T)(Df[k] * (rv.hi + rv.lo));
    else
      rloc[k * BW + lane] = (T)(D[k] * df64_to_double_bits(rv));
  }
}
void launch_restrict_b(int prec, int64_t nflat, const int* gmap, const float* Df, const double* D, const df64* r,
                       void* rloc, cudaStream_t s) {
  if (nflat == 0) return;
  if (prec == DD_PREC_FP32)
    k_restrict_b<float><<<grid_for_b(nflat, 8), 256, 0, s>>>(nflat, gmap, Df, D, r, (float*)rloc);
  else
    k_restrict_b<double><<<grid_for_b(nflat, 8), 256, 0, s>>>(nflat, gmap, Df, D, r, (double*)rloc);
  DD_CHECK_LAUNCH();
}

template <class T>
__global__ void k_restrict_tb(int64_t nflat, const int* __restrict__ gmap, const double* __restrict__ D,
                              const T* __restrict__ r, T* __restrict__ rloc) {
  const int lane = threadIdx.x & 31;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < nflat;
       k += ((int64_t)gridDim.x * blockDim.x) >> 5)
    rloc[k * BW + lane] = (T)D[k] * r[(int64_t)gmap[k] * BW + lane];
}
void launch_restrict_tb(int prec, int64_t nflat, const int* gmap, const double* D, const void* r, void* rloc,
                        cudaStream_t s) {
  if (nflat == 0) return;
  if (prec == DD_PREC_FP32)
    k_restrict_tb<float><<<grid_for_b(nflat, 8), 256, 0, s>>>(nflat, gmap, D, (const float*)r, (float*)rloc);
  else
    k_restrict_tb<double><<<grid_for_b(nflat, 8), 256, 0, s>>>(nflat, gmap, D, (const double*)r, (double*)rloc);
  DD_CHECK_LAUNCH();
}

template <class T>
__global__ void k_wgather_tb(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                             const double* __restrict__ D, const T* __restrict__ uloc, const T* __restrict__ vloc,
                             T* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < n;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    T acc = 0;
    for (int t = ptr[g]; t < ptr[g + 1]; ++t) {
      const int64_t k = idx[t];
      acc = fma((T)D[k], uloc[k * BW + lane] + vloc[k * BW + lane], acc);
    }
    z[g * BW + lane] = acc;
  }
}
void launch_wgather_tb(int prec, int64_t n, const int* ptr, const int* idx, const double* D, const void* uloc,
                       const void* vloc, void* z, cudaStream_t s) {
  if (n == 0) return;
  if (prec == DD_PREC_FP32)
    k_wgather_tb<float><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, D, (const float*)uloc, (const float*)vloc,
                                                         (float*)z);
  else
    k_wgather_tb<double><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, D, (const double*)uloc,
                                                          (const double*)vloc, (double*)z);
  DD_CHECK_LAUNCH();
}

template <class T>
__global__ void k_gather_tb(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                            const T* __restrict__ loc, const T* __restrict__ base, const int64_t* __restrict__ bmap,
                            T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < n;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    T s = base ? base[(bmap ? bmap[g] : g) * BW + lane] : (T)0;
    for (int k = ptr[g]; k < ptr[g + 1]; ++k) s += loc[(int64_t)idx[k] * BW + lane];
    y[g * BW + lane] = s;
  }
}
void launch_gather_tb(int prec, int64_t n, const int* ptr, const int* idx, const void* loc, const void* base,
                      const int64_t* bmap, void* y, cudaStream_t s) {
  if (n == 0) return;
  if (prec == DD_PREC_FP32)
    k_gather_tb<float><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, (const float*)loc, (const float*)base, bmap,
                                                        (float*)y);
  else
    k_gather_tb<double><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, (const double*)loc, (const double*)base,
                                                         bmap, (double*)y);
  DD_CHECK_LAUNCH();
}

template <class T>
__global__ void k_wgather_b(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                            const float* __restrict__ Df, const double* __restrict__ D, const T* __restrict__ uloc,
                            const T* __restrict__ vloc, df64* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < n;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    if (sizeof(T) == 4) {
      // D_k (u + v): exact float products summed in df64
      df64_acc acc;
      for (int t = ptr[g]; t < ptr[g + 1]; ++t) {
        const int64_t k = idx[t];
        acc.fma(df64{Df[k], 0.f}, df64{(float)(uloc[k * BW + lane] + vloc[k * BW + lane]), 0.f});
      }
      z[g * BW + lane] = acc.get();
    } else {
      double acc = 0.0;
      for (int t = ptr[g]; t < ptr[g + 1]; ++t) {
        const int64_t k = idx[t];
        acc = fma(D[k], (double)(uloc[k * BW + lane] + vloc[k * BW + lane]), acc);
      }
      z[g * BW + lane] = df64_from_double_bits(acc);
    }
  }
}
void launch_wgather_b(int prec, int64_t n, const int* ptr, const int* idx, const float* Df, const double* D,
                      const void* uloc, const void* vloc, df64* z, cudaStream_t s) {
  if (n == 0) return;
  if (prec == DD_PREC_FP32)
    k_wgather_b<float><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, Df, D, (const float*)uloc,
                                                        (const float*)vloc, z);
  else
    k_wgather_b<double><<<grid_for_b(n, 8), 256, 0, s>>>(n, ptr, idx, Df, D, (const double*)uloc,
                                                         (const double*)vloc, z);
  DD_CHECK_LAUNCH();
}

template <class T>
__global__ void k_map_b(int64_t n, const int* __restrict__ map, const T* __restrict__ in, T* __restrict__ out,
                        bool scatter) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    if (scatter)
      out[(int64_t)map[i] * BW + lane] = in[i * BW + lane];
    else
      out[i * BW + lane] = in[(int64_t)map[i] * BW + lane];
  }
}
static void map_b(int prec, int64_t n, const int* map, const void* in, void* out, bool scatter, cudaStream_t s) {
  if (n == 0) return;
  if (prec == DD_PREC_FP32)
    k_map_b<float><<<grid_for_b(n, 8), 256, 0, s>>>(n, map, (const float*)in, (float*)out, scatter);
  else
    k_map_b<double><<<grid_for_b(n, 8), 256, 0, s>>>(n, map, (const double*)in, (double*)out, scatter);
  DD_CHECK_LAUNCH();
}
void launch_map_gather_b(int prec, int64_t n, const int* map, const void* in, void* out, cudaStream_t s) {
  map_b(prec, n, map, in, out, false, s);
}
void launch_map_scatter_b(int prec, int64_t n, const int* map, const void* in, void* out, cudaStream_t s) {
  map_b(prec, n, map, in, out, true, s);
}

// ---------------------------------------------------------------------------
// symmetric tiles times BW members (lane = member). Warp w owns the block rows
// b = w (mod warps): it adds T X_bj into out_bi for the tiles of its rows and
// T^T X_bi into out_bj for the tiles of its columns, so every output block has one
// writer and the sums are deterministic. Tiles are read row by row (broadcast loads).
// ---------------------------------------------------------------------------
constexpr int SYMM_WARPS = 4;

template <class T>
__global__ void __launch_bounds__(SYMM_WARPS * 32) k_symm_b(SymTiles A, const int64_t* __restrict__ voff,
                                                            const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_s[];
  T* acc = reinterpret_cast<T*>(smem_s);  // [npad][BW]
  const int mtx = blockIdx.x;
  const int n = A.n[mtx];
  const int nb = (n + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t vo = voff[mtx];
  for (int t = threadIdx.x; t < nb * 32 * BW; t += blockDim.x) acc[t] = (T)0;
  __syncthreads();
  const T* tiles = static_cast<const T*>(A.data) + (size_t)A.toff[mtx] * 1024;
  int t = 0;
  for (int bi = 0; bi < nb; ++bi) {
    for (int bj = bi; bj < nb; ++bj, ++t) {
      const bool own_row = (bi % SYMM_WARPS) == warp;
      const bool own_col = bj != bi && (bj % SYMM_WARPS) == warp;
      if (!own_row && !own_col) continue;
      const T* Tl = tiles + (size_t)t * 1024;
      if (own_row) {
        T xj[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int row = bj * 32 + c;
          xj[c] = row < n ? in[(vo + row) * BW + lane] : (T)0;
        }
        for (int r = 0; r < 32; ++r) {
          const T* tr = Tl + r * 32;
          T a0 = 0, a1 = 0;
#pragma unroll
          for (int c = 0; c < 32; c += 2) {
            a0 = fma(tr[c], xj[c], a0);
            a1 = fma(tr[c + 1], xj[c + 1], a1);
          }
          acc[(bi * 32 + r) * BW + lane] += a0 + a1;
        }
      }
      if (own_col) {
        T ac[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) ac[c] = 0;
        for (int r = 0; r < 32; ++r) {
          const int row = bi * 32 + r;
          const T xi = row < n ? in[(vo + row) * BW + lane] : (T)0;
          const T* tr = Tl + r * 32;
#pragma unroll
          for (int c = 0; c < 32; ++c) ac[c] = fma(tr[c], xi, ac[c]);
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[(bj * 32 + c) * BW + lane] += ac[c];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * BW; i += blockDim.x) out[vo * BW + i] = acc[i];
}

void launch_symm_b(const SymTiles& A, const int64_t* voff, const void* in, void* out, cudaStream_t s) {
  if (A.count == 0) return;
  const int npad = ((A.max_n + 31) / 32) * 32;
  if (A.prec == DD_PREC_FP32) {
    const size_t smem = (size_t)npad * BW * 4;
    max_smem(k_symm_b<float>, smem);
    k_symm_b<float><<<A.count, SYMM_WARPS * 32, smem, s>>>(A, voff, (const float*)in, (float*)out);
  } else if (A.prec == DD_PREC_FP64) {
    const size_t smem = (size_t)npad * BW * 8;
    DD_REQUIRE(smem <= 227 * 1024, "ensemble: local matrix too large for the batched tile kernel");
    max_smem(k_symm_b<double>, smem);
    k_symm_b<double><<<A.count, SYMM_WARPS * 32, smem, s>>>(A, voff, (const double*)in, (double*)out);
  } else {
    throw Error(DD_INVALID_ARG, "ensemble: df64 dense tiles are not supported by the batched path");
  }
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// batched row-major products with BW members (lane = member)
//   k_bmm:   out_m[i] = alpha sum_j A_m[i][j] x_m[j]  -- a warp takes 4 rows, the row
//            entries are loaded by the lanes (coalesced) and broadcast by shuffles
//   k_bmm_t: out_m[j] = alpha sum_i A_m[i][j] x_m[i]  -- a warp takes 8 columns, 4 rows
//            of them per load (lane = row * 8 + column)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ld_x(const T* in, const int* in_map, int64_t io, int j, int lane) {
  const int64_t src = in_map ? (int64_t)in_map[io + j] : io + j;
  return in[src * BW + lane];
}

// STAGE: the item's input rows are first copied to shared memory ([rows][BW]) so the
// inner loop runs on shared-memory loads and register shuffles only
template <class T, bool STAGE>
__global__ void __launch_bounds__(256) k_bmm(const int64_t* __restrict__ row0, const int* __restrict__ cols,
                                             const int64_t* __restrict__ moff, const T* __restrict__ M,
                                             const int64_t* __restrict__ in_off, const int* __restrict__ in_map,
                                             const T* __restrict__ in, const int64_t* __restrict__ out_off,
                                             T* __restrict__ out, T alpha, const T* __restrict__ add) {
  extern __shared__ __align__(16) unsigned char bm_smem[];
  T* xs = reinterpret_cast<T*>(bm_smem);
  const int mi = blockIdx.x;
  const int R = (int)(row0[mi + 1] - row0[mi]), C = cols[mi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t io = in_off[mi], oo = out_off[mi];
  const T* A = M + moff[mi];
  if (blockIdx.y * nw * 4 >= R) return;
  if (STAGE) {
    for (int t = threadIdx.x; t < C * BW; t += blockDim.x) xs[t] = ld_x(in, in_map, io, t / BW, t % BW);
    __syncthreads();
  }
  for (int i0 = (blockIdx.y * nw + warp) * 4; i0 < R; i0 += gridDim.y * nw * 4) {
    T acc[4] = {0, 0, 0, 0};
    for (int j0 = 0; j0 < C; j0 += 32) {
      const int j = j0 + lane;
      T a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = (i0 + k < R && j < C) ? A[(int64_t)(i0 + k) * C + j] : (T)0;
      const int jn = min(32, C - j0);
#pragma unroll 4
      for (int jj = 0; jj < jn; ++jj) {
        const T x = STAGE ? xs[(j0 + jj) * BW + lane] : ld_x(in, in_map, io, j0 + jj, lane);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fma(__shfl_sync(0xffffffffu, a[k], jj), x, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k < R) {
        const int64_t o = (oo + i0 + k) * BW + lane;
        out[o] = alpha * acc[k] + (add ? add[o] : (T)0);
      }
  }
}

template <class T, bool STAGE>
__global__ void __launch_bounds__(256) k_bmm_t(const int64_t* __restrict__ row0, const int* __restrict__ cols,
                                               const int64_t* __restrict__ moff, const T* __restrict__ M,
                                               const int64_t* __restrict__ in_off, const int* __restrict__ in_map,
                                               const T* __restrict__ in, const int64_t* __restrict__ out_off,
                                               T* __restrict__ out, T alpha, const T* __restrict__ add) {
  extern __shared__ __align__(16) unsigned char bm_smem[];
  T* xs = reinterpret_cast<T*>(bm_smem);
  const int mi = blockIdx.x;
  const int R = (int)(row0[mi + 1] - row0[mi]), C = cols[mi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t io = in_off[mi], oo = out_off[mi];
  const T* A = M + moff[mi];
  if (blockIdx.y * nw * 8 >= C) return;
  if (STAGE) {
    for (int t = threadIdx.x; t < R * BW; t += blockDim.x) xs[t] = ld_x(in, in_map, io, t / BW, t % BW);
    __syncthreads();
  }
  const int lr = lane >> 3, lc = lane & 7;
  for (int j0 = (blockIdx.y * nw + warp) * 8; j0 < C; j0 += gridDim.y * nw * 8) {
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i0 = 0; i0 < R; i0 += 4) {
      const int ia = i0 + lr, ja = j0 + lc;
      const T a = (ia < R && ja < C) ? A[(int64_t)ia * C + ja] : (T)0;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int i = i0 + rr;
        const T x = i < R ? (STAGE ? xs[i * BW + lane] : ld_x(in, in_map, io, i, lane)) : (T)0;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fma(__shfl_sync(0xffffffffu, a, rr * 8 + k), x, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (j0 + k < C) {
        const int64_t o = (oo + j0 + k) * BW + lane;
        out[o] = alpha * acc[k] + (add ? add[o] : (T)0);
      }
  }
}

constexpr size_t BMM_STAGE_MAX = 96 * 1024;  // largest staged input slice (bytes)

template <class T>
static void bmm_go(const BatchedRows& B, bool trans, const int64_t* in_off, const int* in_map, const void* in,
                   const int64_t* out_off, void* out, double alpha, const void* add, cudaStream_t s) {
  const int per_block = trans ? 8 * 8 : 8 * 4;  // columns / rows per block pass
  const int extent = trans ? B.max_cols : B.max_rows;
  const int inrows = trans ? B.max_rows : B.max_cols;
  dim3 grid(B.count, std::max(1, std::min(16, (extent + per_block - 1) / per_block)));
  const size_t smem = (size_t)inrows * BW * sizeof(T);
  const bool stage = smem <= BMM_STAGE_MAX;
  const T* Md = static_cast<const T*>(B.data);
  if (trans) {
    if (stage) {
      max_smem(k_bmm_t<T, true>, smem);
      k_bmm_t<T, true><<<grid, 256, smem, s>>>(B.row0, B.cols, B.moff, Md, in_off, in_map, (const T*)in, out_off,
                                               (T*)out, (T)alpha, (const T*)add);
    } else {
      k_bmm_t<T, false><<<grid, 256, 0, s>>>(B.row0, B.cols, B.moff, Md, in_off, in_map, (const T*)in, out_off,
                                             (T*)out, (T)alpha, (const T*)add);
    }
  } else {
    if (stage) {
      max_smem(k_bmm<T, true>, smem);
      k_bmm<T, true><<<grid, 256, smem, s>>>(B.row0, B.cols, B.moff, Md, in_off, in_map, (const T*)in, out_off,
                                             (T*)out, (T)alpha, (const T*)add);
    } else {
      k_bmm<T, false><<<grid, 256, 0, s>>>(B.row0, B.cols, B.moff, Md, in_off, in_map, (const T*)in, out_off,
                                           (T*)out, (T)alpha, (const T*)add);
    }
  }
}

void launch_bmm(const BatchedRows& B, const int64_t* in_off, const int* in_map, const void* in,
                const int64_t* out_off, void* out, double alpha, const void* add, cudaStream_t s) {
  if (B.count == 0) return;
  if (B.prec == DD_PREC_FP32)
    bmm_go<float>(B, false, in_off, in_map, in, out_off, out, alpha, add, s);
  else
    bmm_go<double>(B, false, in_off, in_map, in, out_off, out, alpha, add, s);
  DD_CHECK_LAUNCH();
}

void launch_bmm_t(const BatchedRows& B, const int64_t* in_off, const int* in_map, const void* in,
                  const int64_t* out_off, void* out, double alpha, const void* add, cudaStream_t s) {
  if (B.count == 0) return;
  if (B.prec == DD_PREC_FP32)
    bmm_go<float>(B, true, in_off, in_map, in, out_off, out, alpha, add, s);
  else
    bmm_go<double>(B, true, in_off, in_map, in, out_off, out, alpha, add, s);
  DD_CHECK_LAUNCH();
}

// dense n x n times BW members: warp per row, lanes load the row, shuffles broadcast it
template <class T>
__global__ void __launch_bounds__(256) k_dense_mm(int n, const T* __restrict__ A, const T* __restrict__ x,
                                                  T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
    const T* a = A + (int64_t)row * n;
    T acc0 = 0, acc1 = 0;
    for (int j0 = 0; j0 < n; j0 += 32) {
      const T av = (j0 + lane < n) ? a[j0 + lane] : (T)0;
      const int jn = min(32, n - j0);
      int jj = 0;
      for (; jj + 1 < jn; jj += 2) {
        acc0 = fma(__shfl_sync(0xffffffffu, av, jj), x[(int64_t)(j0 + jj) * BW + lane], acc0);
        acc1 = fma(__shfl_sync(0xffffffffu, av, jj + 1), x[(int64_t)(j0 + jj + 1) * BW + lane], acc1);
      }
      if (jj < jn) acc0 = fma(__shfl_sync(0xffffffffu, av, jj), x[(int64_t)(j0 + jj) * BW + lane], acc0);
    }
    y[(int64_t)row * BW + lane] = acc0 + acc1;
  }
}
void launch_dense_mm(int prec, int n, const void* A, const void* x, void* y, cudaStream_t s) {
  if (n == 0) return;
  const int blocks = std::max(1, std::min(152 * 8, (n * 32 + 255) / 256));
  if (prec == DD_PREC_FP32)
    k_dense_mm<float><<<blocks, 256, 0, s>>>(n, (const float*)A, (const float*)x, (float*)y);
  else
    k_dense_mm<double><<<blocks, 256, 0, s>>>(n, (const double*)A, (const double*)x, (double*)y);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Krylov vectors of the ensemble: per-member dots (lane = member, so a warp's rows
// reduce without shuffles), fixed-order two-stage reductions, device-side stopping
// ---------------------------------------------------------------------------
constexpr int BRB = 256;  // threads per block
constexpr int BND = 4;    // dots per partial record

// partials[blk][d][m], one block reduces its warps in a fixed order
__device__ __forceinline__ void bblock_store(const double* v, int nd, double* partials) {
  __shared__ double sh[BND][BRB / 32][BW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < nd; ++d) sh[d][warp][lane] = v[d];
  __syncthreads();
  for (int t = threadIdx.x; t < nd * BW; t += blockDim.x) {
    const int d = t / BW, m = t % BW;
    double s = 0.0;
    for (int w = 0; w < BRB / 32; ++w) s += sh[d][w][m];
    partials[((int64_t)blockIdx.x * BND + d) * BW + m] = s;
  }
}

// member dots of df64 vectors, accumulated in df64 on the FP32 pipes
__global__ void __launch_bounds__(BRB) k_bdots(int64_t n, const df64* __restrict__ a0, const df64* __restrict__ b0,
                                               const df64* __restrict__ a1, const df64* __restrict__ b1,
                                               double* partials) {
  const int lane = threadIdx.x & 31;
  df64_acc s0, s1;
  for (int64_t i = (blockIdx.x * (int64_t)BRB + threadIdx.x) >> 5; i < n; i += ((int64_t)gridDim.x * BRB) >> 5) {
    s0.fma(a0[i * BW + lane], b0[i * BW + lane]);
    if (a1) s1.fma(a1[i * BW + lane], b1[i * BW + lane]);
  }
  double v[2] = {df64_to_double_bits(s0.get()), df64_to_double_bits(s1.get())};
  bblock_store(v, 2, partials);
}

// x += alpha p ; r -= alpha q ; partial ||r||^2   (per member alpha, df64 arithmetic)
__global__ void __launch_bounds__(BRB) k_baxpy2(int64_t n, const double* __restrict__ sc, df64* __restrict__ x,
                                                const df64* __restrict__ p, df64* __restrict__ r,
                                                const df64* __restrict__ q, double* partials) {
  const int lane = threadIdx.x & 31;
  const df64 alpha = df64_from_double_bits(sc[BS_ALPHA * BW + lane]);
  const df64 malpha = df64_neg(alpha);
  df64_acc rr;
  for (int64_t i = (blockIdx.x * (int64_t)BRB + threadIdx.x) >> 5; i < n; i += ((int64_t)gridDim.x * BRB) >> 5) {
    const int64_t o = i * BW + lane;
    df64_acc xa, ra;
    xa.add(x[o]);
    xa.fma(alpha, p[o]);
    x[o] = xa.get();
    ra.add(r[o]);
    ra.fma(malpha, q[o]);
    const df64 ri = ra.get();
    r[o] = ri;
    rr.fma(ri, ri);
  }
  double v[1] = {df64_to_double_bits(rr.get())};
  bblock_store(v, 1, partials);
}

// one warp, lane = member: sums the block partials in a fixed order and updates the
// member's scalars. Inactive members keep alpha = beta = 0, so their iterates stay fixed.
constexpr int BFIN_WARPS = 32;
__global__ void __launch_bounds__(BFIN_WARPS * 32) k_bfinalize(int nblk, const double* __restrict__ partials,
                                                               double* sc, int op, int flexible,
                                                               const int* __restrict__ its) {
  // warp w sums the blocks w, w + 32, ... (lane = member); warp 0 then adds the 32
  // warp sums in order: a fixed reduction tree
  __shared__ double part[BFIN_WARPS][2][BW];
  {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
    for (int b = w; b < nblk; b += BFIN_WARPS) {
      a0 += partials[((int64_t)b * BND + 0) * BW + l];
      a1 += partials[((int64_t)b * BND + 1) * BW + l];
    }
    part[w][0][l] = a0;
    part[w][1][l] = a1;
  }
  __syncthreads();
  const int m = threadIdx.x;
  if (m >= BW) return;
  double t0 = 0.0, t1 = 0.0;
  for (int w = 0; w < BFIN_WARPS; ++w) {
    t0 += part[w][0][m];
    t1 += part[w][1][m];
  }
  double* S = sc;
  auto at = [&](int slot) -> double& { return S[slot * BW + m]; };
  const bool act = at(BS_ACT) != 0.0;
  if (op == BFIN_RZL) op = *its == 0 ? BFIN_RZ0 : BFIN_RZ;  // device-resident loop: first iteration or not
  switch (op) {
    case BFIN_PQ:
      at(BS_PQ) = t0;
      if (!act) {
        at(BS_ALPHA) = 0.0;
      } else if (!(t0 > 0.0) || !isfinite(t0) || !isfinite(at(BS_RZ))) {
        at(BS_FLAG) = 1.0;
        at(BS_ALPHA) = 0.0;
        at(BS_ACT) = 0.0;
      } else {
        at(BS_ALPHA) = at(BS_RZ) / t0;
      }
      break;
    case BFIN_RR:
      if (act) {
        at(BS_RR) = t0;
        at(BS_ITS) += 1.0;
        if (!isfinite(t0)) {
          at(BS_FLAG) = 1.0;
          at(BS_ACT) = 0.0;
        } else if (t0 < at(BS_RTOL2) * at(BS_REF) * at(BS_REF)) {
          at(BS_ACT) = 0.0;  // converged
        }
      }
      break;
    case BFIN_RZ0:
      at(BS_RZ) = t0;
      if (act && (!(t0 > 0.0) || !isfinite(t0))) {
        at(BS_FLAG) = 1.0;
        at(BS_ACT) = 0.0;
      }
      break;
    case BFIN_RZ: {
      const double num = flexible ? (t0 - t1) : t0;
      const double rz = at(BS_RZ);
      at(BS_BETA) = (act && rz != 0.0) ? num / rz : 0.0;
      at(BS_RZ) = t0;
      if (act && (!(t0 > 0.0) || !isfinite(t0))) {
        at(BS_FLAG) = 1.0;
        at(BS_ACT) = 0.0;
      }
      break;
    }
    case BFIN_BB: {
      // stopping reference and initial activity: ||b|| (or ||r_0||); a zero right-hand
      // side (padding) is solved by x = 0 and never becomes active
      at(BS_BB) = t0;
      at(BS_RR0) = t1;
      at(BS_RR) = t1;
      const bool rhs_ref = at(BS_REF) > 0.0;  // BS_REF holds 1 for ||b||, 0 for ||r_0|| before this step
      double ref = rhs_ref ? sqrt(t0) : sqrt(t1);
      if (ref == 0.0) ref = 1.0;
      at(BS_REF) = ref;
      at(BS_ITS) = 0.0;
      at(BS_ACT) = (t0 > 0.0 && t1 >= at(BS_RTOL2) * ref * ref) ? 1.0 : 0.0;
      break;
    }
    default:
      break;
  }
}

void bvec_dots(int64_t n, const df64* a0, const df64* b0, const df64* a1, const df64* b1, double* partials,
               cudaStream_t s) {
  k_bdots<<<NBLKB, BRB, 0, s>>>(n, a0, b0, a1, b1, partials);
  DD_CHECK_LAUNCH();
}
void bvec_finalize(const double* partials, double* sc, int op, int flexible, cudaStream_t s, const int* its) {
  k_bfinalize<<<1, BFIN_WARPS * 32, 0, s>>>(NBLKB, partials, sc, op, flexible, its);
  DD_CHECK_LAUNCH();
}
void bvec_axpy2(int64_t n, const double* sc, df64* x, const df64* p, df64* r, const df64* q, double* partials,
                cudaStream_t s) {
  k_baxpy2<<<NBLKB, BRB, 0, s>>>(n, sc, x, p, r, q, partials);
  DD_CHECK_LAUNCH();
}

__global__ void k_bsub(int64_t n, const df64* __restrict__ a, const df64* __restrict__ b, df64* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = df64_add(a[i], df64_neg(b[i]));
}
void bvec_sub(int64_t n, const df64* a, const df64* b, df64* y, cudaStream_t s) {
  k_bsub<<<NBLK, BRB, 0, s>>>(n * BW, a, b, y);
  DD_CHECK_LAUNCH();
}

__global__ void k_binit(double* sc, int nrhs, double rtol, int stop_rhs_norm) {
  const int m = threadIdx.x;
  if (m >= BW) return;
  for (int slot = 0; slot < BS_COUNT; ++slot) sc[slot * BW + m] = 0.0;
  sc[BS_RTOL2 * BW + m] = rtol * rtol;
  sc[BS_REF * BW + m] = stop_rhs_norm ? 1.0 : 0.0;
  (void)nrhs;
}
void bvec_init(double* sc, int nrhs, double rtol, int stop_rhs_norm, cudaStream_t s) {
  k_binit<<<1, BW, 0, s>>>(sc, nrhs, rtol, stop_rhs_norm);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// deflation with the basis W shared by the ensemble, as blocked GEMMs in df64:
//   mu = G (W^T Z)             Z: [n][BW]   W: k columns of length n (stride ld)
//   Y = Z + beta Y + s W mu    (per member beta)
// A block takes DROWS rows: the slice of W (16 columns at a time) and of Z is staged in
// shared memory with coalesced loads, so every element of W and Z is read once from HBM.
// ---------------------------------------------------------------------------
constexpr int DROWS = 128;  // rows per block
constexpr int DCOLS = 16;   // basis columns per stage

int defl_blocks(int64_t n) { return (int)((n + DROWS - 1) / DROWS); }

// wpart[b][c][m] = sum over the rows of block b of W[c][i] Z[i][m]  (df64 partials)
__global__ void __launch_bounds__(256) k_bwdots3(int64_t n, int k, const df64* __restrict__ W, int64_t ld,
                                                 const df64* __restrict__ Z, df64* __restrict__ wpart) {
  __shared__ df64 zs[DROWS][BW];      // 32 KiB
  __shared__ df64 ws[DCOLS][DROWS];   // 16 KiB
  const int64_t r0 = (int64_t)blockIdx.x * DROWS;
  const int rows = (int)min((int64_t)DROWS, n - r0);
  for (int t = threadIdx.x; t < DROWS * BW; t += blockDim.x) {
    const int r = t / BW, m = t % BW;
    zs[r][m] = r < rows ? Z[(r0 + r) * BW + m] : df64{0.f, 0.f};
  }
  const int m = threadIdx.x & 31, cw = threadIdx.x >> 5;  // 8 warps: columns cw and cw + 8 of a stage
  for (int c0 = 0; c0 < k; c0 += DCOLS) {
    const int nc = min(DCOLS, k - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < DCOLS * DROWS; t += blockDim.x) {
      const int c = t / DROWS, r = t % DROWS;
      ws[c][r] = (c < nc && r < rows) ? W[(int64_t)(c0 + c) * ld + r0 + r] : df64{0.f, 0.f};
    }
    __syncthreads();
    df64_acc a0, a1;
#pragma unroll 4
    for (int r = 0; r < DROWS; ++r) {
      const df64 z = zs[r][m];
      a0.fma(ws[cw][r], z);
      a1.fma(ws[cw + 8][r], z);
    }
    if (cw < nc) wpart[((int64_t)blockIdx.x * k + c0 + cw) * BW + m] = a0.get();
    if (cw + 8 < nc) wpart[((int64_t)blockIdx.x * k + c0 + cw + 8) * BW + m] = a1.get();
  }
}

// d[c][m] = fixed-order sum of the block partials (one block per column c; warp w takes
// the blocks w, w + 32, ...; warp 0 adds the warp sums in order), written into mu
__global__ void __launch_bounds__(1024) k_bwsum(int nblk, int k, const df64* __restrict__ wpart, double* d) {
  __shared__ df64 part[32][BW];
  const int c = blockIdx.x, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  df64_acc a;
  for (int b = w; b < nblk; b += 32) a.add(wpart[((int64_t)b * k + c) * BW + l]);
  part[w][l] = a.get();
  __syncthreads();
  if (w == 0) {
    df64_acc sum;
    for (int q = 0; q < 32; ++q) sum.add(part[q][l]);
    d[c * BW + l] = df64_to_double_bits(sum.get());
  }
}

// mu[a][m] = sum_c G[a][c] d[c][m] (d read from mu into shared memory first)
__global__ void __launch_bounds__(256) k_bwfinal(int k, const double* __restrict__ G, double* mu) {
  __shared__ double d[MAXK][BW];
  for (int q = threadIdx.x; q < k * BW; q += blockDim.x) d[q / BW][q % BW] = mu[q];
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = w; a < k; a += nw) {
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
    for (; c + 1 < k; c += 2) {
      s0 = fma(G[a * k + c], d[c][l], s0);
      s1 = fma(G[a * k + c + 1], d[c + 1][l], s1);
    }
    if (c < k) s0 = fma(G[a * k + c], d[c][l], s0);
    mu[a * BW + l] = s0 + s1;
  }
}

void bdefl_mu(int64_t n, int k, const df64* W, int64_t ld, const df64* Z, const double* G, df64* wpart, double* mu,
              cudaStream_t s) {
  if (k == 0) return;
  const int nb = defl_blocks(n);
  k_bwdots3<<<nb, 256, 0, s>>>(n, k, W, ld, Z, wpart);
  DD_CHECK_LAUNCH();
  k_bwsum<<<k, 1024, 0, s>>>(nb, k, wpart, mu);
  DD_CHECK_LAUNCH();
  k_bwfinal<<<1, 256, 0, s>>>(k, G, mu);
  DD_CHECK_LAUNCH();
}

// Y = Z + beta Y + sign W mu; warp = 16 rows, lane = member, the sums kept in registers
// while the basis columns pass through shared memory
__global__ void __launch_bounds__(256) k_bpupdate3(int64_t n, int k, const df64* __restrict__ W, int64_t ld,
                                                   const double* __restrict__ mu, const df64* __restrict__ Z,
                                                   df64* __restrict__ Y, const double* __restrict__ sc, int beta_idx,
                                                   double sign_w) {
  __shared__ df64 mus[MAXK][BW];      // 32 KiB
  __shared__ df64 ws[DCOLS][DROWS];   // 16 KiB
  constexpr int RPW = DROWS / 8;      // rows per warp
  for (int q = threadIdx.x; q < k * BW; q += blockDim.x) mus[q / BW][q % BW] = df64_from_double_bits(sign_w * mu[q]);
  const int64_t r0 = (int64_t)blockIdx.x * DROWS;
  const int rows = (int)min((int64_t)DROWS, n - r0);
  const int m = threadIdx.x & 31, w = threadIdx.x >> 5;
  const df64 beta = df64_from_double_bits(beta_idx >= 0 ? sc[beta_idx * BW + m] : 0.0);
  df64_acc acc[RPW];
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const int r = w * RPW + j;
    if (r < rows) {
      const int64_t o = (r0 + r) * BW + m;
      if (Z) acc[j].add(Z[o]);
      if (beta_idx >= 0)
        acc[j].fma(beta, Y[o]);
      else if (!Z)
        acc[j].add(Y[o]);
    }
  }
  for (int c0 = 0; c0 < k; c0 += DCOLS) {
    const int nc = min(DCOLS, k - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < DCOLS * DROWS; t += blockDim.x) {
      const int c = t / DROWS, r = t % DROWS;
      ws[c][r] = (c < nc && r < rows) ? W[(int64_t)(c0 + c) * ld + r0 + r] : df64{0.f, 0.f};
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
      const df64 mc = mus[c0 + c][m];
#pragma unroll
      for (int j = 0; j < RPW; ++j) acc[j].fma(ws[c][w * RPW + j], mc);
    }
  }
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const int r = w * RPW + j;
    if (r < rows) Y[(r0 + r) * BW + m] = acc[j].get();
  }
}

void bdefl_update(int64_t n, int k, const df64* W, int64_t ld, const double* mu, const df64* Z, df64* Y,
                  const double* sc, int beta_idx, double sign_w, cudaStream_t s) {
  if (n == 0) return;
  k_bpupdate3<<<defl_blocks(n), 256, 0, s>>>(n, k, W, ld, mu, Z, Y, sc, beta_idx, sign_w);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

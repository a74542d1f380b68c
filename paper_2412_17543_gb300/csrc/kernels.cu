// Kernels of the Schur-complement operator and the BDDC preconditioner.
//
//  * k_elem_interior / k_elem_interface: the matrix-free Q1 operator of a
//    subdomain (one CTA per subdomain). Each brick's 8x8 matrix is
//    k_e[(hy hz/hx) K1(x)M1(x)M1 + ...] (Sect. 2, Q1 pressure), whose entry for two
//    corners depends only on which axes they differ in, so 8 values per element
//    are formed in shared memory and every output node sums over its <= 8 bricks.
//  * k_symv: batched symmetric GEMV over 32x32 upper tiles (K_II^{-1}, N_i, ...),
//    one CTA per matrix; every warp streams its tiles global->shared with
//    cp.async.bulk (TMA bulk copies completing on an mbarrier), and uses each tile
//    twice (row block and, off the diagonal, column block) with bank-conflict-free
//    skewed shared-memory reads, so each stored element is read from HBM once.
//  * gathers: deterministic interface assembly sum_i R_i^T (.) (a fixed order of
//    the <= 8 copies of an interface dof, no atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "device.h"
#include "policy.cuh"
#include "ptx.cuh"

namespace dd {

// t_I = f_I - ck * (K [0; x_G])_I   (SCHUR: t = (K x)_I; CONDENSE: t = f_I; RECOVER: t = f_I - (K x)_I)
template <class P, int S>
__global__ void __launch_bounds__(256) k_elem_interior(DevMesh m, int mode, const double* __restrict__ xg,
                                                       const double* __restrict__ f, double* __restrict__ tI) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xl = reinterpret_cast<V*>(smem_raw);
  V* kd = xl + m.NL;
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  const int* to = m.type_off + 6 * m.sub_type[s];
  const int64_t io = m.ioff[s];
  // every interior output first gets its base value (0 or f_I)
  for (int l = threadIdx.x; l < m.NL; l += blockDim.x) {
    int cd = code[l];
    if (cd >= 0) tI[io + cd] = (mode == ELEM_SCHUR) ? 0.0 : f[free_index(m, s, l)];
  }
  if (mode == ELEM_CONDENSE) return;
  for (int l = threadIdx.x; l < m.NL; l += blockDim.x) {
    int cd = code[l];
    xl[l] = (cd < 0 && cd != INT16_MIN) ? P::from_d(xg[m.gmap[m.goff[s] + (-1 - cd)]]) : P::zero();
  }
  build_kd_list<P, S>(m, s, m.type_bl + to[4], to[5] - to[4], kd);
  __syncthreads();
  for (int i = to[0] + threadIdx.x; i < to[1]; i += blockDim.x) {
    const int16_t* it = m.type_items + 9 * (size_t)i;
    const int l = it[0];
    const double v = P::to_d(apply_item<P, S>(m, it, xl, kd));
    const int cd = code[l];
    if (mode == ELEM_SCHUR)
      tI[io + cd] = v;
    else
      tI[io + cd] = f[free_index(m, s, l)] - v;
  }
}

// y_G = (K [-s_I; x_G])_G  (SCHUR: x_G given; CONDENSE: x_G = 0)
template <class P, int S>
__global__ void __launch_bounds__(256) k_elem_interface(DevMesh m, int mode, const double* __restrict__ xg,
                                                        const double* __restrict__ sI, double* __restrict__ yloc) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xl = reinterpret_cast<V*>(smem_raw);
  V* kd = xl + m.NL;
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  const int* to = m.type_off + 6 * m.sub_type[s];
  for (int l = threadIdx.x; l < m.NL; l += blockDim.x) {
    int cd = code[l];
    V v = P::zero();
    if (cd >= 0) v = P::from_d(-sI[m.ioff[s] + cd]);
    else if (cd != INT16_MIN && mode == ELEM_SCHUR) v = P::from_d(xg[m.gmap[m.goff[s] + (-1 - cd)]]);
    xl[l] = v;
  }
  build_kd_list<P, S>(m, s, m.type_bl + to[4], to[5] - to[4], kd);
  __syncthreads();
  for (int i = to[2] + threadIdx.x; i < to[3]; i += blockDim.x) {
    const int16_t* it = m.type_items + 9 * (size_t)i;
    const int cd = code[it[0]];
    yloc[m.goff[s] + (-1 - cd)] = P::to_d(apply_item<P, S>(m, it, xl, kd));
  }
}

template <class P>
static void elem_interior_dispatch(const DevMesh& m, int mode, const double* xg, const double* f, double* tI,
                                   size_t smem, cudaStream_t s) {
  if (m.sx == 8 && m.sy == 8 && m.sz == 8)
    k_elem_interior<P, 8><<<m.S, 256, smem, s>>>(m, mode, xg, f, tI);
  else if (m.sx == 4 && m.sy == 4 && m.sz == 4)
    k_elem_interior<P, 4><<<m.S, 256, smem, s>>>(m, mode, xg, f, tI);
  else
    k_elem_interior<P, 0><<<m.S, 256, smem, s>>>(m, mode, xg, f, tI);
}
template <class P>
static void elem_interface_dispatch(const DevMesh& m, int mode, const double* xg, const double* sI, double* yloc,
                                    size_t smem, cudaStream_t s) {
  if (m.sx == 8 && m.sy == 8 && m.sz == 8)
    k_elem_interface<P, 8><<<m.S, 256, smem, s>>>(m, mode, xg, sI, yloc);
  else if (m.sx == 4 && m.sy == 4 && m.sz == 4)
    k_elem_interface<P, 4><<<m.S, 256, smem, s>>>(m, mode, xg, sI, yloc);
  else
    k_elem_interface<P, 0><<<m.S, 256, smem, s>>>(m, mode, xg, sI, yloc);
}

void launch_elem_interior(const DevMesh& m, int mode, const double* xg, const double* f, double* tI,
                          cudaStream_t s) {
  int NE = m.sx * m.sy * m.sz;
  size_t smem = (size_t)(m.NL + NE * 8) * 8;
  if (m.schur_prec == DD_PREC_DF64)
    elem_interior_dispatch<PolDF>(m, mode, xg, f, tI, smem, s);
  else
    elem_interior_dispatch<PolF64>(m, mode, xg, f, tI, smem, s);
  DD_CHECK_LAUNCH();
}

void launch_elem_interface(const DevMesh& m, int mode, const double* xg, const double* sI, double* yloc,
                           cudaStream_t s) {
  int NE = m.sx * m.sy * m.sz;
  size_t smem = (size_t)(m.NL + NE * 8) * 8;
  if (m.schur_prec == DD_PREC_DF64)
    elem_interface_dispatch<PolDF>(m, mode, xg, sI, yloc, smem, s);
  else
    elem_interface_dispatch<PolF64>(m, mode, xg, sI, yloc, smem, s);
  DD_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// batched symmetric tile GEMV
// ---------------------------------------------------------------------------
template <int PREC>
struct TileOps;

template <>
struct TileOps<DD_PREC_FP64> {
  using P = PolF64;
  using V = double;
  static constexpr int BYTES = 8192;
  __device__ static void both_parts(const unsigned char* T, const V* ti, const V* tj, int l, V& row, V& col) {
    row = row_part(T, tj, l);
    col = col_part(T, ti, l);
  }
  // four independent accumulation chains per part (instruction-level parallelism)
  __device__ static V row_part(const unsigned char* T, const V* tv, int l) {
    const double* A = reinterpret_cast<const double*>(T);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 4) {
      int c0 = (cc + l) & 31, c1 = (cc + 1 + l) & 31, c2 = (cc + 2 + l) & 31, c3 = (cc + 3 + l) & 31;
      a0 = ::fma(A[l * 32 + c0], tv[c0], a0);
      a1 = ::fma(A[l * 32 + c1], tv[c1], a1);
      a2 = ::fma(A[l * 32 + c2], tv[c2], a2);
      a3 = ::fma(A[l * 32 + c3], tv[c3], a3);
    }
    return (a0 + a1) + (a2 + a3);
  }
  __device__ static V col_part(const unsigned char* T, const V* tv, int l) {
    const double* A = reinterpret_cast<const double*>(T);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int r = 0; r < 32; r += 4) {
      a0 = ::fma(A[r * 32 + l], tv[r], a0);
      a1 = ::fma(A[(r + 1) * 32 + l], tv[r + 1], a1);
      a2 = ::fma(A[(r + 2) * 32 + l], tv[r + 2], a2);
      a3 = ::fma(A[(r + 3) * 32 + l], tv[r + 3], a3);
    }
    return (a0 + a1) + (a2 + a3);
  }
};

template <>
struct TileOps<DD_PREC_FP32> {
  using P = PolF32;
  using V = float;
  static constexpr int BYTES = 4096;
  __device__ static void both_parts(const unsigned char* T, const V* ti, const V* tj, int l, V& row, V& col) {
    row = row_part(T, tj, l);
    col = col_part(T, ti, l);
  }
  __device__ static V row_part(const unsigned char* T, const V* tv, int l) {
    const float* A = reinterpret_cast<const float*>(T);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 4) {
      int c0 = (cc + l) & 31, c1 = (cc + 1 + l) & 31, c2 = (cc + 2 + l) & 31, c3 = (cc + 3 + l) & 31;
      a0 = fmaf(A[l * 32 + c0], tv[c0], a0);
      a1 = fmaf(A[l * 32 + c1], tv[c1], a1);
      a2 = fmaf(A[l * 32 + c2], tv[c2], a2);
      a3 = fmaf(A[l * 32 + c3], tv[c3], a3);
    }
    return (a0 + a1) + (a2 + a3);
  }
  __device__ static V col_part(const unsigned char* T, const V* tv, int l) {
    const float* A = reinterpret_cast<const float*>(T);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int r = 0; r < 32; r += 4) {
      a0 = fmaf(A[r * 32 + l], tv[r], a0);
      a1 = fmaf(A[(r + 1) * 32 + l], tv[r + 1], a1);
      a2 = fmaf(A[(r + 2) * 32 + l], tv[r + 2], a2);
      a3 = fmaf(A[(r + 3) * 32 + l], tv[r + 3], a3);
    }
    return (a0 + a1) + (a2 + a3);
  }
};

template <>
struct TileOps<DD_PREC_DF64> {
  using P = PolDF;
  using V = df64;
  static constexpr int BYTES = 8192;
  // tile element (r, c) is the float pair at float2 index r * 32 + c
  __device__ static V row_part(const unsigned char* T, const V* tv, int l) {
    const float2* A = reinterpret_cast<const float2*>(T);
    df64_acc a0, a1, a2, a3;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 4) {
      int c0 = (cc + l) & 31, c1 = (cc + 1 + l) & 31, c2 = (cc + 2 + l) & 31, c3 = (cc + 3 + l) & 31;
      float2 e0 = A[l * 32 + c0], e1 = A[l * 32 + c1], e2 = A[l * 32 + c2], e3 = A[l * 32 + c3];
      a0.fma(df64{e0.x, e0.y}, tv[c0]);
      a1.fma(df64{e1.x, e1.y}, tv[c1]);
      a2.fma(df64{e2.x, e2.y}, tv[c2]);
      a3.fma(df64{e3.x, e3.y}, tv[c3]);
    }
    return df64_add(df64_add(a0.get(), a1.get()), df64_add(a2.get(), a3.get()));
  }
  __device__ static V col_part(const unsigned char* T, const V* tv, int l) {
    const float2* A = reinterpret_cast<const float2*>(T);
    df64_acc a0, a1, a2, a3;
#pragma unroll
    for (int r = 0; r < 32; r += 4) {
      float2 e0 = A[r * 32 + l], e1 = A[(r + 1) * 32 + l], e2 = A[(r + 2) * 32 + l], e3 = A[(r + 3) * 32 + l];
      a0.fma(df64{e0.x, e0.y}, tv[r]);
      a1.fma(df64{e1.x, e1.y}, tv[r + 1]);
      a2.fma(df64{e2.x, e2.y}, tv[r + 2]);
      a3.fma(df64{e3.x, e3.y}, tv[r + 3]);
    }
    return df64_add(df64_add(a0.get(), a1.get()), df64_add(a2.get(), a3.get()));
  }
  // both parts of an off-diagonal tile in one pass: eight independent chains
  __device__ static void both_parts(const unsigned char* T, const V* ti, const V* tj, int l, V& row, V& col) {
    const float2* A = reinterpret_cast<const float2*>(T);
    df64_acc r0, r1, r2, r3, q0, q1, q2, q3;
#pragma unroll
    for (int cc = 0; cc < 32; cc += 4) {
      int c0 = (cc + l) & 31, c1 = (cc + 1 + l) & 31, c2 = (cc + 2 + l) & 31, c3 = (cc + 3 + l) & 31;
      float2 e0 = A[l * 32 + c0], e1 = A[l * 32 + c1], e2 = A[l * 32 + c2], e3 = A[l * 32 + c3];
      float2 f0 = A[cc * 32 + l], f1 = A[(cc + 1) * 32 + l], f2 = A[(cc + 2) * 32 + l], f3 = A[(cc + 3) * 32 + l];
      r0.fma(df64{e0.x, e0.y}, tj[c0]);
      q0.fma(df64{f0.x, f0.y}, ti[cc]);
      r1.fma(df64{e1.x, e1.y}, tj[c1]);
      q1.fma(df64{f1.x, f1.y}, ti[cc + 1]);
      r2.fma(df64{e2.x, e2.y}, tj[c2]);
      q2.fma(df64{f2.x, f2.y}, ti[cc + 2]);
      r3.fma(df64{e3.x, e3.y}, tj[c3]);
      q3.fma(df64{f3.x, f3.y}, ti[cc + 3]);
    }
    row = df64_add(df64_add(r0.get(), r1.get()), df64_add(r2.get(), r3.get()));
    col = df64_add(df64_add(q0.get(), q1.get()), df64_add(q2.get(), q3.get()));
  }
};

constexpr int SYMV_WARPS = 4;

__device__ __forceinline__ void tile_coords(int t, int nb, int& bi, int& bj) {
  int b = 0, start = 0;
  while (b < nb && t >= start + (nb - b)) {
    start += nb - b;
    ++b;
  }
  bi = b;
  bj = b + (t - start);
}

// element i of a staged tile as the policy's value type
template <class P>
struct TileElem;
template <>
struct TileElem<PolF32> {
  __device__ static float ld(const unsigned char* T, int i) { return reinterpret_cast<const float*>(T)[i]; }
};
template <>
struct TileElem<PolF64> {
  __device__ static double ld(const unsigned char* T, int i) { return reinterpret_cast<const double*>(T)[i]; }
};
template <>
struct TileElem<PolDF> {
  __device__ static df64 ld(const unsigned char* T, int i) {
    const float2 e = reinterpret_cast<const float2*>(T)[i];
    return {e.x, e.y};
  }
};

template <class P>
__device__ __forceinline__ typename P::V warp_sum(typename P::V v);
template <>
__device__ __forceinline__ float warp_sum<PolF32>(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <>
__device__ __forceinline__ double warp_sum<PolF64>(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <>
__device__ __forceinline__ df64 warp_sum<PolDF>(df64 v) {
  for (int o = 16; o; o >>= 1) {
    df64 u{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df64_add(v, u);
  }
  return v;
}

// diagonal block of height h stored as its packed upper triangle (row r starts at
// off(r) = r h - r (r - 1) / 2): lane l < h returns sum_c T(l, c) x_c. The lower part is
// read by symmetry in a first sweep over r (lanes l > r read the contiguous entries
// T(r, l), at off(r) + l - r), the upper part in a second sweep along the lane's own row.
template <class P, int H>
__device__ __forceinline__ typename P::V packed_diag_sweep(const unsigned char* T, const typename P::V* tv, int l,
                                                           int h) {
  typename P::Acc a0, a1;
  P::init(a0);
  P::init(a1);
  const int hh = H ? H : h;
  int idx = l;
#pragma unroll
  for (int r = 0; r < (H ? H - 1 : 31); ++r) {
    if (!H && r >= hh - 1) break;
    if (l > r && l < hh) P::fma(a0, TileElem<P>::ld(T, idx), tv[r]);
    idx += hh - 1 - r;
  }
  const int base = l * hh - l * (l - 1) / 2;
#pragma unroll
  for (int t = 0; t < (H ? H : 32); ++t) {
    if (!H && t >= hh) break;
    if (l + t < hh) P::fma(a1, TileElem<P>::ld(T, base + t), tv[l + t]);
  }
  return P::add(P::get(a0), P::get(a1));
}

template <class P>
__device__ __forceinline__ typename P::V packed_diag_part(const unsigned char* T, const typename P::V* tv, int l,
                                                          int h) {
  return h == 32 ? packed_diag_sweep<P, 32>(T, tv, l, 32) : packed_diag_sweep<P, 0>(T, tv, l, h);
}

// block of the ragged last w columns (32 rows of wp stored values): lane l returns the row
// part sum_{c<w} T(l, c) x_j[c] and, for l < w, the column part sum_r T(r, l) x_i[r]
template <class P>
__device__ __forceinline__ void packed_ragged_parts(const unsigned char* T, int wp, int w, const typename P::V* ti,
                                                    const typename P::V* tj, int l, typename P::V& row,
                                                    typename P::V& col) {
  typename P::Acc ar;
  P::init(ar);
  col = P::zero();
  for (int c = 0; c < w; ++c) {
    const typename P::V e = TileElem<P>::ld(T, l * wp + c);
    P::fma(ar, e, tj[c]);
    typename P::Acc pc;
    P::init(pc);
    P::fma(pc, e, ti[l]);
    const typename P::V sc = warp_sum<P>(P::get(pc));
    if (l == c) col = sc;
  }
  row = P::get(ar);
}

// Batched symmetric GEMV over the packed panels of SymTiles (one CTA per matrix): each warp
// streams its share of the blocks (round robin) global -> shared through a ring of bulk
// copies completing on mbarriers; an off-diagonal block serves its block row and (by
// symmetry) its block column, so every stored entry is read from HBM once.
template <int PREC, int SYMV_SLOTS>
__global__ void __launch_bounds__(SYMV_WARPS * 32, 5) k_symv(SymTiles A, const int64_t* __restrict__ voff,
                                                          const double* __restrict__ in,
                                                          double* __restrict__ out, int* err) {
  // A.split CTAs per matrix (small batches): CTA q of matrix m takes the blocks of warps
  // q * SYMV_WARPS + w, and the last of the matrix's CTAs to finish adds their partial
  // vectors in CTA order
  using Ops = TileOps<PREC>;
  using P = typename Ops::P;
  using V = typename Ops::V;
  constexpr int EB = PREC == DD_PREC_FP32 ? 4 : 8;
  constexpr int TB = Ops::BYTES;  // the largest block (32 x 32)
  extern __shared__ __align__(128) unsigned char smem_symv[];
  unsigned char* smem_raw = smem_symv;
  const int split = A.split;
  const int m = blockIdx.x / split, q = blockIdx.x % split;
  const int n = A.n[m];
  const PackGeom g = pack_geom(n, EB);
  const int nb = g.nf + (g.w > 0);
  const int npad = nb * 32;
  const int maxpad = ((A.max_n + 31) / 32) * 32;
  unsigned char* slots = smem_raw;                                            // [W][SLOTS][TB]
  uint64_t* bars = reinterpret_cast<uint64_t*>(slots + SYMV_WARPS * SYMV_SLOTS * TB);
  V* tv = reinterpret_cast<V*>(bars + SYMV_WARPS * SYMV_SLOTS);              // [maxpad]
  V* part = tv + maxpad;                                                      // [W][maxpad]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t vo = voff[m];
  for (int i = threadIdx.x; i < npad; i += blockDim.x) tv[i] = (i < n) ? P::from_d(in[vo + i]) : P::from_d(0.0);
  for (int i = threadIdx.x; i < SYMV_WARPS * npad; i += blockDim.x) part[(i / npad) * maxpad + (i % npad)] = P::from_d(0.0);
  if (lane == 0)
    for (int k = 0; k < SYMV_SLOTS; ++k) mbar_init(&bars[warp * SYMV_SLOTS + k], 1);
  fence_mbar_init();
  __syncthreads();

  const int ntl = nb * (nb + 1) / 2;
  const int gw = q * SYMV_WARPS + warp, nw = split * SYMV_WARPS;  // this warp among the matrix's warps
  const int mine = (gw < ntl) ? (ntl - gw + nw - 1) / nw : 0;
  const unsigned char* gm = reinterpret_cast<const unsigned char*>(A.pdata) + (size_t)A.poff[m] * EB;
  unsigned char* wslots = slots + (size_t)warp * SYMV_SLOTS * TB;
  uint64_t* wbars = bars + warp * SYMV_SLOTS;
  auto issue = [&](int k, int slot) {
    int bi, bj;
    tile_coords(gw + k * nw, nb, bi, bj);
    const uint32_t bytes = (uint32_t)pack_tile_elems(g, bi, bj) * EB;
    mbar_arrive_expect_tx(&wbars[slot], bytes);
    bulk_g2s(wslots + (size_t)slot * TB, gm + (size_t)pack_tile_off(g, bi, bj) * EB, bytes, &wbars[slot]);
  };
  if (lane == 0)
    for (int k = 0; k < SYMV_SLOTS && k < mine; ++k) issue(k, k);
  V* mypart = part + warp * maxpad;
  bool ok = true;
  int k = 0;
  for (; k < mine; ++k) {
    const int slot = k % SYMV_SLOTS;
    if (!mbar_wait_bounded(&wbars[slot], (uint32_t)((k / SYMV_SLOTS) & 1), err)) {
      ok = false;
      break;
    }
    int bi, bj;
    tile_coords(gw + k * nw, nb, bi, bj);
    const unsigned char* T = wslots + (size_t)slot * TB;
    if (bi == bj) {
      const int h = bi < g.nf ? 32 : g.w;
      const V r = packed_diag_part<P>(T, tv + bi * 32, lane, h);
      if (lane < h) mypart[bi * 32 + lane] = P::add(mypart[bi * 32 + lane], r);
    } else if (bj < g.nf) {
      V r, c;
      Ops::both_parts(T, tv + bi * 32, tv + bj * 32, lane, r, c);
      mypart[bi * 32 + lane] = P::add(mypart[bi * 32 + lane], r);
      mypart[bj * 32 + lane] = P::add(mypart[bj * 32 + lane], c);
    } else {
      V r, c;
      packed_ragged_parts<P>(T, g.wp, g.w, tv + bi * 32, tv + bj * 32, lane, r, c);
      mypart[bi * 32 + lane] = P::add(mypart[bi * 32 + lane], r);
      if (lane < g.w) mypart[bj * 32 + lane] = P::add(mypart[bj * 32 + lane], c);
    }
    __syncwarp();
    if (lane == 0 && k + SYMV_SLOTS < mine) {
      fence_proxy_async();
      issue(k + SYMV_SLOTS, slot);
    }
  }
  if (!ok) {
    // drain the copies this warp still has in flight (bounded), then leave
    for (int kk = k; kk < mine && kk < k + SYMV_SLOTS; ++kk)
      mbar_wait_bounded(&wbars[kk % SYMV_SLOTS], (uint32_t)((kk / SYMV_SLOTS) & 1), nullptr);
  }
  __syncthreads();
  if (split == 1) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      V s = part[i];
      for (int w = 1; w < SYMV_WARPS; ++w) s = P::add(s, part[w * maxpad + i]);
      out[vo + i] = P::to_d(s);
    }
    return;
  }
  V* sp = reinterpret_cast<V*>(A.spart) + (size_t)blockIdx.x * maxpad;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    V s = part[i];
    for (int w = 1; w < SYMV_WARPS; ++w) s = P::add(s, part[w * maxpad + i]);
    sp[i] = s;
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&A.sticket[m], 1u) == (unsigned)split - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const V* sm0 = reinterpret_cast<const V*>(A.spart) + (size_t)m * split * maxpad;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    V s = sm0[i];
    for (int r = 1; r < split; ++r) s = P::add(s, sm0[(size_t)r * maxpad + i]);
    out[vo + i] = P::to_d(s);
  }
  if (threadIdx.x == 0) A.sticket[m] = 0u;
}

template <int PREC, int SLOTS>
static void symv_launch(const SymTiles& A, const int64_t* voff, const double* in, double* out, int* err,
                        cudaStream_t s) {
  const int maxpad = ((A.max_n + 31) / 32) * 32;
  const size_t vb = (A.prec == DD_PREC_FP32) ? 4 : 8;
  const size_t tb = tile_bytes(A.prec);
  const size_t smem = SYMV_WARPS * SLOTS * tb + SYMV_WARPS * SLOTS * 8 + (size_t)maxpad * vb * (1 + SYMV_WARPS);
  max_smem(k_symv<PREC, SLOTS>, smem);
  k_symv<PREC, SLOTS><<<A.count * std::max(1, A.split), SYMV_WARPS * 32, smem, s>>>(A, voff, in, out, err);
}

template <int PREC>
static void symv_slots(const SymTiles& A, const int64_t* voff, const double* in, double* out, int* err,
                       cudaStream_t s) {
  switch (A.slots) {
    case 3: symv_launch<PREC, 3>(A, voff, in, out, err, s); break;
    case 4: symv_launch<PREC, 4>(A, voff, in, out, err, s); break;
    default: symv_launch<PREC, 2>(A, voff, in, out, err, s);
  }
}

void launch_symv(const SymTiles& A, const int64_t* voff, const double* in, double* out, int* err, cudaStream_t s) {
  if (A.count == 0) return;
  switch (A.prec) {
    case DD_PREC_FP64: symv_slots<DD_PREC_FP64>(A, voff, in, out, err, s); break;
    case DD_PREC_FP32: symv_slots<DD_PREC_FP32>(A, voff, in, out, err, s); break;
    default: symv_slots<DD_PREC_DF64>(A, voff, in, out, err, s);
  }
  DD_CHECK_LAUNCH();
}

// Tiled form from the packed form: tile t of matrix m (32 x 32, zero-padded, diagonal tiles
// with both triangles). One CTA per tile.
template <typename E>
__global__ void k_packed_to_tiles(SymTiles A, const int* __restrict__ tmat, const int* __restrict__ tidx,
                                  E* __restrict__ tiles) {
  const int64_t t = blockIdx.x;
  const int m = tmat[t], ti = tidx[t];
  const int n = A.n[m];
  const PackGeom g = pack_geom(n, sizeof(E) == 4 ? 4 : 8);
  const int nb = g.nf + (g.w > 0);
  int bi, bj;
  tile_coords(ti, nb, bi, bj);
  const E* src = static_cast<const E*>(A.pdata) + A.poff[m] + pack_tile_off(g, bi, bj);
  const int h = bi < g.nf ? 32 : g.w;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int r = e / 32, c = e % 32;
    E v{};
    if (bi == bj) {
      if (r < h && c < h) v = src[r <= c ? tri_index(h, r, c) : tri_index(h, c, r)];
    } else if (bj < g.nf) {
      v = src[r * 32 + c];
    } else if (c < g.w) {
      v = src[r * g.wp + c];
    }
    tiles[t * 1024 + e] = v;
  }
}

void ensure_tiles(DeviceArena& arena, SymTiles& A, cudaStream_t s) {
  if (A.data || A.count == 0) return;
  std::vector<int> n(A.count);
  DD_CUDA(cudaMemcpyAsync(n.data(), A.n, n.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> toff(A.count);
  std::vector<int> tmat, tidx;
  int64_t nt = 0;
  for (int m = 0; m < A.count; ++m) {
    const int nb = (n[m] + 31) / 32;
    toff[m] = nt;
    for (int t = 0; t < nb * (nb + 1) / 2; ++t) {
      tmat.push_back(m);
      tidx.push_back(t);
    }
    nt += (int64_t)nb * (nb + 1) / 2;
  }
  A.ntiles = nt;
  A.toff = arena.upload(toff, s);
  const int* dm = arena.upload(tmat, s);
  const int* di = arena.upload(tidx, s);
  if (nt == 0) return;
  if (A.prec == DD_PREC_FP32) {
    float* d = arena.alloc<float>((size_t)nt * 1024);
    k_packed_to_tiles<float><<<(unsigned)nt, 256, 0, s>>>(A, dm, di, d);
    A.data = d;
  } else if (A.prec == DD_PREC_FP64) {
    double* d = arena.alloc<double>((size_t)nt * 1024);
    k_packed_to_tiles<double><<<(unsigned)nt, 256, 0, s>>>(A, dm, di, d);
    A.data = d;
  } else {
    float2* d = arena.alloc<float2>((size_t)nt * 1024);
    k_packed_to_tiles<float2><<<(unsigned)nt, 256, 0, s>>>(A, dm, di, d);
    A.data = d;
  }
  DD_CHECK_LAUNCH();
}

// Self-test of the bounded-wait path: one thread waits on an mbarrier that nothing arrives
// at (no copy is in flight), gives up after `limit` attempts and raises the error word,
// exactly as the streaming kernels do when a bulk copy never lands.
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbar_init();
  mbar_wait_bounded(&bar, 0u, err, limit);
}

void launch_wait_selftest(int* err, long long limit, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(err, limit);
  DD_CHECK_LAUNCH();
}


// ---------------------------------------------------------------------------
// Fast diagonalization: s = V D^{-1} V^T t with V = Vz (x) Vy (x) Vx, one CTA per subdomain,
// six contractions along one axis each in shared memory (about 14k multiply-adds per
// 8^3 subdomain instead of a 343^2 matrix).
// ---------------------------------------------------------------------------
// out[..j..] = sum_i A(i, j) in[..i..] (transposed) or sum_i A(j, i) in[..i..] along axis `ax`
template <class P>
__device__ __forceinline__ void fdm_contract(const typename P::V* A, int ax, bool trans, const int* n,
                                             const typename P::V* in, typename P::V* out) {
  const int N = n[0] * n[1] * n[2];
  const int na = n[ax];
  const int stride = ax == 0 ? 1 : (ax == 1 ? n[0] : n[0] * n[1]);
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int j = (idx / stride) % na;
    const int base = idx - j * stride;
    typename P::Acc acc[2];
    P::init(acc[0]);
    P::init(acc[1]);
    for (int i = 0; i < na; ++i) {
      typename P::V a = trans ? A[i * 9 + j] : A[j * 9 + i];
      P::fma(acc[i & 1], a, in[base + i * stride]);
    }
    out[idx] = P::add(P::get(acc[0]), P::get(acc[1]));
  }
}

template <class P>
__global__ void __launch_bounds__(128) k_fdm_apply(DevMesh m, const double* __restrict__ tI, double* __restrict__ sI) {
  using V = typename P::V;
  __shared__ V Vs[3][81];
  __shared__ V b0[729], b1[729];
  __shared__ int n[3];
  const int s = blockIdx.x;
  if (threadIdx.x < 3) n[threadIdx.x] = m.fdm_n[3 * s + threadIdx.x];
  for (int t = threadIdx.x; t < 243; t += blockDim.x) Vs[t / 81][t % 81] = ld_fdm<P>(m.fdm_V, (int64_t)s * 243 + t);
  __syncthreads();
  const int N = n[0] * n[1] * n[2];
  const int64_t off = m.ioff[s];
  for (int i = threadIdx.x; i < N; i += blockDim.x) b0[i] = P::from_d(tI[off + i]);
  __syncthreads();
  fdm_contract<P>(Vs[0], 0, true, n, b0, b1);
  __syncthreads();
  fdm_contract<P>(Vs[1], 1, true, n, b1, b0);
  __syncthreads();
  fdm_contract<P>(Vs[2], 2, true, n, b0, b1);
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    typename P::Acc acc;
    P::init(acc);
    P::fma(acc, b1[i], ld_fdm<P>(m.fdm_Dinv, off + i));
    b1[i] = P::get(acc);
  }
  __syncthreads();
  fdm_contract<P>(Vs[0], 0, false, n, b1, b0);
  __syncthreads();
  fdm_contract<P>(Vs[1], 1, false, n, b0, b1);
  __syncthreads();
  fdm_contract<P>(Vs[2], 2, false, n, b1, b0);
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) sI[off + i] = P::to_d(b0[i]);
}

// ---------------------------------------------------------------------------
// Fused Schur-complement application y_i = (K_GG - K_GI K_II^{-1} K_IG) x_i of one
// subdomain per CTA (eq. 6) for the fast-diagonalization local solver: the interior pass
// (t_I = K_IG x_G), the six contractions of K_II^{-1} and the interface pass
// (y_G = K_GG x_G - K_GI s_I) run back to back on shared memory, so the interior
// vectors never leave the SM and the element entries of the boundary-layer elements
// are formed once. The arithmetic and its order are those of k_elem_interior,
// k_fdm_apply and k_elem_interface.
// ---------------------------------------------------------------------------
// The same contractions with an epilogue: EPI 0 stores out[idx], EPI 1 stores
// out[idx] * dv[idx] (the diagonal D^{-1} of the fast diagonalization), EPI 2 stores
// -out[idx] at the local node il[idx] of the subdomain vector xl (the interior values -s_I).
// N7: the 7 x 7 x 7 interior index box (sizes known at compile time); else sizes n[].
template <class P, bool N7, int EPI>
__device__ __forceinline__ void fdm_contract_epi(const typename P::V* A, int ax, bool trans, const int* n,
                                                 const typename P::V* in, typename P::V* out,
                                                 const typename P::V* dv, const int16_t* il) {
  const int n0 = N7 ? 7 : n[0], n1 = N7 ? 7 : n[1], n2 = N7 ? 7 : n[2];
  const int N = n0 * n1 * n2;
  const int na = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
  const int stride = ax == 0 ? 1 : (ax == 1 ? n0 : n0 * n1);
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int j = (idx / stride) % na;
    const int base = idx - j * stride;
    typename P::Acc acc[2];
    P::init(acc[0]);
    P::init(acc[1]);
    if (N7) {
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        typename P::V a = trans ? A[i * 9 + j] : A[j * 9 + i];
        P::fma(acc[i & 1], a, in[base + i * stride]);
      }
    } else {
      // pairs of terms, so that the accumulators stay in registers
      int i = 0;
      for (; i + 1 < na; i += 2) {
        P::fma(acc[0], trans ? A[i * 9 + j] : A[j * 9 + i], in[base + i * stride]);
        P::fma(acc[1], trans ? A[(i + 1) * 9 + j] : A[j * 9 + i + 1], in[base + (i + 1) * stride]);
      }
      if (i < na) P::fma(acc[0], trans ? A[i * 9 + j] : A[j * 9 + i], in[base + i * stride]);
    }
    const typename P::V v = P::add(P::get(acc[0]), P::get(acc[1]));
    if (EPI == 0) {
      out[idx] = v;
    } else if (EPI == 1) {
      typename P::Acc d;
      P::init(d);
      P::fma(d, v, dv[idx]);
      out[idx] = P::get(d);
    } else {
      out[il[idx]] = P::neg(v);
    }
  }
}

template <class P, bool N7>
__device__ __forceinline__ void fdm_solve_fused(const typename P::V* Vs, const int* n, typename P::V* f0,
                                                typename P::V* f1, const typename P::V* dv, const int16_t* il,
                                                typename P::V* xl) {
  fdm_contract_epi<P, N7, 0>(Vs, 0, true, n, f0, f1, dv, il);
  __syncthreads();
  fdm_contract_epi<P, N7, 0>(Vs + 81, 1, true, n, f1, f0, dv, il);
  __syncthreads();
  fdm_contract_epi<P, N7, 1>(Vs + 162, 2, true, n, f0, f1, dv, il);
  __syncthreads();
  fdm_contract_epi<P, N7, 0>(Vs, 0, false, n, f1, f0, dv, il);
  __syncthreads();
  fdm_contract_epi<P, N7, 0>(Vs + 81, 1, false, n, f0, f1, dv, il);
  __syncthreads();
  fdm_contract_epi<P, N7, 2>(Vs + 162, 2, false, n, f1, xl, dv, il);
}

// element-pass item with slots (position in the type's boundary-layer list) * 8 + corner;
// kd holds the 8 entry classes of the listed elements with stride nbl
template <class P, int S>
__device__ __forceinline__ typename P::V apply_citem(const DevMesh& m, const int16_t* it, const typename P::V* xl,
                                                     const typename P::V* kd, const int16_t* bll, int nbl) {
  const int sx = S ? S : m.sx, sy = S ? S : m.sy;
  const int NLx = sx + 1, NLy = sy + 1;
  typename P::Acc acc[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) P::init(acc[t]);
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int v = it[1 + k];
    if (v < 0) break;
    const int b = v >> 3, p = v & 7;
    const int el = bll[b];
    const int ea = el % sx, eb = (el / sx) % sy, ec = el / (sx * sy);
    const int base = ea + NLx * (eb + NLy * ec);
    const typename P::V* kp = kd + b;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int lq = base + (q & 1) + NLx * (((q >> 1) & 1) + NLy * (q >> 2));
      P::fma(acc[q & 3], kp[(p ^ q) * nbl], xl[lq]);
    }
  }
  return P::add(P::add(P::get(acc[0]), P::get(acc[1])), P::add(P::get(acc[2]), P::get(acc[3])));
}

template <class P, int S, int BS>
__global__ void __launch_bounds__(BS) k_schur_fused(DevMesh m, const double* __restrict__ xg,
                                                    double* __restrict__ yloc) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* xl = reinterpret_cast<V*>(smem_raw);  // [NL] local nodal vector
  V* f0 = xl + m.NL;                        // [max_nint] interior vector buffers of the fast diagonalization
  V* f1 = f0 + m.max_nint;
  V* dv = f1 + m.max_nint;                  // [max_nint] D^{-1} of the fast diagonalization
  V* Vs = dv + m.max_nint;                  // [3][81] 1D eigenbases (stride 9)
  V* kd = Vs + 243;                         // [8][nbl] entry classes of the boundary-layer elements
  int16_t* bll = reinterpret_cast<int16_t*>(kd + 8 * m.max_nbl);  // [nbl] boundary-layer elements
  int16_t* il = bll + m.max_nbl;                                   // [max_nint] local node of interior index
  __shared__ int n[3];
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  const int* to = m.type_off + 6 * m.sub_type[s];
  const int nbl = to[5] - to[4];
  const int64_t io = m.ioff[s], go = m.goff[s];
  if (threadIdx.x < 3) n[threadIdx.x] = m.fdm_n[3 * s + threadIdx.x];
  for (int t = threadIdx.x; t < 243; t += blockDim.x) Vs[t] = ld_fdm<P>(m.fdm_V, (int64_t)s * 243 + t);
  // the subdomain's own copies (setup): interface index per local node, the interior entries
  // of D^{-1} (contiguous from ioff[s]) and the boundary-layer element factors in list order,
  // so that every load here is one coalesced level (x_G then one gather through the indices)
  const int* gix = m.sxg + (size_t)s * m.NL;
  constexpr int NLC = (S + 1) * (S + 1) * (S + 1), NLT = (NLC + BS - 1) / BS;
  {
    // all of a thread's codes and indices first, then its x_G values, then the stores
    int cd[NLT], gi[NLT];
#pragma unroll
    for (int u = 0; u < NLT; ++u) {
      const int l = threadIdx.x + u * BS;
      cd[u] = l < NLC ? code[l] : INT16_MIN;
      gi[u] = l < NLC ? gix[l] : -1;
    }
    V xv[NLT];
#pragma unroll
    for (int u = 0; u < NLT; ++u) xv[u] = gi[u] >= 0 ? P::from_d(xg[gi[u]]) : P::zero();
#pragma unroll
    for (int u = 0; u < NLT; ++u) {
      const int l = threadIdx.x + u * BS;
      if (l < NLC) {
        xl[l] = xv[u];
        if (cd[u] >= 0) {
          f0[cd[u]] = P::zero();
          il[cd[u]] = (int16_t)l;
        }
      }
    }
  }
  const int nint = (int)(m.ioff[s + 1] - io);
#pragma unroll
  for (int u = 0; u < NLT; ++u) {
    const int t = threadIdx.x + u * BS;
    if (t < nint) dv[t] = ld_fdm<P>(m.fdm_Dinv, io + t);
  }
  {
    constexpr int NBT = (S * S * S + BS - 1) / BS;  // boundary-layer elements per thread at most
    const V* fac = static_cast<const V*>(m.sfac) + (size_t)s * m.max_nbl * 3;
    V c[NBT][3];
#pragma unroll
    for (int u = 0; u < NBT; ++u) {
      const int t = threadIdx.x + u * BS;
      if (t < nbl) {
        c[u][0] = fac[3 * t];
        c[u][1] = fac[3 * t + 1];
        c[u][2] = fac[3 * t + 2];
      }
    }
#pragma unroll
    for (int u = 0; u < NBT; ++u) {
      const int t = threadIdx.x + u * BS;
      if (t < nbl) {
        bll[t] = m.type_bl[to[4] + t];
#pragma unroll
        for (int d = 0; d < 8; ++d) kd[d * nbl + t] = P::entry(c[u], d);
      }
    }
  }
  __syncthreads();
  // t_I = (K [0; x_G])_I on the interior nodes next to the boundary layer (zero elsewhere)
  for (int i = to[0] + threadIdx.x; i < to[1]; i += blockDim.x) {
    const int16_t* it = m.type_citems + 9 * (size_t)i;
    f0[code[it[0]]] = apply_citem<P, S>(m, it, xl, kd, bll, nbl);
  }
  __syncthreads();
  // s_I = K_II^{-1} t_I = V D^{-1} V^T t_I (V = Vz (x) Vy (x) Vx); the last contraction writes
  // -s_I into the interior entries of the local vector
  if (n[0] == 7 && n[1] == 7 && n[2] == 7)
    fdm_solve_fused<P, true>(Vs, n, f0, f1, dv, il, xl);
  else
    fdm_solve_fused<P, false>(Vs, n, f0, f1, dv, il, xl);
  __syncthreads();
  // y_G = (K [-s_I; x_G])_G
  for (int i = to[2] + threadIdx.x; i < to[3]; i += blockDim.x) {
    const int16_t* it = m.type_citems + 9 * (size_t)i;
    yloc[go + (-1 - code[it[0]])] = P::to_d(apply_citem<P, S>(m, it, xl, kd, bll, nbl));
  }
}

bool schur_fused_available(const DevMesh& m) {
  return m.local_solver == DD_LOCAL_FDM && m.sx == 8 && m.sy == 8 && m.sz == 8 && m.type_citems != nullptr &&
         m.sxg != nullptr && m.sfac != nullptr && m.max_nint > 0 && m.max_nint <= m.NL;
}

template <class P, int BS>
static void schur_fused_bs(const DevMesh& m, const double* xg, double* yloc, size_t smem, cudaStream_t s) {
  max_smem(k_schur_fused<P, 8, BS>, smem);
  k_schur_fused<P, 8, BS><<<m.S, BS, smem, s>>>(m, xg, yloc);
}

void launch_schur_fused(const DevMesh& m, const double* xg, double* yloc, cudaStream_t s) {
  const size_t vb = m.schur_prec == DD_PREC_DF64 ? sizeof(df64) : sizeof(double);
  // interior buffers sized by the largest interior of a subdomain (up to 8^3 on the Neumann
  // boundary, whose face nodes are interior unknowns), so that more CTAs fit on an SM
  const size_t ni = (size_t)m.max_nint;
  const size_t smem = vb * ((size_t)m.NL + 3 * ni + 243 + 8 * (size_t)m.max_nbl) + 2 * ((size_t)m.max_nbl + ni);
  if (m.schur_prec == DD_PREC_DF64) {
    switch (m.schur_threads) {
      case 352: schur_fused_bs<PolDF, 352>(m, xg, yloc, smem, s); break;
      case 416: schur_fused_bs<PolDF, 416>(m, xg, yloc, smem, s); break;
      default: schur_fused_bs<PolDF, 256>(m, xg, yloc, smem, s);
    }
  } else {
    switch (m.schur_threads) {
      case 352: schur_fused_bs<PolF64, 352>(m, xg, yloc, smem, s); break;
      case 416: schur_fused_bs<PolF64, 416>(m, xg, yloc, smem, s); break;
      default: schur_fused_bs<PolF64, 256>(m, xg, yloc, smem, s);
    }
  }
  DD_CHECK_LAUNCH();
}

void launch_kii_apply(const DevMesh& m, const double* tI, double* sI, int* err, cudaStream_t s) {
  if (m.local_solver == DD_LOCAL_FDM) {
    if (m.schur_prec == DD_PREC_DF64)
      k_fdm_apply<PolDF><<<m.S, 128, 0, s>>>(m, tI, sI);
    else
      k_fdm_apply<PolF64><<<m.S, 128, 0, s>>>(m, tI, sI);
    DD_CHECK_LAUNCH();
  } else {
    launch_symv(m.KIIinv, m.ioff, tI, sI, err, s);
  }
}

// ---------------------------------------------------------------------------
// gathers, scatters, BDDC pieces
// ---------------------------------------------------------------------------
__global__ void k_gather(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                         const double* __restrict__ loc, const double* __restrict__ base,
                         const int64_t* __restrict__ bmap, double* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (base) s = base[bmap ? bmap[g] : g];
    for (int k = ptr[g]; k < ptr[g + 1]; ++k) s += loc[idx[k]];
    y[g] = s;
  }
}

static int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

void launch_gather(int64_t n, const int* ptr, const int* idx, const double* loc, const double* base,
                   const int64_t* bmap, double* y, cudaStream_t s) {
  if (n == 0) return;
  k_gather<<<grid_for(n, 256), 256, 0, s>>>(n, ptr, idx, loc, base, bmap, y);
  DD_CHECK_LAUNCH();
}

// dL/dk_e = -lambda_e^T K_e^0 x_e with K_e^0 = K_e / k_e; Dirichlet nodes carry 0
__global__ void k_coef_grad(DevMesh m, const double* __restrict__ x, const double* __restrict__ lam,
                            double* __restrict__ grad, int log_coef) {
  const int64_t E = (int64_t)m.nx * m.ny * m.nz;
  const int64_t Nfx = m.fx1 - m.fx0, Nfy = m.fy1 - m.fy0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int ex = (int)(e % m.nx), ey = (int)((e / m.nx) % m.ny), ez = (int)(e / ((int64_t)m.nx * m.ny));
    double xv[8], lv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int gx = ex + (a & 1), gy = ey + ((a >> 1) & 1), gz = ez + (a >> 2);
      bool fr = gx >= m.fx0 && gx < m.fx1 && gy >= m.fy0 && gy < m.fy1 && gz >= m.fz0 && gz < m.fz1;
      int64_t f = (gx - m.fx0) + Nfx * ((gy - m.fy0) + Nfy * (int64_t)(gz - m.fz0));
      xv[a] = fr ? x[f] : 0.0;
      lv[a] = fr ? lam[f] : 0.0;
    }
    double c[3];
    const double k = m.coef[e];
    c[0] = m.ec[3 * e] / k; c[1] = m.ec[3 * e + 1] / k; c[2] = m.ec[3 * e + 2] / k;
    double kd[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) kd[d] = PolF64::entry(c, d);
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      double row = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) row = fma(kd[p ^ q], xv[q], row);
      s = fma(lv[p], row, s);
    }
    grad[e] = log_coef ? -s * k : -s;  // d/dg_e = k_e d/dk_e for k_e = exp(g_e)
  }
}

void launch_coef_grad(const DevMesh& m, const double* x, const double* lam, double* grad, int log_coef,
                      cudaStream_t s) {
  int64_t E = (int64_t)m.nx * m.ny * m.nz;
  k_coef_grad<<<grid_for(E, 256), 256, 0, s>>>(m, x, lam, grad, log_coef);
  DD_CHECK_LAUNCH();
}

// part[block] = max over this block's elements of |k_e - c_e| / |k_e| (c_e = exp(coef_e) if log)
__global__ void k_coef_mismatch(int64_t E, const double* __restrict__ k, const double* __restrict__ coef, int log,
                                double* __restrict__ part) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double c = log ? exp(coef[e]) : coef[e];
    const double d = fabs(k[e] - c) / fabs(k[e]);
    mx = (d > mx || d != d) ? d : mx;  // a NaN propagates
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = red[threadIdx.x], b = red[threadIdx.x + o];
      red[threadIdx.x] = (b > a || b != b) ? b : a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

void launch_coef_mismatch(const DevMesh& m, const double* coef, int log, double* part, int nblk, cudaStream_t s) {
  const int64_t E = (int64_t)m.nx * m.ny * m.nz;
  k_coef_mismatch<<<nblk, 256, 0, s>>>(E, m.coef, coef, log, part);
  DD_CHECK_LAUNCH();
}

__global__ void k_scatter_recover(DevMesh m, const double* __restrict__ xg, const double* __restrict__ sI,
                                  double* __restrict__ x) {
  const int s = blockIdx.x;
  const int16_t* code = m.lidx + (size_t)s * m.NL;
  for (int l = threadIdx.x; l < m.NL; l += blockDim.x) {
    int cd = code[l];
    if (cd >= 0) x[free_index(m, s, l)] = sI[m.ioff[s] + cd];
  }
  // interface values: each global interface dof written by its first copy's subdomain
  for (int j = threadIdx.x; j < (int)(m.goff[s + 1] - m.goff[s]); j += blockDim.x) {
    int64_t k = m.goff[s] + j;
    int g = m.gmap[k];
    if (m.gidx[m.gptr[g]] == (int)k) x[m.gamma_free[g]] = xg[g];
  }
}

void launch_scatter_recover(const DevMesh& m, const double* xg, const double* sI, double* x, cudaStream_t s) {
  k_scatter_recover<<<m.S, 256, 0, s>>>(m, xg, sI, x);
  DD_CHECK_LAUNCH();
}

__global__ void k_restrict(int64_t nflat, const int* __restrict__ gmap, const double* __restrict__ D,
                           const double* __restrict__ r, double* __restrict__ rloc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nflat; k += (int64_t)gridDim.x * blockDim.x)
    rloc[k] = D[k] * r[gmap[k]];
}

void launch_restrict(int64_t nflat, const int* gmap, const double* D, const double* r, double* rloc,
                     cudaStream_t s) {
  if (nflat == 0) return;
  k_restrict<<<grid_for(nflat, 256), 256, 0, s>>>(nflat, gmap, D, r, rloc);
  DD_CHECK_LAUNCH();
}

// x_j of item m is in[in_map ? in_map[in_off[m] + j] : in_off[m] + j]; the outputs of item m
// start at out_off[m].
// Batched GEMVs over row-major matrices A_m (R_m x C_m). The input slice of item m is
// staged once per block in shared memory, converted to the matrix type T, so FP32
// operators also do FP32 arithmetic (the BDDC preconditioner in FP32 mode).
//   k_bgemv:   y_m = alpha A_m x_m (+ add), warp per row, lanes along the row (coalesced)
//   k_bgemv_t: y_m = alpha A_m^T x_m (+ add), thread per column; the rows are split into
//              blockDim.y slices (slice s takes rows s, s + RS, ...) for tall matrices, and the
//              slice sums are added in slice order
constexpr int BGEMV_T_COLS = 128; // columns per block of k_bgemv_t
constexpr int BG_CHUNK = 8;       // loads a thread issues before using any of them

// k_bgemv: each warp takes B.rows_per_block / 8 rows of one matrix; per row the lanes load
// BG_CHUNK entries (32 apart, coalesced) before the multiply-adds, so every lane keeps
// BG_CHUNK loads in flight
template <class T>
__global__ void __launch_bounds__(256) k_bgemv(const int64_t* __restrict__ row0, const int* __restrict__ cols,
                                               const int64_t* __restrict__ moff, const T* __restrict__ M,
                                               const int64_t* __restrict__ in_off, const int* __restrict__ in_map,
                                               const double* __restrict__ in, const int64_t* __restrict__ out_off,
                                               double* __restrict__ out, double alpha,
                                               const double* __restrict__ add, int rows_per_block) {
  extern __shared__ __align__(16) unsigned char bg_smem[];
  T* xs = reinterpret_cast<T*>(bg_smem);
  const int m = blockIdx.x;
  const int R = (int)(row0[m + 1] - row0[m]), C = cols[m];
  const int r0 = blockIdx.y * rows_per_block;
  if (r0 >= R) return;
  const int64_t io = in_off[m];
  for (int j = threadIdx.x; j < C; j += blockDim.x) xs[j] = (T)in[in_map ? in_map[io + j] : io + j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r1 = min(R, r0 + rows_per_block);
  const int64_t oo = out_off[m];
  for (int i = r0 + warp; i < r1; i += blockDim.x >> 5) {
    const T* a = M + moff[m] + (int64_t)i * C;
    T acc[4] = {0, 0, 0, 0};
    for (int j0 = 0; j0 < C; j0 += 32 * BG_CHUNK) {
      T v[BG_CHUNK];
#pragma unroll
      for (int u = 0; u < BG_CHUNK; ++u) {
        const int j = j0 + u * 32 + lane;
        v[u] = j < C ? a[j] : T(0);
      }
#pragma unroll
      for (int u = 0; u < BG_CHUNK; ++u) {
        const int j = j0 + u * 32 + lane;
        if (j < C) acc[u & 3] = fma(v[u], xs[j], acc[u & 3]);
      }
    }
    T sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) out[oo + i] = alpha * (double)sum + (add ? add[oo + i] : 0.0);
  }
}

template <class T>
static void bgemv_go(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                     const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s) {
  size_t smem = (size_t)std::max(B.max_cols, 1) * sizeof(T);
  if (smem > 48 * 1024) max_smem(k_bgemv<T>, smem);
  const int rpb = std::max(8, B.rows_per_block);
  dim3 grid(B.count, (B.max_rows + rpb - 1) / rpb);
  k_bgemv<T><<<grid, 256, smem, s>>>(B.row0, B.cols, B.moff, static_cast<const T*>(B.data), in_off, in_map, in,
                                      out_off, out, alpha, add, rpb);
}

void launch_bgemv(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                  const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s) {
  if (B.nrows == 0) return;
  if (B.prec == DD_PREC_FP32)
    bgemv_go<float>(B, in_off, in_map, in, out_off, out, alpha, add, s);
  else
    bgemv_go<double>(B, in_off, in_map, in, out_off, out, alpha, add, s);
  DD_CHECK_LAUNCH();
}

// k_bgemv_t: y_m = alpha A_m^T x_m (+ add). Block (m, column block y, row part z): thread
// column j, the block's rows split into blockDim.y slices; each thread loads BG_CHUNK rows of
// its column before the multiply-adds. With gridDim.z > 1 (tall matrices) every row part
// stores its column sums in zpart, and the last of the gridDim.z blocks of (m, y) to finish
// (a per-(m, y) ticket, reset by that block) adds them in row-part order.
template <class T>
__global__ void __launch_bounds__(1024) k_bgemv_t(const int64_t* __restrict__ row0, const int* __restrict__ cols,
                                                  const int64_t* __restrict__ moff, const T* __restrict__ M,
                                                  const int64_t* __restrict__ in_off, const int* __restrict__ in_map,
                                                  const double* __restrict__ in, const int64_t* __restrict__ out_off,
                                                  double* __restrict__ out, double alpha,
                                                  const double* __restrict__ add, int xs_len, T* __restrict__ zpart,
                                                  unsigned* __restrict__ zticket) {
  extern __shared__ __align__(16) unsigned char bg_smem[];
  T* xs = reinterpret_cast<T*>(bg_smem);  // [xs_len]
  T* part = xs + xs_len;                   // [RS][BGEMV_T_COLS]
  __shared__ bool last;
  const int m = blockIdx.x;
  const int R = (int)(row0[m + 1] - row0[m]), C = cols[m];
  if (blockIdx.y * BGEMV_T_COLS >= C) return;  // uniform over the block
  const int RS = blockDim.y, tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BGEMV_T_COLS + tx;
  const int j = blockIdx.y * BGEMV_T_COLS + tx;
  const int ZS = gridDim.z;
  const int rz = (R + ZS - 1) / ZS;
  const int ra = blockIdx.z * rz, rb = min(R, ra + rz);
  const int64_t io = in_off[m];
  for (int i = ra + tid; i < rb; i += BGEMV_T_COLS * RS) xs[i - ra] = (T)in[in_map ? in_map[io + i] : io + i];
  __syncthreads();
  T acc[4] = {0, 0, 0, 0};
  if (j < C) {
    const T* A = M + moff[m] + j;
    for (int i0 = ra + ty; i0 < rb; i0 += RS * BG_CHUNK) {
      T v[BG_CHUNK];
#pragma unroll
      for (int u = 0; u < BG_CHUNK; ++u) {
        const int i = i0 + u * RS;
        v[u] = i < rb ? A[(int64_t)i * C] : T(0);
      }
#pragma unroll
      for (int u = 0; u < BG_CHUNK; ++u) {
        const int i = i0 + u * RS;
        if (i < rb) acc[u & 3] = fma(v[u], xs[i - ra], acc[u & 3]);
      }
    }
  }
  part[ty * BGEMV_T_COLS + tx] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  __syncthreads();
  T v = 0;
  if (ty == 0) {
    v = part[tx];
    for (int q = 1; q < RS; ++q) v += part[q * BGEMV_T_COLS + tx];
  }
  const int64_t oo = out_off[m];
  if (ZS == 1) {
    if (ty == 0 && j < C) out[oo + j] = alpha * (double)v + (add ? add[oo + j] : 0.0);
    return;
  }
  const int64_t slot = (int64_t)m * gridDim.y + blockIdx.y;
  if (ty == 0) zpart[(slot * ZS + blockIdx.z) * BGEMV_T_COLS + tx] = v;
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&zticket[slot], 1u) == (unsigned)ZS - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (ty == 0 && j < C) {
    T sum = 0;
    for (int z = 0; z < ZS; ++z) sum += __ldcg(&zpart[(slot * ZS + z) * BGEMV_T_COLS + tx]);
    out[oo + j] = alpha * (double)sum + (add ? add[oo + j] : 0.0);
  }
  if (tid == 0) zticket[slot] = 0u;
}

template <class T>
static void bgemv_t_go(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                       const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s) {
  const int zs = B.zsplit > 1 && B.zpart ? B.zsplit : 1;
  const int rmax = (B.max_rows + zs - 1) / zs;
  // row slices: one per 32 rows of the tallest row part, at most 8 (1024 threads)
  const int rs = std::min(8, std::max(1, rmax / 32));
  const int xs_len = (std::max(rmax, 1) + 3) / 4 * 4;
  size_t smem = ((size_t)xs_len + (size_t)rs * BGEMV_T_COLS) * sizeof(T);
  if (smem > 48 * 1024) max_smem(k_bgemv_t<T>, smem);
  dim3 grid(B.count, (B.max_cols + BGEMV_T_COLS - 1) / BGEMV_T_COLS, zs);
  k_bgemv_t<T><<<grid, dim3(BGEMV_T_COLS, rs), smem, s>>>(B.row0, B.cols, B.moff, static_cast<const T*>(B.data),
                                                           in_off, in_map, in, out_off, out, alpha, add, xs_len,
                                                           static_cast<T*>(B.zpart), B.zticket);
}

void launch_bgemv_t(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                    const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s) {
  if (B.count == 0) return;
  if (B.prec == DD_PREC_FP32)
    bgemv_t_go<float>(B, in_off, in_map, in, out_off, out, alpha, add, s);
  else
    bgemv_t_go<double>(B, in_off, in_map, in, out_off, out, alpha, add, s);
  DD_CHECK_LAUNCH();
}

// z[g] = sum over copies k of D[k] (uloc[k] + vloc[k])   (eq. 7)
__global__ void k_wgather(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                          const double* __restrict__ D, const double* __restrict__ uloc,
                          const double* __restrict__ vloc, double* __restrict__ z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int t = ptr[g]; t < ptr[g + 1]; ++t) {
      int k = idx[t];
      acc = fma(D[k], uloc[k] + vloc[k], acc);
    }
    z[g] = acc;
  }
}

void launch_wgather(int64_t n, const int* ptr, const int* idx, const double* D, const double* uloc,
                    const double* vloc, double* z, cudaStream_t s) {
  if (n == 0) return;
  k_wgather<<<grid_for(n, 256), 256, 0, s>>>(n, ptr, idx, D, uloc, vloc, z);
  DD_CHECK_LAUNCH();
}

// y = A x for a dense row-major n x n matrix (warp per row)
template <class T>
__global__ void k_dense_gemv(int n, const T* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
    const T* a = A + (int64_t)row * n;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc += (double)a[j] * x[j];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
  }
}

void launch_dense_gemv(int n, int prec, const void* A, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  int blocks = (n * 32 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (prec == DD_PREC_FP32)
    k_dense_gemv<float><<<blocks, 256, 0, s>>>(n, (const float*)A, x, y);
  else
    k_dense_gemv<double><<<blocks, 256, 0, s>>>(n, (const double*)A, x, y);
  DD_CHECK_LAUNCH();
}

__global__ void k_map_gather(int64_t n, const int* __restrict__ map, const double* __restrict__ in,
                             double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[map[i]];
}
__global__ void k_map_scatter(int64_t n, const int* __restrict__ map, const double* __restrict__ in,
                              double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[map[i]] = in[i];
}
void launch_map_gather(int64_t n, const int* map, const double* in, double* out, cudaStream_t s) {
  if (n == 0) return;
  k_map_gather<<<grid_for(n, 256), 256, 0, s>>>(n, map, in, out);
  DD_CHECK_LAUNCH();
}
void launch_map_scatter(int64_t n, const int* map, const double* in, double* out, cudaStream_t s) {
  if (n == 0) return;
  k_map_scatter<<<grid_for(n, 256), 256, 0, s>>>(n, map, in, out);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

// Device arithmetic shared by the single-vector and the batched kernels: the FP64,
// df64 and FP32 policies, the Q1 element entries, subdomain index maps and the
// element work-list helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.h"

namespace dd {

// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------
struct PolF64 {
  using V = double;
  using Acc = double;
  __device__ static V from_d(double d) { return d; }
  __device__ static double to_d(V v) { return v; }
  // ensemble vectors are stored as df64
  __device__ static V from_v(df64 x) { return df64_to_double_bits(x); }
  __device__ static df64 to_v(V v) { return df64_from_double_bits(v); }
  __device__ static V zero() { return 0.0; }
  __device__ static V neg(V v) { return -v; }
  __device__ static void init(Acc& a) { a = 0.0; }
  __device__ static void fma(Acc& a, V k, V x) { a = ::fma(k, x, a); }
  __device__ static V get(const Acc& a) { return a; }
  __device__ static V add(V a, V b) { return a + b; }
  // element entry for corner pair differing on axes d (bit0 x, bit1 y, bit2 z)
  __device__ static V entry(const V* c, int d) {
    double sx = (d & 1) ? -1.0 : 1.0, mx = (d & 1) ? 1.0 : 2.0;
    double sy = (d & 2) ? -1.0 : 1.0, my = (d & 2) ? 1.0 : 2.0;
    double sz = (d & 4) ? -1.0 : 1.0, mz = (d & 4) ? 1.0 : 2.0;
    return c[0] * (sx * my * mz) + c[1] * (mx * sy * mz) + c[2] * (mx * my * sz);
  }
};

struct PolDF {
  using V = df64;
  using Acc = df64_acc;
  __device__ static V from_d(double d) { return df64_from_double(d); }
  __device__ static double to_d(V v) { return df64_to_double(v); }
  __device__ static V from_v(df64 x) { return x; }
  __device__ static df64 to_v(V v) { return v; }
  __device__ static V zero() { return {0.f, 0.f}; }
  __device__ static V neg(V v) { return df64_neg(v); }
  __device__ static void init(Acc& a) { a = df64_acc(); }
  __device__ static void fma(Acc& a, V k, V x) { a.fma(k, x); }
  __device__ static V get(const Acc& a) { return a.get(); }
  __device__ static V add(V a, V b) { return df64_add(a, b); }
  __device__ static V entry(const V* c, int d) {
    // the scalings are +-1, +-2, +-4: exact on both halves
    float sx = (d & 1) ? -1.f : 1.f, mx = (d & 1) ? 1.f : 2.f;
    float sy = (d & 2) ? -1.f : 1.f, my = (d & 2) ? 1.f : 2.f;
    float sz = (d & 4) ? -1.f : 1.f, mz = (d & 4) ? 1.f : 2.f;
    V a = df64_scale_pow2(c[0], sx * my * mz);
    V b = df64_scale_pow2(c[1], mx * sy * mz);
    V e = df64_scale_pow2(c[2], mx * my * sz);
    return df64_add(df64_add(a, b), e);
  }
};

struct PolF32 {
  using V = float;
  using Acc = float;
  __device__ static V from_d(double d) { return (float)d; }
  __device__ static double to_d(V v) { return (double)v; }
  __device__ static V zero() { return 0.f; }
  __device__ static void init(Acc& a) { a = 0.f; }
  __device__ static void fma(Acc& a, V k, V x) { a = fmaf(k, x, a); }
  __device__ static V get(const Acc& a) { return a; }
  __device__ static V add(V a, V b) { return a + b; }
};

template <class P>
__device__ __forceinline__ void load_factors(const DevMesh& m, int64_t e, typename P::V* c);
template <>
__device__ __forceinline__ void load_factors<PolF64>(const DevMesh& m, int64_t e, double* c) {
  c[0] = m.ec[3 * e]; c[1] = m.ec[3 * e + 1]; c[2] = m.ec[3 * e + 2];
}
template <>
__device__ __forceinline__ void load_factors<PolDF>(const DevMesh& m, int64_t e, df64* c) {
  c[0] = m.ec_df[3 * e]; c[1] = m.ec_df[3 * e + 1]; c[2] = m.ec_df[3 * e + 2];
}

__device__ __forceinline__ int64_t free_index(const DevMesh& m, int s, int l) {
  int I = s % m.Sx, J = (s / m.Sx) % m.Sy, K = s / (m.Sx * m.Sy);
  int a = l % m.NLx, b = (l / m.NLx) % m.NLy, c = l / (m.NLx * m.NLy);
  int64_t x = I * m.sx + a - m.fx0, y = J * m.sy + b - m.fy0, z = K * m.sz + c - m.fz0;
  int64_t Nfx = m.fx1 - m.fx0, Nfy = m.fy1 - m.fy0;
  return x + Nfx * (y + Nfy * z);
}

// ---------------------------------------------------------------------------
// Element passes driven by per-subdomain-type work lists. Subdomains with the same
// pattern of interior / interface / absent nodes share lists built on the host:
//   * the boundary-layer elements (those with an interface corner): only they contribute
//     when the input vanishes in the interior (first pass) or the output is taken on the
//     interface (second pass);
//   * output items: node l and up to 8 slots (element * 8 + corner of l in it), sorted by
//     slot count so that the lanes of a warp do the same amount of work.
// S is the subdomain edge in elements (0: taken from the mesh at run time).
// ---------------------------------------------------------------------------
template <class P, int S>
__device__ __forceinline__ void build_kd_list(const DevMesh& m, int s, const int16_t* bll, int nbl,
                                              typename P::V* kd) {
  const int sx = S ? S : m.sx, sy = S ? S : m.sy, sz = S ? S : m.sz;
  const int NE = sx * sy * sz;
  const int I = s % m.Sx, J = (s / m.Sx) % m.Sy, K = s / (m.Sx * m.Sy);
  for (int t = threadIdx.x; t < nbl; t += blockDim.x) {
    const int el = bll[t];
    const int ea = el % sx, eb = (el / sx) % sy, ec = el / (sx * sy);
    const int64_t e = (int64_t)(I * sx + ea) + (int64_t)m.nx * ((J * sy + eb) + (int64_t)m.ny * (K * sz + ec));
    typename P::V c[3];
    load_factors<P>(m, e, c);
#pragma unroll
    for (int d = 0; d < 8; ++d) kd[d * NE + el] = P::entry(c, d);
  }
}

template <class P, int S>
__device__ __forceinline__ typename P::V apply_item(const DevMesh& m, const int16_t* it, const typename P::V* xl,
                                                    const typename P::V* kd) {
  const int sx = S ? S : m.sx, sy = S ? S : m.sy, sz = S ? S : m.sz;
  const int NE = sx * sy * sz;
  const int NLx = sx + 1, NLy = sy + 1;
  typename P::Acc acc[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) P::init(acc[t]);
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
      P::fma(acc[q & 3], kp[(p ^ q) * NE], xl[lq]);
    }
  }
  return P::add(P::add(P::get(acc[0]), P::get(acc[1])), P::add(P::get(acc[2]), P::get(acc[3])));
}

template <class P>
__device__ __forceinline__ typename P::V ld_fdm(const void* base, int64_t i);
template <>
__device__ __forceinline__ double ld_fdm<PolF64>(const void* base, int64_t i) {
  return static_cast<const double*>(base)[i];
}
template <>
__device__ __forceinline__ df64 ld_fdm<PolDF>(const void* base, int64_t i) {
  return static_cast<const df64*>(base)[i];
}

}  // namespace dd

// Shared internals of the GB300 DD solver: error handling, device buffers,
// arithmetic policies (FP64, FP32, and "df64" float pairs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dd_solver.h"

namespace dd {

struct Error : std::runtime_error {
  dd_status code;
  Error(dd_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DD_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw ::dd::Error(e_ == cudaErrorMemoryAllocation ? DD_OOM : DD_CUDA_ERROR,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_) + " at " __FILE__ \
                        ":" + std::to_string(__LINE__));                                      \
  } while (0)

void count_launch();  // process-wide counter of kernel launches (profiling)
int64_t launch_counter();
void add_launches(int64_t n);  // launches made by the device (graph replays)
// raises a kernel's dynamic shared-memory limit once per (kernel, device) and size
// (cudaFuncSetAttribute is a host-side call that costs far more than a launch)
void set_max_smem(const void* func, int bytes);
template <class F>
inline void max_smem(F* func, size_t bytes) {
  set_max_smem(reinterpret_cast<const void*>(func), (int)bytes);
}
#define DD_CHECK_LAUNCH() \
  do {                    \
    ::dd::count_launch(); \
    DD_CUDA(cudaGetLastError()); \
  } while (0)

#define DD_REQUIRE(cond, msg) \
  do {                        \
    if (!(cond)) throw ::dd::Error(DD_INVALID_ARG, msg); \
  } while (0)

// Device allocation owned by a context (freed in the context destructor).
struct DeviceArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <class T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    DD_CUDA(cudaMalloc(&p, n * sizeof(T)));
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) DD_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return p;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
  ~DeviceArena() { release(); }
};

// ---------------------------------------------------------------------------
// df64: an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2), about
// 48 significant bits. Products use the exact FMA-based two-product and sums
// the two-sum of Knuth; both are error-free transformations, so a df64 dot
// product accumulates with a relative error near 2^-44 while running on the
// FP32 pipes (GB300 issues FP64 FMAs at 1/62 of the FP32 rate).
// ---------------------------------------------------------------------------
struct df64 {
  float hi, lo;
};

__host__ __device__ inline df64 df64_from_double(double d) {
  df64 r;
  r.hi = (float)d;
  r.lo = (float)(d - (double)r.hi);
  return r;
}
__host__ __device__ inline double df64_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

#ifdef __CUDACC__
__device__ __forceinline__ df64 df64_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df64 df64_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ df64 df64_add(df64 a, df64 b) {
  df64 s = df64_two_sum(a.hi, b.hi);
  df64 t = df64_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df64_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df64_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 df64_neg(df64 a) { return {-a.hi, -a.lo}; }

// Conversions between double and df64 by bit manipulation, so that the FP64 pipe (1/64 of
// the FP32 rate on this part) is not used for them: hi keeps the top 24 significand bits
// of d (truncated), lo the next 29 bits rounded to a float (I2F and a power-of-two scale).
// Values outside the float exponent range of both parts take the FP64 route.
__device__ __forceinline__ df64 df64_from_double_bits(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned int h = (unsigned int)(u >> 32), l = (unsigned int)u;
  const unsigned int sgn = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7FF);
  if (e == 0 && ((h & 0xFFFFFu) | l) == 0u) return {__uint_as_float(sgn), 0.f};
  const int ef = e - 1023 + 127;  // float exponent of hi
  const int es = e - 1075 + 127;  // float exponent of one unit of lo's 29-bit integer
  if (ef <= 0 || ef >= 255 || es <= 0) return df64_from_double(d);
  const float hi = __uint_as_float(sgn | ((unsigned int)ef << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
  const float lo = __uint2float_rn(l & 0x1FFFFFFFu) * __uint_as_float((unsigned int)es << 23);
  return {hi, sgn ? -lo : lo};
}
// exact widening of a float to double without the FP64 pipe (denormal floats become 0)
__device__ __forceinline__ double double_from_float_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sgn = u & 0x80000000u;
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u) return __hiloint2double((int)sgn, 0);
  if (e == 255u) return (double)f;
  const unsigned int m = u & 0x7FFFFFu;
  return __hiloint2double((int)(sgn | ((e - 127u + 1023u) << 20) | (m >> 3)), (int)(m << 29));
}
// hi + lo in FP64 with one add on the FP64 pipe
__device__ __forceinline__ double df64_to_double_bits(df64 a) {
  return double_from_float_bits(a.hi) + double_from_float_bits(a.lo);
}
__device__ __forceinline__ df64 df64_mul(df64 a, df64 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df64_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 df64_scale_pow2(df64 a, float s) { return {a.hi * s, a.lo * s}; }

// Accumulator for sums of df64 products: the leading parts are added with the
// error-free two-sum, everything of order 2^-24 smaller goes into `c`.
struct df64_acc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void fma(df64 a, df64 b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float t = s + p;
    float bp = t - s;
    float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
  }
  __device__ __forceinline__ void add(df64 a) {
    float t = s + a.hi;
    float bp = t - s;
    float err = (s - (t - bp)) + (a.hi - bp);
    s = t;
    c += err + a.lo;
  }
  __device__ __forceinline__ df64 get() const { return df64_fast_two_sum(s, c); }
};
#endif

}  // namespace dd

// Ensemble constrained-Neumann products U_i = N_i R_i (eq. localCorr) on the 5th-generation
// tensor cores: one CTA per subdomain, D = N_i [rows of a 128-row block] x R_i [32 members]
// accumulated in tensor memory (tcgen05.mma kind::tf32, M = 128, N = 32, K = 8) with the
// 3xTF32 split (a = a_hi + a_lo, a_hi = a with the 13 low mantissa bits cleared; products
// a_hi b_hi + a_hi b_lo + a_lo b_hi), which keeps the FP32 accuracy of the preconditioner.
//
// Operands in shared memory use the canonical K-major layout without swizzle: 8 x 16-byte
// core matrices (8 rows, 4 consecutive k), core matrices adjacent in K at the leading byte
// offset, adjacent in M (or N) at the stride byte offset.
//   A tile (128 rows x 32 k):  [kg 8][mg 16][8][4] floats, LBO 2048 B, SBO 128 B
//   B chunk (32 members x 32 k): [kg 8][ng 4][8][4] floats, LBO 512 B, SBO 128 B
// N_i is kept in HBM once per subdomain as full FP32 rows in the tile order [kc][kg][mg][8][4]
// (expanded on the device from the packed symmetric tiles), so each (k chunk, row block) tile
// is eight contiguous slabs that cp.async.bulk copies straight into the A layout.
#include <cuda_runtime.h>

#include <algorithm>

#include "batch.h"
#include "ptx.cuh"
#include "tc_nmm.h"

namespace dd {

namespace {

constexpr int TC_THREADS = 128;  // 4 warps: each owns 32 TMEM lanes (rows of a block)
constexpr int NST = 2;           // raw A stages in flight

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = smem_u32(p);
  return ((a & 0x3FFFFull) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// kind::tf32, D = F32, A = B = TF32, both K-major, N = 32, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// split 32 floats per thread of a tile: hi in place is not allowed (the raw stage is reused
// by the copy engine), so hi and lo go to the operand buffers
__device__ __forceinline__ void split_tile(const float* raw, float* hi, float* lo, int nfl) {
  for (int i = threadIdx.x * 4; i < nfl; i += TC_THREADS * 4) {
    const float4 v = *reinterpret_cast<const float4*>(raw + i);
    float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
    float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    *reinterpret_cast<float4*>(hi + i) = h;
    *reinterpret_cast<float4*>(lo + i) = l;
  }
}

// One CTA per (matrix, 128-row block): it streams the block's k chunks through a
// two-stage ring of bulk copies, splits each tile and the matching member chunk into
// hi/lo operands, and accumulates D (128 x 32 FP32) in tensor memory. 112 KiB of shared
// memory per CTA, so two CTAs share an SM.
__global__ void __launch_bounds__(TC_THREADS) k_nmm_tc(TcMats A, const int64_t* __restrict__ goff,
                                                      const float* __restrict__ rloc, float* __restrict__ uloc,
                                                      int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* araw = reinterpret_cast<float*>(sm);                                   // [NST][4096]
  float* ahi = araw + NST * 4096;                                               // [2][4096]
  float* alo = ahi + 2 * 4096;                                                  // [2][4096]
  float* bhi = alo + 2 * 4096;                                                  // [2][1024]
  float* blo = bhi + 2 * 1024;                                                  // [2][1024]
  uint64_t* full = reinterpret_cast<uint64_t*>(blo + 2 * 1024);                 // [NST]
  uint64_t* done = full + NST;                                                  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
  const int s = blockIdx.x, mb = blockIdx.y;
  const int n = A.n[s];
  const int mg = (n + 7) / 8;          // 8-row groups
  const int nmb = (mg + 15) / 16;      // 128-row blocks
  if (mb >= nmb) return;               // uniform over the block, before any allocation
  const int T = (n + 31) / 32;         // 32-wide k chunks
  const int nmg = min(16, mg - 16 * mb);
  const float* gA = A.data + A.off[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = goff[s];

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&full[i], 1);
    for (int i = 0; i < 2; ++i) mbar_init(&done[i], 1);
  }
  fence_mbar_init();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // raw tile of k chunk kc: eight slabs of nmg 128-byte core-matrix rows
  const uint32_t slab = (uint32_t)nmg * 128u;
  auto issue = [&](int kc) {
    float* dst = araw + (size_t)(kc % NST) * 4096;
    mbar_arrive_expect_tx(&full[kc % NST], 8u * slab);
    for (int kg = 0; kg < 8; ++kg)
      bulk_g2s(dst + kg * 512, gA + ((size_t)(kc * 8 + kg) * mg + 16 * mb) * 32, slab, &full[kc % NST]);
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < NST && t < T; ++t) issue(t);

  // member chunk of k chunk kc, 8 values per thread: element (member j, row k) of the B
  // operand goes to ((kg * 4 + j / 8) * 8 + j % 8) * 4 + k % 4
  float bv[8];
  auto load_b = [&](int kc) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = threadIdx.x + q * TC_THREADS, k = i >> 5, j = i & 31;
      const int row = kc * 32 + k;
      bv[q] = (kc < T && row < n) ? rloc[(base + row) * BW + j] : 0.f;
    }
  };
  load_b(0);

  bool ok = T > 0;
  int t = 0;
  for (; ok && t < T; ++t) {
    const int sl = t & 1;
    // every thread waits (bounded) for the raw tile and for the MMAs that last read the
    // operand slot; the block leaves together if any wait gave up
    bool mine = mbar_wait_bounded(&full[t % NST], (uint32_t)((t / NST) & 1), err);
    if (mine && t >= 2) mine = mbar_wait_bounded(&done[sl], (uint32_t)(((t - 2) >> 1) & 1), err);
    if (!__syncthreads_and(mine)) {
      ok = false;
      break;
    }
    float* hi = ahi + sl * 4096;
    float* lo = alo + sl * 4096;
    const float* raw = araw + (size_t)(t % NST) * 4096;
    if (nmg == 16) {
      split_tile(raw, hi, lo, 4096);
    } else {
      // partial row block: the slab rows past nmg are zero in both operands
      for (int i = threadIdx.x; i < 4096; i += TC_THREADS) {
        const int g = (i >> 5) & 15;
        const float v = g < nmg ? raw[i] : 0.f;
        const float h = tf32_hi(v);
        hi[i] = h;
        lo[i] = v - h;
      }
    }
    {
      float* bh = bhi + sl * 1024;
      float* bl = blo + sl * 1024;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = threadIdx.x + q * TC_THREADS, k = i >> 5, j = i & 31;
        const int o = (((k >> 2) * 4 + (j >> 3)) * 8 + (j & 7)) * 4 + (k & 3);
        const float h = tf32_hi(bv[q]);
        bh[o] = h;
        bl[o] = bv[q] - h;
      }
    }
    load_b(t + 1);  // next member chunk, in flight during this tile's MMAs
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (t + NST < T) issue(t + NST);  // the raw stage of tile t has been consumed
      tc_fence_after();
      const float* bh = bhi + sl * 1024;
      const float* bl = blo + sl * 1024;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t ah = smem_desc(hi + j * 1024, 2048, 128), al = smem_desc(lo + j * 1024, 2048, 128);
        const uint64_t bh_d = smem_desc(bh + j * 256, 512, 128), bl_d = smem_desc(bl + j * 256, 512, 128);
        mma_tf32(tmem, ah, bh_d, (t > 0 || j > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl_d, 1u);
        mma_tf32(tmem, al, bh_d, 1u);
      }
      mma_commit(&done[sl]);
    }
  }
  if (ok) {
    // the last commit covers every MMA issued before it (T > 0 here)
    const int tl = T - 1;
    if (!mbar_wait_bounded(&done[tl & 1], (uint32_t)((tl >> 1) & 1), err)) ok = false;
  } else if (T > 0) {
    // leave after the copies and MMAs in flight have landed (bounded waits)
    for (int tt = t; tt < T && tt < t + NST; ++tt)
      mbar_wait_bounded(&full[tt % NST], (uint32_t)((tt / NST) & 1), nullptr);
    if (t >= 1) mbar_wait_bounded(&done[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1), nullptr);
  }
  tc_fence_after();
  if (ok) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int row = mb * 128 + warp * 32 + lane;
    if (row < n) {
      float4* o = reinterpret_cast<float4*>(uloc + (base + row) * BW);
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
}

// full rows of N_i in the tile order [kc][kg][mg][8][4] from the packed upper tiles
__global__ void k_expand_tc(SymTiles S, TcMats A) {
  const int s = blockIdx.x;
  const int n = S.n[s];
  const int nb = (n + 31) / 32;
  const int mg = (n + 7) / 8;
  const int ntl = nb * (nb + 1) / 2;
  const float* tiles = static_cast<const float*>(S.data) + (size_t)S.toff[s] * 1024;
  float* out = A.data + A.off[s];
  for (int64_t q = threadIdx.x; q < (int64_t)ntl * 1024; q += blockDim.x) {
    const int t = (int)(q >> 10), e = (int)(q & 1023);
    int bi = 0, start = 0;
    while (t >= start + (nb - bi)) {
      start += nb - bi;
      ++bi;
    }
    const int bj = bi + (t - start);
    const int r = bi * 32 + (e >> 5), c = bj * 32 + (e & 31);
    if (r >= n || c >= n) continue;
    const float v = tiles[q];
    auto put = [&](int row, int col) {
      const int kc = col >> 5, kg = (col & 31) >> 2;
      out[((size_t)(kc * 8 + kg) * mg + (row >> 3)) * 32 + (row & 7) * 4 + (col & 3)] = v;
    };
    put(r, c);
    if (bi != bj) put(c, r);
  }
}

}  // namespace

size_t tc_smem_bytes() {
  return (size_t)(NST * 4096 + 4 * 4096 + 4 * 1024) * sizeof(float) + (NST + 2) * 8 + 16;
}

TcMats build_tc_mats(DeviceArena& arena, const SymTiles& S, const std::vector<int>& n_host, cudaStream_t s) {
  TcMats A;
  A.count = S.count;
  std::vector<int64_t> off(S.count);
  int64_t tot = 0;
  int max_nmb = 1;
  for (int i = 0; i < S.count; ++i) {
    const int n = n_host[i];
    const int mg = (n + 7) / 8, nkc = (n + 31) / 32;
    off[i] = tot;
    tot += (int64_t)nkc * 8 * mg * 32;
    max_nmb = std::max(max_nmb, (mg + 15) / 16);
  }
  A.max_nmb = max_nmb;
  A.n = S.n;
  A.off = arena.upload(off, s);
  A.data = arena.alloc<float>((size_t)std::max<int64_t>(tot, 1));
  DD_CUDA(cudaMemsetAsync(A.data, 0, (size_t)std::max<int64_t>(tot, 1) * sizeof(float), s));
  A.bytes = (double)tot * 4.0;
  k_expand_tc<<<S.count, 256, 0, s>>>(S, A);
  DD_CHECK_LAUNCH();
  return A;
}

void launch_nmm_tc(const TcMats& A, const int64_t* goff, const float* rloc, float* uloc, int* err, cudaStream_t s) {
  if (A.count == 0) return;
  const size_t smem = tc_smem_bytes();
  max_smem(k_nmm_tc, smem);
  k_nmm_tc<<<dim3(A.count, A.max_nmb), TC_THREADS, smem, s>>>(A, goff, rloc, uloc, err);
  DD_CHECK_LAUNCH();
}

}  // namespace dd

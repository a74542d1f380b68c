// Ensemble constrained-Neumann products U_i = N_i R_i (eq. 9) on the 5th-generation
// tensor cores, in a persistent kernel: one CTA per SM walks a list of work items (a
// subdomain and a 128-row block of its N_i, full blocks first), streaming the items'
// 32-wide k chunks through one ring of bulk copies that runs on across item boundaries.
// For each chunk the CTA splits the FP32 tile and the members' chunk into low-precision
// slices, and one thread issues the tcgen05.mma that accumulate D (128 rows x 32 members,
// FP32) in tensor memory; two accumulator slots let the epilogue of an item overlap the
// first products of the next.
//
// Two splits keep the FP32 accuracy of the preconditioner:
//  * 3xTF32 (kind::tf32, K = 8): a = a_hi + a_lo with a_hi = a with the 13 low mantissa
//    bits cleared; products a_hi b_hi + a_hi b_lo + a_lo b_hi. The first two are one
//    MMA with N = 64 (B rows: b_hi then b_lo), the third one with N = 32.
//  * BF16x3 (kind::f16 with bf16 operands, K = 16): a = a0 + a1 + a2, each slice the
//    bf16 rounding of what the previous ones leave; the six products a_i b_j with
//    i + j <= 2 are three MMAs: a0 [b0 b1 b2] (N = 96), a1 [b0 b1] (N = 64), a2 b0 (N = 32).
// The column groups of D are summed in the epilogue.
//
// Operands in shared memory use the canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes, adjacent in K at the leading byte offset (LBO), adjacent
// in M (or N) at the stride byte offset (SBO).
//   TF32 A slice (128 x 32):  [kg 8][mg 16][8][4] floats,  LBO 2048 B, SBO 128 B
//   TF32 B (64 x 32):         [kg 8][ng 8][8][4] floats,   LBO 1024 B, SBO 128 B
//   BF16 A slice (128 x 32):  [kb 4][mg 16][8][8] bf16,    LBO 2048 B, SBO 128 B
//   BF16 B (96 x 32):         [kb 4][ng 12][8][8] bf16,    LBO 1536 B, SBO 128 B
// N_i is kept in HBM once per subdomain as full FP32 rows in the TF32 tile order
// [kc][kg][mg][8][4] (expanded on the device from the packed symmetric tiles), so each
// (k chunk, row block) tile is eight contiguous slabs that cp.async.bulk copies as they are.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "batch.h"
#include "ptx.cuh"
#include "tc_nmm.h"

namespace dd {

namespace {

// warp roles of a CTA: 8 consumer warps (operand splits, epilogue), one thread that issues
// the tensor-core products, one thread that issues the bulk copies
constexpr int NCONS = 256;
constexpr int MMA_WARP = NCONS / 32;
constexpr int PROD_WARP = MMA_WARP + 1;
constexpr int TC_THREADS = NCONS + 64;
constexpr int NST = 5;                   // raw tiles in flight per CTA
constexpr int RAW_A = 16384;             // A tile: 128 rows x 32 k FP32
constexpr int RAW_BYTES = RAW_A + 4096;  // + the members' chunk: 32 rows x 32 members FP32
constexpr int MAXQ = 128;                // work items of one CTA (table in shared memory)

// a work item as the CTA keeps it in shared memory
struct ItemS {
  int64_t base;  // first row of the matrix in the members' local vectors
  int64_t aoff;  // first float of the matrix in TcMats::data
  int n, mg, mb, nmg, T, pad;
};

template <int SCHEME>
struct Tc;
template <>
struct Tc<TC_TF32X3> {
  static constexpr int NA = 2;                // A slices
  static constexpr int A_SLICE = 16384;       // bytes
  static constexpr int B_BYTES = 8192;
  static constexpr int ACC_COLS = 64;         // TMEM columns of one accumulator slot
  static constexpr uint32_t TMEM_COLS = 128;  // two slots
  static constexpr int NPART = 2;             // column groups summed in the epilogue
};
template <>
struct Tc<TC_BF16X3> {
  static constexpr int NA = 3;
  static constexpr int A_SLICE = 8192;
  static constexpr int B_BYTES = 6144;
  static constexpr int ACC_COLS = 128;
  static constexpr uint32_t TMEM_COLS = 256;
  static constexpr int NPART = 3;
};

template <int SCHEME>
constexpr size_t smem_bytes() {
  return (size_t)NST * RAW_BYTES + 2 * (size_t)Tc<SCHEME>::NA * Tc<SCHEME>::A_SLICE + 2 * (size_t)Tc<SCHEME>::B_BYTES +
         MAXQ * sizeof(ItemS) + (2 * NST + 8) * 8 + 16;
}

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = smem_u32(p);
  return ((a & 0x3FFFFull) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptors, M = 128, D = F32, A and B K-major: kind::tf32 (A = B = TF32)
// and kind::f16 (A = B = BF16)
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// three bf16 slices of x: each the round-to-nearest bf16 of what the previous ones leave
__device__ __forceinline__ void bf16_slices(float x, __nv_bfloat16& s0, __nv_bfloat16& s1, __nv_bfloat16& s2) {
  s0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(s0);
  s1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(s1);
  s2 = __float2bfloat16_rn(r2);
}

// ---- operand splits (one 32-wide k chunk) ----
// A tile: float4 index i of the raw tile holds rows (mg = (i >> 3) & 15, rr = i & 7) and
// k = kg * 4 .. kg * 4 + 3 with kg = i >> 7; groups past the block's valid rows are skipped
// (their products only reach accumulator rows that are never stored)
template <int SCHEME>
__device__ __forceinline__ void split_a(const float* rt, unsigned char* a_op, int nmg);
template <>
__device__ __forceinline__ void split_a<TC_TF32X3>(const float* rt, unsigned char* a_op, int nmg) {
  float4* hi = reinterpret_cast<float4*>(a_op);
  float4* lo = reinterpret_cast<float4*>(a_op + Tc<TC_TF32X3>::A_SLICE);
#pragma unroll
  for (int t = 0; t < 1024 / NCONS; ++t) {
    const int i = threadIdx.x + t * NCONS;
    if (((i >> 3) & 15) >= nmg) continue;
    const float4 v = reinterpret_cast<const float4*>(rt)[i];
    const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
    hi[i] = h;
    lo[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
  }
}
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
template <>
__device__ __forceinline__ void split_a<TC_BF16X3>(const float* rt, unsigned char* a_op, int nmg) {
#pragma unroll
  for (int t = 0; t < 1024 / NCONS; ++t) {
    const int i = threadIdx.x + t * NCONS;
    const int kg = i >> 7, mg = (i >> 3) & 15, rr = i & 7;
    if (mg >= nmg) continue;
    const float4 v = reinterpret_cast<const float4*>(rt)[i];
    __nv_bfloat16 s[3][4];
    bf16_slices(v.x, s[0][0], s[1][0], s[2][0]);
    bf16_slices(v.y, s[0][1], s[1][1], s[2][1]);
    bf16_slices(v.z, s[0][2], s[1][2], s[2][2]);
    bf16_slices(v.w, s[0][3], s[1][3], s[2][3]);
    const int e = (((kg >> 1) * 16 + mg) * 64 + rr * 8 + (kg & 1) * 4) * 2;  // byte offset in a slice
#pragma unroll
    for (int sl = 0; sl < 3; ++sl)
      *reinterpret_cast<uint2*>(a_op + sl * Tc<TC_BF16X3>::A_SLICE + e) =
          make_uint2(pack_bf16(s[sl][0], s[sl][1]), pack_bf16(s[sl][2], s[sl][3]));
  }
}

// B chunk: this thread holds rows kq * 4 .. kq * 4 + 3 of the chunk for member j
template <int SCHEME>
__device__ __forceinline__ void split_b(const float (&bv)[4], unsigned char* b_op, int kq, int j);
template <>
__device__ __forceinline__ void split_b<TC_TF32X3>(const float (&bv)[4], unsigned char* b_op, int kq, int j) {
  float4 h = make_float4(tf32_hi(bv[0]), tf32_hi(bv[1]), tf32_hi(bv[2]), tf32_hi(bv[3]));
  float4 l = make_float4(bv[0] - h.x, bv[1] - h.y, bv[2] - h.z, bv[3] - h.w);
  float* B = reinterpret_cast<float*>(b_op);
  *reinterpret_cast<float4*>(B + ((kq * 8 + (j >> 3)) * 8 + (j & 7)) * 4) = h;
  *reinterpret_cast<float4*>(B + ((kq * 8 + 4 + (j >> 3)) * 8 + (j & 7)) * 4) = l;
}
template <>
__device__ __forceinline__ void split_b<TC_BF16X3>(const float (&bv)[4], unsigned char* b_op, int kq, int j) {
  __nv_bfloat16 s[3][4];
#pragma unroll
  for (int r = 0; r < 4; ++r) bf16_slices(bv[r], s[0][r], s[1][r], s[2][r]);
  const int kb = kq >> 1, koff = (kq & 1) * 4;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    const int e = (((kb * 12 + sl * 4 + (j >> 3)) * 8 + (j & 7)) * 8 + koff) * 2;
    *reinterpret_cast<uint2*>(b_op + e) = make_uint2(pack_bf16(s[sl][0], s[sl][1]), pack_bf16(s[sl][2], s[sl][3]));
  }
}

// the products of one k chunk into the accumulator at TMEM address dt
template <int SCHEME>
__device__ __forceinline__ void issue_mma(uint32_t dt, const unsigned char* a_op, const unsigned char* b_op, int kc);
template <>
__device__ __forceinline__ void issue_mma<TC_TF32X3>(uint32_t dt, const unsigned char* a_op,
                                                     const unsigned char* b_op, int kc) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {  // K = 8 per instruction
    const uint64_t ah = smem_desc(a_op + j * 4096, 2048, 128);
    const uint64_t al = smem_desc(a_op + Tc<TC_TF32X3>::A_SLICE + j * 4096, 2048, 128);
    const uint64_t b = smem_desc(b_op + j * 2048, 1024, 128);
    mma_tf32(dt, ah, b, idesc_tf32(64), (kc > 0 || j > 0) ? 1u : 0u);  // a_hi [b_hi b_lo]
    mma_tf32(dt, al, b, idesc_tf32(32), 1u);                           // a_lo b_hi
  }
}
template <>
__device__ __forceinline__ void issue_mma<TC_BF16X3>(uint32_t dt, const unsigned char* a_op,
                                                     const unsigned char* b_op, int kc) {
  constexpr int AS = Tc<TC_BF16X3>::A_SLICE;
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // K = 16 per instruction
    const uint64_t b = smem_desc(b_op + j * 3072, 1536, 128);
    mma_f16(dt, smem_desc(a_op + j * 4096, 2048, 128), b, idesc_bf16(96), (kc > 0 || j > 0) ? 1u : 0u);
    mma_f16(dt, smem_desc(a_op + AS + j * 4096, 2048, 128), b, idesc_bf16(64), 1u);
    mma_f16(dt, smem_desc(a_op + 2 * AS + j * 4096, 2048, 128), b, idesc_bf16(32), 1u);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded mbarrier wait that also gives up once another role of the CTA has given up
__device__ __forceinline__ bool wait_tc(uint64_t* bar, uint32_t parity, int* err, volatile int* abort) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  if (err) atomicExch(err, (int)DD_TIMEOUT);
  *abort = 1;
  return false;
}

// Persistent, warp-specialized kernel. CTA b takes the items b, b + gridDim.x, ... (at
// most MAXQ); its tiles g = 0, 1, ... (item q, k chunk kc) pass through raw stage g % NST,
// operand slot g % 2 and accumulator slot q % 2:
//   producer thread: waits until the consumers have split the stage's previous tile
//     (empty), then bulk-copies the A tile and the members' chunk (full);
//   consumer warps: wait for the tile (full) and for the products that last read the
//     operand slot (done), split into the slot, release the stage (empty) and hand the
//     slot to the tensor cores (opready); after the first tile of an item they drain the
//     previous item's accumulator (accf), free it (acce) and store its rows;
//   MMA thread: waits for the operands (opready) and, at an item's first tile, for its
//     accumulator slot to be drained (acce); issues the products and commits them to
//     done, and at the item's last tile to accf.
// Every wait is bounded: on a timeout the CTA records DD_TIMEOUT, the other roles stop at
// their next wait, and the CTA waits (bounded) for its copies and products in flight,
// frees its tensor memory and returns.
template <int SCHEME>
__global__ void __launch_bounds__(TC_THREADS, 1) k_nmm_tc(TcMats A, const int64_t* __restrict__ goff,
                                                         const float* __restrict__ rloc, float* __restrict__ uloc,
                                                         int* err) {
  using P = Tc<SCHEME>;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* raw = sm;                                                // [NST][RAW_BYTES]
  unsigned char* opA = raw + (size_t)NST * RAW_BYTES;                     // [2][NA][A_SLICE]
  unsigned char* opB = opA + 2 * (size_t)P::NA * P::A_SLICE;              // [2][B_BYTES]
  ItemS* items = reinterpret_cast<ItemS*>(opB + 2 * (size_t)P::B_BYTES);  // [MAXQ]
  uint64_t* full = reinterpret_cast<uint64_t*>(items + MAXQ);             // [NST] tile landed
  uint64_t* empty = full + NST;                                           // [NST] tile split
  uint64_t* opready = empty + NST;                                        // [2] operands written
  uint64_t* done = opready + 2;                                           // [2] the slot's products complete
  uint64_t* accf = done + 2;                                              // [2] an item's accumulator complete
  uint64_t* acce = accf + 2;                                              // [2] accumulator drained
  int* ctl = reinterpret_cast<int*>(acce + 2);  // TMEM address, abort flag, tiles issued, last committed tile
  volatile int* abort = ctl + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nq = min(MAXQ, (A.n_items - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
  if (nq <= 0) return;  // uniform over the block, before any barrier or allocation

  for (int q = tid; q < nq; q += TC_THREADS) {
    const int2 it = A.items[(int)blockIdx.x + q * (int)gridDim.x];
    ItemS I;
    I.n = A.n[it.x];
    I.mg = (I.n + 7) / 8;
    I.mb = it.y;
    I.nmg = min(16, I.mg - 16 * I.mb);
    I.T = (I.n + 31) / 32;
    I.base = goff[it.x];
    I.aoff = A.off[it.x];
    I.pad = 0;
    items[q] = I;
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCONS);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&opready[i], NCONS);
      mbar_init(&done[i], 1);
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], NCONS);
    }
    ctl[1] = 0;
    ctl[2] = 0;
    ctl[3] = -1;
  }
  fence_mbar_init();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(ctl)),
                 "r"(P::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = (uint32_t)ctl[0];

  if (warp == PROD_WARP) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int q = 0; q < nq && ok; ++q) {
        const ItemS I = items[q];
        const float* gA = A.data + I.aoff;
        const uint32_t slab = (uint32_t)I.nmg * 128u;
        for (int kc = 0; kc < I.T; ++kc, ++g) {
          const int st = g % NST;
          if (g >= NST && !wait_tc(&empty[st], (uint32_t)(((g / NST) - 1) & 1), err, abort)) {
            ok = false;
            break;
          }
          unsigned char* dst = raw + (size_t)st * RAW_BYTES;
          const int vb = min(32, I.n - kc * 32);  // members' rows of this chunk inside the matrix
          mbar_arrive_expect_tx(&full[st], 8u * slab + (uint32_t)vb * 128u);
          for (int kg = 0; kg < 8; ++kg)
            bulk_g2s(dst + kg * 2048, gA + ((size_t)(kc * 8 + kg) * I.mg + 16 * I.mb) * 32, slab, &full[st]);
          bulk_g2s(dst + RAW_A, rloc + (I.base + kc * 32) * BW, (uint32_t)vb * 128u, &full[st]);
          ctl[2] = g + 1;
        }
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int q = 0; q < nq && ok; ++q) {
        const int T = items[q].T;
        if (q >= 2 && !wait_tc(&acce[q & 1], (uint32_t)(((q - 2) >> 1) & 1), err, abort)) break;
        const uint32_t dt = tmem + (uint32_t)((q & 1) * P::ACC_COLS);
        for (int kc = 0; kc < T; ++kc, ++g) {
          const int slot = g & 1;
          if (!wait_tc(&opready[slot], (uint32_t)((g >> 1) & 1), err, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          issue_mma<SCHEME>(dt, opA + (size_t)slot * P::NA * P::A_SLICE, opB + (size_t)slot * P::B_BYTES, kc);
          mma_commit(&done[slot]);
          if (kc == T - 1) mma_commit(&accf[q & 1]);
          ctl[3] = g;
        }
      }
    }
  } else {
    // consumers: warp kq holds rows kq * 4 .. kq * 4 + 3 of each members' chunk
    const int kq = warp;
    auto drain = [&](const ItemS& J, int qj) -> bool {
      const bool w = __all_sync(0xffffffffu, wait_tc(&accf[qj & 1], (uint32_t)((qj >> 1) & 1), err, abort));
      if (!w) return false;
      tc_fence_after();
      const int lb = (warp & 3) * 32, half = warp >> 2;
      float acc[16], v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
#pragma unroll
      for (int p = P::NPART - 1; p >= 0; --p) {  // smallest terms first
        tmem_ld16(tmem + ((uint32_t)lb << 16) + (uint32_t)((qj & 1) * P::ACC_COLS + p * 32 + half * 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] += v[i];
      }
      tc_fence_before();
      mbar_arrive(&acce[qj & 1]);
      const int row = J.mb * 128 + lb + lane;
      if (row < J.n) {
        float4* o = reinterpret_cast<float4*>(uloc + (J.base + row) * BW + half * 16);
#pragma unroll
        for (int c = 0; c < 4; ++c) o[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
      }
      return true;
    };
    int g = 0;
    bool ok = true;
    for (int q = 0; q < nq && ok; ++q) {
      const ItemS I = items[q];
      for (int kc = 0; kc < I.T; ++kc, ++g) {
        const int st = g % NST, slot = g & 1;
        // every lane polls; the warp continues only if all its lanes' waits succeeded
        bool w = wait_tc(&full[st], (uint32_t)((g / NST) & 1), err, abort);
        if (g >= 2) w = wait_tc(&done[slot], (uint32_t)(((g - 2) >> 1) & 1), err, abort) && w;
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        const unsigned char* rs = raw + (size_t)st * RAW_BYTES;
        split_a<SCHEME>(reinterpret_cast<const float*>(rs), opA + (size_t)slot * P::NA * P::A_SLICE, I.nmg);
        const float* rb = reinterpret_cast<const float*>(rs + RAW_A);
        const int vb = min(32, I.n - kc * 32);
        float bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = kq * 4 + r;
          bv[r] = row < vb ? rb[row * BW + lane] : 0.f;
        }
        split_b<SCHEME>(bv, opB + (size_t)slot * P::B_BYTES, kq, lane);
        fence_proxy_async();
        mbar_arrive(&opready[slot]);
        mbar_arrive(&empty[st]);
        if (kc == 0 && q > 0 && !drain(items[q - 1], q - 1)) {
          ok = false;
          break;
        }
      }
    }
    if (ok) drain(items[nq - 1], nq - 1);
  }
  __syncthreads();
  if (*abort && tid == 0) {
    // leave after the copies and products in flight have landed (bounded waits): the
    // last tile issued into each stage, and the last committed products
    const int issued = ctl[2];
    for (int st = 0; st < NST; ++st) {
      const int t = issued - 1 - (((issued - 1 - st) % NST) + NST) % NST;
      if (t >= 0) mbar_wait_bounded(&full[st], (uint32_t)((t / NST) & 1), nullptr);
    }
    if (ctl[3] >= 0) mbar_wait_bounded(&done[ctl[3] & 1], (uint32_t)((ctl[3] >> 1) & 1), nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::TMEM_COLS) : "memory");
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

TcMats build_tc_mats(DeviceArena& arena, const SymTiles& S, const std::vector<int>& n_host, cudaStream_t s) {
  TcMats A;
  A.count = S.count;
  std::vector<int64_t> off(S.count);
  int64_t tot = 0;
  int max_nmb = 1;
  // work items (matrix, 128-row block), full blocks first so that a static round-robin
  // over the CTAs spreads them evenly
  std::vector<std::pair<int, int2>> items;
  for (int i = 0; i < S.count; ++i) {
    const int n = n_host[i];
    const int mg = (n + 7) / 8, nkc = (n + 31) / 32;
    off[i] = tot;
    tot += (int64_t)nkc * 8 * mg * 32;
    const int nmb = (mg + 15) / 16;
    max_nmb = std::max(max_nmb, nmb);
    if (n > 0)
      for (int mb = 0; mb < nmb; ++mb) items.push_back({std::min(16, mg - 16 * mb), make_int2(i, mb)});
  }
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<int2> it(items.size());
  for (size_t k = 0; k < items.size(); ++k) it[k] = items[k].second;
  A.max_nmb = max_nmb;
  A.n = S.n;
  A.off = arena.upload(off, s);
  A.n_items = (int)it.size();
  A.items = arena.upload(it, s);
  A.data = arena.alloc<float>((size_t)std::max<int64_t>(tot, 1));
  DD_CUDA(cudaMemsetAsync(A.data, 0, (size_t)std::max<int64_t>(tot, 1) * sizeof(float), s));
  A.bytes = (double)tot * 4.0;
  k_expand_tc<<<S.count, 256, 0, s>>>(S, A);
  DD_CHECK_LAUNCH();
  return A;
}

static int sm_count() {
  static std::mutex mu;
  static int dev_cached = -1, count = 0;
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev != dev_cached) {
    DD_CUDA(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    dev_cached = dev;
  }
  return count;
}

void launch_nmm_tc(const TcMats& A, const int64_t* goff, const float* rloc, float* uloc, int* err, int scheme,
                   cudaStream_t s) {
  if (A.n_items == 0) return;
  // one persistent CTA per SM, more when an SM would hold more than MAXQ items
  const int grid = std::max(std::min(A.n_items, sm_count()), (A.n_items + MAXQ - 1) / MAXQ);
  if (scheme == TC_BF16X3) {
    max_smem(k_nmm_tc<TC_BF16X3>, smem_bytes<TC_BF16X3>());
    k_nmm_tc<TC_BF16X3><<<grid, TC_THREADS, smem_bytes<TC_BF16X3>(), s>>>(A, goff, rloc, uloc, err);
  } else {
    max_smem(k_nmm_tc<TC_TF32X3>, smem_bytes<TC_TF32X3>());
    k_nmm_tc<TC_TF32X3><<<grid, TC_THREADS, smem_bytes<TC_TF32X3>(), s>>>(A, goff, rloc, uloc, err);
  }
  DD_CHECK_LAUNCH();
}

}  // namespace dd

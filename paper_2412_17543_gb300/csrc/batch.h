// Ensemble (multi-right-hand-side) kernels: every vector of the batched path holds the
// members of an ensemble interleaved, v[i * BW + m] for row i and member m, so that a
// warp's lanes are the members of one row (coalesced 128/256-byte rows, one index
// lookup per row shared by all members). The ensemble is padded to BW members; padded
// members carry zero right-hand sides and stay inactive.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"
#include "device.h"
#include "loop.h"
#include "tc_nmm.h"

namespace dd {

constexpr int BW = 32;  // ensemble block width (members per row, one per lane)
constexpr int NBLKB = 152 * 8;  // fixed reduction grid of the ensemble kernels (deterministic partials)

// per-member device scalars, slot-major: sc[slot * BW + m]
enum {
  BS_RZ = 0, BS_PQ, BS_ALPHA, BS_RR, BS_BETA, BS_BB, BS_FLAG, BS_ACT, BS_REF, BS_RTOL2, BS_ITS, BS_RR0,
  BS_COUNT = 16
};
// BFIN_RZL: BFIN_RZ0 when the device iteration count *its is 0, else BFIN_RZ
enum { BFIN_PQ = 1, BFIN_RR, BFIN_RZ0, BFIN_RZ, BFIN_BB, BFIN_RZL };

// scratch of the batched operators, interleaved [rows][BW]: the Krylov and local vectors
// of the Schur operator in df64 (float pairs: the ensemble's steps run on the FP32 pipes,
// FP64 only at the boundary), the BDDC vectors in the preconditioner's type (float for
// FP32, double for FP64)
struct BatchWork {
  DeviceArena arena;
  df64 *tI = nullptr, *sI = nullptr, *yloc = nullptr;
  double* kii_tmp = nullptr;          // [n_int][BW] doubles (dense K_II^{-1} only)
  float* D1f = nullptr;               // level-1 BDDC weights as floats
  void *rloc = nullptr, *uloc = nullptr, *vloc = nullptr, *gloc = nullptr, *gC = nullptr, *uC = nullptr;
  void *gI2 = nullptr, *u0I2 = nullptr, *rl2 = nullptr, *r2 = nullptr, *rloc2 = nullptr, *uloc2 = nullptr,
       *vloc2 = nullptr, *gloc2 = nullptr, *g3 = nullptr, *u3 = nullptr, *z2 = nullptr, *uI2 = nullptr;
  df64 *xg = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *p = nullptr, *q = nullptr, *bvec = nullptr;
  df64 *F = nullptr, *X = nullptr;    // [n_free][BW]
  double* sc = nullptr;               // [BS_COUNT][BW]
  double* sc_host = nullptr;          // pinned mirror
  double* partials = nullptr;         // [NBLKB][4][BW]
  df64* wpart = nullptr;              // [deflation blocks][MAXK][BW]
  double* mu = nullptr;               // [MAXK][BW]
  LoopCtl* ctl = nullptr;             // device-resident loop control
  LoopCtl* ctl_host = nullptr;        // pinned mirror
  double* alphas = nullptr;           // [maxit] member 0's step lengths
  // members per pass of the element kernels and per block of the fast diagonalization
  // (launch shapes chosen by timing at the first ensemble call), and their timings (ms)
  int elem_rc = 8, fdm_rc = 8;
  float elem_ms[3] = {0.f, 0.f, 0.f}, fdm_ms[2] = {0.f, 0.f};
  // symmetric products of the ensemble (level-1 N_i; level-2 K_II^{-1} and N): tensor-core
  // operand copy, the kernel in use, and the selection timings (SIMT, 3xTF32, BF16x3)
  struct SymOp {
    TcMats tc;
    int kind = DD_ENS_SIMT;  // DD_ENS_SIMT, DD_ENS_TC (3xTF32) or DD_ENS_BF16X3
    float ms[3] = {0.f, 0.f, 0.f};
  } op[3];
};
enum { BOP_N1 = 0, BOP_KII2 = 1, BOP_N2 = 2 };

// ---- layout ----
// out[i * BW + m] = m < nrhs ? F[m * n + i] : 0   (F member-major, as the caller passes it)
void launch_pack_in(int64_t n, int nrhs, const double* F, df64* out, cudaStream_t s);
// X[m * n + i] = in[i * BW + m] for m < nrhs
void launch_pack_out(int64_t n, int nrhs, const df64* in, double* X, cudaStream_t s);
void launch_to_float(int64_t n, const double* in, float* out, cudaStream_t s);

// ---- Schur-complement operator (interleaved counterparts of the single-vector kernels) ----
// rc: members per pass of the element kernels (4, 8 or 16; used for 8^3 subdomains, df64)
void launch_elem_interior_b(const DevMesh& m, int mode, const df64* xg, const df64* f, df64* tI, int rc,
                            cudaStream_t s);
void launch_elem_interface_b(const DevMesh& m, int mode, const df64* xg, const df64* sI, df64* yloc, int rc,
                             cudaStream_t s);
// tmp: [n_int][BW] doubles, used by the dense local solver only; rc: members per block of
// the fast diagonalization (4 or 8, df64)
void launch_kii_apply_b(const DevMesh& m, const df64* tI, df64* sI, double* tmp, int rc, cudaStream_t s);
void launch_gather_b(int64_t n, const int* ptr, const int* idx, const df64* loc, const df64* base,
                     const int64_t* bmap, df64* y, cudaStream_t s);
void launch_scatter_recover_b(const DevMesh& m, const df64* xg, const df64* sI, df64* x, cudaStream_t s);

// ---- BDDC (T = float or double by prec) ----
// symmetric tiles times a block of BW members: out_m = A_m in_m
void launch_symm_b(const SymTiles& A, const int64_t* voff, const void* in, void* out, cudaStream_t s);
// rloc[k][.] = D_k r[gmap[k]][.]  (Df: the weights as floats, used by the FP32 preconditioner)
void launch_restrict_b(int prec, int64_t nflat, const int* gmap, const float* Df, const double* D, const df64* r,
                       void* rloc, cudaStream_t s);
// per item m: out[(out_off[m]+i)][.] = alpha * sum_j M_m[i][j] x_j[.] (+ add), x_j = in[in_map?..][.]
void launch_bmm(const BatchedRows& B, const int64_t* in_off, const int* in_map, const void* in,
                const int64_t* out_off, void* out, double alpha, const void* add, cudaStream_t s);
// transposed: out[(out_off[m]+j)][.] = alpha * sum_i M_m[i][j] x_i[.] (+ add)
void launch_bmm_t(const BatchedRows& B, const int64_t* in_off, const int* in_map, const void* in,
                  const int64_t* out_off, void* out, double alpha, const void* add, cudaStream_t s);
// y[g][.] = sum over copies of loc[idx[k]][.]  (BDDC coarse / level-2 gathers, type by prec)
void launch_gather_tb(int prec, int64_t n, const int* ptr, const int* idx, const void* loc, const void* base,
                      const int64_t* bmap, void* y, cudaStream_t s);
// typed counterparts for a level whose residual is already in the preconditioner type
void launch_restrict_tb(int prec, int64_t nflat, const int* gmap, const double* D, const void* r, void* rloc,
                        cudaStream_t s);
void launch_wgather_tb(int prec, int64_t n, const int* ptr, const int* idx, const double* D, const void* uloc,
                       const void* vloc, void* z, cudaStream_t s);
// z[g][.] = sum over copies k of D_k (u_k + v_k)   (level-1 combine into the df64 Krylov vector)
void launch_wgather_b(int prec, int64_t n, const int* ptr, const int* idx, const float* Df, const double* D,
                      const void* uloc, const void* vloc, df64* z, cudaStream_t s);
void launch_dense_mm(int prec, int n, const void* A, const void* x, void* y, cudaStream_t s);
void launch_map_gather_b(int prec, int64_t n, const int* map, const void* in, void* out, cudaStream_t s);
void launch_map_scatter_b(int prec, int64_t n, const int* map, const void* in, void* out, cudaStream_t s);

// ---- Krylov vectors, per member (df64 storage and arithmetic) ----
void bvec_dots(int64_t n, const df64* a0, const df64* b0, const df64* a1, const df64* b1, double* partials,
               cudaStream_t s);
void bvec_finalize(const double* partials, double* sc, int op, int flexible, cudaStream_t s,
                   const int* its = nullptr);
void bvec_axpy2(int64_t n, const double* sc, df64* x, const df64* p, df64* r, const df64* q, double* partials,
                cudaStream_t s);
void bvec_sub(int64_t n, const df64* a, const df64* b, df64* y, cudaStream_t s);
void bvec_init(double* sc, int nrhs, double rtol, int stop_rhs_norm, cudaStream_t s);
// deflation with the shared basis (df64 copy W, k columns of length n, stride ld):
// mu[j][m] = sum_l G[j][l] sum_i W[l][i] Z[i][m]; wpart: [defl_blocks(n)][MAXK][BW] scratch
int defl_blocks(int64_t n);
void bdefl_mu(int64_t n, int k, const df64* W, int64_t ld, const df64* Z, const double* G, df64* wpart, double* mu,
              cudaStream_t s);
// Y[i][m] = Z[i][m] + beta_m Y[i][m] + sign_w sum_j W[j][i] mu[j][m]  (Z NULL: Y += sign_w W mu;
// beta_idx < 0: no beta term)
void bdefl_update(int64_t n, int k, const df64* W, int64_t ld, const double* mu, const df64* Z, df64* Y,
                  const double* sc, int beta_idx, double sign_w, cudaStream_t s);

}  // namespace dd

// Device-side data of the DD solver and the launch wrappers of its kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace dd {

constexpr int TILE = 32;  // symmetric matrices are stored as 32x32 upper tiles

// Batched symmetric matrices. Streamed form ("packed panels", read by k_symv): each
// matrix is cut into 32-row block rows; block row b holds its diagonal block as the packed
// upper triangle (row-major), then the full 32 x 32 blocks to its right, then the block of
// the ragged last w = n % 32 columns (32 rows of w values padded to a multiple of 16
// bytes); the ragged last block row is its packed w x w triangle padded likewise. Only the
// padding to 16 bytes (the bulk-copy granule) is stored beyond the n(n+1)/2 entries.
// Tiled form (read by the ensemble kernels, built from the packed form on the first
// ensemble call): upper-triangular 32x32 tiles (bi <= bj, row-major over the tile pairs;
// each tile row-major, zero-padded). FP64: doubles; FP32: floats; DF64: (hi, lo) pairs.
struct SymTiles {
  int prec = DD_PREC_FP64;
  int count = 0;
  int max_n = 0;
  const int* n = nullptr;         // [count] dimension of each matrix
  const int64_t* poff = nullptr;  // [count] first element of each matrix in the packed form
  const void* pdata = nullptr;    // packed form
  int64_t pelems = 0;             // elements of the packed form
  int slots = 2;                  // bulk-copy ring depth per warp of k_symv (2, 3 or 4; tuned at setup)
  int split = 1;                  // CTAs per matrix of k_symv (small batches; tuned at setup)
  void* spart = nullptr;          // [count * split][padded n] partial vectors (split > 1)
  unsigned* sticket = nullptr;    // [count] counters, 0 between launches
  const int64_t* toff = nullptr;  // [count] first tile of each matrix (tiled form, nullptr until built)
  const void* data = nullptr;     // tiled form
  int64_t ntiles = 0;
};

// Geometry of one matrix in the packed form (element counts; eb = bytes per element).
struct PackGeom {
  int nf, w, wp, dw;  // full block rows, ragged width, padded ragged width, padded ragged triangle
};
__host__ __device__ inline PackGeom pack_geom(int n, int eb) {
  const int g = 16 / eb;  // elements per 16 bytes
  PackGeom p;
  p.nf = n / 32;
  p.w = n % 32;
  p.wp = (p.w + g - 1) / g * g;
  p.dw = (p.w * (p.w + 1) / 2 + g - 1) / g * g;
  return p;
}
__host__ __device__ inline int64_t pack_row_off(const PackGeom& p, int b) {
  const int64_t rc = p.w ? 32 * p.wp : 0;
  return (int64_t)b * (528 + rc) + 1024 * ((int64_t)b * (p.nf - 1) - (int64_t)b * (b - 1) / 2);
}
__host__ __device__ inline int64_t pack_tile_off(const PackGeom& p, int bi, int bj) {
  const int64_t r = pack_row_off(p, bi);
  if (bi == bj) return r;
  return r + 528 + 1024 * (int64_t)((bj < p.nf ? bj : p.nf) - bi - 1);
}
__host__ __device__ inline int pack_tile_elems(const PackGeom& p, int bi, int bj) {
  if (bi == bj) return bi < p.nf ? 528 : p.dw;
  return bj < p.nf ? 1024 : 32 * p.wp;
}
__host__ __device__ inline int64_t pack_total(const PackGeom& p) { return pack_row_off(p, p.nf) + (p.w ? p.dw : 0); }
// index of (r, c), c >= r, in a packed upper triangle of size h
__host__ __device__ inline int tri_index(int h, int r, int c) { return r * h - r * (r - 1) / 2 + (c - r); }

inline size_t tile_bytes(int prec) { return prec == DD_PREC_FP32 ? 4096 : 8192; }

// A batch of row-major matrices (for batched GEMVs): item m has rows row0[m] ..
// row0[m+1] - 1 of a flat row space and cols[m] columns; its matrix starts at element moff[m].
struct BatchedRows {
  int prec = DD_PREC_FP64;
  int64_t nrows = 0;
  int count = 0;
  int max_cols = 0;
  int max_rows = 0;
  const int64_t* row0 = nullptr;
  const int* cols = nullptr;
  const int64_t* moff = nullptr;
  const void* data = nullptr;
  int rows_per_block = 32;        // k_bgemv: rows of one matrix per block (8 warps)
  int zsplit = 1;                 // k_bgemv_t: row parts per matrix (combined in the kernel); tuned at setup
  void* zpart = nullptr;          // [count][column blocks][zsplit][128] partial sums (zsplit > 1)
  unsigned* zticket = nullptr;    // [count][column blocks] counters, 0 between launches
};

// Level-1 geometry and Schur-complement operator (Sect. 3.1).
struct DevMesh {
  int nx, ny, nz, sx, sy, sz, Sx, Sy, Sz, S;
  int fx0, fx1, fy0, fy1, fz0, fz1;
  int NLx, NLy, NLz, NL;
  int64_t n_free, n_gamma, n_int;
  int64_t n_flat;           // sum of the subdomains' local interface sizes (host copy of goff[S])
  const int16_t* lidx;
  const int* sub_type;      // [S] work-list type of each subdomain
  const int* type_off;      // [types][6]: first/last item of the interior pass, of the interface pass,
                            //             first/last boundary-layer element
  const int16_t* type_items;  // items: node, then 8 slots (element * 8 + corner, -1 = none)
  const int16_t* type_bl;     // boundary-layer element ids
  const int16_t* type_citems; // the items with slots (position in the type's boundary-layer list) * 8 + corner
  int max_nbl;                // largest boundary-layer list of a subdomain type
  int max_nint = 0;           // largest interior (unknowns not on the interface) of a subdomain
  int schur_threads;          // threads per CTA of the fused Schur kernel (256, 352 or 416; tuned at setup)
  const int64_t* ioff;
  const int64_t* goff;
  const int* gmap;
  const int* gptr;
  const int* gidx;
  const int64_t* gamma_free;
  const double* ec;     // [E][3] FP64 element factors k hy hz/(36 hx), ...
  const double* coef;   // [E] element coefficients k_e (FP64)
  const df64* ec_df;    // [E][3] same as float pairs
  SymTiles KIIinv;         // dense representation (local_solver == DD_LOCAL_DENSE)
  int schur_prec;
  int local_solver;         // DD_LOCAL_DENSE or DD_LOCAL_FDM
  const int* fdm_n;         // [S][3] sizes of the interior index sets per axis (<= 9)
  const void* fdm_V;        // [S][3][81] 1D generalized eigenvectors, stride 9 (df64 or double)
  const void* fdm_Dinv;     // [n_int] inverse eigenvalue sums, indexed like interior vectors
  // per-subdomain copies read by the fused Schur kernel in one coalesced level each
  // (8^3-element subdomains with the fast-diagonalization solver only; else null):
  const int* sxg = nullptr;     // [S][NL] interface index of each local node (-1: not on the interface)
  const void* sfac = nullptr;   // [S][max_nbl][3] factors of the boundary-layer elements in the
                                // order of the type's list (df64 or double, as schur_prec)
};

// One BDDC level (Sect. 3.2): weights, constrained Neumann operator N, coarse basis
// Phi on the interface, coarse maps. Used for level 1 and level 2.
struct DevBDDC {
  int S;
  int64_t n_gamma;
  int n_coarse;
  int64_t n_flat;          // sum of local interface sizes
  int64_t n_cflat;         // sum of local coarse sizes
  const int64_t* goff;
  const int* gmap;
  const int* gsub;         // flat local interface position -> subdomain
  const int* gptr;
  const int* gidx;
  const double* D;         // flat weights
  SymTiles N;
  BatchedRows PhiT;        // Phi_i^T: nc x nG per subdomain (rows = local coarse dofs)
  const int64_t* coff;
  const int* cmap;         // flat local coarse -> global coarse dof
  const int* cptr;
  const int* cidx;
  int prec;
};

// Level-2 extras (three-level BDDC, Sect. 3.2): interior correction and extension.
struct DevLevel2 {
  DevBDDC b;
  int64_t n_int;
  const int64_t* ioff;
  const int* imap;          // flat interior -> level-1 coarse dof
  const int* gam_c;         // level-2 interface -> level-1 coarse dof
  const int64_t* gam_c64;   // same, 64-bit (gather base map)
  SymTiles KIIinv;
  BatchedRows E;            // nI x nG per group (K_II^{-1} K_IG)
  const void* KC3inv;       // n3 x n3 dense, prec of b
  int n3;
};

// Scratch buffers of the operators (device).
struct Work {
  double* tI;      // [n_int] level-1 interior
  double* sI;      // [n_int]
  double* yloc;    // [n_flat] level-1 local interface
  double* rloc;    // [n_flat]
  double* uloc;    // [n_flat]
  double* vloc;    // [n_flat]
  double* gloc;    // [n_cflat]
  double* gC;      // [n_coarse]
  double* uC;      // [n_coarse]
  // level 2
  double* gI2;     // [n_int2]
  double* u0I2;    // [n_int2]
  double* rl2;     // [n_flat2]
  double* r2;      // [n_gamma2]
  double* rloc2;   // [n_flat2]
  double* uloc2;   // [n_flat2]
  double* vloc2;   // [n_flat2]
  double* gloc2;   // [n_cflat2]
  double* g3;      // [n3]
  double* u3;      // [n3]
  double* z2;      // [n_gamma2]
  double* uI2;     // [n_int2]
  int* err;        // device error word (bounded waits)
};

enum ElemMode { ELEM_SCHUR = 0, ELEM_CONDENSE = 1, ELEM_RECOVER = 2 };

// ---- launch wrappers (kernels.cu) ----
void launch_elem_interior(const DevMesh& m, int mode, const double* xg, const double* f, double* tI, cudaStream_t s);
void launch_elem_interface(const DevMesh& m, int mode, const double* xg, const double* sI, double* yloc,
                           cudaStream_t s);
// s_I = K_II^{-1} t_I for every subdomain (dense tiles or fast diagonalization)
void launch_kii_apply(const DevMesh& m, const double* tI, double* sI, int* err, cudaStream_t s);
// fused Schur application (one CTA per subdomain) for the fast-diagonalization solver of 8^3 subdomains
bool schur_fused_available(const DevMesh& m);
void launch_schur_fused(const DevMesh& m, const double* xg, double* yloc, cudaStream_t s);
void launch_symv(const SymTiles& A, const int64_t* voff, const double* in, double* out, int* err, cudaStream_t s);
// builds the tiled form of A from its packed form (once; the ensemble kernels read tiles)
void ensure_tiles(DeviceArena& arena, SymTiles& A, cudaStream_t s);
void launch_wait_selftest(int* err, long long limit, cudaStream_t s);
// y[g] = (base ? base[bmap ? bmap[g] : g] : 0) + sum over copies of loc[idx[k]]
void launch_gather(int64_t n, const int* ptr, const int* idx, const double* loc, const double* base,
                   const int64_t* bmap, double* y, cudaStream_t s);
// grad[e] = -lambda_e^T K_e^0 x_e (coefficient gradient of the adjoint)
void launch_coef_grad(const DevMesh& m, const double* x, const double* lam, double* grad, int log_coef,
                      cudaStream_t s);
// part[b] (b < nblk) = block maxima of |k_e - c_e| / |k_e| (c_e = exp(coef_e) when log)
void launch_coef_mismatch(const DevMesh& m, const double* coef, int log, double* part, int nblk, cudaStream_t s);
void launch_scatter_recover(const DevMesh& m, const double* xg, const double* sI, double* x, cudaStream_t s);
void launch_restrict(int64_t nflat, const int* gmap, const double* D, const double* r, double* rloc, cudaStream_t s);
void launch_dense_gemv(int n, int prec, const void* A, const double* x, double* y, cudaStream_t s);
// per item m: out[out_off[m]+i] = alpha * sum_j M_m[i][j] x_j (+ add[out_off[m]+i]),
// x_j = in[in_map ? in_map[in_off[m]+j] : in_off[m]+j]
void launch_bgemv(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                  const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s);
// per item m: out[out_off[m]+j] = alpha * sum_i M_m[i][j] x_i (+ add[out_off[m]+j]) (transposed product)
void launch_bgemv_t(const BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                    const int64_t* out_off, double* out, double alpha, const double* add, cudaStream_t s);
// z[g] = sum over copies k of D[k] (uloc[k] + vloc[k])
void launch_wgather(int64_t n, const int* ptr, const int* idx, const double* D, const double* uloc,
                    const double* vloc, double* z, cudaStream_t s);
void launch_map_gather(int64_t n, const int* map, const double* in, double* out, cudaStream_t s);
void launch_map_scatter(int64_t n, const int* map, const double* in, double* out, cudaStream_t s);

// vector kernels for the Krylov loop (vecops in kernels.cu)
struct Scalars;  // device-resident scalars of PCG
}  // namespace dd

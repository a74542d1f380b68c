// Krylov-vector kernels (vecops.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace dd {

constexpr int NBLK = 304;   // reduction grid: 2 blocks per SM of GB300 (fixed => deterministic sums)
constexpr int MAXDOT = 4;   // dot products per partial record
constexpr int MAXK = 128;   // maximum deflation basis size

// device scalar slots of PCG
enum {
  SC_RZ = 0, SC_PQ, SC_ALPHA, SC_RR, SC_BETA, SC_BB, SC_FLAG, SC_COUNT = 16
};
// FIN_RZL: FIN_RZ0 when the device iteration count *its is 0, else FIN_RZ
enum { FIN_PQ = 1, FIN_RR, FIN_RZ0, FIN_RZ, FIN_BB, FIN_RZL };

void vec_dots(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1, const double* a2,
              const double* b2, double* partials, cudaStream_t s);
void vec_finalize(const double* partials, double* sc, int op, int flexible, cudaStream_t s,
                  const int* its = nullptr);
void vec_axpy2(int64_t n, const double* sc, double* x, const double* p, double* r, const double* q, double* partials,
               cudaStream_t s);
// the same with vec_finalize done by the last block of the launch (ticket: a device counter,
// zero between launches; the calls sharing one ticket must be ordered on one stream)
void vec_dots_fin(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1,
                  double* partials, double* sc, int op, int flexible, unsigned* ticket, cudaStream_t s,
                  const int* its = nullptr);
void vec_axpy2_fin(int64_t n, double* sc, double* x, const double* p, double* r, const double* q, double* partials,
                   unsigned* ticket, cudaStream_t s);
void vec_sub(int64_t n, const double* a, const double* b, double* y, cudaStream_t s);
// out = in - mean(in) (in == out allowed); partials: [NBLK * MAXDOT] scratch
void vec_sub_mean(int64_t n, const double* in, double* out, double* partials, cudaStream_t s);
// deflation with the basis stored as df64 (float pairs), and the conversion
void to_df64(int64_t n, const double* in, df64* out, cudaStream_t s);
// mu with the basis as df64 (V: k columns, stride ld); wpart: [defl_df_part_rows(n)][MAXK],
// ticket: [defl_df_tickets(n)] counters, zero before the first call (each call leaves them zero)
int defl_df_blocks(int64_t n);
int defl_df_part_rows(int64_t n);  // rows of MAXK doubles that wpart needs
int defl_df_tickets(int64_t n);    // ticket counters (zeroed once) that the dots need
void defl_mu_df(int64_t n, int k, const df64* V, int64_t ld, const double* v, const double* Ginv, double* wpart,
                double* mu, unsigned* ticket, cudaStream_t s);
void defl_update_df(int64_t n, int k, const df64* W, int64_t ld, const double* mu, const double* z, double* y,
                    const double* sc, int beta_idx, double sign_w, cudaStream_t s);
// the update with an FP32-stored basis (exact entries of a basis rounded to FP32 values)
void defl_update_f(int64_t n, int k, const float* W, int64_t ld, const double* mu, const double* z, double* y,
                   const double* sc, int beta_idx, double sign_w, cudaStream_t s);
// wf = (float)w; w takes the rounded values; *changed = 1 if any entry changed (not cleared here)
void round_to_f32(int64_t n, double* w, float* wf, int* changed, cudaStream_t s);
void gram(int64_t n, int na, const double* const* X, int nb, const double* const* Y, double* part, double* C,
          cudaStream_t s);
void lincomb(int64_t n, int m, const double* const* V, const double* Yc, int kc, double* const* out, cudaStream_t s);
void zdiff(int64_t n, const double* z0, const double* z1, double inv_alpha, double* out, cudaStream_t s);

}  // namespace dd

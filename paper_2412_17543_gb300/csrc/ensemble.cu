// Ensemble solves: BW (= 32) independent right-hand-side sequences that share the
// matrix, the BDDC preconditioner and one recycled deflation basis W, advanced as
// one block. Every operator application streams the operator data once for all
// members; each member runs its own deflated PCG (own alpha, beta and stopping test,
// decided on the device), and a member that has converged keeps its iterate
// (alpha = 0) while the others continue. The basis W is shared: it is built from the
// search vectors of member 0 (V = [W, P of member 0]) with the single-sequence
// recycling update (Sect. 4.2), and every member is deflated by it (Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "batch.h"
#include "context.h"

namespace dd {

void free_batch_work(BatchWork* bw) {
  if (!bw) return;
  if (bw->sc_host) cudaFreeHost(bw->sc_host);
  if (bw->ctl_host) cudaFreeHost(bw->ctl_host);
  delete bw;
}

namespace {

// The symmetric products of the ensemble (level-1 N_i, level-2 K_II^{-1} and N) run on
// the tensor cores (3xTF32 or BF16x3 splits) or on CUDA-core tiles. With DD_ENS_AUTO the
// kernels run on the context's own operators (three timed launches each after a warm-up)
// and the fastest is kept: the autotuning step of the ensemble path.
void apply_sym_b(dd_ctx* c, int which, const SymTiles& S, const int64_t* voff, const void* in, void* out,
                 cudaStream_t s) {
  const BatchWork::SymOp& o = c->bw->op[which];
  if (o.kind == DD_ENS_SIMT)
    launch_symm_b(S, voff, in, out, s);
  else
    launch_nmm_tc(o.tc, voff, (const float*)in, (float*)out, c->w.err,
                  o.kind == DD_ENS_BF16X3 ? TC_BF16X3 : TC_TF32X3, s);
}

// mean time of three launches of f after one warm-up (ms)
template <class F>
float time_ms(F&& f, cudaStream_t s) {
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  f();
  DD_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < 3; ++r) f();
  DD_CUDA(cudaEventRecord(e1, s));
  DD_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 3.f;
}

void select_op(dd_ctx* c, int which, const SymTiles& S, const int64_t* voff, void* in, void* out, int64_t rows,
               cudaStream_t s) {
  BatchWork::SymOp& o = c->bw->op[which];
  const int mode = c->opt.ens_nmm;
  o.kind = DD_ENS_SIMT;
  if (S.prec != DD_PREC_FP32 || mode == DD_ENS_SIMT || S.count == 0) return;
  std::vector<int> nh(S.count);
  DD_CUDA(cudaMemcpyAsync(nh.data(), S.n, nh.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  o.tc = build_tc_mats(c->bw->arena, S, nh, s);
  if (mode == DD_ENS_TC || mode == DD_ENS_BF16X3) {
    o.kind = mode;
    return;
  }
  const int npad = ((S.max_n + 31) / 32) * 32;
  const bool simt_fits = (size_t)npad * BW * sizeof(float) <= 227 * 1024;  // CUDA-core tiles hold the vector
  DD_CUDA(cudaMemsetAsync(in, 0, (size_t)rows * BW * sizeof(float), s));
  const int kinds[3] = {DD_ENS_SIMT, DD_ENS_TC, DD_ENS_BF16X3};
  int best = -1;
  for (int v = 0; v < 3; ++v) {
    o.ms[v] = 0.f;
    if (v == 0 && !simt_fits) continue;
    o.kind = kinds[v];
    o.ms[v] = time_ms([&] { apply_sym_b(c, which, S, voff, in, out, s); }, s);
    if (best < 0 || o.ms[v] < o.ms[best]) best = v;
  }
  check_err(c, s);
  o.kind = kinds[best];
  if (which == BOP_N1 && o.kind != DD_ENS_SIMT) {
    // tensor-core work of one level-1 launch as issued: per (subdomain, 128-row block) and
    // 32-wide k chunk, 128 x 32 x N multiply-adds with N = 64 + 32 (3xTF32: a_hi [b_hi b_lo],
    // a_lo b_hi) or 96 + 64 + 32 (BF16x3: the six slice products i + j <= 2)
    const double nsum = o.kind == DD_ENS_BF16X3 ? 192.0 : 96.0;
    double fl = 0.0;
    for (int i = 0; i < S.count; ++i)
      fl += (double)((nh[i] + 127) / 128) * ((nh[i] + 31) / 32) * 128.0 * 32.0 * nsum * 2.0;
    c->prof_flops[DD_PROF_ENS_N] = fl;
  }
}


// launch shapes of the Schur operator of the ensemble: members per pass of the element
// kernels (4, 8, 16) and per block of the fast diagonalization (4, 8), taken from the
// options or else each timed on the context's own mesh (df64 operator on 8^3 subdomains;
// other meshes keep 8)
void select_shapes(dd_ctx* c, cudaStream_t s) {
  BatchWork& B = *c->bw;
  const DevMesh& m = c->mesh;
  if (m.schur_prec != DD_PREC_DF64 || !(m.sx == 8 && m.sy == 8 && m.sz == 8)) return;
  const int64_t n = c->n_gamma;
  DD_CUDA(cudaMemsetAsync(B.p, 0, (size_t)n * BW * sizeof(df64), s));
  DD_CUDA(cudaMemsetAsync(B.sI, 0, (size_t)std::max<int64_t>(m.n_int, 1) * BW * sizeof(df64), s));
  if (c->opt.ens_elem_rc) {
    B.elem_rc = c->opt.ens_elem_rc;
  } else {
    const int rcs[3] = {4, 8, 16};
    int best = 1;
    for (int v = 0; v < 3; ++v) {
      B.elem_ms[v] = time_ms([&] { launch_elem_interface_b(m, ELEM_SCHUR, B.p, B.sI, B.yloc, rcs[v], s); }, s);
      if (B.elem_ms[v] < B.elem_ms[best]) best = v;
    }
    B.elem_rc = rcs[best];
  }
  if (m.local_solver == DD_LOCAL_FDM) {
    if (c->opt.ens_fdm_rc) {
      B.fdm_rc = c->opt.ens_fdm_rc;
    } else {
      for (int v = 0; v < 2; ++v)
        B.fdm_ms[v] = time_ms([&] { launch_kii_apply_b(m, B.sI, B.tI, B.kii_tmp, v == 0 ? 4 : 8, s); }, s);
      B.fdm_rc = B.fdm_ms[0] < B.fdm_ms[1] ? 4 : 8;
    }
  }
  check_err(c, s);
}

void select_ops(dd_ctx* c, cudaStream_t s) {
  BatchWork& B = *c->bw;
  select_shapes(c, s);
  select_op(c, BOP_N1, c->b1.N, c->b1.goff, B.rloc, B.uloc, c->b1.n_flat, s);
  if (c->levels == 3) {
    const DevLevel2& L = c->l2;
    select_op(c, BOP_KII2, L.KIIinv, L.ioff, B.gI2, B.u0I2, L.n_int, s);
    select_op(c, BOP_N2, L.b.N, L.b.goff, B.rloc2, B.uloc2, L.b.n_flat, s);
  }
}

BatchWork& batch_work(dd_ctx* c, cudaStream_t s) {
  if (c->bw) return *c->bw;
  // the ensemble kernels read the symmetric operators as 32 x 32 tiles: build that form from
  // the packed panels once (kept by the context)
  ensure_tiles(c->arena, c->b1.N, s);
  if (c->mesh.local_solver != DD_LOCAL_FDM) ensure_tiles(c->arena, c->mesh.KIIinv, s);
  if (c->levels == 3) {
    ensure_tiles(c->arena, c->l2.KIIinv, s);
    ensure_tiles(c->arena, c->l2.b.N, s);
  }
  auto B = std::make_unique<BatchWork>();
  DeviceArena& A = B->arena;
  const DevMesh& m = c->mesh;
  const int64_t n = c->n_gamma;
  auto dvec = [&](int64_t rows) { return A.alloc<df64>((size_t)std::max<int64_t>(rows, 1) * BW); };
  auto tvec = [&](int prec, int64_t rows) -> void* {
    return prec == DD_PREC_FP32 ? (void*)A.alloc<float>((size_t)std::max<int64_t>(rows, 1) * BW)
                                : (void*)A.alloc<double>((size_t)std::max<int64_t>(rows, 1) * BW);
  };
  B->tI = dvec(m.n_int);
  B->sI = dvec(m.n_int);
  B->yloc = dvec(c->b1.n_flat);
  if (m.local_solver != DD_LOCAL_FDM) B->kii_tmp = A.alloc<double>((size_t)std::max<int64_t>(m.n_int, 1) * BW);
  B->D1f = A.alloc<float>((size_t)std::max<int64_t>(c->b1.n_flat, 1));
  launch_to_float(c->b1.n_flat, c->b1.D, B->D1f, s);
  const int pp = c->b1.prec;
  B->rloc = tvec(pp, c->b1.n_flat);
  B->uloc = tvec(pp, c->b1.n_flat);
  B->vloc = tvec(pp, c->b1.n_flat);
  B->gloc = tvec(pp, c->b1.n_cflat);
  B->gC = tvec(pp, c->b1.n_coarse);
  B->uC = tvec(pp, c->b1.n_coarse);
  if (c->levels == 3) {
    const DevLevel2& L = c->l2;
    const int p2 = L.b.prec;
    B->gI2 = tvec(p2, L.n_int);
    B->u0I2 = tvec(p2, L.n_int);
    B->uI2 = tvec(p2, L.n_int);
    B->rl2 = tvec(p2, L.b.n_flat);
    B->rloc2 = tvec(p2, L.b.n_flat);
    B->uloc2 = tvec(p2, L.b.n_flat);
    B->vloc2 = tvec(p2, L.b.n_flat);
    B->r2 = tvec(p2, L.b.n_gamma);
    B->z2 = tvec(p2, L.b.n_gamma);
    B->gloc2 = tvec(p2, L.b.n_cflat);
    B->g3 = tvec(p2, L.n3);
    B->u3 = tvec(p2, L.n3);
  }
  B->xg = dvec(n);
  B->r = dvec(n);
  B->z = dvec(n);
  B->zold = dvec(n);
  B->p = dvec(n);
  B->q = dvec(n);
  B->bvec = dvec(n);
  B->F = dvec(c->n_free);
  B->X = dvec(c->n_free);
  B->sc = A.alloc<double>((size_t)BS_COUNT * BW);
  B->partials = A.alloc<double>((size_t)NBLKB * 4 * BW);
  B->wpart = A.alloc<df64>((size_t)defl_blocks(std::max<int64_t>(n, 1)) * MAXK * BW);
  B->mu = A.alloc<double>((size_t)MAXK * BW);
  DD_CUDA(cudaMallocHost(&B->sc_host, (size_t)BS_COUNT * BW * sizeof(double)));
  B->ctl = A.alloc<LoopCtl>(1);
  B->alphas = A.alloc<double>((size_t)c->opt.maxit);
  DD_CUDA(cudaMallocHost(&B->ctl_host, sizeof(LoopCtl)));
  c->bw = B.release();
  select_ops(c, s);
  return *c->bw;
}

// ---- operators on BW members ----
void schur_b(dd_ctx* c, const df64* x, df64* y, cudaStream_t s) {
  ProfScope ps(c, DD_PROF_ENS_SCHUR, s);
  BatchWork& B = *c->bw;
  launch_elem_interior_b(c->mesh, ELEM_SCHUR, x, nullptr, B.tI, B.elem_rc, s);
  launch_kii_apply_b(c->mesh, B.tI, B.sI, B.kii_tmp, B.fdm_rc, s);
  launch_elem_interface_b(c->mesh, ELEM_SCHUR, x, B.sI, B.yloc, B.elem_rc, s);
  launch_gather_b(c->n_gamma, c->mesh.gptr, c->mesh.gidx, B.yloc, nullptr, nullptr, y, s);
}

void condense_b(dd_ctx* c, const df64* f, df64* b, cudaStream_t s) {
  BatchWork& B = *c->bw;
  launch_elem_interior_b(c->mesh, ELEM_CONDENSE, nullptr, f, B.tI, B.elem_rc, s);
  launch_kii_apply_b(c->mesh, B.tI, B.sI, B.kii_tmp, B.fdm_rc, s);
  launch_elem_interface_b(c->mesh, ELEM_CONDENSE, nullptr, B.sI, B.yloc, B.elem_rc, s);
  launch_gather_b(c->n_gamma, c->mesh.gptr, c->mesh.gidx, B.yloc, f, c->mesh.gamma_free, b, s);
}

void recover_b(dd_ctx* c, const df64* f, const df64* xg, df64* x, cudaStream_t s) {
  BatchWork& B = *c->bw;
  launch_elem_interior_b(c->mesh, ELEM_RECOVER, xg, f, B.tI, B.elem_rc, s);
  launch_kii_apply_b(c->mesh, B.tI, B.sI, B.kii_tmp, B.fdm_rc, s);
  launch_scatter_recover_b(c->mesh, xg, B.sI, x, s);
}

// The same fork as the single path: the coarse correction (Phi_i^T r_i, the coarse solve,
// Phi_i u_C) on the context's high-priority side stream beside the local products N_i r_i;
// in level 2, K_II^{-1} g_I and the level-3 correction on two more side streams.
struct ForkB {
  cudaStream_t side;
  cudaEvent_t f, j;
  cudaStream_t begin(cudaStream_t s) const {
    if (!side) return s;
    DD_CUDA(cudaEventRecord(f, s));
    DD_CUDA(cudaStreamWaitEvent(side, f, 0));
    return side;
  }
  void end(cudaStream_t s) const {
    if (!side) return;
    DD_CUDA(cudaEventRecord(j, side));
    DD_CUDA(cudaStreamWaitEvent(s, j, 0));
  }
};

template <class CoarseFn>
void bddc_b(dd_ctx* c, const DevBDDC& b, const df64* r, df64* z, void* rloc, void* uloc, void* vloc, void* gloc,
            void* gC, void* uC, CoarseFn coarse, cudaStream_t s) {
  launch_restrict_b(b.prec, b.n_flat, b.gmap, c->bw->D1f, b.D, r, rloc, s);
  const ForkB fk{c->s_coarse, c->ev_fork, c->ev_join};
  const cudaStream_t sc = fk.begin(s);
  launch_bmm(b.PhiT, b.goff, nullptr, rloc, b.coff, gloc, 1.0, nullptr, sc);    // Phi_i^T r_i
  launch_gather_tb(b.prec, b.n_coarse, b.cptr, b.cidx, gloc, nullptr, nullptr, gC, sc);
  coarse(gC, uC, sc);
  launch_bmm_t(b.PhiT, b.coff, b.cmap, uC, b.goff, vloc, 1.0, nullptr, sc);     // Phi_i R_Ci u_C
  {
    ProfScope pk(c, DD_PROF_ENS_N, s);
    apply_sym_b(c, BOP_N1, b.N, b.goff, rloc, uloc, s);                        // u_i = N_i r_i
  }
  fk.end(s);
  launch_wgather_b(b.prec, b.n_gamma, b.gptr, b.gidx, c->bw->D1f, b.D, uloc, vloc, z, s);
}

// level-2 BDDC on the coarse system of the ensemble (same steps as the single path)
void level2_b(dd_ctx* c, const void* g, void* u, cudaStream_t s) {
  DevLevel2& L = c->l2;
  BatchWork& B = *c->bw;
  const int p2 = L.b.prec;
  const ForkB f0{c->s_aux[0], c->ev_aux[0], c->ev_aux[1]};
  const ForkB f1{c->s_aux[1], c->ev_aux[2], c->ev_aux[3]};
  launch_map_gather_b(p2, L.n_int, L.imap, g, B.gI2, s);
  const cudaStream_t s0 = f0.begin(s);
  apply_sym_b(c, BOP_KII2, L.KIIinv, L.ioff, B.gI2, B.u0I2, s0);
  launch_bmm_t(L.E, L.ioff, nullptr, B.gI2, L.b.goff, B.rl2, -1.0, nullptr, s);  // -K_GI K_II^{-1} g_I
  launch_gather_tb(p2, L.b.n_gamma, L.b.gptr, L.b.gidx, B.rl2, g, L.gam_c64, B.r2, s);
  {
    // level-2 interface BDDC on r2 (vectors in the preconditioner type), exact level 3
    const DevBDDC& b = L.b;
    launch_restrict_tb(p2, b.n_flat, b.gmap, b.D, B.r2, B.rloc2, s);
    const cudaStream_t s1 = f1.begin(s);
    launch_bmm(b.PhiT, b.goff, nullptr, B.rloc2, b.coff, B.gloc2, 1.0, nullptr, s1);
    launch_gather_tb(p2, b.n_coarse, b.cptr, b.cidx, B.gloc2, nullptr, nullptr, B.g3, s1);
    launch_dense_mm(p2, L.n3, L.KC3inv, B.g3, B.u3, s1);
    launch_bmm_t(b.PhiT, b.coff, b.cmap, B.u3, b.goff, B.vloc2, 1.0, nullptr, s1);
    apply_sym_b(c, BOP_N2, b.N, b.goff, B.rloc2, B.uloc2, s);
    f1.end(s);
    launch_wgather_tb(p2, b.n_gamma, b.gptr, b.gidx, b.D, B.uloc2, B.vloc2, B.z2, s);
  }
  f0.end(s);
  launch_bmm(L.E, L.b.goff, L.b.gmap, B.z2, L.ioff, B.uI2, -1.0, B.u0I2, s);  // u0 - K_II^{-1} K_IG z
  launch_map_scatter_b(p2, L.n_int, L.imap, B.uI2, u, s);
  launch_map_scatter_b(p2, L.b.n_gamma, L.gam_c, B.z2, u, s);
}

void precond_b(dd_ctx* c, const df64* r, df64* z, cudaStream_t s) {
  ProfScope ps(c, DD_PROF_ENS_PRECOND, s);
  BatchWork& B = *c->bw;
  bddc_b(c, c->b1, r, z, B.rloc, B.uloc, B.vloc, B.gloc, B.gC, B.uC,
         [&](const void* g, void* u, cudaStream_t ss) {
           if (c->levels == 2)
             launch_dense_mm(c->b1.prec, c->b1.n_coarse, c->KCinv, g, u, ss);
           else
             level2_b(c, g, u, ss);
         },
         s);
}

void copy_b(df64* dst, const df64* src, int64_t rows, cudaStream_t s) {
  DD_CUDA(cudaMemcpyAsync(dst, src, (size_t)rows * BW * sizeof(df64), cudaMemcpyDeviceToDevice, s));
}

// deflated PCG (Algorithm 1) for every member; returns the worst member status
dd_status pcg_solve_b(dd_ctx* c, dd_recycle* st, double rtol, bool record, int nrhs, dd_stats* stats,
                      cudaStream_t s) {
  BatchWork& B = *c->bw;
  const int64_t n = c->n_gamma;
  const dd_options& o = c->opt;
  const int k = st->k;
  const df64* W = k ? st->Wd : nullptr;
  const df64* AW = k ? st->AWd : nullptr;
  auto host_sc = [&]() {
    DD_CUDA(cudaMemcpyAsync(B.sc_host, B.sc, (size_t)BS_COUNT * BW * sizeof(double), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
  };
  auto hs = [&](int slot, int m) { return B.sc_host[slot * BW + m]; };
  bvec_init(B.sc, nrhs, rtol, o.stop_rhs_norm, s);
  if (k) {
    // x_0 = x_{-1} + W (W^T A W)^{-1} W^T (b - A x_{-1})  (shared W, per-member mu)
    schur_b(c, B.xg, B.q, s);
    bvec_sub(n, B.bvec, B.q, B.r, s);
    bdefl_mu(n, k, W, n, B.r, st->Ginv, B.wpart, B.mu, s);
    bdefl_update(n, k, W, n, B.mu, nullptr, B.xg, B.sc, -1, 1.0, s);
  }
  schur_b(c, B.xg, B.q, s);
  bvec_sub(n, B.bvec, B.q, B.r, s);
  bvec_dots(n, B.bvec, B.bvec, B.r, B.r, B.partials, s);
  bvec_finalize(B.partials, B.sc, BFIN_BB, 0, s);
  // member 0 feeds the recycling histories while it is active
  launch_loop_begin_b(B.ctl, B.sc, o.maxit, record && st->hmax > 0 ? 1 : 0, s);
  // p enters the first update p = z + beta p - W mu with beta = 0
  DD_CUDA(cudaMemsetAsync(B.p, 0, (size_t)n * BW * sizeof(df64), s));
  const bool rec = record && st->hmax > 0;
  const int flex = o.flexible;
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool in_graph) {
    if (flex) copy_b(B.zold, B.z, n, bs);
    precond_b(c, B.r, B.z, bs);
    if (rec) launch_record_col0(B.ctl, B.z, st->Z, n, st->hmax, 1, bs);
    bvec_dots(n, B.r, B.z, flex ? B.r : nullptr, flex ? B.zold : nullptr, B.partials, bs);
    bvec_finalize(B.partials, B.sc, BFIN_RZL, flex, bs, &B.ctl->its);
    if (k) bdefl_mu(n, k, AW, n, B.z, st->Ginv, B.wpart, B.mu, bs);
    bdefl_update(n, k, W, n, B.mu, B.z, B.p, B.sc, BS_BETA, -1.0, bs);
    schur_b(c, B.p, B.q, bs);
    bvec_dots(n, B.p, B.q, nullptr, nullptr, B.partials, bs);
    bvec_finalize(B.partials, B.sc, BFIN_PQ, 0, bs);
    if (rec) {
      launch_record_col0(B.ctl, B.p, st->P, n, st->hmax, 0, bs);
      launch_record_col0(B.ctl, B.q, st->AP, n, st->hmax, 0, bs);
    }
    bvec_axpy2(n, B.sc, B.xg, B.p, B.r, B.q, B.partials, bs);
    bvec_finalize(B.partials, B.sc, BFIN_RR, 0, bs);
    launch_loop_check_b(B.ctl, B.sc, B.alphas, h, in_graph, bs);
  };
  const std::vector<uint64_t> key = {2,
                                     (uint64_t)k,
                                     (uint64_t)rec,
                                     (uint64_t)st->hmax,
                                     (uint64_t)flex,
                                     (uint64_t)(uintptr_t)W,
                                     (uint64_t)(uintptr_t)AW,
                                     (uint64_t)(uintptr_t)st->Ginv,
                                     (uint64_t)(uintptr_t)st->P,
                                     (uint64_t)(uintptr_t)st->AP,
                                     (uint64_t)(uintptr_t)st->Z};
  st->loop.run(key, body, B.ctl, B.ctl_host, o.loop_graph && !c->prof_on, s);
  const LoopCtl L = *B.ctl_host;
  st->alphas.assign(rec ? (size_t)L.nalpha : 0, 0.0);
  if (rec && L.nalpha > 0)
    DD_CUDA(cudaMemcpyAsync(st->alphas.data(), B.alphas, (size_t)L.nalpha * sizeof(double), cudaMemcpyDeviceToHost,
                            s));
  host_sc();
  dd_status status = L.status == LOOP_NOT_CONVERGED ? DD_NOT_CONVERGED : DD_OK;
  for (int m = 0; m < nrhs; ++m) {
    if (hs(BS_FLAG, m) != 0.0) status = DD_BREAKDOWN;
    if (stats) {
      stats[m].iters = (int)hs(BS_ITS, m);
      stats[m].rel_res0 = std::sqrt(hs(BS_RR0, m)) / hs(BS_REF, m);
      stats[m].rel_res = std::sqrt(hs(BS_RR, m)) / hs(BS_REF, m);
      stats[m].recycled_k = k;
      stats[m].frozen = (int)st->frozen;
    }
  }
  return status;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_recycle_create_batch(dd_ctx* c, int32_t k, int32_t strategy, double freeze_tol, dd_recycle** out) {
  dd_status rc = dd_recycle_create(c, k, strategy, freeze_tol, out);
  if (rc != DD_OK) return rc;
  rc = guard_call([&] {
    dd_recycle* st = *out;
    st->nrhs = BW;
    st->xg_prev_b = st->arena.alloc<df64>((size_t)c->n_gamma * BW);
    DD_CUDA(cudaMemset(st->xg_prev_b, 0, (size_t)c->n_gamma * BW * sizeof(df64)));
  });
  if (rc != DD_OK) {
    dd_recycle_destroy(*out);
    *out = nullptr;
  }
  return rc;
}

// operator-level ensemble calls (interface vectors, member-major [nrhs][n_gamma])
static dd_status batch_op(dd_ctx* c, int32_t nrhs, const double* X, double* Y, void* stream, bool precond,
                          const char* what) {
  if (!c || !X || !Y || nrhs < 1 || nrhs > BW) {
    set_last_error(std::string(what) + ": invalid argument");
    return DD_INVALID_ARG;
  }
  if (!precond && c->mesh.local_solver != DD_LOCAL_FDM && c->mesh.schur_prec == DD_PREC_DF64) {
    set_last_error(std::string(what) + ": dense K_II^{-1} needs schur_prec FP64 for ensembles");
    return DD_INVALID_ARG;
  }
  return guard_call([&] {
    cudaStream_t s = (cudaStream_t)stream;
    BatchWork& B = batch_work(c, s);
    launch_pack_in(c->n_gamma, nrhs, X, B.p, s);
    if (precond)
      precond_b(c, B.p, B.q, s);
    else
      schur_b(c, B.p, B.q, s);
    launch_pack_out(c->n_gamma, nrhs, B.q, Y, s);
    check_err(c, s);
  });
}

dd_status dd_schur_apply_batch(dd_ctx* c, int32_t nrhs, const double* X, double* Y, void* stream) {
  return batch_op(c, nrhs, X, Y, stream, false, "dd_schur_apply_batch");
}

dd_status dd_precond_apply_batch(dd_ctx* c, int32_t nrhs, const double* R, double* Z, void* stream) {
  return batch_op(c, nrhs, R, Z, stream, true, "dd_precond_apply_batch");
}

dd_status dd_solve_batch(dd_ctx* c, int32_t nrhs, const double* F, double* X, double rtol, dd_recycle* st,
                         dd_stats* stats, void* stream) {
  if (!c || !F || !X || !st || st->ctx != c || st->nrhs != BW || nrhs < 1 || nrhs > BW || !(rtol > 0.0)) {
    set_last_error("dd_solve_batch: invalid argument");
    return DD_INVALID_ARG;
  }
  if (c->neumann) {
    set_last_error("dd_solve_batch: the pure-Neumann case (no Dirichlet face) is solved by dd_solve only");
    return DD_INVALID_ARG;
  }
  if (c->mesh.local_solver != DD_LOCAL_FDM && c->mesh.schur_prec == DD_PREC_DF64) {
    set_last_error("dd_solve_batch: dense K_II^{-1} needs schur_prec FP64 for ensembles");
    return DD_INVALID_ARG;
  }
  dd_status result = DD_OK;
  dd_status gs = guard_call([&] {
    cudaStream_t s = (cudaStream_t)stream;
    BatchWork& B = batch_work(c, s);
    DD_CUDA(cudaEventRecord(c->ev0, s));
    launch_pack_in(c->n_free, nrhs, F, B.F, s);
    condense_b(c, B.F, B.bvec, s);
    copy_b(B.xg, st->xg_prev_b, c->n_gamma, s);
    const bool record = st->kmax > 0 && !st->frozen;
    result = pcg_solve_b(c, st, rtol, record, nrhs, stats, s);
    recover_b(c, B.F, B.xg, B.X, s);
    copy_b(st->xg_prev_b, B.xg, c->n_gamma, s);
    if (record && (result == DD_OK || result == DD_NOT_CONVERGED)) {
      ProfScope pr(c, DD_PROF_RECYCLE, s);
      recycle_update(c, st, (int)st->alphas.size(), s);
    } else
      st->step++;
    launch_pack_out(c->n_free, nrhs, B.X, X, s);
    DD_CUDA(cudaEventRecord(c->ev1, s));
    check_err(c, s);
    if (c->prof_on) c->harvest();
    if (stats) {
      float ms = 0.f;
      DD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      for (int m = 0; m < nrhs; ++m) {
        stats[m].ms = ms;
        stats[m].frozen = (int)st->frozen;
      }
    }
  });
  if (gs != DD_OK) return gs;
  if (result != DD_OK) set_last_error(result == DD_NOT_CONVERGED ? "maxit reached" : "PCG breakdown");
  return result;
}

}  // extern "C"

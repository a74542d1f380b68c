// Context, device uploads, operator applications and the deflated PCG solve
// (Algorithm 1) with Krylov subspace recycling (Sect. 4.2), behind the C ABI of
// include/dd_solver.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>

#include "common.h"
#include "device.h"
#include "hostla.h"
#include "setup.h"
#include "vecops.h"
#include "context.h"
#include "batch.h"
#include "recycle.h"

using namespace dd;

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
namespace dd {
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_counter() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_max_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& have = done[{func, dev}];
  if (have >= bytes) return;
  DD_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  have = bytes;
}
}  // namespace dd

// ---------------------------------------------------------------------------
// uploads
// ---------------------------------------------------------------------------
namespace dd {

SymTiles upload_sym(DeviceArena& A, const std::vector<const double*>& mats, const std::vector<int>& dims, int prec,
                    cudaStream_t s) {
  SymTiles T;
  T.prec = prec;
  T.count = (int)mats.size();
  const int eb = prec == DD_PREC_FP32 ? 4 : 8;
  std::vector<int64_t> poff(T.count);
  int64_t ne = 0;
  int maxn = 0;
  for (int m = 0; m < T.count; ++m) {
    poff[m] = ne;
    ne += pack_total(pack_geom(dims[m], eb));
    maxn = std::max(maxn, dims[m]);
  }
  T.pelems = ne;
  T.max_n = maxn;
  std::vector<unsigned char> buf((size_t)ne * eb, 0);
  auto put = [&](int64_t at, double v) {
    unsigned char* d = buf.data() + (size_t)at * eb;
    if (prec == DD_PREC_FP64) {
      std::memcpy(d, &v, 8);
    } else if (prec == DD_PREC_FP32) {
      float f = (float)v;
      std::memcpy(d, &f, 4);
    } else {  // float pair (hi, lo)
      df64 x = df64_from_double(v);
      std::memcpy(d, &x.hi, 4);
      std::memcpy(d + 4, &x.lo, 4);
    }
  };
#pragma omp parallel for schedule(dynamic, 16)
  for (int m = 0; m < T.count; ++m) {
    const int n = dims[m];
    const PackGeom g = pack_geom(n, eb);
    const int nb = g.nf + (g.w > 0);
    const double* M = mats[m];
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) {
        const int64_t o = poff[m] + pack_tile_off(g, bi, bj);
        const int h = bi < g.nf ? 32 : g.w;
        if (bi == bj) {
          for (int r = 0; r < h; ++r)
            for (int c = r; c < h; ++c) put(o + tri_index(h, r, c), M[(size_t)(bi * 32 + r) * n + bi * 32 + c]);
        } else if (bj < g.nf) {
          for (int r = 0; r < 32; ++r)
            for (int c = 0; c < 32; ++c) put(o + r * 32 + c, M[(size_t)(bi * 32 + r) * n + bj * 32 + c]);
        } else {
          for (int r = 0; r < 32; ++r)
            for (int c = 0; c < g.w; ++c) put(o + r * g.wp + c, M[(size_t)(bi * 32 + r) * n + bj * 32 + c]);
        }
      }
  }
  T.n = A.upload(dims, s);
  T.poff = A.upload(poff, s);
  unsigned char* d = A.alloc<unsigned char>(buf.size());
  DD_CUDA(cudaMemcpy(d, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  T.pdata = d;
  return T;
}

// Row batch of row-major matrices (rows x cols per item); transposed: stores M^T of every item.
BatchedRows upload_rows(DeviceArena& A, const std::vector<const double*>& mats, const std::vector<int>& rows,
                        const std::vector<int>& cols, int prec, bool transpose, cudaStream_t s) {
  BatchedRows B;
  B.prec = prec;
  const size_t cnt = mats.size();
  std::vector<int64_t> row0(cnt + 1, 0), moff(cnt);
  std::vector<int> ncol(cnt);
  int64_t tot = 0;
  for (size_t m = 0; m < cnt; ++m) {
    int R = transpose ? cols[m] : rows[m], C = transpose ? rows[m] : cols[m];
    row0[m + 1] = row0[m] + R;
    ncol[m] = C;
    moff[m] = tot;
    tot += (int64_t)R * C;
    B.max_cols = std::max(B.max_cols, C);
    B.max_rows = std::max(B.max_rows, R);
  }
  B.nrows = row0[cnt];
  B.count = (int)cnt;
  std::vector<double> buf(tot);
  for (size_t m = 0; m < cnt; ++m) {
    int R0 = rows[m], C0 = cols[m];
    for (int i = 0; i < R0; ++i)
      for (int j = 0; j < C0; ++j) {
        double v = mats[m][(size_t)i * C0 + j];
        if (transpose)
          buf[moff[m] + (int64_t)j * R0 + i] = v;
        else
          buf[moff[m] + (int64_t)i * C0 + j] = v;
      }
  }
  if (prec == DD_PREC_FP32) {
    std::vector<float> f(buf.begin(), buf.end());
    float* d = A.alloc<float>(f.size());
    DD_CUDA(cudaMemcpy(d, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    B.data = d;
  } else {
    double* d = A.alloc<double>(buf.size());
    DD_CUDA(cudaMemcpy(d, buf.data(), buf.size() * 8, cudaMemcpyHostToDevice));
    B.data = d;
  }
  B.row0 = A.upload(row0, s);
  B.cols = A.upload(ncol, s);
  B.moff = A.upload(moff, s);
  return B;
}

void upload_bddc(DeviceArena& A, const Level& L, int prec, DevBDDC& b, cudaStream_t s) {
  b.S = L.S;
  b.n_gamma = L.n_gamma;
  b.n_coarse = L.n_coarse;
  b.n_flat = L.goff[L.S];
  b.n_cflat = L.coff[L.S];
  b.prec = prec;
  b.goff = A.upload(L.goff, s);
  b.gmap = A.upload(L.gmap, s);
  std::vector<int> gsub(b.n_flat);
  std::vector<double> D(b.n_flat);
  std::vector<int> cmap(b.n_cflat);
  for (int i = 0; i < L.S; ++i) {
    for (int64_t k = L.goff[i]; k < L.goff[i + 1]; ++k) {
      gsub[k] = i;
      D[k] = L.sub[i].D[k - L.goff[i]];
    }
    for (int c = 0; c < L.sub[i].nc; ++c) cmap[L.coff[i] + c] = L.sub[i].cmap[c];
  }
  b.gsub = A.upload(gsub, s);
  b.D = A.upload(D, s);
  b.gptr = A.upload(L.gptr, s);
  b.gidx = A.upload(L.gidx, s);
  b.coff = A.upload(L.coff, s);
  b.cmap = A.upload(cmap, s);
  b.cptr = A.upload(L.cptr, s);
  b.cidx = A.upload(L.cidx, s);
  std::vector<const double*> Ns, Ps;
  std::vector<int> nG, nc;
  for (int i = 0; i < L.S; ++i) {
    Ns.push_back(L.sub[i].N.data());
    Ps.push_back(L.sub[i].Phi.data());
    nG.push_back(L.sub[i].nG);
    nc.push_back(L.sub[i].nc);
  }
  b.N = upload_sym(A, Ns, nG, prec == DD_PREC_FP32 ? DD_PREC_FP32 : DD_PREC_FP64, s);
  int rp = prec == DD_PREC_FP32 ? DD_PREC_FP32 : DD_PREC_FP64;
  b.PhiT = upload_rows(A, Ps, nG, nc, rp, true, s);
}

const void* upload_dense(DeviceArena& A, const std::vector<double>& M, int prec) {
  if (prec == DD_PREC_FP32) {
    std::vector<float> f(M.begin(), M.end());
    float* d = A.alloc<float>(f.size());
    DD_CUDA(cudaMemcpy(d, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    return d;
  }
  double* d = A.alloc<double>(M.size());
  DD_CUDA(cudaMemcpy(d, M.data(), M.size() * 8, cudaMemcpyHostToDevice));
  return d;
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
void schur_apply(dd_ctx* c, const double* x, double* y, cudaStream_t s) {
  ProfScope ps(c, DD_PROF_SCHUR, s);
  if (schur_fused_available(c->mesh)) {
    launch_schur_fused(c->mesh, x, c->w.yloc, s);
    launch_gather(c->n_gamma, c->mesh.gptr, c->mesh.gidx, c->w.yloc, nullptr, nullptr, y, s);
    return;
  }
  launch_elem_interior(c->mesh, ELEM_SCHUR, x, nullptr, c->w.tI, s);
  {
    ProfScope pk(c, DD_PROF_SYMV_KII, s);
    launch_kii_apply(c->mesh, c->w.tI, c->w.sI, c->w.err, s);
  }
  launch_elem_interface(c->mesh, ELEM_SCHUR, x, c->w.sI, c->w.yloc, s);
  launch_gather(c->n_gamma, c->mesh.gptr, c->mesh.gidx, c->w.yloc, nullptr, nullptr, y, s);
}

void condense(dd_ctx* c, const double* f, double* b, cudaStream_t s) {
  launch_elem_interior(c->mesh, ELEM_CONDENSE, nullptr, f, c->w.tI, s);
  launch_kii_apply(c->mesh, c->w.tI, c->w.sI, c->w.err, s);
  launch_elem_interface(c->mesh, ELEM_CONDENSE, nullptr, c->w.sI, c->w.yloc, s);
  launch_gather(c->n_gamma, c->mesh.gptr, c->mesh.gidx, c->w.yloc, f, c->mesh.gamma_free, b, s);
}

void recover(dd_ctx* c, const double* f, const double* xg, double* x, cudaStream_t s) {
  launch_elem_interior(c->mesh, ELEM_RECOVER, xg, f, c->w.tI, s);
  launch_kii_apply(c->mesh, c->w.tI, c->w.sI, c->w.err, s);
  launch_scatter_recover(c->mesh, xg, c->w.sI, x, s);
}

// A side stream and the two events that fork work onto it and join it back.
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t f = nullptr, j = nullptr;
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

// BDDC of one level on an interface residual r -> z, with a coarse solver callback.
// The coarse correction (Phi_i^T D_i R_i r, the coarse solve, Phi_i u_C) does not depend on
// the local products N_i D_i R_i r: with a fork it is issued on a high-priority side
// stream, so that its short, latency-bound launches run while the N_i product streams from
// HBM, and the two branches meet before the weighted gather. Each kernel computes the same
// values in either order.
template <class CoarseFn>
void bddc_apply(dd_ctx* c, const DevBDDC& b, const double* r, double* z, double* rloc, double* uloc, double* vloc,
                double* gloc, double* gC, double* uC, CoarseFn coarse, cudaStream_t s, const Fork& fk) {
  launch_restrict(b.n_flat, b.gmap, b.D, r, rloc, s);
  cudaStream_t sc = fk.begin(s);
  launch_bgemv(b.PhiT, b.goff, nullptr, rloc, b.coff, gloc, 1.0, nullptr, sc);  // Phi_i^T D_i R_i r
  launch_gather(b.n_coarse, b.cptr, b.cidx, gloc, nullptr, nullptr, gC, sc);
  coarse(gC, uC, sc);
  launch_bgemv_t(b.PhiT, b.coff, b.cmap, uC, b.goff, vloc, 1.0, nullptr, sc);  // Phi_i R_Ci u_C
  {
    ProfScope pk(c, &b == &c->b1 ? DD_PROF_SYMV_N : DD_PROF_COUNT, s);
    launch_symv(b.N, b.goff, rloc, uloc, c->w.err, s);
  }
  fk.end(s);
  launch_wgather(b.n_gamma, b.gptr, b.gidx, b.D, uloc, vloc, z, s);
}

// three-level: BDDC for the whole coarse system K_C u = g (interior correction, interface BDDC,
// extension). On the coarse branch it is the critical path of the preconditioner, so its
// independent pieces run on two more side streams: u0 = K_II^{-1} g_I beside the interface
// correction and the level-2 BDDC, and the level-3 coarse correction beside the level-2
// local products.
void level2_apply(dd_ctx* c, const double* g, double* u, cudaStream_t s) {
  DevLevel2& L = c->l2;
  Work& w = c->w;
  const bool par = c->s_aux[0] != nullptr;
  const Fork f0{par ? c->s_aux[0] : nullptr, c->ev_aux[0], c->ev_aux[1]};
  const Fork f1{par ? c->s_aux[1] : nullptr, c->ev_aux[2], c->ev_aux[3]};
  launch_map_gather(L.n_int, L.imap, g, w.gI2, s);
  const cudaStream_t s0 = f0.begin(s);
  launch_symv(L.KIIinv, L.ioff, w.gI2, w.u0I2, w.err, s0);
  launch_bgemv_t(L.E, L.ioff, nullptr, w.gI2, L.b.goff, w.rl2, -1.0, nullptr, s);  // -K_GI K_II^{-1} g_I
  launch_gather(L.b.n_gamma, L.b.gptr, L.b.gidx, w.rl2, g, L.gam_c64, w.r2, s);  // g[gam_c] + sum of copies
  bddc_apply(c, L.b, w.r2, w.z2, w.rloc2, w.uloc2, w.vloc2, w.gloc2, w.g3, w.u3,
             [&](const double* g3, double* u3, cudaStream_t ss) { launch_dense_gemv(L.n3, L.b.prec, L.KC3inv, g3, u3, ss); },
             s, f1);
  f0.end(s);
  launch_bgemv(L.E, L.b.goff, L.b.gmap, w.z2, L.ioff, w.uI2, -1.0, w.u0I2, s);  // u0 - K_II^{-1} K_IG z
  launch_map_scatter(L.n_int, L.imap, w.uI2, u, s);
  launch_map_scatter(L.b.n_gamma, L.gam_c, w.z2, u, s);
}

void precond_apply(dd_ctx* c, const double* r, double* z, cudaStream_t s) {
  ProfScope ps(c, DD_PROF_PRECOND, s);
  Work& w = c->w;
  bddc_apply(c, c->b1, r, z, w.rloc, w.uloc, w.vloc, w.gloc, w.gC, w.uC,
             [&](const double* g, double* u, cudaStream_t ss) {
               if (c->levels == 2)
                 launch_dense_gemv(c->b1.n_coarse, c->b1.prec, c->KCinv, g, u, ss);
               else
                 level2_apply(c, g, u, ss);
             },
             s, Fork{c->s_coarse, c->ev_fork, c->ev_join});
}

// z = M^{-1} r as the PCG sees it: without a Dirichlet face the constant interface vector
// is the null-space column of the deflation basis, and z is kept orthogonal to it (its mean
// removed) so the search directions are too
void precond_z(dd_ctx* c, const double* r, double* z, cudaStream_t s) {
  precond_apply(c, r, z, s);
  if (c->neumann) vec_sub_mean(c->n_gamma, z, z, c->partials, s);
}

// Reads the context's device error word (set by a bounded wait that gave up) and clears
// it, so that a failure is reported once and later calls on the context start clean.
void check_err(dd_ctx* c, cudaStream_t s) {
  int e = 0;
  DD_CUDA(cudaMemcpyAsync(&e, c->w.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  if (e) {
    DD_CUDA(cudaMemsetAsync(c->w.err, 0, sizeof(int), s));
    DD_CUDA(cudaStreamSynchronize(s));
    throw Error((dd_status)e, "a bounded device-side wait timed out");
  }
}

template <class F>
dd_status guard(F&& f) {
  try {
    f();
    return DD_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return DD_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return DD_INVALID_ARG;
  }
}

// Work lists of the element passes, one set per distinct pattern of interior /
// interface / absent nodes among the subdomains (a handful: interior subdomains and
// those touching each part of the Dirichlet boundary).
struct WorkLists {
  std::vector<int> sub_type;          // [S]
  std::vector<int> type_off;          // [types][6]
  std::vector<int16_t> items;         // [items][9]
  std::vector<int16_t> bl;            // boundary-layer element ids
  std::vector<int16_t> citems;        // items with slots (position in the type's boundary-layer list) * 8 + corner
  int max_nbl = 0;                    // largest boundary-layer list of a type
};

WorkLists build_work_lists(const Mesh1& M) {
  const int sx = M.sx, sy = M.sy, sz = M.sz, NE = sx * sy * sz;
  DD_REQUIRE(8 * NE <= 32767, "subdomain too large for the element work lists (8 * elements > 32767)");
  WorkLists W;
  W.sub_type.resize(M.S);
  std::map<std::vector<int8_t>, int> types;
  std::vector<int8_t> pat(M.NL);
  for (int s = 0; s < M.S; ++s) {
    const int16_t* code = M.lidx.data() + (size_t)s * M.NL;
    for (int l = 0; l < M.NL; ++l) pat[l] = code[l] >= 0 ? 1 : (code[l] == INT16_MIN ? 0 : 2);
    auto it = types.find(pat);
    if (it != types.end()) {
      W.sub_type[s] = it->second;
      continue;
    }
    const int t = (int)types.size();
    types.emplace(pat, t);
    W.sub_type[s] = t;
    auto node = [&](int a, int b, int c) { return a + M.NLx * (b + M.NLy * c); };
    // boundary-layer elements: at least one interface corner
    std::vector<char> isbl(NE, 0);
    const int bl0 = (int)W.bl.size();
    for (int el = 0; el < NE; ++el) {
      const int ea = el % sx, eb = (el / sx) % sy, ec = el / (sx * sy);
      for (int q = 0; q < 8 && !isbl[el]; ++q)
        if (pat[node(ea + (q & 1), eb + ((q >> 1) & 1), ec + (q >> 2))] == 2) isbl[el] = 1;
      if (isbl[el]) W.bl.push_back((int16_t)el);
    }
    // output items of one pass: nodes of kind `want` with their boundary-layer slots
    auto pass = [&](int want, int& b, int& e) {
      std::vector<std::array<int16_t, 9>> its;
      for (int c = 0; c < M.NLz; ++c)
        for (int bb = 0; bb < M.NLy; ++bb)
          for (int a = 0; a < M.NLx; ++a) {
            const int l = node(a, bb, c);
            if (pat[l] != want) continue;
            std::array<int16_t, 9> it;
            it.fill(-1);
            it[0] = (int16_t)l;
            int k = 0;
            for (int p = 0; p < 8; ++p) {
              const int ea = a - (p & 1), eb = bb - ((p >> 1) & 1), ec = c - (p >> 2);
              if (ea < 0 || eb < 0 || ec < 0 || ea >= sx || eb >= sy || ec >= sz) continue;
              const int el = ea + sx * (eb + sy * ec);
              if (!isbl[el]) continue;
              it[1 + k++] = (int16_t)(el * 8 + p);
            }
            if (k > 0) its.push_back(it);
          }
      auto cnt = [](const std::array<int16_t, 9>& x) {
        int k = 0;
        while (k < 8 && x[1 + k] >= 0) ++k;
        return k;
      };
      std::stable_sort(its.begin(), its.end(), [&](const auto& x, const auto& y) { return cnt(x) > cnt(y); });
      b = (int)(W.items.size() / 9);
      for (auto& x : its) W.items.insert(W.items.end(), x.begin(), x.end());
      e = (int)(W.items.size() / 9);
    };
    int o[6];
    pass(1, o[0], o[1]);
    pass(2, o[2], o[3]);
    o[4] = bl0;
    o[5] = (int)W.bl.size();
    W.type_off.insert(W.type_off.end(), o, o + 6);
    // the same items with each element named by its position in this type's boundary-layer
    // list, so that a kernel can keep the element entries of these elements only
    std::vector<int> blpos(NE, -1);
    for (int t = o[4]; t < o[5]; ++t) blpos[W.bl[t]] = t - o[4];
    W.max_nbl = std::max(W.max_nbl, o[5] - o[4]);
    W.citems.resize(W.items.size());
    for (int i = o[0]; i < o[3]; ++i) {
      W.citems[9 * (size_t)i] = W.items[9 * (size_t)i];
      for (int k = 1; k < 9; ++k) {
        const int16_t v = W.items[9 * (size_t)i + k];
        W.citems[9 * (size_t)i + k] = v < 0 ? v : (int16_t)(blpos[v >> 3] * 8 + (v & 7));
      }
    }
  }
  return W;
}

// mean device time of three launches of f after one warm-up (ms)
template <class F>
float time_launches(F&& f, cudaStream_t s) {
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

// Launch shapes of the two per-iteration kernels that stream the most, timed on this
// context's own operators: the bulk-copy ring depth of the batched symmetric products
// (level-1 N_i, and dense K_II^{-1}) and the block size of the fused Schur kernel.
constexpr int SYMV_WARPS_HOST = 4;  // warps per CTA of k_symv

void tune_shapes(dd_ctx* c, cudaStream_t s) {
  Work& w = c->w;
  DD_CUDA(cudaMemsetAsync(w.rloc, 0, c->b1.n_flat * sizeof(double), s));
  DD_CUDA(cudaMemsetAsync(w.tI, 0, c->mesh.n_int * sizeof(double), s));
  DD_CUDA(cudaMemsetAsync(c->p, 0, c->n_gamma * sizeof(double), s));
  auto tune_sym = [&](SymTiles& A, const int64_t* voff, const double* in, double* out, float* ms) {
    if (A.count < 152) return;  // a small batch leaves most SMs idle whatever the ring depth
    float best = 0.f;
    int pick = 2;
    for (int sl : {2, 3, 4}) {
      A.slots = sl;
      const float t = time_launches([&] { launch_symv(A, voff, in, out, w.err, s); }, s);
      ms[sl - 2] = t;
      if (sl == 2 || t < best) {
        best = t;
        pick = sl;
      }
    }
    A.slots = pick;
  };
  tune_sym(c->b1.N, c->b1.goff, w.rloc, w.uloc, c->info.tune_symv_ms);
  if (c->mesh.local_solver != DD_LOCAL_FDM) tune_sym(c->mesh.KIIinv, c->mesh.ioff, w.tI, w.sI, c->info.tune_kii_ms);
  if (schur_fused_available(c->mesh)) {
    float best = 0.f;
    int pick = 256, i = 0;
    for (int bs : {256, 352, 416}) {
      c->mesh.schur_threads = bs;
      const float t = time_launches([&] { launch_schur_fused(c->mesh, c->p, w.yloc, s); }, s);
      c->info.tune_schur_ms[i++] = t;
      if (bs == 256 || t < best) {
        best = t;
        pick = bs;
      }
    }
    c->mesh.schur_threads = pick;
  }
  // the batched products of the coarse levels (level-1 Phi, level-2 K_II^{-1}, E, N, Phi):
  // rows per block of the row-wise GEMV, row parts of the column-wise GEMV, CTAs per matrix
  // of the symmetric products
  auto zero = [&](void* p, size_t bytes) { if (p && bytes) DD_CUDA(cudaMemsetAsync(p, 0, bytes, s)); };
  auto tune_rows = [&](BatchedRows& B, const int64_t* in_off, const int* in_map, const double* in,
                       const int64_t* out_off, double* out, double alpha, const double* add) {
    if (B.count == 0) return;
    float best = 0.f;
    int pick = 32;
    for (int rpb : {32, 16, 8}) {
      B.rows_per_block = rpb;
      const float t = time_launches([&] { launch_bgemv(B, in_off, in_map, in, out_off, out, alpha, add, s); }, s);
      if (rpb == 32 || t < best) {
        best = t;
        pick = rpb;
      }
    }
    B.rows_per_block = pick;
  };
  // Row parts of the column-wise GEMV and CTAs per matrix of the symmetric products change
  // the order of the sums, so they follow from the sizes alone (never from timings): runs
  // and contexts stay bitwise reproducible. Target: about two blocks per SM.
  auto split_cols = [&](BatchedRows& B) {
    if (B.count == 0) return;
    const int ycols = (B.max_cols + 127) / 128;
    const int want = (2 * 152 + B.count * ycols - 1) / (B.count * ycols);
    B.zsplit = std::max(1, std::min({8, want, B.max_rows / 64}));
    if (B.zsplit > 1 && !B.zpart) {
      const size_t eb = B.prec == DD_PREC_FP32 ? 4 : 8;
      B.zpart = c->arena.alloc<unsigned char>((size_t)B.count * ycols * 8 * 128 * eb);
      B.zticket = c->arena.alloc<unsigned>((size_t)B.count * ycols);
      zero(B.zticket, (size_t)B.count * ycols * sizeof(unsigned));
    }
  };
  auto split_sym = [&](SymTiles& A) {
    if (A.count == 0 || A.count >= 152) return;
    const int nb = (A.max_n + 31) / 32;
    const int want = (2 * 152 + A.count - 1) / A.count;
    A.split = std::max(1, std::min({8, want, nb * (nb + 1) / 2 / SYMV_WARPS_HOST}));
    if (A.split > 1 && !A.spart) {
      const int maxpad = nb * 32;
      A.spart = c->arena.alloc<unsigned char>((size_t)A.count * 8 * maxpad * 8);
      A.sticket = c->arena.alloc<unsigned>((size_t)A.count);
      zero(A.sticket, (size_t)A.count * sizeof(unsigned));
    }
  };
  zero(w.uC, c->b1.n_coarse * sizeof(double));
  tune_rows(c->b1.PhiT, c->b1.goff, nullptr, w.rloc, c->b1.coff, w.gloc, 1.0, nullptr);
  split_cols(c->b1.PhiT);
  if (c->levels == 3) {
    DevLevel2& L = c->l2;
    zero(w.z2, L.b.n_gamma * sizeof(double));
    zero(w.u0I2, L.n_int * sizeof(double));
    zero(w.rloc2, L.b.n_flat * sizeof(double));
    split_cols(L.E);
    tune_rows(L.E, L.b.goff, L.b.gmap, w.z2, L.ioff, w.uI2, -1.0, w.u0I2);
    tune_rows(L.b.PhiT, L.b.goff, nullptr, w.rloc2, L.b.coff, w.gloc2, 1.0, nullptr);
    split_cols(L.b.PhiT);
    split_sym(L.KIIinv);
    split_sym(L.b.N);
  }
  c->info.symv_slots = c->b1.N.slots;
  c->info.schur_threads = schur_fused_available(c->mesh) ? c->mesh.schur_threads : 0;
  check_err(c, s);
}

}  // namespace dd

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* dd_last_error(void) { return g_last_error.c_str(); }

dd_status dd_default_options(dd_options* o) {
  if (!o) return DD_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->levels = 3;
  o->coarse_group = 4;
  o->use_corners = o->use_edges = o->use_faces = 1;
  o->adaptive = 0;
  o->tau = 10.0;
  o->max_eig_per_face = 10;
  o->weights = DD_WEIGHTS_DIAG;
  o->precond_prec = DD_PREC_FP64;
  o->schur_prec = DD_PREC_FP64;
  o->flexible = 0;
  o->reorth = 0;
  o->stop_rhs_norm = 1;
  o->maxit = 500;
  o->local_solver = DD_LOCAL_AUTO;
  o->ens_nmm = DD_ENS_AUTO;
  o->ens_elem_rc = 0;
  o->ens_fdm_rc = 0;
  o->loop_graph = 1;
  o->zero_initial_guess = 0;
  o->adaptive_solver = DD_EIG_DENSE;
  o->lobpcg_iters = 15;
  return DD_OK;
}

void dd_abi_struct_sizes(size_t* sizes) {
  if (!sizes) return;
  sizes[0] = sizeof(dd_mesh_desc);
  sizes[1] = sizeof(dd_options);
  sizes[2] = sizeof(dd_info_t);
  sizes[3] = sizeof(dd_stats);
  sizes[4] = sizeof(dd_kernel_prof);
}

dd_status dd_setup(const dd_mesh_desc* md, const dd_options* opt, void* stream, dd_ctx** out) {
  if (!md || !opt || !out) {
    g_last_error = "dd_setup: NULL argument";
    return DD_INVALID_ARG;
  }
  *out = nullptr;
  return guard([&] {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    DD_REQUIRE(opt->precond_prec == DD_PREC_FP64 || opt->precond_prec == DD_PREC_FP32,
               "precond_prec must be FP64 or FP32");
    DD_REQUIRE(opt->schur_prec == DD_PREC_FP64 || opt->schur_prec == DD_PREC_DF64, "schur_prec must be FP64 or DF64");
    DD_REQUIRE(opt->maxit >= 1, "maxit must be positive");
    DD_REQUIRE(opt->ens_nmm >= DD_ENS_AUTO && opt->ens_nmm <= DD_ENS_BF16X3,
               "ens_nmm must be AUTO, SIMT, TC or BF16X3");
    DD_REQUIRE(opt->ens_elem_rc == 0 || opt->ens_elem_rc == 4 || opt->ens_elem_rc == 8 || opt->ens_elem_rc == 16,
               "ens_elem_rc must be 0, 4, 8 or 16");
    DD_REQUIRE(opt->ens_fdm_rc == 0 || opt->ens_fdm_rc == 4 || opt->ens_fdm_rc == 8, "ens_fdm_rc must be 0, 4 or 8");
    DD_REQUIRE(opt->loop_graph == 0 || opt->loop_graph == 1, "loop_graph must be 0 or 1");
    DD_REQUIRE(opt->zero_initial_guess == 0 || opt->zero_initial_guess == 1, "zero_initial_guess must be 0 or 1");
    auto H = std::make_unique<HostSetup>();
    build_host_setup(*md, *opt, *H);
    auto c = std::make_unique<dd_ctx>();
    c->opt = *opt;
    c->levels = H->levels;
    c->neumann = H->neumann;
    const Mesh1& M = H->mesh;
    DeviceArena& A = c->arena;
    c->n_free = M.n_free;
    if (c->neumann) c->fc = A.alloc<double>((size_t)std::max<int64_t>(M.n_free, 1));
    c->n_gamma = H->l1.n_gamma;
    c->gamma_free_host = M.gamma_free;
    // ---- level-1 mesh / Schur operator ----
    DevMesh& dm = c->mesh;
    std::vector<double> elem_madds, elem_nbl;  // per subdomain type (for the profiling counts)
    std::vector<int> elem_type;
    dm.nx = M.nx; dm.ny = M.ny; dm.nz = M.nz; dm.sx = M.sx; dm.sy = M.sy; dm.sz = M.sz;
    dm.Sx = M.Sx; dm.Sy = M.Sy; dm.Sz = M.Sz; dm.S = M.S;
    dm.fx0 = M.fx0; dm.fx1 = M.fx1; dm.fy0 = M.fy0; dm.fy1 = M.fy1; dm.fz0 = M.fz0; dm.fz1 = M.fz1;
    dm.NLx = M.NLx; dm.NLy = M.NLy; dm.NLz = M.NLz; dm.NL = M.NL;
    dm.n_free = M.n_free;
    dm.n_gamma = H->l1.n_gamma;
    dm.n_int = H->l1.ioff[M.S];
    dm.n_flat = H->l1.goff[M.S];
    dm.schur_prec = opt->schur_prec;
    dm.lidx = A.upload(M.lidx, s);
    {
      WorkLists W = build_work_lists(M);
      // multiply-adds of the element passes of one Schur application per subdomain type
      // (8 per occupied slot of an output item) and the elements whose entries are formed
      const int ntypes = (int)W.type_off.size() / 6;
      elem_madds.assign(ntypes, 0.0);
      elem_nbl.assign(ntypes, 0.0);
      for (int t = 0; t < ntypes; ++t) {
        const int* o = W.type_off.data() + 6 * t;
        for (int i = o[0]; i < o[3]; ++i)
          for (int k = 1; k < 9; ++k) elem_madds[t] += W.items[9 * (size_t)i + k] >= 0 ? 8.0 : 0.0;
        elem_nbl[t] = o[5] - o[4];
      }
      elem_type = W.sub_type;
      dm.sub_type = A.upload(W.sub_type, s);
      dm.type_off = A.upload(W.type_off, s);
      dm.type_items = A.upload(W.items, s);
      dm.type_bl = A.upload(W.bl, s);
      dm.type_citems = A.upload(W.citems, s);
      dm.max_nbl = W.max_nbl;
      for (int i = 0; i < M.S; ++i)
        dm.max_nint = std::max(dm.max_nint, (int)(H->l1.ioff[i + 1] - H->l1.ioff[i]));
      dm.schur_threads = 256;
      if (H->local_solver == DD_LOCAL_FDM && M.sx == 8 && M.sy == 8 && M.sz == 8) {
        // the fused Schur kernel's per-subdomain copies: each local node's interface index, and
        // the factors of the boundary-layer elements in the order of the type's list
        std::vector<int> sxg((size_t)M.S * M.NL, -1);
        std::vector<double> sf((size_t)M.S * W.max_nbl * 3, 0.0);
        for (int i = 0; i < M.S; ++i) {
          const int16_t* code = M.lidx.data() + (size_t)i * M.NL;
          for (int l = 0; l < M.NL; ++l)
            if (code[l] < 0 && code[l] != INT16_MIN)
              sxg[(size_t)i * M.NL + l] = H->l1.gmap[H->l1.goff[i] + (-1 - code[l])];
          const int* o = W.type_off.data() + 6 * W.sub_type[i];
          const int I = i % M.Sx, J = (i / M.Sx) % M.Sy, K = i / (M.Sx * M.Sy);
          for (int t = o[4]; t < o[5]; ++t) {
            const int el = W.bl[t], ea = el % M.sx, eb = (el / M.sx) % M.sy, ec = el / (M.sx * M.sy);
            const size_t e = (size_t)(I * M.sx + ea) + (size_t)M.nx * ((J * M.sy + eb) + (size_t)M.ny * (K * M.sz + ec));
            double* d = sf.data() + ((size_t)i * W.max_nbl + (t - o[4])) * 3;
            d[0] = M.ecx[e];
            d[1] = M.ecy[e];
            d[2] = M.ecz[e];
          }
        }
        dm.sxg = A.upload(sxg, s);
        if (opt->schur_prec == DD_PREC_DF64) {
          std::vector<df64> sfd(sf.size());
          for (size_t t = 0; t < sf.size(); ++t) sfd[t] = df64_from_double(sf[t]);
          dm.sfac = A.upload(sfd, s);
        } else {
          dm.sfac = A.upload(sf, s);
        }
      }
    }
    dm.ioff = A.upload(H->l1.ioff, s);
    dm.goff = A.upload(H->l1.goff, s);
    dm.gmap = A.upload(H->l1.gmap, s);
    dm.gptr = A.upload(H->l1.gptr, s);
    dm.gidx = A.upload(H->l1.gidx, s);
    dm.gamma_free = A.upload(M.gamma_free, s);
    {
      size_t E = M.ecx.size();
      std::vector<double> ec(3 * E);
      std::vector<df64> ecd(3 * E);
      for (size_t e = 0; e < E; ++e) {
        ec[3 * e] = M.ecx[e]; ec[3 * e + 1] = M.ecy[e]; ec[3 * e + 2] = M.ecz[e];
        for (int t = 0; t < 3; ++t) ecd[3 * e + t] = df64_from_double(ec[3 * e + t]);
      }
      dm.ec = A.upload(ec, s);
      dm.ec_df = A.upload(ecd, s);
      std::vector<double> kc(E, 1.0);  // E = number of elements
      if (md->coef) std::copy(md->coef, md->coef + E, kc.begin());
      dm.coef = A.upload(kc, s);
    }
    dm.local_solver = H->local_solver;
    if (H->local_solver == DD_LOCAL_FDM) {
      // 1D eigenbases padded to 9x9 per axis, and D^{-1} indexed like the interior vectors
      std::vector<int> fn((size_t)3 * M.S);
      std::vector<double> Vd((size_t)243 * M.S, 0.0), Dd((size_t)dm.n_int);
      for (int i = 0; i < M.S; ++i) {
        const FdmSub& F = H->fdm[i];
        for (int a = 0; a < 3; ++a) {
          fn[3 * i + a] = F.n[a];
          for (int r = 0; r < F.n[a]; ++r)
            for (int q = 0; q < F.n[a]; ++q) Vd[(size_t)243 * i + 81 * a + 9 * r + q] = F.V[a][(size_t)r * F.n[a] + q];
        }
        std::copy(F.Dinv.begin(), F.Dinv.end(), Dd.begin() + H->l1.ioff[i]);
      }
      dm.fdm_n = A.upload(fn, s);
      if (opt->schur_prec == DD_PREC_DF64) {
        std::vector<df64> Vf(Vd.size()), Df(Dd.size());
        for (size_t t = 0; t < Vd.size(); ++t) Vf[t] = df64_from_double(Vd[t]);
        for (size_t t = 0; t < Dd.size(); ++t) Df[t] = df64_from_double(Dd[t]);
        dm.fdm_V = A.upload(Vf, s);
        dm.fdm_Dinv = A.upload(Df, s);
      } else {
        dm.fdm_V = A.upload(Vd, s);
        dm.fdm_Dinv = A.upload(Dd, s);
      }
      dm.KIIinv.count = 0;
    } else {
      std::vector<const double*> mats;
      std::vector<int> dims;
      for (int i = 0; i < M.S; ++i) {
        mats.push_back(H->l1.sub[i].KIIinv.data());
        dims.push_back(H->l1.sub[i].nI);
      }
      dm.KIIinv = upload_sym(A, mats, dims, opt->schur_prec == DD_PREC_DF64 ? DD_PREC_DF64 : DD_PREC_FP64, s);
    }
    // ---- level-1 BDDC ----
    upload_bddc(A, H->l1, opt->precond_prec, c->b1, s);
    int pp = opt->precond_prec;
    Work& w = c->w;
    w.tI = A.alloc<double>(dm.n_int);
    w.sI = A.alloc<double>(dm.n_int);
    w.yloc = A.alloc<double>(c->b1.n_flat);
    w.rloc = A.alloc<double>(c->b1.n_flat);
    w.uloc = A.alloc<double>(c->b1.n_flat);
    w.vloc = A.alloc<double>(c->b1.n_flat);
    w.gloc = A.alloc<double>(c->b1.n_cflat);
    w.gC = A.alloc<double>(c->b1.n_coarse);
    w.uC = A.alloc<double>(c->b1.n_coarse);
    w.err = A.alloc<int>(1);
    DD_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
    if (c->levels == 2) {
      c->KCinv = upload_dense(A, H->KCinv, pp);
    } else {
      DevLevel2& L = c->l2;
      upload_bddc(A, H->l2, pp, L.b, s);
      L.n_int = H->l2.ioff[H->l2.S];
      L.ioff = A.upload(H->l2.ioff, s);
      L.imap = A.upload(H->imap2, s);
      L.gam_c = A.upload(H->gam2_c, s);
      L.gam_c64 = A.upload(std::vector<int64_t>(H->gam2_c.begin(), H->gam2_c.end()), s);
      std::vector<const double*> Ks, Es;
      std::vector<int> nI, nG;
      for (int j = 0; j < H->l2.S; ++j) {
        Ks.push_back(H->l2.sub[j].KIIinv.data());
        Es.push_back(H->l2.sub[j].E.data());
        nI.push_back(H->l2.sub[j].nI);
        nG.push_back(H->l2.sub[j].nG);
      }
      L.KIIinv = upload_sym(A, Ks, nI, pp == DD_PREC_FP32 ? DD_PREC_FP32 : DD_PREC_FP64, s);
      L.E = upload_rows(A, Es, nI, nG, pp == DD_PREC_FP32 ? DD_PREC_FP32 : DD_PREC_FP64, false, s);
      L.n3 = H->l2.n_coarse;
      L.KC3inv = upload_dense(A, H->KC3inv, pp);
      w.gI2 = A.alloc<double>(L.n_int);
      w.u0I2 = A.alloc<double>(L.n_int);
      w.uI2 = A.alloc<double>(L.n_int);
      w.rl2 = A.alloc<double>(L.b.n_flat);
      w.rloc2 = A.alloc<double>(L.b.n_flat);
      w.uloc2 = A.alloc<double>(L.b.n_flat);
      w.vloc2 = A.alloc<double>(L.b.n_flat);
      w.r2 = A.alloc<double>(L.b.n_gamma);
      w.z2 = A.alloc<double>(L.b.n_gamma);
      w.gloc2 = A.alloc<double>(L.b.n_cflat);
      w.g3 = A.alloc<double>(L.n3);
      w.u3 = A.alloc<double>(L.n3);
    }
    // ---- Krylov buffers ----
    int64_t nG = c->n_gamma;
    c->xg = A.alloc<double>(nG);
    c->r = A.alloc<double>(nG);
    c->z = A.alloc<double>(nG);
    c->zold = A.alloc<double>(nG);
    c->p = A.alloc<double>(nG);
    c->q = A.alloc<double>(nG);
    c->bvec = A.alloc<double>(nG);
    c->tmp = A.alloc<double>(nG);
    c->sc = A.alloc<double>(SC_COUNT);
    c->ctl = A.alloc<LoopCtl>(1);
    c->alphas = A.alloc<double>((size_t)opt->maxit);
    c->partials = A.alloc<double>(NBLK * MAXDOT);
    c->wpart = A.alloc<double>((size_t)std::max<int64_t>(NBLK, defl_df_part_rows(c->n_gamma)) * MAXK);
    c->mu = A.alloc<double>(MAXK);
    c->fticket = A.alloc<unsigned>(1);
    DD_CUDA(cudaMemsetAsync(c->fticket, 0, sizeof(unsigned), s));
    c->wticket = A.alloc<unsigned>(defl_df_tickets(c->n_gamma));
    DD_CUDA(cudaMemsetAsync(c->wticket, 0, defl_df_tickets(c->n_gamma) * sizeof(unsigned), s));
    c->gram_part = A.alloc<double>((size_t)NBLK * 4096);
    c->gram_out = A.alloc<double>(4096);
    c->ybuf = A.alloc<double>(128 * 128);
    c->ptrs = A.alloc<const double*>(512);
    DD_CUDA(cudaMallocHost(&c->sc_host, SC_COUNT * sizeof(double)));
    DD_CUDA(cudaMallocHost(&c->ctl_host, sizeof(LoopCtl)));
    DD_CUDA(cudaEventCreate(&c->ev0));
    DD_CUDA(cudaEventCreate(&c->ev1));
    {
      int least = 0, greatest = 0;
      DD_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      DD_CUDA(cudaStreamCreateWithPriority(&c->s_coarse, cudaStreamNonBlocking, greatest));
      DD_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      DD_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
      for (auto& a : c->s_aux) DD_CUDA(cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, greatest));
      for (auto& e : c->ev_aux) DD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    DD_CUDA(cudaStreamSynchronize(s));
    {
      // algorithmic bytes of one K_II^{-1} application: the operator data read once and the
      // vectors in and out (dense: packed triangles; FDM: 1D eigenbases and D^{-1})
      double kii = 0, nn = 0, nne = 0;
      for (int i = 0; i < M.S; ++i) {
        double a = H->l1.sub[i].nI, g = H->l1.sub[i].nG;
        if (H->local_solver == DD_LOCAL_FDM) {
          const FdmSub& F = H->fdm[i];
          kii += (F.n[0] * F.n[0] + F.n[1] * F.n[1] + F.n[2] * F.n[2]) * 8.0 + a * 8.0 + 2 * a * 8.0;
        } else {
          kii += a * (a + 1) / 2 * 8.0 + 2 * a * 8.0;
        }
        nn += g * (g + 1) / 2 * (pp == DD_PREC_FP32 ? 4.0 : 8.0) + 2 * g * 8.0;
        // ensemble: the same matrix once, the members' vectors in the preconditioner type
        nne += g * (g + 1) / 2 * (pp == DD_PREC_FP32 ? 4.0 : 8.0) + 2 * g * BW * (pp == DD_PREC_FP32 ? 4.0 : 8.0);
      }
      c->prof_bytes[DD_PROF_SYMV_KII] = kii;
      c->prof_bytes[DD_PROF_SYMV_N] = nn;
      c->prof_bytes[DD_PROF_ENS_N] = nne;
      // Schur application: multiply-adds of the element passes and of K_II^{-1} (fast
      // diagonalization: six 1D contractions and the diagonal; dense: the symmetric product),
      // and the data it must stream: x, the element factors of the boundary-layer elements,
      // the K_II^{-1} data, the local maps, the local results and the assembled y
      double sm = 0.0, sb = 0.0;
      const double n_flat = (double)H->l1.goff[M.S], n_g = (double)c->n_gamma;
      for (int i = 0; i < M.S; ++i) {
        const int t = elem_type[i];
        sm += elem_madds[t];
        sb += elem_nbl[t] * 3 * 8.0 + M.NL * 2.0;
        const double a = H->l1.sub[i].nI;
        if (H->local_solver == DD_LOCAL_FDM) {
          const FdmSub& F = H->fdm[i];
          sm += 2.0 * a * (F.n[0] + F.n[1] + F.n[2]) + a;
          sb += 243 * 8.0 + a * 8.0;
        } else {
          sm += a * a;
          sb += a * (a + 1) / 2 * 8.0;
        }
      }
      sb += n_g * 8.0 + n_flat * (8.0 + 4.0) + n_flat * (8.0 + 8.0 + 4.0) + n_g * (8.0 + 4.0);
      c->prof_flops[DD_PROF_SCHUR] = 2.0 * sm;
      c->prof_bytes[DD_PROF_SCHUR] = sb;
      // BDDC application: every operator once per use (N_i packed, Phi^T twice, and at three
      // levels K_II^{-1} packed, E twice, N, Phi^T twice, dense K_C3^{-1}) and the vectors
      // (r, z and the local and coarse copies, 8 bytes each)
      auto level_bytes = [&](const Level& L, int prec) {
        const double eb = prec == DD_PREC_FP32 ? 4.0 : 8.0;
        const double lf = (double)L.goff[L.S], lc = (double)L.coff[L.S];
        double b = 0.0;
        for (int i = 0; i < L.S; ++i) {
          const double g = L.sub[i].nG, nc = L.sub[i].nc;
          b += g * (g + 1) / 2 * eb + 2.0 * g * nc * eb;
        }
        return b + 8.0 * (3.0 * (double)L.n_gamma + 6.0 * lf + 3.0 * lc);
      };
      double pb = level_bytes(H->l1, pp);
      if (c->levels == 3) {
        const double eb = pp == DD_PREC_FP32 ? 4.0 : 8.0;
        pb += level_bytes(H->l2, pp);
        for (int j = 0; j < H->l2.S; ++j) {
          const double a = H->l2.sub[j].nI, g = H->l2.sub[j].nG;
          pb += a * (a + 1) / 2 * eb + 2.0 * a * g * eb + 8.0 * 4.0 * a;
        }
        pb += (double)H->l2.n_coarse * H->l2.n_coarse * eb;
      } else {
        pb += (double)H->l1.n_coarse * H->l1.n_coarse * (pp == DD_PREC_FP32 ? 4.0 : 8.0);
      }
      c->prof_bytes[DD_PROF_PRECOND] = pb;
    }
    c->info.n_free = c->n_free;
    c->info.n_gamma = c->n_gamma;
    c->info.n_sub = M.S;
    c->info.n_coarse = H->l1.n_coarse;
    c->info.n_adaptive = H->l1.n_adaptive;
    c->info.n_sub2 = c->levels == 3 ? H->l2.S : 0;
    c->info.n_coarse3 = c->levels == 3 ? H->l2.n_coarse : 0;
    c->info.local_solver = H->local_solver;
    c->info.neumann = c->neumann ? 1 : 0;
    tune_shapes(c.get(), s);
    c->info.device_bytes = (int64_t)A.bytes;
    c->info.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = c.release();
  });
}

void dd_destroy(dd_ctx* c) { delete c; }

dd_status dd_plan(const dd_mesh_desc* md, const dd_options* opt, dd_info_t* info, int64_t* nodes,
                  int64_t capacity) {
  if (!md || !opt || !info) {
    g_last_error = "dd_plan: NULL argument";
    return DD_INVALID_ARG;
  }
  return guard([&] {
    DD_REQUIRE(!(opt->adaptive && opt->adaptive_solver == DD_EIG_LOBPCG),
               "dd_plan: adaptive_solver LOBPCG runs on the device (use dd_setup)");
    HostSetup H;
    build_host_setup(*md, *opt, H);
    std::memset(info, 0, sizeof(*info));
    info->n_free = H.mesh.n_free;
    info->n_gamma = H.l1.n_gamma;
    info->n_sub = H.mesh.S;
    info->n_coarse = H.l1.n_coarse;
    info->n_adaptive = H.l1.n_adaptive;
    info->neumann = H.neumann ? 1 : 0;
    info->n_sub2 = H.levels == 3 ? H.l2.S : 0;
    info->n_coarse3 = H.levels == 3 ? H.l2.n_coarse : 0;
    info->local_solver = H.local_solver;
    info->setup_seconds = H.setup_seconds;
    if (nodes) {
      DD_REQUIRE(capacity >= H.l1.n_gamma, "dd_plan: node buffer too small");
      std::copy(H.mesh.gamma_free.begin(), H.mesh.gamma_free.end(), nodes);
    }
  });
}

dd_status dd_get_info(const dd_ctx* c, dd_info_t* info) {
  if (!c || !info) return DD_INVALID_ARG;
  *info = c->info;
  if (c->bw) {
    info->ens_nmm = c->bw->op[BOP_N1].kind;
    for (int v = 0; v < 3; ++v) info->ens_nmm_ms[v] = c->bw->op[BOP_N1].ms[v];
    info->ens_elem_rc = c->bw->elem_rc;
    info->ens_fdm_rc = c->bw->fdm_rc;
  }
  return DD_OK;
}

dd_status dd_interface_nodes(const dd_ctx* c, int64_t* nodes) {
  if (!c || !nodes) return DD_INVALID_ARG;
  std::copy(c->gamma_free_host.begin(), c->gamma_free_host.end(), nodes);
  return DD_OK;
}

dd_status dd_schur_apply(dd_ctx* c, const double* x, double* y, void* stream) {
  if (!c || !x || !y) return DD_INVALID_ARG;
  return guard([&] { schur_apply(c, x, y, (cudaStream_t)stream); check_err(c, (cudaStream_t)stream); });
}

dd_status dd_precond_apply(dd_ctx* c, const double* r, double* z, void* stream) {
  if (!c || !r || !z) return DD_INVALID_ARG;
  return guard([&] { precond_apply(c, r, z, (cudaStream_t)stream); check_err(c, (cudaStream_t)stream); });
}

dd_status dd_condense(dd_ctx* c, const double* f, double* b, void* stream) {
  if (!c || !f || !b) return DD_INVALID_ARG;
  return guard([&] { condense(c, f, b, (cudaStream_t)stream); check_err(c, (cudaStream_t)stream); });
}

dd_status dd_recover(dd_ctx* c, const double* f, const double* xg, double* x, void* stream) {
  if (!c || !f || !xg || !x) return DD_INVALID_ARG;
  return guard([&] { recover(c, f, xg, x, (cudaStream_t)stream); check_err(c, (cudaStream_t)stream); });
}

dd_status dd_selftest_bounded_wait(dd_ctx* c, int64_t polls, void* stream) {
  if (!c || polls < 1) {
    g_last_error = "dd_selftest_bounded_wait: invalid argument";
    return DD_INVALID_ARG;
  }
  return guard([&] {
    launch_wait_selftest(c->w.err, (long long)polls, (cudaStream_t)stream);
    check_err(c, (cudaStream_t)stream);
  });
}

dd_status dd_recycle_create(dd_ctx* c, int32_t k, int32_t strategy, double freeze_tol, dd_recycle** out) {
  if (!c || !out || k < 0 || k > MAXK - 1 || strategy < DD_B1 || strategy > DD_B4) {
    g_last_error = "dd_recycle_create: invalid argument";
    return DD_INVALID_ARG;
  }
  return guard([&] {
    auto st = std::make_unique<dd_recycle>();
    st->ctx = c;
    st->kmax = k;
    st->strategy = strategy;
    st->freeze_tol = freeze_tol;
    int64_t n = c->n_gamma;
    st->xg_prev = st->arena.alloc<double>(n);
    DD_CUDA(cudaMemset(st->xg_prev, 0, n * sizeof(double)));
    if (k > 0) {
      st->W = st->arena.alloc<double>((size_t)k * n);
      st->AW = st->arena.alloc<double>((size_t)k * n);
      st->MAW = st->arena.alloc<double>((size_t)k * n);
      st->W2 = st->arena.alloc<double>((size_t)k * n);
      st->AW2 = st->arena.alloc<double>((size_t)k * n);
      st->MAW2 = st->arena.alloc<double>((size_t)k * n);
      st->Wd = st->arena.alloc<df64>((size_t)k * n);
      st->AWd = st->arena.alloc<df64>((size_t)k * n);
      st->Ginv = st->arena.alloc<double>((size_t)k * k);
      st->WWinv = st->arena.alloc<double>((size_t)k * k);
      st->hmax = std::min(c->opt.maxit + 1, std::max(16, 128 - k));
      st->P = st->arena.alloc<double>((size_t)st->hmax * n);
      st->AP = st->arena.alloc<double>((size_t)st->hmax * n);
      st->Z = st->arena.alloc<double>((size_t)(st->hmax + 1) * n);
      st->MAP = st->arena.alloc<double>((size_t)st->hmax * n);
    }
    *out = st.release();
  });
}

void dd_recycle_destroy(dd_recycle* st) { delete st; }

}  // extern "C"

// ---------------------------------------------------------------------------
// deflated PCG (Algorithm 1) and the recycling update
// ---------------------------------------------------------------------------
namespace dd {

// df64 copies of the basis used by the deflation kernels
void refresh_df(dd_ctx* c, dd_recycle* st, cudaStream_t s) {
  if (st->k == 0) return;
  const int64_t kn = (int64_t)st->k * c->n_gamma;
  to_df64(kn, st->W, st->Wd, s);
  to_df64(kn, st->AW, st->AWd, s);
}

// With an FP32 preconditioner the per-iteration update p = z + beta p - W mu streams the
// basis as FP32: W is rounded to FP32-representable values (another basis of the same span
// up to rounding; deflation is exact for whichever basis it uses) and A W is recomputed for
// the rounded basis by the Schur operator (df64), so that the projection stays exact for
// the stored W. Single sequences only (the ensemble streams W in df64). Returns whether W
// changed; with `force` A W is recomputed in any case.
bool use_f32_basis(const dd_ctx* c, const dd_recycle* st) {
  return c->opt.precond_prec == DD_PREC_FP32 && st->nrhs == 0;
}
bool basis_to_f32(dd_ctx* c, dd_recycle* st, cudaStream_t s, bool force) {
  const int64_t n = c->n_gamma;
  const int k = st->k;
  if (!st->Wf) {
    st->Wf = st->arena.alloc<float>((size_t)st->kmax * n);
    st->rflag = st->arena.alloc<int>(1);
  }
  DD_CUDA(cudaMemsetAsync(st->rflag, 0, sizeof(int), s));
  round_to_f32((int64_t)k * n, st->W, st->Wf, st->rflag, s);
  int changed = 0;
  DD_CUDA(cudaMemcpyAsync(&changed, st->rflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  if (changed || force)
    for (int j = 0; j < k; ++j) schur_apply(c, st->W + (size_t)j * n, st->AW + (size_t)j * n, s);
  st->wf_valid = true;
  return changed != 0;
}

// Device work space of the recycling update, allocated once per recycle state.
void recycle_work(dd_recycle* st) {
  if (st->rptr) return;
  st->rptr = st->arena.alloc<void*>(REC_PTRS);
  st->rblk = st->arena.alloc<short2>(3 * REC_BLOCKS);
  st->rpart = st->arena.alloc<double>((size_t)REC_CHUNKS * REC_BLOCKS * 16);
  st->rout = st->arena.alloc<double>((size_t)2 * REC_BLOCKS * 16);
  st->rY = st->arena.alloc<double>((size_t)REC_MAXM * REC_MAXM);
  st->ralpha = st->arena.alloc<double>(REC_MAXM);
}

// Host image of the pointer table and block lists, uploaded with one copy.
struct RecTables {
  std::vector<void*> ptr = std::vector<void*>(REC_PTRS, nullptr);
  std::vector<short2> blk = std::vector<short2>(3 * REC_BLOCKS, short2{0, 0});
  void upload(dd_recycle* st, cudaStream_t s) {
    DD_CUDA(cudaMemcpyAsync(st->rptr, ptr.data(), ptr.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
    DD_CUDA(cudaMemcpyAsync(st->rblk, blk.data(), blk.size() * sizeof(short2), cudaMemcpyHostToDevice, s));
  }
};

// Scatters the upper 4 x 4 blocks of a Gram product into the full symmetric m x m matrix.
void blocks_to_sym(int m, const std::vector<short2>& q, const double* vals, std::vector<double>& M) {
  for (size_t t = 0; t < q.size(); ++t)
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) {
        const int a = 4 * q[t].x + u, b = 4 * q[t].y + v;
        if (a >= m || b >= m || a > b) continue;
        M[(size_t)a * m + b] = M[(size_t)b * m + a] = vals[t * 16 + 4 * u + v];
      }
}

// G = W^T A W (symmetric, df64 products) and its inverse; with re-orthogonalization also
// (W^T W)^{-1}. The df64 copies of W and A W used by the deflation kernels are refreshed
// unless the caller wrote them already.
void refresh_gram(dd_ctx* c, dd_recycle* st, cudaStream_t s, bool df_done = false) {
  const int k = st->k;
  st->G_host.clear();
  if (k == 0) return;
  recycle_work(st);
  const int64_t n = c->n_gamma;
  RecTables tab;
  for (int j = 0; j < k; ++j) {
    tab.ptr[j] = (void*)(st->W + (size_t)j * n);
    tab.ptr[REC_MAXM + j] = (void*)(st->AW + (size_t)j * n);
  }
  const std::vector<short2> q = gram_block_list(k, 0);
  std::copy(q.begin(), q.end(), tab.blk.begin());
  tab.upload(st, s);
  const double* const* P = reinterpret_cast<const double* const*>(st->rptr);
  gram_blocks(n, k, P, P + REC_MAXM, st->rblk, (int)q.size(), true, st->rpart, st->rout, s);
  const bool reo = c->opt.reorth != 0;
  if (reo) gram_blocks(n, k, P, P, st->rblk, (int)q.size(), true, st->rpart, st->rout + REC_BLOCKS * 16, s);
  std::vector<double> hv((size_t)2 * REC_BLOCKS * 16);
  DD_CUDA(cudaMemcpyAsync(hv.data(), st->rout, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  std::vector<double> G((size_t)k * k, 0.0), Gi((size_t)k * k);
  blocks_to_sym(k, q, hv.data(), G);
  if (!la::spd_inverse(k, G.data(), Gi.data())) {
    // basis numerically dependent: drop it (plain PCG until it is rebuilt)
    st->k = 0;
    return;
  }
  st->G_host = G;
  DD_CUDA(cudaMemcpyAsync(st->Ginv, Gi.data(), Gi.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (reo) {
    std::vector<double> WW((size_t)k * k, 0.0), WWi((size_t)k * k);
    blocks_to_sym(k, q, hv.data() + REC_BLOCKS * 16, WW);
    if (!la::spd_inverse(k, WW.data(), WWi.data())) {
      st->k = 0;
      st->G_host.clear();
      return;
    }
    DD_CUDA(cudaMemcpyAsync(st->WWinv, WWi.data(), WWi.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (!df_done) refresh_df(c, st, s);
  DD_CUDA(cudaStreamSynchronize(s));
}

// Recycling after a solve with l search vectors (Sect. 4.2).
void recycle_update(dd_ctx* c, dd_recycle* st, int l, cudaStream_t s) {
  st->step++;
  if (st->kmax == 0 || st->frozen || l == 0) return;
  int64_t n = c->n_gamma;
  int R = st->kmax;
  l = std::min(l, st->hmax);
  if (st->strategy == DD_B1 || st->strategy == DD_B2) {
    // basis of search vectors (B1: first R, then frozen; B2: last R)
    std::vector<const double*> Vs, AVs;
    for (int j = 0; j < st->k; ++j) {
      Vs.push_back(st->W + (size_t)j * n);
      AVs.push_back(st->AW + (size_t)j * n);
    }
    for (int j = 0; j < l; ++j) {
      Vs.push_back(st->P + (size_t)j * n);
      AVs.push_back(st->AP + (size_t)j * n);
    }
    int m = (int)Vs.size();
    int first = (st->strategy == DD_B1) ? 0 : std::max(0, m - R);
    int last = (st->strategy == DD_B1) ? std::min(m, R) : m;
    int kn = last - first;
    for (int j = 0; j < kn; ++j) {
      DD_CUDA(cudaMemcpyAsync(st->W2 + (size_t)j * n, Vs[first + j], n * 8, cudaMemcpyDeviceToDevice, s));
      DD_CUDA(cudaMemcpyAsync(st->AW2 + (size_t)j * n, AVs[first + j], n * 8, cudaMemcpyDeviceToDevice, s));
    }
    std::swap(st->W, st->W2);
    std::swap(st->AW, st->AW2);
    st->k = kn;
    st->wf_valid = false;
    if (st->strategy == DD_B1 && kn >= R) st->frozen = true;
    refresh_gram(c, st, s);
    return;
  }
  // B3 / B4: harmonic Ritz vectors of V = [W, P]  (eq. 15)
  recycle_work(st);
  const int k = st->k;
  const int m = k + l;
  DD_REQUIRE(m <= REC_MAXM, "recycling: more than 128 columns in V = [W, P]");
  if (k > 0 && (int)st->G_host.size() != k * k) refresh_gram(c, st, s);  // e.g. after a checkpoint import
  // M^{-1} A p_j = (z_j - z_{j+1}) / alpha_j, and one preconditioner application for the last
  DD_CUDA(cudaMemcpyAsync(st->ralpha, st->alphas.data(), (size_t)l * sizeof(double), cudaMemcpyHostToDevice, s));
  zdiff_all(n, l - 1, st->Z, st->ralpha, st->MAP, s);
  precond_z(c, st->AP + (size_t)(l - 1) * n, st->MAP + (size_t)(l - 1) * n, s);
  // F = V^T A V: the leading block W^T A W is G of the current basis; the rest in df64.
  // Gh = (AV)^T M^{-1} (AV): df64 for an FP64 preconditioner; for an FP32 one the vectors
  // M^{-1} A v carry FP32 accuracy only and the products accumulate in FP32 per stage.
  RecTables tab;
  for (int j = 0; j < m; ++j) {
    const bool w = j < k;
    const size_t off = (size_t)(w ? j : j - k) * n;
    tab.ptr[j] = (void*)((w ? st->W : st->P) + off);
    tab.ptr[REC_MAXM + j] = (void*)((w ? st->AW : st->AP) + off);
    tab.ptr[2 * REC_MAXM + j] = (void*)((w ? st->MAW : st->MAP) + off);
  }
  const std::vector<short2> qF = gram_block_list(m, k), qG = gram_block_list(m, 0);
  std::copy(qF.begin(), qF.end(), tab.blk.begin());
  std::copy(qG.begin(), qG.end(), tab.blk.begin() + REC_BLOCKS);
  tab.upload(st, s);
  const double* const* PV = reinterpret_cast<const double* const*>(st->rptr);
  const bool gh_df = c->opt.precond_prec == DD_PREC_FP64;
  gram_blocks(n, m, PV, PV + REC_MAXM, st->rblk, (int)qF.size(), true, st->rpart, st->rout, s);
  gram_blocks(n, m, PV + REC_MAXM, PV + 2 * REC_MAXM, st->rblk + REC_BLOCKS, (int)qG.size(), gh_df, st->rpart,
              st->rout + REC_BLOCKS * 16, s);
  std::vector<double> hv((size_t)2 * REC_BLOCKS * 16);
  DD_CUDA(cudaMemcpyAsync(hv.data(), st->rout, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  std::vector<double> F((size_t)m * m, 0.0), Gh((size_t)m * m, 0.0);
  blocks_to_sym(m, qF, hv.data(), F);
  blocks_to_sym(m, qG, hv.data() + REC_BLOCKS * 16, Gh);
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) F[(size_t)a * m + b] = st->G_host[(size_t)a * k + b];
  // The pencil's eigenpairs do not depend on the scaling of V's columns, and the search
  // vectors shrink with the residual by many orders of magnitude: scale the columns to unit
  // A-norm, D = diag(F)^{-1/2}, then restrict to the numerically nonsingular part of D F D =
  // Q L Q^T, T = D Q_r L_r^{-1/2} (so that only numerically dependent directions are dropped)
  std::vector<double> dsc(m);
  for (int a = 0; a < m; ++a) dsc[a] = F[(size_t)a * m + a] > 0.0 ? 1.0 / std::sqrt(F[(size_t)a * m + a]) : 0.0;
  std::vector<double> Fw(F);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) Fw[(size_t)a * m + b] *= dsc[a] * dsc[b];
  // Numerical rank of D F D at the accuracy of the pencil's data: with an FP32 preconditioner
  // the vectors M^{-1} A v carry about 1e-7 relative error, which a direction with eigenvalue
  // lam of D F D amplifies by 1/lam in T^T Gh T; directions below 1e-5 would produce spurious
  // harmonic Ritz values (and B4 would select the largest of them). FP64 data: 1e-12.
  const double rank_tol = c->opt.precond_prec == DD_PREC_FP32 ? 1e-5 : 1e-12;
  int r = 0;
  std::vector<double> T;
  {
    // When a Cholesky factor D F D = L L^T certifies lambda_min(D F D) >= 1 / ||L^{-1}||_F^2 >
    // rank_tol * ||D F D||_F >= rank_tol * lambda_max, no direction is dropped and T = D L^{-T}
    // spans the same pencil as the eigenvector form below (one eigen-decomposition less).
    std::vector<double> L(Fw), Li((size_t)m * m);
    double fro = 0.0;
    for (double v : Fw) fro += v * v;
    fro = std::sqrt(fro);
    bool full_rank = la::cholesky(m, L.data());
    if (full_rank) {
      la::tri_inv_lower(m, L.data(), Li.data());
      double li2 = 0.0;
      for (double v : Li) li2 += v * v;
      full_rank = li2 > 0.0 && 1.0 / li2 > rank_tol * fro;
    }
    if (full_rank) {
      r = m;
      T.assign((size_t)m * m, 0.0);
      for (int a = 0; a < m; ++a)
        for (int j = 0; j < m; ++j) T[(size_t)a * m + j] = dsc[a] * Li[(size_t)j * m + a];  // D L^{-T}
    } else {
      // restrict to the numerically nonsingular part: D F D = Q Lam Q^T, T = D Q_r Lam_r^{-1/2}
      std::vector<double> lam(m), Q((size_t)m * m);
      la::sym_eig(m, Fw.data(), lam.data(), Q.data());
      double lmax = lam[m - 1];
      std::vector<int> keep;
      for (int a = 0; a < m; ++a)
        if (lam[a] > rank_tol * lmax) keep.push_back(a);
      r = (int)keep.size();
      if (r == 0) return;
      T.assign((size_t)m * r, 0.0);
      for (int a = 0; a < m; ++a)
        for (int j = 0; j < r; ++j) T[(size_t)a * r + j] = dsc[a] * Q[(size_t)a * m + keep[j]] / std::sqrt(lam[keep[j]]);
    }
  }
  // C = T^T Gh T
  std::vector<double> GT((size_t)m * r), Cm((size_t)r * r);
  la::gemm_nn(m, r, m, Gh.data(), T.data(), GT.data());
  std::fill(Cm.begin(), Cm.end(), 0.0);
  for (int a = 0; a < m; ++a) {
    const double* Ta = T.data() + (size_t)a * r;
    const double* Ga = GT.data() + (size_t)a * r;
    for (int i = 0; i < r; ++i) {
      const double t = Ta[i];
      double* Ci = Cm.data() + (size_t)i * r;
      for (int j = 0; j < r; ++j) Ci[j] += t * Ga[j];
    }
  }
  std::vector<double> th(r), U((size_t)r * r);
  la::sym_eig(r, Cm.data(), th.data(), U.data());
  int kn = std::min(R, r);
  std::vector<int> sel(kn);
  for (int j = 0; j < kn; ++j) sel[j] = (st->strategy == DD_B4) ? (r - 1 - j) : j;
  std::vector<double> theta(kn);
  for (int j = 0; j < kn; ++j) theta[j] = th[sel[j]];
  if ((int)st->theta.size() == R && kn == R) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j < R; ++j) {
      num += (theta[j] - st->theta[j]) * (theta[j] - st->theta[j]);
      den += theta[j] * theta[j];
    }
    if (std::sqrt(num) <= st->freeze_tol * std::sqrt(den)) st->frozen = true;  // eq. 16
  }
  st->theta = theta;
  // Y = T U_sel (m x kn)
  std::vector<double> Y((size_t)m * kn, 0.0), Us((size_t)r * kn);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < kn; ++j) Us[(size_t)i * kn + j] = U[(size_t)i * r + sel[j]];
  la::gemm_nn(m, kn, r, T.data(), Us.data(), Y.data());
  // W = V Y, A W = (A V) Y in df64 (their df64 copies written alongside), M^{-1} A W = (M^{-1} A V) Y
  DD_CUDA(cudaMemcpyAsync(st->rY, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  for (int j = 0; j < kn; ++j) {
    tab.ptr[3 * REC_MAXM + j] = (void*)(st->W2 + (size_t)j * n);
    tab.ptr[4 * REC_MAXM + j] = (void*)(st->AW2 + (size_t)j * n);
    tab.ptr[5 * REC_MAXM + j] = (void*)(st->MAW2 + (size_t)j * n);
    tab.ptr[6 * REC_MAXM + j] = (void*)(st->Wd + (size_t)j * n);
    tab.ptr[7 * REC_MAXM + j] = (void*)(st->AWd + (size_t)j * n);
  }
  DD_CUDA(cudaMemcpyAsync(st->rptr + 3 * REC_MAXM, tab.ptr.data() + 3 * REC_MAXM, 5 * REC_MAXM * sizeof(void*),
                          cudaMemcpyHostToDevice, s));
  double* const* PO = reinterpret_cast<double* const*>(st->rptr);
  df64* const* PD = reinterpret_cast<df64* const*>(st->rptr);
  const bool f32 = use_f32_basis(c, st);
  // an FP32-valued basis is formed in FP32 accumulation: it is rounded to floats next, and
  // whichever basis results, A W is then computed for exactly it
  lincomb_src(n, m, kn, PV, st->rY, PO + 3 * REC_MAXM, f32 ? nullptr : PD + 6 * REC_MAXM, !f32, s);
  if (!f32) lincomb_src(n, m, kn, PV + REC_MAXM, st->rY, PO + 4 * REC_MAXM, PD + 7 * REC_MAXM, true, s);
  lincomb_src(n, m, kn, PV + 2 * REC_MAXM, st->rY, PO + 5 * REC_MAXM, nullptr, gh_df, s);
  std::swap(st->W, st->W2);
  std::swap(st->AW, st->AW2);
  std::swap(st->MAW, st->MAW2);
  st->k = kn;
  if (f32) {
    // W rounded to FP32 values and A W recomputed for it; M^{-1} A W stays the combination
    // (it only enters the next harmonic Ritz problem, at the FP32 preconditioner's accuracy)
    basis_to_f32(c, st, s, true);
    refresh_gram(c, st, s);
  } else {
    st->wf_valid = false;
    refresh_gram(c, st, s, true);
  }
}


// Algorithm 1 on A x_G = b with initial guess in c->xg; returns iterations.
dd_status pcg_solve(dd_ctx* c, dd_recycle* st, double rtol, bool record, dd_stats* stats, cudaStream_t s) {
  const int64_t n = c->n_gamma;
  const dd_options& o = c->opt;
  const int k = st ? st->k : 0;
  const df64* Wd = k ? st->Wd : nullptr;
  const df64* AWd = k ? st->AWd : nullptr;
  const float* Wf = (k && st->wf_valid) ? st->Wf : nullptr;
  DD_CUDA(cudaMemsetAsync(c->sc, 0, SC_COUNT * sizeof(double), s));
  // deflation of one iteration streams A W (df64) and W (df64 or FP32) once each, and z, p
  // (read) and p (written); the Krylov dots r^T z (and r^T z_old) run in the same window
  c->prof_bytes[DD_PROF_DEFL] =
      ((double)k * (8.0 + (Wf ? 4.0 : 8.0)) + 3.0 * 8.0 + (o.flexible ? 4.0 : 2.0) * 8.0) * (double)n;
  if (k) {
    // x_0 = x_{-1} + W (W^T A W)^{-1} W^T (b - A x_{-1})   (assures W^T r_0 = 0)
    schur_apply(c, c->xg, c->q, s);
    vec_sub(n, c->bvec, c->q, c->r, s);
    defl_mu_df(n, k, Wd, n, c->r, st->Ginv, c->wpart, c->mu, c->wticket, s);
    defl_update_df(n, k, Wd, n, c->mu, nullptr, c->xg, c->sc, -1, 1.0, s);
  }
  schur_apply(c, c->xg, c->q, s);
  vec_sub(n, c->bvec, c->q, c->r, s);
  vec_dots(n, c->bvec, c->bvec, c->r, c->r, nullptr, nullptr, c->partials, s);
  vec_finalize(c->partials, c->sc, FIN_BB, 0, s);
  launch_loop_begin(c->ctl, c->sc, rtol, o.maxit, o.stop_rhs_norm, s);
  // p enters the first update p = z + beta p - W mu with beta = 0
  DD_CUDA(cudaMemsetAsync(c->p, 0, n * sizeof(double), s));
  const bool rec = record && st && st->hmax > 0;
  const bool reo = k && o.reorth;
  const int flex = o.flexible;
  // one iteration of Algorithm 1 in the order z = M^{-1} r, beta, p = z + beta p - W mu,
  // q = A p, alpha, x += alpha p, r -= alpha q, stopping test (first pass: beta = 0)
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle h, bool in_graph) {
    if (flex) DD_CUDA(cudaMemcpyAsync(c->zold, c->z, n * sizeof(double), cudaMemcpyDeviceToDevice, bs));
    precond_z(c, c->r, c->z, bs);
    if (rec) launch_record(c->ctl, c->z, st->Z, n, st->hmax, 1, bs);
    {
      // the deflation dots (AW)^T z and the Krylov dots r^T z (r^T z_old) only read z: the
      // former run on the side stream while the latter finalize beta on the main stream
      ProfScope pd(c, k ? DD_PROF_DEFL : DD_PROF_COUNT, bs);
      const Fork fk{k ? c->s_coarse : nullptr, c->ev_fork, c->ev_join};
      const cudaStream_t sd = fk.begin(bs);
      if (k) defl_mu_df(n, k, AWd, n, c->z, st->Ginv, c->wpart, c->mu, c->wticket, sd);
      vec_dots_fin(n, c->r, c->z, flex ? c->r : nullptr, flex ? c->zold : nullptr, c->partials, c->sc, FIN_RZL, flex,
                   c->fticket, bs, &c->ctl->its);
      fk.end(bs);
      if (Wf)
        defl_update_f(n, k, Wf, n, c->mu, c->z, c->p, c->sc, SC_BETA, -1.0, bs);
      else
        defl_update_df(n, k, Wd, n, c->mu, c->z, c->p, c->sc, SC_BETA, -1.0, bs);
    }
    schur_apply(c, c->p, c->q, bs);
    vec_dots_fin(n, c->p, c->q, nullptr, nullptr, c->partials, c->sc, FIN_PQ, 0, c->fticket, bs);
    if (rec) {
      launch_record(c->ctl, c->p, st->P, n, st->hmax, 0, bs);
      launch_record(c->ctl, c->q, st->AP, n, st->hmax, 0, bs);
    }
    vec_axpy2_fin(n, c->sc, c->xg, c->p, c->r, c->q, c->partials, c->fticket, bs);
    if (reo) {
      // r -= W (W^T W)^{-1} W^T r  (Algorithm 1, optional re-orthogonalization), then ||r||^2 again
      defl_mu_df(n, k, Wd, n, c->r, st->WWinv, c->wpart, c->mu, c->wticket, bs);
      defl_update_df(n, k, Wd, n, c->mu, nullptr, c->r, c->sc, -1, -1.0, bs);
      vec_dots_fin(n, c->r, c->r, nullptr, nullptr, c->partials, c->sc, FIN_RR, 0, c->fticket, bs);
    }
    launch_loop_check(c->ctl, c->sc, c->alphas, h, in_graph, bs);
  };
  // everything the captured body bakes into its launches
  const std::vector<uint64_t> key = {1,
                                     (uint64_t)k,
                                     (uint64_t)rec,
                                     (uint64_t)(st ? st->hmax : 0),
                                     (uint64_t)reo,
                                     (uint64_t)flex,
                                     (uint64_t)(uintptr_t)Wd,
                                     (uint64_t)(uintptr_t)AWd,
                                     (uint64_t)(uintptr_t)Wf,
                                     (uint64_t)(uintptr_t)(st ? st->Ginv : nullptr),
                                     (uint64_t)(uintptr_t)(st ? st->WWinv : nullptr),
                                     (uint64_t)(uintptr_t)(st ? st->P : nullptr),
                                     (uint64_t)(uintptr_t)(st ? st->AP : nullptr),
                                     (uint64_t)(uintptr_t)(st ? st->Z : nullptr),
                                     (uint64_t)c->neumann};
  (st ? st->loop : c->loop).run(key, body, c->ctl, c->ctl_host, o.loop_graph && !c->prof_on, s);
  const LoopCtl L = *c->ctl_host;
  const int its = L.its;
  const double rel = L.rel;
  const dd_status status =
      L.status == LOOP_BREAKDOWN ? DD_BREAKDOWN : (L.status == LOOP_NOT_CONVERGED ? DD_NOT_CONVERGED : DD_OK);
  if (stats) stats->rel_res0 = L.rel0;
  // the step lengths feed the recycling update (M^{-1} A p_j from consecutive z)
  if (st) st->alphas.assign(record ? (size_t)L.nalpha : 0, 0.0);
  if (st && record && L.nalpha > 0) {
    DD_CUDA(cudaMemcpyAsync(st->alphas.data(), c->alphas, (size_t)L.nalpha * sizeof(double), cudaMemcpyDeviceToHost,
                            s));
    DD_CUDA(cudaStreamSynchronize(s));
  }
  if (stats) {
    stats->iters = its;
    stats->rel_res = rel;
    stats->recycled_k = k;
    stats->frozen = st ? (int)st->frozen : 0;
  }
  return status;
}

}  // namespace dd

extern "C" {

dd_status dd_solve(dd_ctx* c, const double* f, double* x, double rtol, dd_recycle* st, dd_stats* stats, void* stream) {
  if (!c || !f || !x || !st || st->ctx != c || !(rtol > 0.0)) {
    g_last_error = "dd_solve: invalid argument";
    return DD_INVALID_ARG;
  }
  dd_status result = DD_OK;
  dd_status gs = guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    DD_CUDA(cudaEventRecord(c->ev0, s));
    if (c->neumann) {
      // pure Neumann: the load vector projected onto the range of K (its mean removed)
      vec_sub_mean(c->n_free, f, c->fc, c->partials, s);
      f = c->fc;
    }
    condense(c, f, c->bvec, s);
    // initial guess: the previous solution (Sect. 5) or zero
    if (c->opt.zero_initial_guess)
      DD_CUDA(cudaMemsetAsync(c->xg, 0, c->n_gamma * 8, s));
    else
      DD_CUDA(cudaMemcpyAsync(c->xg, st->xg_prev, c->n_gamma * 8, cudaMemcpyDeviceToDevice, s));
    bool record = st->kmax > 0 && !st->frozen;
    result = pcg_solve(c, st, rtol, record, stats, s);
    recover(c, f, c->xg, x, s);
    if (c->neumann) vec_sub_mean(c->n_free, x, x, c->partials, s);  // the mean-free representative
    // a breakdown (non-finite or non-positive PCG scalars, e.g. from a non-finite load
    // vector) leaves the recycle state as it was: previous solution, basis and histories
    if (result != DD_BREAKDOWN)
      DD_CUDA(cudaMemcpyAsync(st->xg_prev, c->xg, c->n_gamma * 8, cudaMemcpyDeviceToDevice, s));
    if (record && (result == DD_OK || result == DD_NOT_CONVERGED)) {
      ProfScope pr(c, DD_PROF_RECYCLE, s);
      recycle_update(c, st, (int)st->alphas.size(), s);
    } else {
      st->step++;
    }
    DD_CUDA(cudaEventRecord(c->ev1, s));
    check_err(c, s);
    if (c->prof_on) c->harvest();
    if (stats) {
      float ms = 0.f;
      DD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      stats->ms = ms;
      stats->frozen = (int)st->frozen;
    }
  });
  if (gs != DD_OK) return gs;
  if (result != DD_OK) g_last_error = result == DD_NOT_CONVERGED ? "maxit reached" : "PCG breakdown";
  return result;
}

dd_status dd_profile(dd_ctx* c, int32_t enable, dd_kernel_prof* prof, int64_t* launches, void* stream) {
  if (!c) return DD_INVALID_ARG;
  return guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (prof || launches) {
      DD_CUDA(cudaStreamSynchronize(s));
      c->harvest();
    }
    if (prof) {
      for (int k = 0; k < DD_PROF_COUNT; ++k) {
        prof[k].ms = c->prof_ms[k];
        prof[k].launches = c->prof_n[k];
        prof[k].alg_bytes = c->prof_bytes[k];
        prof[k].alg_flops = c->prof_flops[k];
        c->prof_ms[k] = 0;
        c->prof_n[k] = 0;
      }
    }
    if (launches) *launches = g_launches.exchange(0);
    c->prof_on = enable != 0;
  });
}

dd_status dd_coef_mismatch(dd_ctx* c, const double* coef, int32_t coef_is_log, double* max_rel_diff, void* stream) {
  if (!c || !coef || !max_rel_diff || (coef_is_log != 0 && coef_is_log != 1)) {
    g_last_error = "dd_coef_mismatch: invalid argument";
    return DD_INVALID_ARG;
  }
  return guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    launch_coef_mismatch(c->mesh, coef, coef_is_log, c->partials, NBLK, s);
    std::vector<double> part(NBLK);
    DD_CUDA(cudaMemcpyAsync(part.data(), c->partials, NBLK * sizeof(double), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    double mx = 0.0;
    for (double v : part) mx = (v > mx || v != v) ? v : mx;
    *max_rel_diff = mx;
  });
}

dd_status dd_adjoint(dd_ctx* c, const double* grad_x, const double* x, double* grad_f, double* grad_coef,
                     int32_t coef_grad_log, double rtol, dd_recycle* st, dd_stats* stats, void* stream) {
  if (!c || !grad_x || !grad_f || (grad_coef && !x) || !(rtol > 0.0) || (st && st->ctx != c) ||
      (coef_grad_log != 0 && coef_grad_log != 1)) {
    g_last_error = "dd_adjoint: invalid argument";
    return DD_INVALID_ARG;
  }
  if (c->neumann) {
    g_last_error = "dd_adjoint: the pure-Neumann case (no Dirichlet face) has no adjoint solve";
    return DD_INVALID_ARG;
  }
  dd_status result = DD_OK;
  dd_status gs = guard([&] {
    cudaStream_t s = (cudaStream_t)stream;
    DD_CUDA(cudaEventRecord(c->ev0, s));
    // lambda = K^{-1} grad_x: the same condensation, deflated PCG (basis of st, not updated) and recovery
    condense(c, grad_x, c->bvec, s);
    DD_CUDA(cudaMemsetAsync(c->xg, 0, c->n_gamma * sizeof(double), s));
    result = pcg_solve(c, st, rtol, false, stats, s);
    recover(c, grad_x, c->xg, grad_f, s);
    if (grad_coef) launch_coef_grad(c->mesh, x, grad_f, grad_coef, coef_grad_log, s);
    DD_CUDA(cudaEventRecord(c->ev1, s));
    check_err(c, s);
    if (c->prof_on) c->harvest();
    if (stats) {
      float ms = 0.f;
      DD_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      stats->ms = ms;
    }
  });
  if (gs != DD_OK) return gs;
  if (result != DD_OK) g_last_error = result == DD_NOT_CONVERGED ? "maxit reached" : "PCG breakdown";
  return result;
}

// Checkpoint layout (host bytes): header, theta[ntheta], x_prev[n_gamma], then for k > 0
// W, AW, MAW [k][n_gamma] and Ginv, WWinv [k][k] (all FP64, little-endian as in memory).
struct RecycleHeader {
  char magic[8];
  int64_t n_gamma;
  int32_t kmax, strategy, k, frozen, step, ntheta;
  double freeze_tol;
};

static size_t recycle_bytes(const dd_recycle* st) {
  size_t n = (size_t)st->ctx->n_gamma, k = (size_t)st->k;
  return sizeof(RecycleHeader) + st->theta.size() * 8 + n * 8 + (k ? (3 * k * n + 2 * k * k) * 8 : 0);
}

dd_status dd_recycle_export(const dd_recycle* st, void* host_buf, size_t* bytes) {
  if (!st || !bytes) {
    g_last_error = "dd_recycle_export: NULL argument";
    return DD_INVALID_ARG;
  }
  return guard([&] {
    size_t need = recycle_bytes(st);
    if (!host_buf) {
      *bytes = need;
      return;
    }
    DD_REQUIRE(*bytes >= need, "dd_recycle_export: buffer too small");
    *bytes = need;
    unsigned char* p = static_cast<unsigned char*>(host_buf);
    RecycleHeader h{};
    std::memcpy(h.magic, "DDRCY01", 8);
    h.n_gamma = st->ctx->n_gamma;
    h.kmax = st->kmax; h.strategy = st->strategy; h.k = st->k; h.frozen = st->frozen; h.step = st->step;
    h.ntheta = (int32_t)st->theta.size();
    h.freeze_tol = st->freeze_tol;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    std::memcpy(p, st->theta.data(), st->theta.size() * 8);
    p += st->theta.size() * 8;
    const size_t n = (size_t)h.n_gamma, k = (size_t)st->k;
    DD_CUDA(cudaMemcpy(p, st->xg_prev, n * 8, cudaMemcpyDeviceToHost));
    p += n * 8;
    if (k) {
      for (const double* src : {st->W, st->AW, st->MAW}) {
        DD_CUDA(cudaMemcpy(p, src, k * n * 8, cudaMemcpyDeviceToHost));
        p += k * n * 8;
      }
      DD_CUDA(cudaMemcpy(p, st->Ginv, k * k * 8, cudaMemcpyDeviceToHost));
      p += k * k * 8;
      if (st->ctx->opt.reorth) DD_CUDA(cudaMemcpy(p, st->WWinv, k * k * 8, cudaMemcpyDeviceToHost));
      else std::memset(p, 0, k * k * 8);
    }
  });
}

dd_status dd_recycle_import(dd_ctx* c, const void* host_buf, size_t bytes, dd_recycle** out) {
  if (!c || !host_buf || !out) {
    g_last_error = "dd_recycle_import: NULL argument";
    return DD_INVALID_ARG;
  }
  *out = nullptr;
  RecycleHeader h;
  if (bytes < sizeof h) {
    g_last_error = "dd_recycle_import: buffer too small";
    return DD_INVALID_ARG;
  }
  std::memcpy(&h, host_buf, sizeof h);
  if (std::memcmp(h.magic, "DDRCY01", 8) != 0 || h.n_gamma != c->n_gamma || h.k < 0 || h.k > h.kmax) {
    g_last_error = "dd_recycle_import: not a checkpoint of this problem";
    return DD_INVALID_ARG;
  }
  dd_recycle* st = nullptr;
  dd_status rc = dd_recycle_create(c, h.kmax, h.strategy, h.freeze_tol, &st);
  if (rc != DD_OK) return rc;
  rc = guard([&] {
    st->k = h.k;
    st->frozen = h.frozen != 0;
    st->step = h.step;
    DD_REQUIRE(bytes >= recycle_bytes(st) + (size_t)h.ntheta * 8 - st->theta.size() * 8,
               "dd_recycle_import: truncated checkpoint");
    const unsigned char* p = static_cast<const unsigned char*>(host_buf) + sizeof h;
    st->theta.assign(reinterpret_cast<const double*>(p), reinterpret_cast<const double*>(p) + h.ntheta);
    p += (size_t)h.ntheta * 8;
    const size_t n = (size_t)h.n_gamma, k = (size_t)h.k;
    DD_CUDA(cudaMemcpy(st->xg_prev, p, n * 8, cudaMemcpyHostToDevice));
    p += n * 8;
    if (k) {
      for (double* dst : {st->W, st->AW, st->MAW}) {
        DD_CUDA(cudaMemcpy(dst, p, k * n * 8, cudaMemcpyHostToDevice));
        p += k * n * 8;
      }
      DD_CUDA(cudaMemcpy(st->Ginv, p, k * k * 8, cudaMemcpyHostToDevice));
      p += k * k * 8;
      DD_CUDA(cudaMemcpy(st->WWinv, p, k * k * 8, cudaMemcpyHostToDevice));
      // a basis saved from an FP32-basis state is FP32-representable and comes back as it
      // was; any other is rounded here and its A W and Gram matrices recomputed
      if (use_f32_basis(c, st) && (st->strategy == DD_B3 || st->strategy == DD_B4) &&
          basis_to_f32(c, st, nullptr, false))
        refresh_gram(c, st, nullptr);
      else
        refresh_df(c, st, nullptr);
      DD_CUDA(cudaStreamSynchronize(nullptr));
    }
  });
  if (rc != DD_OK) {
    delete st;
    return rc;
  }
  *out = st;
  return DD_OK;
}

}  // extern "C"

namespace dd {
void set_last_error(const std::string& msg) { g_last_error = msg; }
// Read access to a context's Schur-operator data and error word for other translation units.
const DevMesh* context_mesh(const dd_ctx* c) { return c ? &c->mesh : nullptr; }
int* context_err(dd_ctx* c) { return c ? c->w.err : nullptr; }
}  // namespace dd

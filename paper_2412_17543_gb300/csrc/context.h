// Internal state of a solver context and of a recycle state, shared by the
// translation units of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.h"
#include "device.h"
#include "loop.h"
#include "vecops.h"

namespace dd {
struct BatchWork;
void free_batch_work(BatchWork* bw);
}  // namespace dd

using dd::DevBDDC;
using dd::DeviceArena;
using dd::DevLevel2;
using dd::DevMesh;
using dd::Work;

struct dd_ctx {
  dd_options opt{};
  dd_info_t info{};
  DeviceArena arena;
  std::vector<int64_t> gamma_free_host;
  int64_t n_free = 0, n_gamma = 0;
  int levels = 2;
  bool neumann = false;         // no Dirichlet face: solutions are the mean-free representatives
  double* fc = nullptr;         // [n_free] the consistent (mean-free) load vector (neumann)
  DevMesh mesh{};
  DevBDDC b1{};
  DevLevel2 l2{};
  const void* KCinv = nullptr;
  Work w{};
  dd::BatchWork* bw = nullptr;  // ensemble workspace (allocated by the first batched solve)
  // Krylov buffers
  double *xg = nullptr, *r = nullptr, *z = nullptr, *zold = nullptr, *p = nullptr, *q = nullptr, *bvec = nullptr;
  double* tmp = nullptr;
  double* sc = nullptr;        // device scalars [SC_COUNT]
  double* sc_host = nullptr;   // pinned mirror
  dd::LoopCtl* ctl = nullptr;       // device-resident loop control
  dd::LoopCtl* ctl_host = nullptr;  // pinned mirror
  double* alphas = nullptr;         // [maxit] step lengths of the last solve
  dd::LoopGraph loop;               // captured PCG loop of solves without a recycle state
  double* partials = nullptr;  // [NBLK*MAXDOT]
  double* wpart = nullptr;     // [NBLK*MAXK]
  double* mu = nullptr;        // [MAXK]
  unsigned* wticket = nullptr;  // block ticket of the one-launch deflation dots (0 between launches)
  unsigned* fticket = nullptr;  // block ticket of the dot products that finalize in the same launch
  double* gram_part = nullptr; // [NBLK*4096]
  double* gram_out = nullptr;  // [4096]
  double* ybuf = nullptr;      // [128*128] combination coefficients
  const double** ptrs = nullptr;  // device pointer table for gram / lincomb
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // second (high-priority) stream of the BDDC coarse correction and its fork/join events
  cudaStream_t s_coarse = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // two more side streams for the independent pieces of the level-2 BDDC, and their events
  cudaStream_t s_aux[2] = {nullptr, nullptr};
  cudaEvent_t ev_aux[4] = {nullptr, nullptr, nullptr, nullptr};
  // profiling: events around timed launches, harvested after a synchronization
  bool prof_on = false;
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[DD_PROF_COUNT] = {0};
  int64_t prof_n[DD_PROF_COUNT] = {0};
  double prof_bytes[DD_PROF_COUNT] = {0};
  double prof_flops[DD_PROF_COUNT] = {0};
  cudaEvent_t get_event() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    DD_CUDA(cudaEventCreate(&e));
    return e;
  }
  void harvest() {  // caller has synchronized the stream
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        prof_ms[p.cls] += ms;
        prof_n[p.cls] += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~dd_ctx() {
    if (bw) dd::free_batch_work(bw);
    if (sc_host) cudaFreeHost(sc_host);
    if (ctl_host) cudaFreeHost(ctl_host);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (s_coarse) cudaStreamDestroy(s_coarse);
    for (auto e : ev_aux)
      if (e) cudaEventDestroy(e);
    for (auto a : s_aux)
      if (a) cudaStreamDestroy(a);
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

namespace dd {
// times the launches issued on `s` during its lifetime when profiling is on
struct ProfScope {
  dd_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(dd_ctx* c_, int cls_, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    if (c->prof_on && cls >= 0 && cls < DD_PROF_COUNT) {
      a = c->get_event();
      b = c->get_event();
      DD_CUDA(cudaEventRecord(a, s));
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEventRecord(b, s);
      c->pending.push_back({cls, a, b});
    }
  }
};
}  // namespace dd

struct dd_recycle {
  dd_ctx* ctx = nullptr;
  int kmax = 0, strategy = DD_B4;
  double freeze_tol = 1e-5;
  int k = 0;
  bool frozen = false;
  int step = 0;
  DeviceArena arena;
  double *W = nullptr, *AW = nullptr, *MAW = nullptr;       // [kmax][n_gamma]
  double *W2 = nullptr, *AW2 = nullptr, *MAW2 = nullptr;    // next basis
  dd::df64 *Wd = nullptr, *AWd = nullptr;                   // df64 copies of W, AW (deflation kernels)
  float* Wf = nullptr;        // FP32 copy of W when W holds FP32-representable values (FP32 preconditioner)
  bool wf_valid = false;      // the per-iteration update streams Wf
  int* rflag = nullptr;       // device flag of the rounding kernel
  double* Ginv = nullptr;                                   // [kmax*kmax] (W^T A W)^{-1}
  double* WWinv = nullptr;                                  // [kmax*kmax] (W^T W)^{-1}
  std::vector<double> theta;
  double* xg_prev = nullptr;                                // [n_gamma]
  int nrhs = 0;                                             // ensemble width (0: single sequence)
  dd::df64* xg_prev_b = nullptr;                            // [n_gamma][BW] previous ensemble solutions (df64)
  bool have_prev = false;
  int hmax = 0;
  double *P = nullptr, *AP = nullptr, *Z = nullptr, *MAP = nullptr;  // histories [hmax][n_gamma]
  std::vector<double> alphas;
  dd::LoopGraph loop;                                       // captured PCG loop of this sequence
  // recycling-update work space (allocated on first use) and the host copy of G = W^T A W
  void** rptr = nullptr;                                    // [REC_PTRS] device pointer table
  short2* rblk = nullptr;                                   // [3][REC_BLOCKS] Gram block lists
  double *rpart = nullptr, *rout = nullptr;                 // Gram partials and results
  double *rY = nullptr, *ralpha = nullptr;                  // combination coefficients, step lengths
  std::vector<double> G_host;                               // [k*k] of the current basis
};


namespace dd {
// operators and steps of one solve (solver.cu)
void schur_apply(dd_ctx* c, const double* x, double* y, cudaStream_t s);
void precond_apply(dd_ctx* c, const double* r, double* z, cudaStream_t s);
void recycle_update(dd_ctx* c, dd_recycle* st, int l, cudaStream_t s);
void check_err(dd_ctx* c, cudaStream_t s);
void set_last_error(const std::string& msg);
void free_batch_work(BatchWork* bw);

// runs f, mapping exceptions to a status and the thread-local last error
template <class F>
dd_status guard_call(F&& f) {
  try {
    f();
    return DD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return DD_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return DD_INVALID_ARG;
  }
}
}  // namespace dd

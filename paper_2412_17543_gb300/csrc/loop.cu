// Device-resident PCG loop control and its CUDA graph (conditional WHILE node).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "batch.h"
#include "loop.h"
#include "vecops.h"

namespace dd {

namespace {

__global__ void k_loop_begin(LoopCtl* ctl, const double* __restrict__ sc, double rtol, int maxit, int stop_rhs_norm) {
  // same stopping reference as the residual test of every iteration: ||b|| or ||r_0||
  const double bnorm = sqrt(sc[SC_BB]);
  const double r0 = sqrt(sc[SC_RR]);
  double ref = stop_rhs_norm ? bnorm : r0;
  if (ref == 0.0) ref = 1.0;
  const double rel = r0 / ref;
  ctl->rtol = rtol;
  ctl->ref = ref;
  ctl->rel0 = rel;
  ctl->rel = rel;
  ctl->its = 0;
  ctl->maxit = maxit;
  // a non-finite right-hand side or initial residual is a breakdown, not convergence
  const bool finite = isfinite(rel) && isfinite(ref);
  ctl->status = finite ? LOOP_OK : LOOP_BREAKDOWN;
  ctl->go = (finite && rel >= rtol) ? 1 : 0;
  ctl->rec0 = 0;
  ctl->nalpha = 0;
}

__global__ void k_loop_gate(const LoopCtl* ctl, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, ctl->go ? 1u : 0u);
}

__global__ void k_loop_check(LoopCtl* ctl, const double* __restrict__ sc, double* alphas,
                             cudaGraphConditionalHandle h, int in_graph) {
  const int its = ctl->its + 1;
  ctl->its = its;
  if (its - 1 < ctl->maxit) alphas[its - 1] = sc[SC_ALPHA];
  ctl->nalpha = its;
  int go = 1;
  if (sc[SC_FLAG] != 0.0) {
    ctl->status = LOOP_BREAKDOWN;
    go = 0;
  } else {
    const double rel = sqrt(sc[SC_RR]) / ctl->ref;
    ctl->rel = rel;
    if (!isfinite(rel)) {
      ctl->status = LOOP_BREAKDOWN;
      go = 0;
    } else if (rel < ctl->rtol) {
      go = 0;
    } else if (its >= ctl->maxit) {
      ctl->status = LOOP_NOT_CONVERGED;
      go = 0;
    }
  }
  ctl->go = go;
  if (in_graph) cudaGraphSetConditional(h, (unsigned)go);
}

__global__ void k_loop_begin_b(LoopCtl* ctl, const double* __restrict__ scb, int maxit, int rec0) {
  int any = 0;
  for (int m = 0; m < BW; ++m) any |= scb[BS_ACT * BW + m] != 0.0;
  ctl->its = 0;
  ctl->maxit = maxit;
  ctl->status = LOOP_OK;
  ctl->go = any;
  ctl->rec0 = (rec0 && scb[BS_ACT * BW + 0] != 0.0) ? 1 : 0;
  ctl->nalpha = 0;
}

__global__ void k_loop_check_b(LoopCtl* ctl, const double* __restrict__ scb, double* alphas,
                               cudaGraphConditionalHandle h, int in_graph) {
  const int its = ctl->its + 1;
  ctl->its = its;
  if (ctl->rec0) {
    // member 0 was active during this iteration: its alpha feeds the recycling update
    if (ctl->nalpha < ctl->maxit) alphas[ctl->nalpha] = scb[BS_ALPHA * BW + 0];
    ctl->nalpha += 1;
    ctl->rec0 = scb[BS_ACT * BW + 0] != 0.0 ? 1 : 0;
  }
  int any = 0;
  for (int m = 0; m < BW; ++m) any |= scb[BS_ACT * BW + m] != 0.0;
  int go = any;
  if (any && its >= ctl->maxit) {
    ctl->status = LOOP_NOT_CONVERGED;
    go = 0;
  }
  ctl->go = go;
  if (in_graph) cudaGraphSetConditional(h, (unsigned)go);
}

__global__ void k_record(const LoopCtl* __restrict__ ctl, const double* __restrict__ src, double* __restrict__ dst,
                         int64_t n, int limit, int inclusive) {
  const int its = ctl->its;
  if (inclusive ? its > limit : its >= limit) return;
  double* d = dst + (int64_t)its * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = src[i];
}

__global__ void k_record_col0(const LoopCtl* __restrict__ ctl, const df64* __restrict__ src, double* __restrict__ dst,
                              int64_t n, int limit, int inclusive) {
  const int its = ctl->its;
  if (!ctl->rec0 || (inclusive ? its > limit : its >= limit)) return;
  double* d = dst + (int64_t)its * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = df64_to_double_bits(src[i * BW]);
}

}  // namespace

void launch_loop_begin(LoopCtl* ctl, const double* sc, double rtol, int maxit, int stop_rhs_norm, cudaStream_t s) {
  k_loop_begin<<<1, 1, 0, s>>>(ctl, sc, rtol, maxit, stop_rhs_norm);
  DD_CHECK_LAUNCH();
}
void launch_loop_check(LoopCtl* ctl, const double* sc, double* alphas, cudaGraphConditionalHandle h, bool in_graph,
                       cudaStream_t s) {
  k_loop_check<<<1, 1, 0, s>>>(ctl, sc, alphas, h, in_graph ? 1 : 0);
  DD_CHECK_LAUNCH();
}
void launch_loop_begin_b(LoopCtl* ctl, const double* scb, int maxit, int rec0, cudaStream_t s) {
  k_loop_begin_b<<<1, 1, 0, s>>>(ctl, scb, maxit, rec0);
  DD_CHECK_LAUNCH();
}
void launch_loop_check_b(LoopCtl* ctl, const double* scb, double* alphas, cudaGraphConditionalHandle h,
                         bool in_graph, cudaStream_t s) {
  k_loop_check_b<<<1, 1, 0, s>>>(ctl, scb, alphas, h, in_graph ? 1 : 0);
  DD_CHECK_LAUNCH();
}
void launch_record(const LoopCtl* ctl, const double* src, double* dst, int64_t n, int limit, int inclusive,
                   cudaStream_t s) {
  if (n == 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * 152);
  k_record<<<(unsigned)blocks, 256, 0, s>>>(ctl, src, dst, n, limit, inclusive);
  DD_CHECK_LAUNCH();
}
void launch_record_col0(const LoopCtl* ctl, const df64* src, double* dst, int64_t n, int limit, int inclusive,
                        cudaStream_t s) {
  if (n == 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * 152);
  k_record_col0<<<(unsigned)blocks, 256, 0, s>>>(ctl, src, dst, n, limit, inclusive);
  DD_CHECK_LAUNCH();
}

LoopGraph::~LoopGraph() {
  reset();
  if (cap_) cudaStreamDestroy(cap_);
}

void LoopGraph::reset() {
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  exec_ = nullptr;
  graph_ = nullptr;
  key_.clear();
}

void LoopGraph::run(const std::vector<uint64_t>& key, const Body& body, LoopCtl* ctl, LoopCtl* ctl_host,
                    bool use_graph, cudaStream_t s, const std::function<void()>& after_pass) {
  if (use_graph) {
    if (!exec_ || key != key_) {
      reset();
      if (!cap_) DD_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
      DD_CUDA(cudaGraphCreate(&graph_, 0));
      cudaGraphConditionalHandle h;
      DD_CUDA(cudaGraphConditionalHandleCreate(&h, graph_, 0, 0));
      // gate node: the condition starts from ctl->go, which the stream set before the launch
      cudaGraphNode_t gate;
      {
        const LoopCtl* cctl = ctl;
        void* args[] = {(void*)&cctl, (void*)&h};
        cudaKernelNodeParams kp{};
        kp.func = (void*)k_loop_gate;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        kp.extra = nullptr;
        DD_CUDA(cudaGraphAddKernelNode(&gate, graph_, nullptr, 0, &kp));
      }
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cond;
      DD_CUDA(cudaGraphAddNode(&cond, graph_, &gate, nullptr, 1, &cp));
      cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
      DD_CUDA(cudaStreamBeginCaptureToGraph(cap_, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      const int64_t l0 = launch_counter();
      try {
        body(cap_, h, true);
      } catch (...) {
        cudaGraph_t g2 = nullptr;
        cudaStreamEndCapture(cap_, &g2);
        cudaGetLastError();
        reset();
        throw;
      }
      // captured launches are counted when the graph runs them
      body_launches_ = launch_counter() - l0;
      add_launches(-body_launches_);
      cudaGraph_t g2 = nullptr;
      DD_CUDA(cudaStreamEndCapture(cap_, &g2));
      // kernel nodes keep the priority of the stream they were captured from (the BDDC
      // coarse branch runs ahead of the level-1 N_i blocks, as in the host-issued loop)
      DD_CUDA(cudaGraphInstantiate(&exec_, graph_, cudaGraphInstantiateFlagUseNodePriority));
      key_ = key;
      ++captures_;
    }
    DD_CUDA(cudaGraphLaunch(exec_, s));
    DD_CUDA(cudaMemcpyAsync(ctl_host, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    add_launches(1 + (int64_t)ctl_host->its * body_launches_);  // gate + iterations
    return;
  }
  DD_CUDA(cudaMemcpyAsync(ctl_host, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  while (ctl_host->go) {
    body(s, cudaGraphConditionalHandle{}, false);
    DD_CUDA(cudaMemcpyAsync(ctl_host, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
    DD_CUDA(cudaStreamSynchronize(s));
    if (after_pass) after_pass();
  }
}

}  // namespace dd

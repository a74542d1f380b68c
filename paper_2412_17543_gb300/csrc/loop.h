// Device-resident PCG loop (Algorithm 1): the iteration count, the stopping test and the
// continue flag live in device memory, so a whole solve runs as one launch of a CUDA graph
// whose conditional WHILE node repeats the captured iteration body until a kernel at the
// end of the body clears the flag. The same body can also be issued pass by pass on a
// stream, reading the flag back after each pass (profiling mode: events around operators).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "common.h"

namespace dd {

enum { LOOP_OK = 0, LOOP_NOT_CONVERGED = 1, LOOP_BREAKDOWN = 2 };

struct LoopCtl {
  double rtol;    // relative tolerance of the stopping test
  double ref;     // ||b|| or ||r_0|| (single sequence; the ensemble keeps one per member)
  double rel0;    // relative residual of the initial guess
  double rel;     // relative residual after the last iteration
  int its;        // completed iterations
  int maxit;      // iteration limit
  int status;     // LOOP_*
  int go;         // 1 while the loop continues
  int rec0;       // ensemble: member 0 still feeds the recycling histories
  int nalpha;     // alphas recorded (single sequence: its)
};

// stopping test of the single sequence before the first iteration (sc: the PCG scalars
// after the initial residual; alphas are written per iteration by the check)
void launch_loop_begin(LoopCtl* ctl, const double* sc, double rtol, int maxit, int stop_rhs_norm, cudaStream_t s);
// end of one iteration: its += 1, alpha recorded, stop on breakdown, convergence or maxit
void launch_loop_check(LoopCtl* ctl, const double* sc, double* alphas, cudaGraphConditionalHandle h, bool in_graph,
                       cudaStream_t s);
// ensemble: the members' device flags decide; member 0's alphas are recorded while it is active
void launch_loop_begin_b(LoopCtl* ctl, const double* scb, int maxit, int rec0, cudaStream_t s);
void launch_loop_check_b(LoopCtl* ctl, const double* scb, double* alphas, cudaGraphConditionalHandle h,
                         bool in_graph, cudaStream_t s);
// dst + its * n <- src when its < limit (inclusive: its <= limit), its read on the device
void launch_record(const LoopCtl* ctl, const double* src, double* dst, int64_t n, int limit, int inclusive,
                   cudaStream_t s);
// member 0 of an interleaved df64 ensemble vector into dst + its * n, when ctl->rec0 and
// its < limit (inclusive: its <= limit)
void launch_record_col0(const LoopCtl* ctl, const df64* src, double* dst, int64_t n, int limit, int inclusive,
                        cudaStream_t s);

// One captured loop: the graph is rebuilt when the key (everything the body bakes into
// its launches: sizes, basis width, buffer addresses, flags) changes.
class LoopGraph {
 public:
  using Body = std::function<void(cudaStream_t, cudaGraphConditionalHandle, bool in_graph)>;
  LoopGraph() = default;
  LoopGraph(const LoopGraph&) = delete;
  LoopGraph& operator=(const LoopGraph&) = delete;
  ~LoopGraph();
  // runs body while ctl->go (set on the stream before the call); ctl_host: pinned mirror,
  // current on return
  void run(const std::vector<uint64_t>& key, const Body& body, LoopCtl* ctl, LoopCtl* ctl_host, bool use_graph,
           cudaStream_t s, const std::function<void()>& after_pass = {});
  int captures() const { return captures_; }

 private:
  void reset();
  std::vector<uint64_t> key_;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
  cudaStream_t cap_ = nullptr;  // capture stream: the caller's stream may be the legacy default stream
  int captures_ = 0;
  int64_t body_launches_ = 0;  // kernel launches of one captured iteration
};

}  // namespace dd

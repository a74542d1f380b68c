// Schur-complement application without any device allocation on the call path:
// the scratch vectors live in a file-scope static device array (see
// dd_schur_apply_noalloc in include/dd_solver.h for limits and semantics).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.h"
#include "device.h"

namespace dd {
const DevMesh* context_mesh(const dd_ctx* c);
int* context_err(dd_ctx* c);
void set_last_error(const std::string& msg);
}  // namespace dd

namespace {

constexpr size_t kScratchDoubles = DD_NOALLOC_SCRATCH_BYTES / sizeof(double);

// Shared by every call on a device; every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
double* scratch_address() {
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw dd::Error(DD_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw dd::Error(DD_CUDA_ERROR, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" dd_status dd_schur_apply_noalloc(dd_ctx* ctx, const double* x, double* y, void* stream) {
  if (!ctx || !x || !y) {
    dd::set_last_error("dd_schur_apply_noalloc: NULL argument");
    return DD_INVALID_ARG;
  }
  try {
    const dd::DevMesh& m = *dd::context_mesh(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n_int = (size_t)m.n_int;
    const size_t n_flat = (size_t)m.n_flat;  // host copy, fixed at setup: no device read-back
    const size_t need = 2 * n_int + n_flat;
    if (need > kScratchDoubles)
      throw dd::Error(DD_INVALID_ARG, "dd_schur_apply_noalloc: problem needs " + std::to_string(need * 8) +
                                          " bytes of scratch, the static array holds " +
                                          std::to_string(kScratchDoubles * 8));
    double* base = scratch_address();
    double* tI = base;
    double* sI = base + n_int;
    double* yloc = base + 2 * n_int;
    // stream-ordered launches only: the call returns without waiting for the GPU. A bounded
    // wait that gives up in these kernels sets the context's error word, which the next
    // entry point of the context that reads it reports as DD_TIMEOUT.
    dd::launch_elem_interior(m, dd::ELEM_SCHUR, x, nullptr, tI, s);
    dd::launch_kii_apply(m, tI, sI, dd::context_err(ctx), s);
    dd::launch_elem_interface(m, dd::ELEM_SCHUR, x, sI, yloc, s);
    dd::launch_gather(m.n_gamma, m.gptr, m.gidx, yloc, nullptr, nullptr, y, s);
    return DD_OK;
  } catch (const dd::Error& err) {
    dd::set_last_error(err.what());
    return err.code;
  } catch (const std::exception& err) {
    dd::set_last_error(err.what());
    return DD_INVALID_ARG;
  }
}

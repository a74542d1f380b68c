// Tensor-core (tcgen05) ensemble products U_i = N_i R_i of the constrained-Neumann
// operators (tc_nmm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.h"
#include "device.h"

namespace dd {

// operand splits of the tensor-core products (FP32 accuracy from low-precision slices)
enum { TC_TF32X3 = 0, TC_BF16X3 = 1 };

// full FP32 rows of every N_i in the tcgen05 operand tile order, and the work items
struct TcMats {
  int count = 0;
  int max_nmb = 1;              // most 128-row blocks of a matrix
  int n_items = 0;              // (matrix, 128-row block) items, full blocks first
  const int2* items = nullptr;  // [n_items] (matrix, block) (device)
  const int* n = nullptr;       // [count] local interface sizes (device)
  const int64_t* off = nullptr; // [count] first float of each matrix (device)
  float* data = nullptr;
  double bytes = 0;             // stored bytes
};

// expands the packed FP32 symmetric tiles S (device) into TcMats; n_host = S's sizes
TcMats build_tc_mats(DeviceArena& arena, const SymTiles& S, const std::vector<int>& n_host, cudaStream_t s);
// uloc[(goff[i] + r) * BW + m] = sum_c N_i[r][c] rloc[(goff[i] + c) * BW + m] on tcgen05
// with the split `scheme` (TC_TF32X3 or TC_BF16X3); a persistent CTA per SM
void launch_nmm_tc(const TcMats& A, const int64_t* goff, const float* rloc, float* uloc, int* err, int scheme,
                   cudaStream_t s);

}  // namespace dd

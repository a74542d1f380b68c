// Tensor-core (tcgen05) ensemble products U_i = N_i R_i of the constrained-Neumann
// operators (tc_nmm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.h"
#include "device.h"

namespace dd {

// full FP32 rows of every N_i in the tcgen05 operand tile order
struct TcMats {
  int count = 0;
  int max_nmb = 1;              // most 128-row blocks of a matrix (grid height)
  const int* n = nullptr;       // [count] local interface sizes (device)
  const int64_t* off = nullptr; // [count] first float of each matrix (device)
  float* data = nullptr;
  double bytes = 0;             // stored bytes
};

// expands the packed FP32 symmetric tiles S (device) into TcMats; n_host = S's sizes
TcMats build_tc_mats(DeviceArena& arena, const SymTiles& S, const std::vector<int>& n_host, cudaStream_t s);
// uloc[(goff[i] + r) * BW + m] = sum_c N_i[r][c] rloc[(goff[i] + c) * BW + m]  (3xTF32 on tcgen05)
void launch_nmm_tc(const TcMats& A, const int64_t* goff, const float* rloc, float* uloc, int* err, cudaStream_t s);
size_t tc_smem_bytes();

}  // namespace dd

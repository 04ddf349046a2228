// Rank-predictor MLP shared declarations.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "common.h"

#define IFMM_MLP_IN 9
#define IFMM_MLP_NWEIGHTS 9025

#define CKM(x)                                                                                         \
  do {                                                                                                 \
    cudaError_t e_ = (x);                                                                              \
    if (e_ != cudaSuccess) throw ::ifmm::Error(IFMM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace ifmm {
// forward pass of the weights d_w (device) over ns feature rows d_x (device);
// predictions to d_y (device), enqueued on s (no synchronization, no
// allocation); work: mlp_predict_floats(ns) floats of device memory for the
// hidden activations
size_t mlp_predict_floats(int ns);
void mlp_predict_device(const float* d_w, const float* d_x, float* d_y, int ns, cudaStream_t s, float* work);
}  // namespace ifmm

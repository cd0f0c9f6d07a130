// Training launchers (maximum likelihood, Eq. 2): loss and gradient of the
// mean code length in bits per dimension, and the Adam update.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"

namespace nlc {

size_t train_ws_bytes(const Dims& d, long long n_px, int sm_count);
cudaError_t launch_loss_grad(const Dims& d, const float* w, const float* wt, const uint8_t* batch,
                             int N, int H,
                             int W, float* loss, float* grad, void* ws, int sm_count,
                             cudaStream_t s);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, long long t, cudaStream_t s);

}  // namespace nlc

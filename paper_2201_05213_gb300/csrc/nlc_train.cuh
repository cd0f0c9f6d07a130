// Training launchers (maximum likelihood, Eq. 2): loss and gradient of the
// mean code length in bits per dimension, and the Adam update.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"

namespace nlc {

size_t train_ws_bytes(const Dims& d, long long n_px, int sm_count);
// FP32 SIMT path.  dparams == nullptr: loss (bits per dimension) and its
// gradient; else the gradient of sum(dparams * network outputs) (loss
// untouched).
cudaError_t launch_loss_grad(const Dims& d, const float* w, const float* wt, const uint8_t* batch,
                             int N, int H, int W, const float* dparams, float* loss, float* grad,
                             void* ws, int sm_count, cudaStream_t s);
// Sums per-CTA gradient slots (and loss partials, if part_l and loss are
// non-null) in a fixed order.
cudaError_t launch_reduce_grad(const float* part_g, const float* part_l, int nblk, int n_w, int ldw,
                               long long n_px, float* grad, float* loss, cudaStream_t s);
// Whether the FP32 SIMT training kernel's tiles fit in one CTA.
bool simt_train_fits(const Dims& d);
// BF16 tensor-core path (tcgen05), same contract; fits: whether the model's
// tiles fit in one CTA's shared memory.
bool tc_train_fits(const Dims& d);
size_t tc_train_ws_bytes(const Dims& d, long long n_px, int sm_count);
cudaError_t launch_tc_train(const Dims& d, const uint16_t* umma, const float* bias,
                            const uint8_t* batch, int N, int H, int W, const float* dparams,
                            float* loss, float* grad, void* ws, int sm_count, int* status,
                            cudaStream_t s);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, long long t, cudaStream_t s);

}  // namespace nlc

// Throughput of the special-function unit (MUFU) for the instruction pair
// that dominates the decoder's symbol search: one logistic term is
// rcp.approx(1 + ex2.approx(z)), two MUFU operations.  The kernel runs
// eight independent chains of that pair per thread at full occupancy, so
// that the MUFU pipe, not latency, bounds it; the measured rate is the
// denominator of the decoder's MUFU roofline.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nlc.h"
#include "nlc_common.cuh"

namespace nlc {

constexpr int kProbeThreads = 512;
constexpr int kProbeChains = 8;

__device__ float g_mufu_sink;

__global__ void __launch_bounds__(kProbeThreads) mufu_rate_kernel(int iters) {
  float x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; c++)
    x[c] = 0.05f + 0.1f * (float)c + 1e-7f * (float)(threadIdx.x + blockIdx.x);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) {
      // x stays in (0, 1): ex2 in (1, 2), the reciprocal in (1/3, 1/2)
      x[c] = rcp_approx(__fadd_rn(1.f, ex2_approx(x[c])));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; c++) s = __fadd_rn(s, x[c]);
  if (s == 12345.f) g_mufu_sink = s;  // never true; keeps the chains live
}

}  // namespace nlc

using namespace nlc;

extern "C" int nlc_measure_mufu(int iters, nlc_stream stream, double* h_ops_per_s, double* h_ms) {
  if (iters < 1 || !h_ops_per_s) return NLC_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NLC_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mufu_rate_kernel, kProbeThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return NLC_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return NLC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NLC_ERR_CUDA;
  }
  int rc = NLC_OK;
  mufu_rate_kernel<<<grid, kProbeThreads, 0, s>>>(iters / 8 + 1);  // warm-up
  cudaEventRecord(e0, s);
  mufu_rate_kernel<<<grid, kProbeThreads, 0, s>>>(iters);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
    rc = NLC_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double ops = 2.0 * kProbeChains * (double)iters * grid * kProbeThreads;
  *h_ops_per_s = ops / (ms * 1e-3);
  if (h_ms) *h_ms = ms;
  return NLC_OK;
}

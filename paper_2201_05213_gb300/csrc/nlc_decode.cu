// Launchers of the wavefront decoder (Algorithm 1, Section 3) and its plain
// build; the device code is in nlc_decode_kernel.cuh.
#include "nlc_decode_kernel.cuh"

namespace nlc {

// The instrumented build's kernels (nlc_decode_prof.cu).
const void* decode_fn_prof(int prec, bool win);

static int decode_threads_of(int prec) {
  return prec == PREC_BF16 ? decode_threads<PREC_BF16>() : decode_threads<PREC_FP32>();
}

size_t decode_smem_bytes(const Dims& d, int n_units) {
  return tile_smem_bytes(d, n_units, decode_threads_of(d.prec) / kGW, true);
}

// The kernel for a launch; prof selects the instrumented build (decoding
// only: the sampler is never profiled).
static const void* decode_fn(int prec, bool sample = false, bool win = false, bool prof = false) {
  if (prof && !sample) return decode_fn_prof(prec, win);
  if (win)
    return sample ? (const void*)decode_kernel<PREC_BF16, true, true, false>
                  : (const void*)decode_kernel<PREC_BF16, false, true, false>;
  if (sample)
    return prec == PREC_BF16 ? (const void*)decode_kernel<PREC_BF16, true, false, false>
                             : (const void*)decode_kernel<PREC_FP32, true, false, false>;
  return prec == PREC_BF16 ? (const void*)decode_kernel<PREC_BF16, false, false, false>
                           : (const void*)decode_kernel<PREC_FP32, false, false, false>;
}

int decode_max_grid(const DeviceModel& m, int n_units, int sm_count, bool sample, bool win) {
  const size_t smem = decode_smem_bytes(m.d, n_units);
  // both builds (plain and instrumented) get the attribute, so that a plan
  // set up before profiling was switched on can launch either; the grid is
  // the smaller of their co-resident counts
  int best = -1;
  for (int prof = 0; prof < (sample ? 1 : 2); prof++) {
    const void* fn = decode_fn(m.d.prec, sample, win, prof != 0);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, decode_threads_of(m.d.prec),
                                                      smem) != cudaSuccess)
      return 0;
    best = best < 0 ? per : (per < best ? per : best);
  }
  return best * sm_count;
}

cudaError_t launch_decode(const DeviceModel& m, const CodecBufs& b, const uint8_t* in,
                          const unsigned long long* d_offsets, int layout, int patch, int sched,
                          int T, int grid, cudaStream_t s, bool set_attr) {
  cudaError_t e;
  if (b.n_images == 0) return cudaSuccess;
  if ((e = launch_parse(m, b, in, d_offsets, layout, patch, s)) != cudaSuccess) return e;
  if (b.n_units == 0) return cudaSuccess;
  if ((e = cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
  if (b.times != nullptr && b.n_times > 0 &&
      (e = cudaMemsetAsync(b.times, 0, (size_t)b.n_times * sizeof(unsigned long long), s)) !=
          cudaSuccess)
    return e;
  DecodeArgs a;
  a.m = m;
  a.units = b.units;
  a.n_units = b.n_units;
  a.layout = layout;
  a.sched = sched;
  a.T = T;
  a.in = in;
  a.st = b.st;
  a.bar = b.bar;
  a.status = b.status;
  a.prof = b.prof;
  a.times = b.times;
  a.n_times = b.n_times;
  a.ring = b.ring;
  a.spin_limit = b.spin_limit ? b.spin_limit : kSpinLimit;
  a.mma_limit = b.mma_limit ? b.mma_limit : kMbarSpin;
  const bool win = b.ring != nullptr && sched == SCHED_WAVEFRONT;
  const size_t smem = decode_smem_bytes(m.d, b.n_units);
  const void* fn = decode_fn(m.d.prec, false, win, b.prof != nullptr);
  const int nt = decode_threads_of(m.d.prec);
  if (set_attr &&
      (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return e;
  a.seed = 0;
  void* args[] = {&a};
  if (grid > 1) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(nt), args, smem, s);
  return cudaLaunchKernel(fn, dim3(1), dim3(nt), args, smem, s);
}

cudaError_t launch_sample(const DeviceModel& m, const CodecBufs& b, int sched, int T, int grid,
                          unsigned long long seed, cudaStream_t s) {
  cudaError_t e;
  if (b.n_units == 0) return cudaSuccess;
  if ((e = cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
  DecodeArgs a;
  a.m = m;
  a.units = b.units;
  a.n_units = b.n_units;
  a.layout = 1;
  a.sched = sched;
  a.T = T;
  a.in = nullptr;
  a.st = nullptr;
  a.bar = b.bar;
  a.status = b.status;
  a.prof = nullptr;
  a.times = nullptr;
  a.n_times = 0;
  a.seed = seed;
  a.ring = b.ring;
  a.spin_limit = b.spin_limit ? b.spin_limit : kSpinLimit;
  a.mma_limit = b.mma_limit ? b.mma_limit : kMbarSpin;
  const bool win = b.ring != nullptr && sched == SCHED_WAVEFRONT;
  const size_t smem = decode_smem_bytes(m.d, b.n_units);
  const void* fn = decode_fn(m.d.prec, true, win);
  const int nt = decode_threads_of(m.d.prec);
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  void* args[] = {&a};
  if (grid > 1) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(nt), args, smem, s);
  return cudaLaunchKernel(fn, dim3(1), dim3(nt), args, smem, s);
}

}  // namespace nlc

// Shared device-side definitions of the nlc CUDA library (sm_103a).
//
// Everything that decides a frequency table is written with explicitly
// rounded intrinsics and the library is compiled with -fmad=false, so the
// table of a pixel is a pure function of its inputs: the encoder (all pixels
// in parallel) and the decoder (one wavefront per step) compute identical
// tables, which the rANS round trip requires (Section 4: the paper reuses
// the decoder's inference in the encoder for the same reason).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nlc {

constexpr uint32_t kRansL = 1u << 23;   // rANS state interval [2^23, 2^31)
constexpr int kMq = 65280;              // 2^16 - 256 counts spread by the CDF
constexpr int kMaxK = 16;               // mixture components
constexpr int kMaxR = 4;                // residual blocks
constexpr int kMaxH = 3;                // horizon
constexpr int kMaxC = 64;               // channels of the local network
constexpr int kThreads = 256;           // threads of the codec kernels
constexpr int kWarps = kThreads / 32;

enum Status {
  ST_OK = 0,
  ST_ARG = 1,
  ST_CAPACITY = 2,
  ST_CORRUPT = 3,
  ST_WEIGHTS = 4,
  ST_CUDA = 5,
  ST_TIMEOUT = 6,
  ST_UNSUPPORTED = 7,
};

enum Precision { PREC_FP32 = 0, PREC_BF16 = 1 };
enum Schedule { SCHED_RASTER = 0, SCHED_WAVEFRONT = 1 };

// Model dimensions.  F = 6h(h+1) context features (2h(h+1) pixels x RGB),
// Fp = F rounded up to a multiple of 16, NO = 10K network outputs, NOp = NO
// rounded up to a multiple of 16, ldP = NOp + 1 (row stride of the per-pixel
// outputs in shared memory; odd, against bank conflicts).
// shear = 1: the first layer is evaluated as the sheared kernels of Section
// 3.1 (Fig. 5) over the h+1 rows of the h(h+2) sheared columns before the
// pixel's own (Ws = h(h+2) pixels, 3 Ws features per window row, stored in
// rows of Fsp features, zero past 3 Ws); the network runs in BF16 (prec =
// PREC_BF16).
struct Dims {
  int h, C, R, K;
  int F, Fp, NO, NOp, ldP;
  int prec;
  int shear, Ws, Fsp;
};

// Sheared first layer, window row dd (0 = top): its taps sit at window
// columns qa .. qa + n - 1 (n = 2h+1 above the pixel's row, h in it), qa =
// Ws - (h+1)(h-dd) - h, i.e. features [3 qa, 3 (qa + n)); its MMAs cover
// the features [8 c_lo, 8 c_lo + 16 ks) (whole 8-feature chunks, K = 16 per
// MMA), the rest of the window row holds only zero weights.
__host__ __device__ __forceinline__ void shear_krange(int h, int Ws, int dd, int& c_lo, int& ks) {
  const int qa = Ws - (h + 1) * (h - dd) - h, n = dd < h ? 2 * h + 1 : h;
  c_lo = (3 * qa) / 8;
  ks = (3 * (qa + n) - 8 * c_lo + 15) / 16;
}
// Features per stored window row: every MMA's range inside it.
__host__ __device__ __forceinline__ int shear_row_features_n(int h) {
  const int Ws = h * (h + 2);
  int f = 0;
  for (int dd = 0; dd <= h; dd++) {
    int c, k;
    shear_krange(h, Ws, dd, c, k);
    f = f > 8 * c + 16 * k ? f : 8 * c + 16 * k;
  }
  return f;
}
// Offset (BF16 elements) of window row dd's kernel tile [C][16 ks] among the
// sheared tiles, and their total (dd = h + 1).
__host__ __device__ __forceinline__ int shear_tile_off(const Dims& d, int dd) {
  int off = 0;
  for (int e = 0; e < dd; e++) {
    int c, k;
    shear_krange(d.h, d.Ws, e, c, k);
    off += d.C * 16 * k;
  }
  return off;
}

// Precision byte of a container (and of the model's hash): 0 FP32, 1 BF16,
// 2 BF16 with the sheared first layer.
__host__ __device__ __forceinline__ int prec_code(const Dims& d) { return d.shear ? 2 : d.prec; }

// One coding unit (a whole image or one patch of it).
struct Unit {
  uint8_t* img;          // image base (decode: output; encode: input), HWC uint8
  long long px_base;     // pixels of all preceding units of the batch
  int img_W;             // image width (row stride = 3 * img_W bytes)
  int y0, x0, Hu, Wu;    // unit origin and size inside its image
  int stream_base;       // index of the unit's first rANS stream
  int start_step;        // global step at which the unit's local step 0 runs
  int image;             // image index in the batch
  int ring_row;          // rows of all preceding units (the sheared decoder's ring rows)
  long long img_px_base; // pixels of all preceding images (raster output order)
};

// Byte offsets of the packed weight blobs inside the device weight buffer.
struct WeightView {
  const float* simt;            // FP32: W0T[F][C] b0[C] {W1T[C][C] b1 W2T[C][C] b2}xR WHT[C][NOp] bH[NOp]
  const uint16_t* umma;         // BF16 UMMA tiles (see nlc_model.cuh)
  const float* bias;            // BF16 path biases: b0[C] {b1 b2}xR bH[NOp]
  int simt_floats;
  int umma_halves;
};

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Approximate 2^x and 1/x (PTX ex2.approx / rcp.approx): deterministic
// single MUFU instructions.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint8_t ld_cg_u8(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(v) : "l"(p));
  return (uint8_t)v;
}
__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014): the k-th output (k = 0, 1, ...) of the generator seeded
// with `seed` is the mixing function applied to seed + (k + 1) * gamma,
// gamma = 0x9E3779B97F4A7C15.  Used as a counter-based generator: the
// sampler's uniform 16-bit value of channel c of pixel (y, x) of image n is
// the top 16 bits of output k = ((n * 2^21 + y) * 2^21 + x) * 3 + c.
__host__ __device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                                     unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint32_t sample_u16(unsigned long long seed, int image, int y,
                                                        int x, int c) {
  const unsigned long long k =
      ((((unsigned long long)image << 21) + (unsigned long long)y) << 21) + (unsigned long long)x;
  return (uint32_t)(splitmix64_at(seed, 3ull * k + (unsigned long long)c) >> 48);
}

// The GPU's global nanosecond timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Asynchronous global -> shared copies (cp.async): no register receives the
// data, so nothing waits for it before cp_async_wait_all.  16 bytes through
// L2 only (both addresses 16-byte aligned), or 4 bytes (4-byte aligned)
// that read nothing and write zeros when !ok.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc),
               "r"(ok ? 4 : 0)
               : "memory");
}
// Waits for the calling thread's copies; other threads see them after a
// barrier that includes it.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch, split in two so that a CTA can
// do work that needs no other CTA's results between arriving and waiting.
// Arrival is a fire-and-forget atomic add to a counter that grows
// monotonically (generation g completes at nblocks * g arrivals, so it never
// needs a reset inside the launch); waiters poll the counter.  The wait is
// bounded: after kSpinLimit polls a CTA records ST_TIMEOUT and sets bit 31
// of the counter (kBarPoison), which releases every waiting CTA at once and
// tells it to leave its loop.  Counts stay below 2^31 (the host caps
// nblocks * steps).
constexpr unsigned kSpinLimit = 1u << 25;
constexpr unsigned kBarPoison = 0x80000000u;

// One thread of the CTA, after the CTA's writes (a __syncthreads() must
// precede): a release reduction, cumulative over the CTA's writes that the
// barrier made visible to that thread, with no wait for a reply.  The
// release holds the issuing warp until those writes are visible at GPU
// scope, so the caller issues it from a warp with nothing else to do.
__device__ __forceinline__ void grid_arrive(unsigned* count) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}

// Thread 0 waits until nblocks * target CTAs have arrived; then the whole CTA
// synchronises.  Returns false if the decode must stop (a timeout here or
// elsewhere).
__device__ __forceinline__ bool grid_wait(unsigned* count, unsigned nblocks, unsigned target,
                                          int* status, int* s_flag, unsigned limit = kSpinLimit) {
  if (threadIdx.x == 0 && *s_flag == 0) {
    const unsigned goal = nblocks * target;
    unsigned it = 0;
    for (;;) {
      const unsigned c = ld_acquire_gpu(count);
      if (c & kBarPoison) {
        *s_flag = 1;
        break;
      }
      if (c >= goal) break;
      if (++it > limit) {
        set_status(status, ST_TIMEOUT);
        atomicOr(count, kBarPoison);
        *s_flag = 1;
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  return *s_flag == 0;
}

// Front of a unit at its local step tau.
//   wavefront (Section 3): rows i with j = tau - (h+1) i in [0, Wu)
//   raster: the single pixel tau of the unit in raster order.
struct Front {
  int i_lo, n;  // first row and number of pixels
};

__device__ __forceinline__ Front unit_front(const Unit& u, int t, int h, int sched) {
  Front f{0, 0};
  int tau = t - u.start_step;
  if (tau < 0) return f;
  if (sched == SCHED_WAVEFRONT) {
    int o = h + 1;
    int hi = tau / o;
    if (hi > u.Hu - 1) hi = u.Hu - 1;
    int num = tau - u.Wu + 1;  // i >= ceil(num / o)
    int lo = num <= 0 ? 0 : (num + o - 1) / o;
    if (hi >= lo) { f.i_lo = lo; f.n = hi - lo + 1; }
  } else {
    if (tau < u.Hu * u.Wu) { f.i_lo = tau / u.Wu; f.n = 1; }
  }
  return f;
}

__device__ __forceinline__ int front_col(const Unit& u, int t, int i, int h, int sched) {
  int tau = t - u.start_step;
  return sched == SCHED_WAVEFRONT ? tau - (h + 1) * i : tau % u.Wu;
}

}  // namespace nlc

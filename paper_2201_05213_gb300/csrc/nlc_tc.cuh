// BF16 local network on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// A tile is M = 128 pixels.  Each layer is one chain of
// tcgen05.mma.cta_group::1.kind::f16 instructions (K = 16 per instruction,
// FP32 accumulation in TMEM columns [0, 128)) issued by one thread; the
// accumulator is read back with tcgen05.ld by all warps (warp w reads TMEM
// lanes 32(w%4)..+31, i.e. its rows, and 8-column chunks w/4, w/4 + NP, ...),
// bias/ELU/residual are applied in registers, and the next layer's A
// operand stays in tensor memory: each thread writes its row's BF16 pairs
// with tcgen05.st into columns [128, 128 + C/2) (lane m = row m, column
// 128 + k/2 = elements k, k+1), which the next tcgen05.mma reads as its A
// operand (8 columns per K step).  The first layer's A operand (the context
// tile) and every B operand (the weights) are in shared memory, in the
// canonical no-swizzle K-major layout:
//   element (r, k) of an R x Kd matrix at
//   ((r/8) * (Kd/8) + k/8) * 64 + (r%8) * 8 + (k%8)   (BF16 elements)
// i.e. 8x8 core matrices of 128 contiguous bytes; the leading-dimension byte
// offset (next core matrix along K) is 128 and the stride-dimension byte
// offset (next 8-row group) is Kd/8 * 128.
//
// Network input: the integer 2v-255 (exact in BF16); the 1/255 of the scaled
// pixel value (2v-255)/255 is folded into the first-layer weights.  The
// residual stream stays in FP32 registers; only layer inputs are BF16.
#pragma once

#include <cuda_bf16.h>

#include "nlc_common.cuh"
#include "nlc_model.cuh"

namespace nlc {

constexpr int kTcM = 128;
constexpr int kTileMax = 128;
constexpr int kTmemCols = 256;  // accumulator [0, 128), A operand [128, 128 + C/2)
constexpr int kAcol = 128;       // first TMEM column of the A operand
constexpr unsigned kMbarSpin = 1u << 22;

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Rows of the sheared decoder's window tile: a tile of 128 output rows reads
// window rows m .. m + h (h <= 3), rounded up to a multiple of 8.
constexpr int kWinRows = 136;

struct TcPlan {
  int w0, w1[kMaxR], w2[kMaxR], wh, w0s, bias, p, mbar, tslot, sdesc, end;
};

// Sheared first layer: at most 8 MMAs (7 for h = 3); their (A, B)
// descriptors for both A layouts, built once per CTA, behind a count.
constexpr int kShearMaxMma = 8;

__host__ __device__ inline TcPlan tc_plan(const Dims& d) {
  TcPlan p;
  int o = 0;
  p.w0 = o;
  o += d.C * d.Fp * 2;
  for (int r = 0; r < kMaxR; r++) {
    p.w1[r] = o;
    if (r < d.R) o += d.C * d.C * 2;
    p.w2[r] = o;
    if (r < d.R) o += d.C * d.C * 2;
  }
  p.wh = o;
  o += d.NOp * d.C * 2;
  // sheared first layer: h+1 tiles [C][16 ks(dd)], one per window row (top
  // first), each only over the window row's tap range
  p.w0s = o;
  if (d.shear) o += shear_tile_off(d, d.h + 1) * 2;
  p.bias = o;
  o += (d.C + 2 * d.R * d.C + d.NOp) * 4;
  o = align_up(o, 128);
  p.p = o;  // P[m][ldP] FP32, aliased with the BF16 context tile(s) X
  int pbytes = kTcM * d.ldP * 4, xbytes = kTcM * d.Fp * 2;
  if (d.shear) {
    const int per_px = (d.h + 1) * kTcM * d.Fsp * 2, win = d.Fsp * kWinRows * 2;
    xbytes = per_px > win ? per_px : win;
  }
  o += pbytes > xbytes ? pbytes : xbytes;
  o = align_up(o, 16);
  p.mbar = o;
  o += 8;
  p.tslot = o;
  o += 8;
  p.sdesc = o;  // [0]: count (set by tc_setup for every model); then (a_px, a_win, b) per MMA
  o += 8;
  if (d.shear) o += 3 * 8 * kShearMaxMma;
  p.end = align_up(o, 128);
  return p;
}

__host__ __device__ inline size_t tc_smem_bytes(const Dims& d) { return (size_t)tc_plan(d).end; }
// BF16 weight tiles: the tap-ordered first layer, the residual blocks and the
// head (umma_plain_halves), then, for a sheared model, the sheared first layer.
__host__ __device__ inline size_t umma_plain_halves(const Dims& d) {
  return (size_t)d.C * d.Fp + 2 * (size_t)d.R * d.C * d.C + (size_t)d.NOp * d.C;
}
__host__ __device__ inline size_t umma_halves(const Dims& d) {
  return umma_plain_halves(d) + (d.shear ? (size_t)shear_tile_off(d, d.h + 1) : 0);
}
__host__ __device__ inline size_t bias_floats(const Dims& d) { return (size_t)d.C + 2 * (size_t)d.R * d.C + d.NOp; }

struct TcSmem {
  unsigned char* base;
  uint16_t* X;
  float* P;
  float* bias;
  uint64_t* mbar;
  uint32_t* tslot;
  uint64_t* sdesc;  // sheared first layer's descriptors (thread 0 only)
  uint32_t tmem;
  uint32_t phase;
  int ok;
  unsigned mma_limit;  // polls of an MMA completion before a timeout is recorded
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ __forceinline__ int umma_off(int r, int k, int Kd) {
  return ((r >> 3) * (Kd >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ TcSmem tc_carve(const Dims& d, unsigned char* smem) {
  TcPlan p = tc_plan(d);
  TcSmem t;
  t.base = smem;
  t.X = reinterpret_cast<uint16_t*>(smem + p.p);
  t.P = reinterpret_cast<float*>(smem + p.p);
  t.bias = reinterpret_cast<float*>(smem + p.bias);
  t.mbar = reinterpret_cast<uint64_t*>(smem + p.mbar);
  t.tslot = reinterpret_cast<uint32_t*>(smem + p.tslot);
  t.sdesc = reinterpret_cast<uint64_t*>(smem + p.sdesc);
  t.tmem = 0;
  t.phase = 0;
  t.ok = 1;
  t.mma_limit = kMbarSpin;
  return t;
}

// --- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, relative LBO, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase,
                                          unsigned limit = kMbarSpin) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Non-blocking test of an mbarrier phase, at most `limit` times.
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t phase, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}

// 32 consecutive FP32 columns of this thread's TMEM lane (one load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// The columns c0 .. c0 + ch - 1 (ch = 8, 16, 24 or 32) of this thread's lane.
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, int ch, float (&v)[32]) {
  if (ch == 32) {
    tmem_ld32(taddr, v);
  } else {
#pragma unroll
    for (int g = 0; g < 4; g++) {
      if (g < ch / 8) {
        float u[8];
        tmem_ld8(taddr + (uint32_t)(8 * g), u);
#pragma unroll
        for (int e = 0; e < 8; e++) v[8 * g + e] = u[e];
      }
    }
  }
}

// --- setup / teardown -------------------------------------------------------
__device__ __forceinline__ void tc_setup(TcSmem& t) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(t.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    t.sdesc[0] = 0;  // the sheared layer's descriptors are built on first use
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(t.tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  t.tmem = *t.tslot;
  t.phase = 0;
  t.ok = 1;
}

__device__ __forceinline__ void tc_teardown(TcSmem& t) {
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem),
                 "r"(kTmemCols)
                 : "memory");
}

__device__ __forceinline__ void tc_load_weights(const Dims& d, const WeightView& w, TcSmem& t) {
  const int nh = w.umma_halves;  // multiple of 64 (core matrices)
  const uint4* src = reinterpret_cast<const uint4*>(w.umma);
  uint4* dst = reinterpret_cast<uint4*>(t.base);
  for (int i = threadIdx.x; i < nh / 8; i += blockDim.x) dst[i] = src[i];
  const int nb = (int)bias_floats(d);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) t.bias[i] = w.bias[i];
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// --- gather ------------------------------------------------------------------
// X(m, k) = 2v - 255 for feature k = 3p + c of tap p, 0 outside the unit and
// for F <= k < Fp.  One lane per (pixel m, context row r): row r < h is image
// row i - h + r over columns j-h .. j+h, row h is row i over columns j-h ..
// j-1 (the taps of Eq. 3 in raster order).  A row's 3(2h+1) (or 3h) bytes are
// contiguous in the image and are features k0 = 3 r (2h+1) onwards, so the
// lane reads the aligned 32-bit words that hold at least one byte of the row
// inside the unit (never a word without a byte of the image), realigns them
// with funnel shifts and writes the features.  A warp covers 8 pixels x 4
// rows, so the four rows' stores of one feature index fall on different banks.
template <bool kCoherent>
__device__ __noinline__ void tc_gather(const Unit* units, const PixSlot* slots, const Dims& d,
                                       TcSmem& t, int n_valid) {
  const int h = d.h, Fp = d.Fp, F = d.F, w2 = 2 * h + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane >> 3;
  for (int mb = 8 * warp; mb < n_valid; mb += 8 * (int)(blockDim.x >> 5)) {
    const int m = mb + (lane & 7);
    if (r > h || m >= n_valid) continue;
    const PixSlot s = slots[m];
    const Unit u = units[s.unit];
    const int y = r < h ? s.i - h + r : s.i;
    const int ncol = r < h ? w2 : h;  // pixels of this row's window
    const int k0 = 3 * r * w2;
    // window columns x = j - h + c, c in [0, ncol); inside the unit: [ca, cb)
    const int x0 = s.j - h;
    const int ca = x0 < 0 ? -x0 : 0;
    const int cb = min(ncol, u.Wu - x0);
    const bool row_ok = y >= 0 && y < u.Hu && ca < cb;
    uint32_t wv[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
    uint32_t sh = 0;
    if (row_ok) {
      const uintptr_t row = (uintptr_t)(u.img + ((long long)(u.y0 + y) * u.img_W + u.x0) * 3);
      const uintptr_t lo = row + (uintptr_t)(3 * (long long)x0);  // window start
      const uintptr_t a = lo + 3 * ca, b = lo + 3 * cb;         // bytes inside the unit
      const uintptr_t w0 = lo & ~(uintptr_t)3;
      sh = 8u * (uint32_t)(lo & 3);
#pragma unroll
      for (int q = 0; q < 6; q++) {
        const uintptr_t wa = w0 + 4 * q;
        if (wa + 4 > a && wa < b) {
          const uint32_t* p = reinterpret_cast<const uint32_t*>(wa);
          wv[q] = kCoherent ? ld_cg_u32(p) : *p;
        }
      }
    }
    uint32_t al[6];
#pragma unroll
    for (int q = 0; q < 6; q++) al[q] = __funnelshift_r(wv[q], wv[q + 1], sh);
    uint16_t* X = t.X;
#pragma unroll
    for (int q = 0; q < 3 * (2 * kMaxH + 1); q++) {
      const int c = q / 3;
      if (c < ncol) {
        const int v = (int)((al[q >> 2] >> (8 * (q & 3))) & 0xFFu);
        const float x = (row_ok && c >= ca && c < cb) ? (float)(2 * v - 255) : 0.f;
        X[umma_off(m, k0 + q, Fp)] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
      }
    }
    if (r == h)
      for (int k = F; k < Fp; k++) X[umma_off(m, k, Fp)] = 0;
  }
}

// --- sheared first layer (Section 3.1, Fig. 5) ---------------------------------
// Window row dd (0 = top, h = the pixel's own row) of pixel (i, j) at
// wavefront step t = j + (h+1) i: unit row i - h + dd, the Ws = h(h+2)
// sheared columns t - Ws .. t - 1, i.e. image columns j0 .. j0 + Ws - 1 with
// j0 = j + (h+1)(h - dd) - Ws; feature 3q + c is channel c of window column
// q (2v - 255, 0 outside the unit), features 3 Ws .. Fsp - 1 are 0.  The
// sheared kernels give the taps of Eq. 3 their weights and every other
// window position 0, so the layer equals the masked one.

// Writes the Fsp features of one window row (3 Ws bytes at the realigned
// words al[], zero outside columns [ca, cb) of the window) as BF16 8-feature
// chunks: chunk kc to dst(kc).
template <class Dst>
__device__ __forceinline__ void shear_row_features(const uint32_t (&al)[12], int Ws, int Fsp,
                                                   int ca, int cb, bool ok, Dst dst) {
#pragma unroll
  for (int kc = 0; kc < 7; kc++) {  // Fsp <= 56
    if (kc >= Fsp / 8) break;
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float xv[2];
#pragma unroll
      for (int f = 0; f < 2; f++) {
        const int k = 8 * kc + e + f, q = k / 3;
        const int v = (int)((al[(k >> 2) < 12 ? (k >> 2) : 11] >> (8 * (k & 3))) & 0xFFu);
        xv[f] = (k < 3 * Ws && ok && q >= ca && q < cb) ? (float)(2 * v - 255) : 0.f;
      }
      pk[e / 2] = pack_bf16(xv[0], xv[1]);
    }
    *dst(kc) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// Per-pixel window rows: h+1 tiles [128][Fsp] (canonical K-major), tile dd
// at X + dd * 128 * Fsp.  One lane per (pixel m, window row dd), reading the
// aligned 32-bit words that hold at least one byte of the row inside the
// unit, as tc_gather does.
template <bool kCoherent>
__device__ __noinline__ void tc_gather_shear_px(const Unit* units, const PixSlot* slots,
                                                const Dims& d, TcSmem& t, int n_valid) {
  const int h = d.h, Ws = d.Ws, Fsp = d.Fsp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int dd = lane >> 3;
  for (int mb = 8 * warp; mb < n_valid; mb += 8 * (int)(blockDim.x >> 5)) {
    const int m = mb + (lane & 7);
    if (dd > h || m >= n_valid) continue;
    const PixSlot s = slots[m];
    const Unit u = units[s.unit];
    const int y = s.i - h + dd;
    const int x0 = s.j + (h + 1) * (h - dd) - Ws;
    const int ca = x0 < 0 ? -x0 : 0;
    const int cb = min(Ws, u.Wu - x0);
    const bool row_ok = y >= 0 && ca < cb;
    uint32_t wv[13];
#pragma unroll
    for (int q = 0; q < 13; q++) wv[q] = 0u;
    uint32_t sh = 0;
    if (row_ok) {
      const uintptr_t row = (uintptr_t)(u.img + ((long long)(u.y0 + y) * u.img_W + u.x0) * 3);
      const uintptr_t lo = row + (uintptr_t)(3 * (long long)x0);
      const uintptr_t a = lo + 3 * ca, b = lo + 3 * cb;
      const uintptr_t w0 = lo & ~(uintptr_t)3;
      sh = 8u * (uint32_t)(lo & 3);
#pragma unroll
      for (int q = 0; q < 13; q++) {
        const uintptr_t wa = w0 + 4 * q;
        if (wa + 4 > a && wa < b) {
          const uint32_t* p = reinterpret_cast<const uint32_t*>(wa);
          wv[q] = kCoherent ? ld_cg_u32(p) : *p;
        }
      }
    }
    uint32_t al[12];
#pragma unroll
    for (int q = 0; q < 12; q++) al[q] = __funnelshift_r(wv[q], wv[q + 1], sh);
    uint16_t* X = t.X + (size_t)dd * kTcM * Fsp;
    shear_row_features(al, Ws, Fsp, ca, cb, row_ok, [&](int kc) {
      return reinterpret_cast<uint4*>(X + umma_off(m, 8 * kc, Fsp));
    });
  }
}

// Bytes of a unit row in the sheared ring: the pixel of sheared column c is
// stored twice, at slots c mod 16 and c mod 16 + 16 (3 bytes each), so that
// the Ws <= 15 columns before any column are one contiguous byte range.
constexpr int kRingRowBytes = 96;

// Window tile of a sheared wavefront step, K-chunk-major: feature k of window
// row rho at X + (k/8) * kWinRows * 8 + rho * 8 + k % 8 (BF16), so that
// consecutive rows are 16 bytes apart and the A operand of window row dd of
// output row m is the tile started dd rows further.  wrow[rho] = (unit, unit
// row) of window row rho (unit -1: a zero row); the decoded pixels come from
// the units' sheared rings (unit u's row r at ring + 96 (u.ring_row + r)).
static __device__ __noinline__ void tc_gather_shear_win(const Unit* units, const int2* wrow,
                                                        const uint8_t* ring, const Dims& d,
                                                        TcSmem& t, int step, int n_rows) {
  const int h = d.h, Ws = d.Ws, nch = d.Fsp / 8;
  // window columns step - Ws .. step - 1: ring bytes from 3 ((step - Ws) mod 16);
  // feature k of a window row is byte k of that range
  const int c0 = step - Ws;
  const int b0 = 3 * (c0 & 15);
  uint16_t* X = t.X;
  // one item per (window row, 8-feature chunk); rows past n_rows feed only
  // output rows that hold no pixel and are left as they are
  for (int it = threadIdx.x; it < n_rows * nch; it += blockDim.x) {
    const int rho = it / nch, kc = it - rho * nch;
    const int2 wr = wrow[rho];
    uint32_t w0 = 0u, w1 = 0u, w2 = 0u;
    int ca = 0, cb = 0;
    const int bs = b0 + 8 * kc;  // first ring byte of the chunk (<= 85)
    if (wr.x >= 0 && wr.y >= 0 && 8 * kc < 3 * Ws) {
      const Unit u = units[wr.x];
      const int j0 = c0 - (h + 1) * wr.y;  // image column of window column 0
      ca = j0 < 0 ? -j0 : 0;
      cb = min(Ws, u.Wu - j0);
      if (ca < cb) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(
            ring + (long long)kRingRowBytes * (u.ring_row + wr.y) + (bs & ~3));
        w0 = ld_cg_u32(src);
        w1 = ld_cg_u32(src + 1);
        if ((bs & ~3) + 8 < kRingRowBytes) w2 = ld_cg_u32(src + 2);
      }
    }
    const uint32_t sh = 8u * (uint32_t)(bs & 3);
    const uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float xv[2];
#pragma unroll
      for (int f = 0; f < 2; f++) {
        const int k = 8 * kc + e + f, q = k / 3;
        const uint32_t byte = ((e + f) < 4 ? lo >> (8 * (e + f)) : hi >> (8 * (e + f - 4))) & 0xFFu;
        xv[f] = (k < 3 * Ws && q >= ca && q < cb) ? (float)(2 * (int)byte - 255) : 0.f;
      }
      pk[e / 2] = pack_bf16(xv[0], xv[1]);
    }
    *reinterpret_cast<uint4*>(X + (size_t)kc * kWinRows * 8 + (size_t)rho * 8) =
        make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// The sheared first layer: for window rows dd = 0..h, ks(dd) MMAs of A = the
// tap range of window row dd of every output row against B = its sheared
// kernel tile, accumulated in one chain (the same instructions for both A
// layouts, so the per-pixel and the window tile give the same bits).
__device__ __forceinline__ void tc_issue_shear(const TcSmem& t, const TcPlan& pl, const Dims& d,
                                               bool win) {
  if (threadIdx.x == 0) {
    fence_after_sync();
    uint64_t* sd = t.sdesc;
    if (sd[0] == 0) {  // first use by this CTA: every MMA's descriptors
      int n = 0;
      for (int dd = 0; dd <= d.h; dd++) {
        int c_lo, ks;
        shear_krange(d.h, d.Ws, dd, c_lo, ks);
        // window tile: rows 16 bytes apart, K chunks kWinRows rows apart
        const uint32_t w_lbo = (uint32_t)kWinRows * 16u;
        const uint32_t aw = smem_u32(t.X) + 16u * (uint32_t)dd + (uint32_t)c_lo * w_lbo;
        // per-pixel tile dd, canonical
        const uint32_t ap = smem_u32(t.X + (size_t)dd * kTcM * d.Fsp) + 128u * (uint32_t)c_lo;
        const uint32_t p_sbo = (uint32_t)(d.Fsp / 8) * 128u;
        const uint32_t b = smem_u32(t.base + pl.w0s) + (uint32_t)(shear_tile_off(d, dd) * 2);
        const uint32_t b_sbo = (uint32_t)(2 * ks) * 128u;
        for (int k = 0; k < ks; k++, n++) {
          sd[1 + 3 * n] = umma_desc(ap + 256u * (uint32_t)k, 128u, p_sbo);
          sd[2 + 3 * n] = umma_desc(aw + 2u * w_lbo * (uint32_t)k, w_lbo, 128u);
          sd[3 + 3 * n] = umma_desc(b + 256u * (uint32_t)k, 128u, b_sbo);
        }
      }
      sd[0] = (uint64_t)n;
    }
    const uint32_t idesc = idesc_bf16(kTcM, d.C);
    const int n = (int)sd[0];
    for (int k = 0; k < n; k++)
      mma_bf16(t.tmem, sd[(win ? 2 : 1) + 3 * k], sd[3 + 3 * k], idesc, k > 0 ? 1u : 0u);
    mma_commit(t.mbar);
  }
}

// --- network -----------------------------------------------------------------
__device__ __forceinline__ void tc_issue(const TcSmem& t, uint32_t a_off, uint32_t b_off, int Kd,
                                         int N) {
  if (threadIdx.x == 0) {
    fence_after_sync();
    const uint32_t sbo = (uint32_t)(Kd / 8) * 128u;
    const uint64_t da = umma_desc(smem_u32(t.base + a_off), 128u, sbo);
    const uint64_t db = umma_desc(smem_u32(t.base + b_off), 128u, sbo);
    const uint32_t idesc = idesc_bf16(kTcM, N);
    const uint32_t tm = t.tmem;
    // K step s starts 256 bytes further: +16 in the descriptors' address
    // field (Kd <= 80: at most 5 steps)
    mma_bf16(tm, da, db, idesc, 0u);
    if (Kd / 16 > 1) mma_bf16(tm, da + 16, db + 16, idesc, 1u);
    if (Kd / 16 > 2) mma_bf16(tm, da + 32, db + 32, idesc, 1u);
    if (Kd / 16 > 3) mma_bf16(tm, da + 48, db + 48, idesc, 1u);
    if (Kd / 16 > 4) mma_bf16(tm, da + 64, db + 64, idesc, 1u);
    mma_commit(t.mbar);
  }
}

// Layers 1..: A from tensor memory (columns kAcol + 8 s for K step s).
__device__ __forceinline__ void mma_bf16_ta(uint32_t dtm, uint32_t atm, uint64_t bd,
                                            uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
      "r"(atm), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_issue_ta(const TcSmem& t, uint32_t b_off, int Kd, int N) {
  if (threadIdx.x == 0) {
    fence_after_sync();
    const uint64_t db = umma_desc(smem_u32(t.base + b_off), 128u, (uint32_t)(Kd / 8) * 128u);
    const uint32_t idesc = idesc_bf16(kTcM, N);
    const uint32_t tm = t.tmem, ta = t.tmem + (uint32_t)kAcol;
    mma_bf16_ta(tm, ta, db, idesc, 0u);  // Kd = C <= 64: at most 4 steps
    if (Kd / 16 > 1) mma_bf16_ta(tm, ta + 8u, db + 16, idesc, 1u);
    if (Kd / 16 > 2) mma_bf16_ta(tm, ta + 16u, db + 32, idesc, 1u);
    if (Kd / 16 > 3) mma_bf16_ta(tm, ta + 24u, db + 48, idesc, 1u);
    mma_commit(t.mbar);
  }
}

// A wait that gives up after t.mma_limit polls reports the timeout, then
// waits (bounded by the default limit) for the MMAs it issued, so that no
// tensor-core write is in flight when the caller goes on or frees its
// tensor memory.
__device__ __forceinline__ bool tc_wait(TcSmem& t) {
  // a reduced limit counts non-blocking tests (a blocking try_wait may
  // itself suspend until the phase completes)
  bool ok = t.mma_limit >= kMbarSpin ? mbar_wait(t.mbar, t.phase)
                                     : mbar_test(t.mbar, t.phase, t.mma_limit);
  if (!ok) mbar_wait(t.mbar, t.phase);
  t.phase ^= 1u;
  fence_after_sync();
  return ok;
}

__device__ __forceinline__ float elu_tc(float x) {
  return x > 0.f ? x : __fsub_rn(ex2_approx(__fmul_rn(x, 1.4426950408889634f)), 1.f);
}

// Writes 8 BF16 values (A-operand elements k0..k0+7 of this thread's row)
// to tensor memory at taddr (4 columns), without waiting (tmem_wait_st).
__device__ __forceinline__ void tmem_st8_bf16(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(pack_bf16(v[0], v[1])), "r"(pack_bf16(v[2], v[3])), "r"(pack_bf16(v[4], v[5])),
               "r"(pack_bf16(v[6], v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane, without waiting:
// the registers hold the values only after tmem_wait_ld() and tmem_touch().
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Orders every use of r after the preceding tmem_wait_ld (the registers pass
// through an asm that the compiler cannot move above the wait).
__device__ __forceinline__ void tmem_touch(uint32_t (&r)[8]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]));
}

// Runs the whole network on the tile in X; P[m][ldP] = head outputs.
//
// Epilogues: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the
// 8-column chunks c = w/4, w/4 + NP, ... (NP = NT/128 column parts), issuing
// all its loads before one wait.  With pc non-null, thread 0 adds its cycles
// from MMA issue to completion to pc[14] and those of the epilogues (TMEM
// loads, bias/ELU, operand stores, CTA barriers) to pc[15].
template <int NT>
__device__ __noinline__ bool tc_network(const Dims& d, TcSmem& t, int n_valid, long long* pc,
                                        bool win = false) {
  constexpr int NP = NT / 128;                // column parts
  constexpr int CH = (kMaxC / 8 + NP - 1) / NP;  // chunks of the hidden width per thread
  constexpr int HB = 4;                       // head chunks per load batch
  const TcPlan pl = tc_plan(d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;
  const int part = warp >> 2;
  // a warp whose 32 TMEM lanes hold no valid pixel skips its epilogue
  const bool live = 32 * (warp & 3) < n_valid;
  const uint32_t tl = t.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t ta = tl + (uint32_t)kAcol;  // this warp's lanes of the A operand
  const int C = d.C, nc = C / 8;
  float a[CH][8];
  bool ok = true;
  const bool pr = pc != nullptr && threadIdx.x == 0;
  long long ck = pr ? clock64() : 0;
  auto tick = [&](int slot) {
    if (pr) {
      const long long n_ = clock64();
      pc[slot] += n_ - ck;
      ck = n_;
    }
  };
  // epilogue of a hidden layer: v = acc + bias (+ residual), H = ELU(v)
  auto hidden = [&](const float* bias, int mode) {  // 0: a = v, 1: a += v, 2: H only
    if (live) {
      uint32_t r[CH][8];
#pragma unroll
      for (int i = 0; i < CH; i++)
        if (part + NP * i < nc) tmem_ld8_nw(tl + (uint32_t)(8 * (part + NP * i)), r[i]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < CH; i++) {
        const int c = part + NP * i;
        if (c < nc) {
          tmem_touch(r[i]);
          float u[8];
#pragma unroll
          for (int e = 0; e < 8; e++) {
            const float v = __fadd_rn(__uint_as_float(r[i][e]), bias[8 * c + e]);
            if (mode == 0) a[i][e] = v;
            if (mode == 1) a[i][e] = __fadd_rn(a[i][e], v);
            u[e] = elu_tc(mode == 2 ? v : a[i][e]);
          }
          tmem_st8_bf16(ta + (uint32_t)(4 * c), u);
        }
      }
      tmem_wait_st();
    }
    fence_before_sync();
    __syncthreads();
  };

  // layer 0: a = X W0^T + b0
  fence_async_smem();
  __syncthreads();
  tick(15);
  if (d.shear) tc_issue_shear(t, pl, d, win);
  else tc_issue(t, (uint32_t)pl.p, (uint32_t)pl.w0, d.Fp, C);
  ok &= tc_wait(t);
  tick(14);
  // The hidden layers' epilogues in order, each followed by the next layer's
  // MMAs: layer 0 (H = ELU(a)), then per residual block r the inner layer
  // (hidden = ELU(H W1^T + b1)) and the outer one (a += H W2^T + b2, H =
  // ELU(a)); the last one is followed by the head, P = H WH^T + bH.  (One
  // loop over the layers: written out per block, the same steps left the
  // coding function, compiled in the same unit, with three times the spills.)
  const int n_hidden = 1 + 2 * d.R;
  for (int l = 0; l < n_hidden; l++) {
    // layer l's biases: b0 at 0, then b1, b2 of block r at C + 2 r C, C + (2 r + 1) C
    hidden(l == 0 ? t.bias : t.bias + C + (l - 1) * C, l == 0 ? 0 : ((l - 1) % 2 == 0 ? 2 : 1));
    tick(15);
    const int nl = l + 1;  // the layer issued next
    if (nl == n_hidden)
      tc_issue_ta(t, (uint32_t)pl.wh, C, d.NOp);
    else
      tc_issue_ta(t, (uint32_t)((nl - 1) % 2 == 0 ? pl.w1[(nl - 1) / 2] : pl.w2[(nl - 1) / 2]), C, C);
    ok &= tc_wait(t);
    tick(14);
  }

  // head epilogue: P = acc + bH, in batches of HB chunks
  const float* bh = t.bias + C + 2 * d.R * C;
  if (live) {
    const int nh = d.NOp / 8;
    float* o = t.P + (size_t)row * d.ldP;
    for (int c0 = part; c0 < nh; c0 += NP * HB) {
      uint32_t r[HB][8];
#pragma unroll
      for (int i = 0; i < HB; i++)
        if (c0 + NP * i < nh) tmem_ld8_nw(tl + (uint32_t)(8 * (c0 + NP * i)), r[i]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < HB; i++) {
        const int c = c0 + NP * i;
        if (c < nh) {
          tmem_touch(r[i]);
#pragma unroll
          for (int e = 0; e < 8; e++) o[8 * c + e] = __fadd_rn(__uint_as_float(r[i][e]), bh[8 * c + e]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  tick(15);
  return all_ok;
}

cudaError_t launch_repack_umma(const Dims& d, const float* w, uint16_t* umma, float* bias,
                               cudaStream_t s);

}  // namespace nlc

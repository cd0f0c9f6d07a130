// Maximum-likelihood training (Eq. 2) of a BF16 model on the 5th-generation
// tensor cores: forward, mixture likelihood and adjoint of one 128-pixel tile
// per step of a persistent loop, every contraction a tcgen05.mma chain with
// FP32 accumulation in tensor memory.
//
// Per tile (pixels p, layers l with weights W_l[o][i]):
//   forward   Y_l = X_l W_l^T  (A = activations, B = weights, both K-major)
//   adjoint   dX_l = dY_l W_l  (A = dY K-major, B = W_l read MN-major)
//   weights   dW_l = dY_l^T X_l (A = dY read MN-major, B = X_l read MN-major)
//   biases    db_l = dY_l^T 1   (A = dY read MN-major, B = a 16 x 16 tile of ones)
// so every operand stays in its natural pixel-row layout in shared memory
// (8 x 8 core matrices of 128 contiguous bytes, K-major for the forward) and
// the transposes are the instruction descriptor's transpose bits.  For an
// MN-major operand the descriptor's leading byte offset is the stride of
// core matrices along K and the stride byte offset their stride along M/N.
// The weight-gradient chains use M = 128 rows of which the first n_out are
// the layer's outputs (the others read the neighbouring core matrices and
// are discarded).  Each layer's weight and bias gradients are added to the
// CTA's own FP32 slot in global memory after its chain completes (every
// element by one thread, tiles in a fixed order), and a second kernel sums
// the slots in a fixed order: the result is deterministic.
//
// Activations: the integer 2v-255 as the first layer's input (the 1/255 is
// folded into W0, so its gradient is scaled by 1/255 on the way out), then
// u = ELU(a) and v = ELU(z) in BF16; ELU'(t) = 1 for t > 0 and ELU(t) + 1
// otherwise, taken from the stored BF16 activation.  The residual stream and
// its gradient stay in FP32 registers.  The mixture likelihood and its
// gradient with respect to the 10K network outputs are FP32; the outputs are
// read straight from tensor memory (two threads per pixel, each holding
// every other mixture component) and the gradient is stored in BF16 as the
// A operand of the head's adjoint.  256 threads per CTA: each thread owns a
// pixel row and half of its columns, within the register budget.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"
#include "nlc_model.cuh"
#include "nlc_tc.cuh"
#include "nlc_train.cuh"

namespace nlc {

constexpr int kTT = 256;                  // threads (8 warps)
constexpr int kTTM = 128;                 // pixels per tile (the MMA's M)
constexpr int kParts = kTT / kTTM;        // threads per pixel row (column parts)
constexpr uint32_t kTTCols = 512;         // tensor-memory columns
constexpr uint32_t kColAcc = 0;           // forward / adjoint accumulator (N <= 160)
constexpr uint32_t kColDW = 256;          // weight-gradient accumulator (N <= Fp <= 80)
constexpr uint32_t kColDB = 384;          // bias-gradient accumulator (N = 16)
constexpr uint32_t kColRes = 400;         // residual stream / its gradient (FP32, C <= 64)
constexpr int kCompPerThread = (kMaxK + kParts - 1) / kParts;
constexpr int kChunks = (kMaxC / 8 + kParts - 1) / kParts;  // 8-column chunks per thread
constexpr int kLbStride = kMaxK + 1;  // per-row table of l_k (odd: rows on different banks)

// Byte offsets of the shared-memory regions.  Residual block r's tiles are
// at w1 + r * wstride (W1) and w1 + r * wstride + wstride / 2 (W2): plain
// arithmetic, so that no offset table has to live in local memory.
struct TTPlan {
  int w0, w1, wstride, wh;  // BF16 weight tiles (the decoder's layout)
  int bias, ones, u, gx, g2, xe, red, slots, taps, mbar, tslot, end;
  bool fits;
};

__host__ __device__ inline int tile_bytes(int ncol) { return kTTM * ncol * 2; }

__host__ __device__ inline TTPlan tt_plan(const Dims& d) {
  Dims dp_ = d;
  dp_.shear = 0;  // the trainer's tiles: the plain layout (no sheared first layer)
  const TcPlan tp = tc_plan(dp_);
  TTPlan p;
  p.w0 = tp.w0;
  p.w1 = tp.w1[0];
  p.wstride = 4 * d.C * d.C;
  p.wh = tp.wh;
  int o = tp.bias;
  p.bias = o;
  o += (d.C + 2 * d.R * d.C + d.NOp) * 4;
  o = align_up(o, 128);
  p.ones = o;  // 16 x 16 BF16 ones
  o += 512;
  p.u = o;  // 2R+1 activation tiles [128][C]
  o += (2 * d.R + 1) * tile_bytes(d.C);
  // gradient region: X during the forward, then dP [128][NOp] with the
  // likelihood's per-row table [128][17], then G and G2 [128][C]
  p.gx = o;
  p.g2 = o + tile_bytes(d.C);
  const int dp = tile_bytes(d.NOp);
  p.red = o + dp;
  int need = dp + kTTM * kLbStride * 4;
  if (need < 2 * tile_bytes(d.C)) need = 2 * tile_bytes(d.C);
  if (need < tile_bytes(d.Fp)) need = tile_bytes(d.Fp);
  // X for the first layer's weight gradient, gathered again after the
  // adjoint: into the activation tiles when they are large enough
  if ((2 * d.R + 1) * tile_bytes(d.C) >= tile_bytes(d.Fp)) {
    p.xe = p.u;
  } else {
    p.xe = o + tile_bytes(d.C);
    if (need < tile_bytes(d.C) + tile_bytes(d.Fp)) need = tile_bytes(d.C) + tile_bytes(d.Fp);
  }
  // the weight-gradient chains read up to (128 - n_out)/8 core matrices
  // past a gradient tile's end (discarded rows): keep them inside the block
  o += need + 1024;
  o = align_up(o, 16);
  p.slots = o;  // (image, i, j, valid) per pixel
  o += kTTM * 16;
  p.taps = o;  // (dy, dx) of the context taps (Eq. 3), 2h(h+1) <= 24
  o += 24 * 8;
  p.mbar = o;
  o += 8;
  p.tslot = o;
  o += 8;
  p.end = align_up(o, 128);
  p.fits = p.end <= 227 * 1024 && d.NOp <= 160 && d.Fp <= 80;
  return p;
}

bool tc_train_fits(const Dims& d) { return tt_plan(d).fits; }

size_t tc_train_ws_bytes(const Dims& d, long long n_px, int sm_count) {
  const size_t nw = (size_t)d.C * d.F + d.C + (size_t)d.R * (2 * d.C * d.C + 2 * d.C) +
                    (size_t)d.NO * d.C + d.NO;
  const long long t = (n_px + kTTM - 1) / kTTM;
  const size_t g = (size_t)(t < sm_count ? (t < 1 ? 1 : t) : sm_count);
  return (g * ((nw + 3) & ~(size_t)3) + g + 64) * 4;
}

struct SmOp {
  uint32_t addr, lbo, sbo, kstep;
};
// A natural tile T[rows][ncol] (canonical K-major layout) as the K-major
// operand (rows = M or N, K = columns) ...
__device__ __forceinline__ SmOp op_k(uint32_t addr, int ncol) {
  return SmOp{addr, 128u, (uint32_t)(ncol / 8) * 128u, 256u};
}
// ... and as the MN-major operand (K = rows, M or N = columns): the leading
// byte offset is then the stride of core matrices along K (8-row groups) and
// the stride byte offset their stride along M/N (measured with a probe of
// both assignments on GB300).
__device__ __forceinline__ SmOp op_mn(uint32_t addr, int ncol) {
  return SmOp{addr, (uint32_t)(ncol / 8) * 128u, 128u, (uint32_t)(ncol / 8) * 256u};
}

// nk chained MMAs (K = 16 each) D[128][N] (+)= A B, issued by thread 0.
__device__ __forceinline__ void tt_mma(uint32_t dtm, SmOp a, bool a_mn, SmOp b, bool b_mn, int N,
                                       int nk, bool accumulate) {
  const uint32_t idesc =
      idesc_bf16(kTTM, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
  for (int s = 0; s < nk; s++) {
    const uint64_t da = umma_desc(a.addr + (uint32_t)s * a.kstep, a.lbo, a.sbo);
    const uint64_t db = umma_desc(b.addr + (uint32_t)s * b.kstep, b.lbo, b.sbo);
    mma_bf16(dtm, da, db, idesc, (accumulate || s > 0) ? 1u : 0u);
  }
}

__device__ __forceinline__ void tt_store8(unsigned char* base, int ncol, int row, int c8,
                                          const float (&v)[8]) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + 2 * umma_off(row, 8 * c8, ncol)) = q;
}

__device__ __forceinline__ void tt_load8(const unsigned char* base, int ncol, int row, int c8,
                                         float (&v)[8]) {
  const uint4 q = *reinterpret_cast<const uint4*>(base + 2 * umma_off(row, 8 * c8, ncol));
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int e = 0; e < 4; e++) {
    v[2 * e] = __uint_as_float(w[e] << 16);
    v[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
  }
}

// ELU with e^x - 1 through ex2.approx (absolute error ~1e-7, below the BF16
// rounding of the stored activation)
__device__ __forceinline__ float elu_t(float x) {
  return x > 0.f ? x : __fsub_rn(ex2_approx(__fmul_rn(x, 1.4426950408889634f)), 1.f);
}
// ELU'(t) from the stored activation u = ELU(t)
__device__ __forceinline__ float elu_d_from_act(float u) { return u > 0.f ? 1.f : u + 1.f; }

// X tile [128][Fp] (K-major): feature 3p + c of pixel m = 2v - 255 of channel
// c of context tap p (Eq. 3), 0 outside the image and for F <= k < Fp and for
// rows past the batch.  Pixel m's (image, row, column, valid) come from the
// tile's slot table and tap p's offsets from taps[p], so that no index is
// divided per feature; thread t handles pixel t mod 128.
__device__ __noinline__ void tt_gather(const Dims& d, const uint8_t* __restrict__ batch, int H,
                                       int W, const int4* slots, const int2* taps,
                                       unsigned char* X) {
  const int ntap = d.F / 3, Fp = d.Fp;
  uint16_t* x = reinterpret_cast<uint16_t*>(X);
  const int m = threadIdx.x & (kTTM - 1);
  const int4 sl = slots[m];
  const long long base = ((long long)sl.x * H) * W;
  for (int p = threadIdx.x / kTTM; 3 * p < Fp; p += kTT / kTTM) {
    float v[3] = {0.f, 0.f, 0.f};
    if (sl.w != 0 && p < ntap) {
      const int2 t = taps[p];
      const int ii = sl.y + t.x, jj = sl.z + t.y;
      if (ii >= 0 && ii < H && jj >= 0 && jj < W) {
        const uint8_t* px = batch + (base + (long long)ii * W + jj) * 3;
        v[0] = (float)(2 * (int)px[0] - 255);
        v[1] = (float)(2 * (int)px[1] - 255);
        v[2] = (float)(2 * (int)px[2] - 255);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
      if (3 * p + c < Fp)
        x[umma_off(m, 3 * p + c, Fp)] = __bfloat16_as_ushort(__float2bfloat16_rn(v[c]));
  }
}

// Adds the weight gradient of one layer (D rows o < n_out, columns i < n_in
// of the weight-gradient accumulator, times `scale`) and its bias gradient
// (column 0 of the bias accumulator) to the CTA's slot (16-byte aligned rows
// when n_in and ld are multiples of 4).  All tensor-memory loads, then all
// global loads, then the stores: one memory round trip per layer.
constexpr int kFlushChunks = (80 / 8 + kParts - 1) / kParts;  // n_in <= 80
__device__ __noinline__ void tt_flush(uint32_t tmem, int n_out, int n_in, int ld, float scale,
                         float* __restrict__ gW, float* __restrict__ gb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, part = warp >> 2;
  const int o = 32 * q + lane;
  if (32 * q >= n_out) return;  // whole warp outside the layer's outputs
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  const int nch = (n_in + 7) / 8;
  uint32_t r[kFlushChunks][8];
#pragma unroll
  for (int i = 0; i < kFlushChunks; i++)
    if (part + kParts * i < nch) tmem_ld8_nw(tl + kColDW + 8 * (part + kParts * i), r[i]);
  uint32_t rb[8];
  if (part == 0) tmem_ld8_nw(tl + kColDB, rb);
  tmem_wait_ld();
  if (o >= n_out) return;
  float* row = gW + (size_t)o * ld;
  float4 g[kFlushChunks][2];
#pragma unroll
  for (int i = 0; i < kFlushChunks; i++) {
    const int c = part + kParts * i;
    if (c < nch && 8 * c + 8 <= n_in) {
      g[i][0] = *reinterpret_cast<const float4*>(row + 8 * c);
      g[i][1] = *reinterpret_cast<const float4*>(row + 8 * c + 4);
    }
  }
  const float gbo = part == 0 ? gb[o] : 0.f;
#pragma unroll
  for (int i = 0; i < kFlushChunks; i++) {
    const int c = part + kParts * i;
    if (c >= nch) continue;
    tmem_touch(r[i]);
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; e++) v[e] = __fmul_rn(__uint_as_float(r[i][e]), scale);
    if (8 * c + 8 <= n_in) {
      float4 a = g[i][0], b = g[i][1];
      a.x = __fadd_rn(a.x, v[0]);
      a.y = __fadd_rn(a.y, v[1]);
      a.z = __fadd_rn(a.z, v[2]);
      a.w = __fadd_rn(a.w, v[3]);
      b.x = __fadd_rn(b.x, v[4]);
      b.y = __fadd_rn(b.y, v[5]);
      b.z = __fadd_rn(b.z, v[6]);
      b.w = __fadd_rn(b.w, v[7]);
      *reinterpret_cast<float4*>(row + 8 * c) = a;
      *reinterpret_cast<float4*>(row + 8 * c + 4) = b;
    } else {  // ragged last chunk
      for (int e = 0; e < 8 && 8 * c + e < n_in; e++) row[8 * c + e] = __fadd_rn(row[8 * c + e], v[e]);
    }
  }
  if (part == 0) {
    tmem_touch(rb);
    gb[o] = __fadd_rn(gbo, __uint_as_float(rb[0]));
  }
}

// 8 FP32 columns of this thread's lane to tensor memory (no wait).
__device__ __forceinline__ void tmem_st8_f32(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}

// Forward epilogue of a hidden layer for this thread's row and column chunks
// (8 columns each): v = acc + b; mode 0: a = v, 1: a += v (a, the residual
// stream, kept in FP32 in tensor memory), 2: hidden layer; out = BF16
// ELU(mode 2 ? v : a).
__device__ __noinline__ void tt_fwd_epi(uint32_t tl, const float* __restrict__ b, int mode,
                                        unsigned char* out, int C, int row, int part) {
#pragma unroll 1
  for (int c = part; c < C / 8; c += kParts) {
    uint32_t r[8], ra[8];
    tmem_ld8_nw(tl + kColAcc + 8 * c, r);
    if (mode == 1) tmem_ld8_nw(tl + kColRes + 8 * c, ra);
    tmem_wait_ld();
    tmem_touch(r);
    if (mode == 1) tmem_touch(ra);
    float a[8], u[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const float v = __fadd_rn(__uint_as_float(r[e]), b[8 * c + e]);
      a[e] = mode == 1 ? __fadd_rn(__uint_as_float(ra[e]), v) : v;
      u[e] = elu_t(a[e]);
    }
    if (mode != 2) tmem_st8_f32(tl + kColRes + 8 * c, a);
    tt_store8(out, C, row, c, u);
  }
  tmem_wait_st();
}

// Adjoint epilogue: g = acc * ELU'(act) (act: this row of a BF16 activation
// tile); mode 0: ga = g, 1: ga += g (ga, the residual stream's gradient, in
// FP32 in tensor memory), 2: g alone; out = BF16 (mode 2 ? g : ga).
__device__ __noinline__ void tt_bwd_epi(uint32_t tl, const unsigned char* act, int mode,
                                        unsigned char* out, int C, int row, int part) {
#pragma unroll 1
  for (int c = part; c < C / 8; c += kParts) {
    uint32_t r[8], ra[8];
    tmem_ld8_nw(tl + kColAcc + 8 * c, r);
    if (mode == 1) tmem_ld8_nw(tl + kColRes + 8 * c, ra);
    float u[8];
    tt_load8(act, C, row, c, u);
    tmem_wait_ld();
    tmem_touch(r);
    if (mode == 1) tmem_touch(ra);
    float o[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const float g = __fmul_rn(__uint_as_float(r[e]), elu_d_from_act(u[e]));
      o[e] = mode == 1 ? __fadd_rn(__uint_as_float(ra[e]), g) : g;
    }
    if (mode != 2) tmem_st8_f32(tl + kColRes + 8 * c, o);
    tt_store8(out, C, row, c, o);
  }
  tmem_wait_st();
}

// The likelihood gradient dP of this thread's row (components k = part,
// part + kParts, ...; each component's 10 outputs read from tensor memory),
// as a BF16 row of the [128][NOp] tile DP; MODE 1 takes dP from dparams.
// Returns this row's -log p (nats) for part 0 of a valid row, else 0.
template <int MODE>
__device__ __noinline__ float tt_likelihood(const Dims& d, uint32_t tcol, const float* bh,
                                            float* lb, uint16_t* DP, int row, int part,
                                            bool valid, const uint8_t* px, float scale,
                                            const float* dparams, long long q) {
  const int K = d.K, NO = d.NO, NOp = d.NOp;
  float nll = 0.f;
  // the 10 outputs of component k of this thread's row (+ bias)
  auto load_comp = [&](int k, float (&pr)[10]) {
    uint32_t x[10];
#pragma unroll
    for (int g = 0; g < 10; g++)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                   : "=r"(x[g])
                   : "r"(tcol + (uint32_t)(g * K + k))
                   : "memory");
    tmem_wait_ld();
#pragma unroll
    for (int g = 0; g < 10; g++) {
      asm volatile("" : "+r"(x[g]));
      pr[g] = __fadd_rn(__uint_as_float(x[g]), bh[g * K + k]);
    }
  };
  auto row_lse = [&]() {  // log-sum-exp of lb[0 .. K)
    float mx = -INFINITY;
    for (int k = 0; k < K; k++) mx = fmaxf(mx, lb[k]);
    float se = 0.f;
    for (int k = 0; k < K; k++) se = __fadd_rn(se, exp_f(__fsub_rn(lb[k], mx)));
    return __fadd_rn(mx, log_f(se));
  };
  if (MODE == 0) {
    const int v[3] = {valid ? (int)px[0] : 0, valid ? (int)px[1] : 0, valid ? (int)px[2] : 0};
    const float xr = __fdiv_rn((float)(2 * v[0] - 255), 255.f);
    const float xg = __fdiv_rn((float)(2 * v[1] - 255), 255.f);
    // log pi_k = logit_k - LSE(logits)
#pragma unroll 1
    for (int k = part; k < K; k += kParts) {
      uint32_t x;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                   : "=r"(x)
                   : "r"(tcol + (uint32_t)k)
                   : "memory");
      tmem_wait_ld();
      asm volatile("" : "+r"(x));
      lb[k] = __fadd_rn(__uint_as_float(x), bh[k]);
    }
    __syncthreads();
    const float lse_pi = row_lse();
    __syncthreads();
    // locations m_c (coupled), log-scales, the channel log-masses, and with
    // want_d the derivatives of each channel's log-mass with respect to its
    // location (dlm) and log-scale (dll)
    auto comp_terms = [&](const float (&pr)[10], float (&co)[3], float (&dlm)[3],
                          float (&dll)[3], bool want_d) {
      float lk = 0.f;
#pragma unroll
      for (int c = 0; c < 3; c++) co[c] = tanh_f(pr[7 + c]);
      const float m3[3] = {pr[1], __fadd_rn(pr[2], __fmul_rn(co[0], xr)),
                           __fadd_rn(__fadd_rn(pr[3], __fmul_rn(co[1], xr)), __fmul_rn(co[2], xg))};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float ls = fmaxf(pr[4 + c], -7.f);
        const float inv = exp_f(-ls), mc = m3[c];
        if (!want_d) {
          lk = __fadd_rn(lk, log_bin_mass_f(mc, inv, bin_log_width(ls, inv), v[c]));
          continue;
        }
        // sigma(-a) = 1/(1 + e^a), sigma(b) = 1/(1 + e^-b) through the MUFU
        // (a gradient, not a frequency table: the approximations only
        // perturb it by ~1e-6 relative)
        if (v[c] == 0) {
          const float aa = __fmul_rn(__fsub_rn(edge_f(1), mc), inv);
          const float sa = rcp_approx(__fadd_rn(1.f, exp_f(aa)));
          dlm[c] = -inv * sa;
          dll[c] = -aa * sa;
        } else if (v[c] == 255) {
          const float bb = __fmul_rn(__fsub_rn(edge_f(255), mc), inv);
          const float sb = rcp_approx(__fadd_rn(1.f, exp_f(-bb)));
          dlm[c] = inv * sb;
          dll[c] = bb * sb;
        } else {
          const float aa = __fmul_rn(__fsub_rn(edge_f(v[c] + 1), mc), inv);
          const float bb = __fmul_rn(__fsub_rn(edge_f(v[c]), mc), inv);
          const float dd = __fmul_rn(2.f / 255.f, inv);
          // 1/(e^d - 1): Taylor series of e^d - 1 for d < 1/8 (no cancellation)
          float em1;
          if (dd < 0.125f) {
            float p = __fmaf_rn(dd, 1.f / 120.f, 1.f / 24.f);
            p = __fmaf_rn(p, dd, 1.f / 6.f);
            p = __fmaf_rn(p, dd, 0.5f);
            p = __fmaf_rn(p, dd, 1.f);
            em1 = __fmul_rn(dd, p);
          } else {
            em1 = __fsub_rn(exp_f(dd), 1.f);
          }
          const float gk = rcp_approx(em1);
          const float sa = rcp_approx(__fadd_rn(1.f, exp_f(aa)));
          const float sb = rcp_approx(__fadd_rn(1.f, exp_f(-bb)));
          dlm[c] = -inv * (sa - sb);
          dll[c] = -aa * sa + bb * sb - gk * dd;
        }
      }
      return lk;
    };
    // l_k = log pi_k + sum_c log P_c,k
#pragma unroll 1
    for (int k = part; k < K; k += kParts) {
      float pr[10], co[3], dlm[3], dll[3];
      load_comp(k, pr);
      lb[k] = __fadd_rn(__fsub_rn(pr[0], lse_pi), comp_terms(pr, co, dlm, dll, false));
    }
    __syncthreads();
    const float lse = row_lse();  // log p(pixel)
    if (valid && part == 0) nll = -lse;
    const float sc = valid ? scale : 0.f;
#pragma unroll 1
    for (int k = part; k < K; k += kParts) {
      float pr[10], co[3], dlm[3], dll[3];
      load_comp(k, pr);
      comp_terms(pr, co, dlm, dll, true);
      const float rho = valid ? exp_f(__fsub_rn(lb[k], lse)) : 0.f;
      const float pi = exp_f(__fsub_rn(pr[0], lse_pi));
      float gk[10];
      gk[0] = sc * (pi - rho);
      const float dmR = -rho * dlm[0], dmG = -rho * dlm[1], dmB = -rho * dlm[2];
      gk[1] = sc * dmR;
      gk[2] = sc * dmG;
      gk[3] = sc * dmB;
#pragma unroll
      for (int c = 0; c < 3; c++) gk[4 + c] = pr[4 + c] > -7.f ? sc * (-rho * dll[c]) : 0.f;
      gk[7] = sc * dmG * xr * (1.f - co[0] * co[0]);
      gk[8] = sc * dmB * xr * (1.f - co[1] * co[1]);
      gk[9] = sc * dmB * xg * (1.f - co[2] * co[2]);
#pragma unroll
      for (int g = 0; g < 10; g++)
        DP[umma_off(row, g * K + k, NOp)] = __bfloat16_as_ushort(__float2bfloat16_rn(gk[g]));
    }
  } else {
#pragma unroll 1
    for (int k = part; k < K; k += kParts) {
#pragma unroll
      for (int g = 0; g < 10; g++) {
        const float gv = valid ? dparams[q * NO + g * K + k] : 0.f;
        DP[umma_off(row, g * K + k, NOp)] = __bfloat16_as_ushort(__float2bfloat16_rn(gv));
      }
    }
  }
  if (part == 0)
    for (int c = NO; c < NOp; c++) DP[umma_off(row, c, NOp)] = 0;
  return nll;
}

// MODE 0: dP = gradient of the mean code length in bits per dimension of the
// batch (Eq. 2), the loss summed per CTA into part_l; MODE 1: dP = the given
// upstream gradient dparams [n_px][10K] (raster order of the batch).  The
// per-thread state between phases (the residual stream and its gradient)
// lives in tensor memory, so that each phase's function keeps its own
// registers.
template <int MODE>
__global__ void __launch_bounds__(kTT, 1)
    tc_train_kernel(Dims d, const uint16_t* __restrict__ umma, const float* __restrict__ bias,
                    const uint8_t* __restrict__ batch, int N, int H, int W,
                    const float* __restrict__ dparams, float* __restrict__ part_g,
                    float* __restrict__ part_l, int n_w, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const TTPlan pl = tt_plan(d);
  const int C = d.C, R = d.R, NO = d.NO, NOp = d.NOp, Fp = d.Fp, F = d.F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = warp >> 2;
  const int row = 32 * (warp & 3) + lane;
  float* sbias = reinterpret_cast<float*>(sm + pl.bias);
  float* red = reinterpret_cast<float*>(sm + pl.red);
  int4* slots = reinterpret_cast<int4*>(sm + pl.slots);
  int2* taps = reinterpret_cast<int2*>(sm + pl.taps);
  for (int p = threadIdx.x; p < d.F / 3; p += blockDim.x) {
    int dy, dx;
    tap_offset(p, d.h, dy, dx);
    taps[p] = make_int2(dy, dx);
  }
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + pl.mbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + pl.tslot);
  // weights (BF16 tiles) and biases
  {
    const int nh = (int)umma_plain_halves(d);  // a sheared model trains the same weights
    const uint4* src = reinterpret_cast<const uint4*>(umma);
    uint4* dst = reinterpret_cast<uint4*>(sm);
    for (int i = threadIdx.x; i < nh / 8; i += blockDim.x) dst[i] = src[i];
    const int nb = (int)bias_floats(d);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sbias[i] = bias[i];
    uint16_t* ones = reinterpret_cast<uint16_t*>(sm + pl.ones);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) ones[i] = 0x3F80u;  // BF16 1.0
  }
  // this CTA's gradient slot (stride n_w rounded up to 4 floats)
  float* gW = part_g + (size_t)blockIdx.x * ((n_w + 3) & ~3);
  for (int i = threadIdx.x; i < n_w; i += blockDim.x) gW[i] = 0.f;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTTCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t s0 = smem_u32(sm);
  uint32_t phase = 0;
  bool ok = true;
  auto wait_mma = [&]() {  // the same outcome in every thread
    if (threadIdx.x == 0) mma_commit(mbar);
    const bool done = mbar_wait(mbar, phase);
    phase ^= 1u;
    fence_after_sync();
    return __syncthreads_and(done ? 1 : 0) != 0;
  };
  auto sync_for_mma = [&]() {  // smem stores and TMEM accesses before the next MMA
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  };
  const SmOp ones_op{s0 + (uint32_t)pl.ones, 128u, 256u, 0u};

  // canonical offsets of the FP32 gradient
  const size_t ob0 = (size_t)C * F, oblk = ob0 + C, blk = 2 * (size_t)C * C + 2 * C;
  const size_t oWH = oblk + (size_t)R * blk, obH = oWH + (size_t)NO * C;
  const long long n_px = (long long)N * H * W, HW = (long long)H * W;
  const long long ntiles = (n_px + kTTM - 1) / kTTM;
  const float scale = 1.f / (0.6931471805599453f * 3.f * (float)n_px);
  float loss = 0.f;
  unsigned char* U = sm + pl.u;
  const int tb = tile_bytes(C);
  const uint32_t uoff = s0 + pl.u;

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long q0 = tile * kTTM;
    if (threadIdx.x < kTTM) {
      const long long q = q0 + threadIdx.x;
      int4 sv = make_int4(0, 0, 0, 0);
      if (q < n_px) {
        const long long rr = q % HW;
        sv = make_int4((int)(q / HW), (int)(rr / W), (int)(rr % W), 1);
      }
      slots[threadIdx.x] = sv;
    }
    __syncthreads();  // the slots (and, on the first tile, the taps)
    tt_gather(d, batch, H, W, slots, taps, sm + pl.gx);
    sync_for_mma();

    // ---------------- forward ----------------
    if (threadIdx.x == 0)
      tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, Fp), false, op_k(s0 + pl.w0, Fp), false, C, Fp / 16,
             false);
    ok &= wait_mma();
    tt_fwd_epi(tl, sbias, 0, U, C, row, part);
    sync_for_mma();
    for (int r = 0; r < R && ok; r++) {
      const float* b1 = sbias + C + 2 * r * C;
      const uint32_t w1 = s0 + pl.w1 + r * pl.wstride, w2 = w1 + pl.wstride / 2;
      if (threadIdx.x == 0)
        tt_mma(tmem + kColAcc, op_k(uoff + (2 * r) * tb, C), false, op_k(w1, C), false, C, C / 16,
               false);
      ok &= wait_mma();
      tt_fwd_epi(tl, b1, 2, U + (2 * r + 1) * tb, C, row, part);
      sync_for_mma();
      if (threadIdx.x == 0)
        tt_mma(tmem + kColAcc, op_k(uoff + (2 * r + 1) * tb, C), false, op_k(w2, C), false, C,
               C / 16, false);
      ok &= wait_mma();
      tt_fwd_epi(tl, b1 + C, 1, U + (2 * r + 2) * tb, C, row, part);
      sync_for_mma();
    }
    if (threadIdx.x == 0)
      tt_mma(tmem + kColAcc, op_k(uoff + (2 * R) * tb, C), false, op_k(s0 + pl.wh, C), false, NOp,
             C / 16, false);
    ok &= wait_mma();
    if (!ok) break;

    // ---------------- likelihood gradient dP -> BF16 tile [128][NOp] ----------------
    {
      const int4 sl = slots[row];
      const bool valid = sl.w != 0;
      const uint8_t* px =
          valid ? batch + ((long long)sl.x * HW + (long long)sl.y * W + sl.z) * 3 : batch;
      loss = __fadd_rn(loss, tt_likelihood<MODE>(
                                 d, tl + kColAcc, sbias + C + 2 * R * C,
                                 reinterpret_cast<float*>(sm + pl.red) + row * kLbStride,
                                 reinterpret_cast<uint16_t*>(sm + pl.gx), row, part, valid, px,
                                 scale, dparams, q0 + row));
    }
    sync_for_mma();

    // ---------------- adjoint ----------------
    // head: dH = dP WH, dWH = dP^T u_R, dbH = dP^T 1
    if (threadIdx.x == 0) {
      tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, NOp), false, op_mn(s0 + pl.wh, C), true, C,
             NOp / 16, false);
      tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, NOp), true, op_mn(uoff + (2 * R) * tb, C), true, C,
             kTTM / 16, false);
      tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, NOp), true, ones_op, false, 16, kTTM / 16, false);
    }
    ok &= wait_mma();
    tt_bwd_epi(tl, U + (2 * R) * tb, 0, sm + pl.gx, C, row, part);  // da_R = dH * ELU'(a_R)
    tt_flush(tmem, NO, C, C, 1.f, gW + oWH, gW + obH);
    sync_for_mma();
    for (int r = R - 1; r >= 0 && ok; r--) {
      const size_t oW1 = oblk + r * blk, ob1 = oW1 + (size_t)C * C;
      const size_t oW2 = ob1 + C, ob2 = oW2 + (size_t)C * C;
      const uint32_t w1 = s0 + pl.w1 + r * pl.wstride, w2 = w1 + pl.wstride / 2;
      // dv = da W2, dW2 = da^T v_r, db2 = da^T 1  (da in G)
      if (threadIdx.x == 0) {
        tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, C), false, op_mn(w2, C), true, C, C / 16, false);
        tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, C), true, op_mn(uoff + (2 * r + 1) * tb, C), true,
               C, kTTM / 16, false);
        tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, C), true, ones_op, false, 16, kTTM / 16, false);
      }
      ok &= wait_mma();
      tt_bwd_epi(tl, U + (2 * r + 1) * tb, 2, sm + pl.g2, C, row, part);  // dz = dv * ELU'(z)
      tt_flush(tmem, C, C, C, 1.f, gW + oW2, gW + ob2);
      sync_for_mma();
      // du = dz W1, dW1 = dz^T u_r, db1 = dz^T 1  (dz in G2)
      if (threadIdx.x == 0) {
        tt_mma(tmem + kColAcc, op_k(s0 + pl.g2, C), false, op_mn(w1, C), true, C, C / 16, false);
        tt_mma(tmem + kColDW, op_mn(s0 + pl.g2, C), true, op_mn(uoff + (2 * r) * tb, C), true, C,
               kTTM / 16, false);
        tt_mma(tmem + kColDB, op_mn(s0 + pl.g2, C), true, ones_op, false, 16, kTTM / 16, false);
      }
      ok &= wait_mma();
      tt_bwd_epi(tl, U + (2 * r) * tb, 1, sm + pl.gx, C, row, part);  // da_r = da + du * ELU'(a_r)
      tt_flush(tmem, C, C, C, 1.f, gW + oW1, gW + ob1);
      sync_for_mma();
    }
    if (!ok) break;
    // first layer: dW0 = da_0^T X / 255 (X gathered again), db0 = da_0^T 1
    tt_gather(d, batch, H, W, slots, taps, sm + pl.xe);
    sync_for_mma();
    if (threadIdx.x == 0) {
      tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, C), true, op_mn(s0 + pl.xe, Fp), true, Fp,
             kTTM / 16, false);
      tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, C), true, ones_op, false, 16, kTTM / 16, false);
    }
    ok &= wait_mma();
    tt_flush(tmem, C, F, F, 1.f / 255.f, gW, gW + ob0);
    sync_for_mma();
  }
  if (!ok && threadIdx.x == 0) set_status(status, ST_TIMEOUT);
  // per-CTA loss (nats), fixed order over the 128 row owners
  if (MODE == 0) {
    __syncthreads();
    if (part == 0) red[row] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int i = 0; i < kTTM; i++) t = __fadd_rn(t, red[i]);
      part_l[blockIdx.x] = t;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTTCols)
                 : "memory");
}

cudaError_t launch_tc_train(const Dims& d, const uint16_t* umma, const float* bias,
                            const uint8_t* batch, int N, int H, int W, const float* dparams,
                            float* loss, float* grad, void* ws, int sm_count, int* status,
                            cudaStream_t s) {
  const TTPlan pl = tt_plan(d);
  if (!pl.fits) return cudaErrorInvalidConfiguration;
  const int n_w = (int)((size_t)d.C * d.F + d.C + (size_t)d.R * (2 * d.C * d.C + 2 * d.C) +
                        (size_t)d.NO * d.C + d.NO);
  const long long n_px = (long long)N * H * W;
  const long long tiles = (n_px + kTTM - 1) / kTTM;
  const int g = (int)(tiles < sm_count ? (tiles < 1 ? 1 : tiles) : sm_count);
  const void* fn = dparams ? (const void*)tc_train_kernel<1> : (const void*)tc_train_kernel<0>;
  cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.end);
  if (e != cudaSuccess) return e;
  const int ldw = (n_w + 3) & ~3;
  float* part_g = reinterpret_cast<float*>(ws);
  float* part_l = part_g + (size_t)g * ldw;
  if (dparams)
    tc_train_kernel<1><<<g, kTT, pl.end, s>>>(d, umma, bias, batch, N, H, W, dparams, part_g,
                                              part_l, n_w, status);
  else
    tc_train_kernel<0><<<g, kTT, pl.end, s>>>(d, umma, bias, batch, N, H, W, nullptr, part_g,
                                              part_l, n_w, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_grad(part_g, dparams ? nullptr : part_l, g, n_w, ldw, n_px, grad, loss, s);
}

}  // namespace nlc

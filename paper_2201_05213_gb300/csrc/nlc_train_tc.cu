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
// read straight from tensor memory (four threads per pixel, each holding
// every fourth mixture component) and the gradient is stored in BF16 as the
// A operand of the head's adjoint.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"
#include "nlc_model.cuh"
#include "nlc_tc.cuh"
#include "nlc_train.cuh"

namespace nlc {

constexpr int kTT = 512;                  // threads (16 warps)
constexpr int kTTM = 128;                 // pixels per tile (the MMA's M)
constexpr uint32_t kTTCols = 512;         // tensor-memory columns
constexpr uint32_t kColAcc = 0;           // forward / adjoint accumulator (N <= 160)
constexpr uint32_t kColDW = 256;          // weight-gradient accumulator (N <= Fp <= 80)
constexpr uint32_t kColDB = 384;          // bias-gradient accumulator (N = 16)
constexpr int kCompPerThread = (kMaxK + 3) / 4;

struct TTPlan {
  int w0, w1[kMaxR], w2[kMaxR], wh;  // BF16 weight tiles (the decoder's layout)
  int bias, ones, u, gx, g2, xe, red, slots, mbar, tslot, end;
  bool fits;
};

__host__ __device__ inline int tile_bytes(int ncol) { return kTTM * ncol * 2; }

__host__ __device__ inline TTPlan tt_plan(const Dims& d) {
  const TcPlan tp = tc_plan(d);
  TTPlan p;
  p.w0 = tp.w0;
  for (int r = 0; r < kMaxR; r++) {
    p.w1[r] = tp.w1[r];
    p.w2[r] = tp.w2[r];
  }
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
  // likelihood's reduction scratch, then G and G2 [128][C]
  p.gx = o;
  p.g2 = o + tile_bytes(d.C);
  const int dp = tile_bytes(d.NOp);
  p.red = o + dp;
  int need = dp + 4 * kTTM * 4;
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
  return (g * nw + g + 64) * 4;
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

__device__ __forceinline__ float elu_t(float x) { return x > 0.f ? x : expm1f(x); }
// ELU'(t) from the stored activation u = ELU(t)
__device__ __forceinline__ float elu_d_from_act(float u) { return u > 0.f ? 1.f : u + 1.f; }

// X tile [128][Fp] (K-major): feature 3p + c of pixel m = 2v - 255 of channel
// c of context tap p (Eq. 3), 0 outside the image and for F <= k < Fp and for
// rows past the batch.
__device__ void tt_gather(const Dims& d, const uint8_t* __restrict__ batch, int H, int W,
                          long long n_px, long long q0, unsigned char* X) {
  const int ntap = d.F / 3, Fp = d.Fp, h = d.h;
  uint16_t* x = reinterpret_cast<uint16_t*>(X);
  const long long HW = (long long)H * W;
  for (int it = threadIdx.x; it < kTTM * (Fp / 3 + 1); it += blockDim.x) {
    const int m = it % kTTM, p = it / kTTM;
    if (3 * p >= Fp) continue;
    const long long q = q0 + m;
    float v[3] = {0.f, 0.f, 0.f};
    if (q < n_px && p < ntap) {
      const long long n = q / HW, rr = q % HW;
      const int i = (int)(rr / W), j = (int)(rr % W);
      int dy, dx;
      tap_offset(p, h, dy, dx);
      const int ii = i + dy, jj = j + dx;
      if (ii >= 0 && ii < H && jj >= 0 && jj < W) {
        const uint8_t* px = batch + (n * HW + (long long)ii * W + jj) * 3;
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
// (column 0 of the bias accumulator) to the CTA's slot.
__device__ void tt_flush(uint32_t tmem, int n_out, int n_in, int ld, float scale,
                         float* __restrict__ gW, float* __restrict__ gb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, part = warp >> 2;
  const int o = 32 * q + lane;
  if (32 * q >= n_out) return;  // whole warp outside the layer's outputs
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  const int nch = (n_in + 7) / 8;
  for (int c = part; c < nch; c += 4) {
    float v[8];
    tmem_ld8(tl + kColDW + 8 * c, v);
    if (o < n_out) {
#pragma unroll
      for (int e = 0; e < 8; e++)
        if (8 * c + e < n_in) {
          float* g = gW + (size_t)o * ld + 8 * c + e;
          *g = __fadd_rn(*g, __fmul_rn(v[e], scale));
        }
    }
  }
  if (part == 0) {
    float v[8];
    tmem_ld8(tl + kColDB, v);
    if (o < n_out) gb[o] = __fadd_rn(gb[o], v[0]);
  }
}

// MODE 0: dP = gradient of the mean code length in bits per dimension of the
// batch (Eq. 2), the loss summed per CTA into part_l; MODE 1: dP = the given
// upstream gradient dparams [n_px][10K] (raster order of the batch).
template <int MODE>
__global__ void __launch_bounds__(kTT, 1)
    tc_train_kernel(Dims d, const uint16_t* __restrict__ umma, const float* __restrict__ bias,
                    const uint8_t* __restrict__ batch, int N, int H, int W,
                    const float* __restrict__ dparams, float* __restrict__ part_g,
                    float* __restrict__ part_l, int n_w, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const TTPlan pl = tt_plan(d);
  const int C = d.C, R = d.R, K = d.K, NO = d.NO, NOp = d.NOp, Fp = d.Fp, F = d.F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q4 = warp & 3, part = warp >> 2;
  const int row = 32 * q4 + lane;
  float* sbias = reinterpret_cast<float*>(sm + pl.bias);
  float* red = reinterpret_cast<float*>(sm + pl.red);
  int4* slots = reinterpret_cast<int4*>(sm + pl.slots);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + pl.mbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + pl.tslot);
  // weights (BF16 tiles) and biases
  {
    const int nh = (int)umma_halves(d);
    const uint4* src = reinterpret_cast<const uint4*>(umma);
    uint4* dst = reinterpret_cast<uint4*>(sm);
    for (int i = threadIdx.x; i < nh / 8; i += blockDim.x) dst[i] = src[i];
    const int nb = (int)bias_floats(d);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sbias[i] = bias[i];
    uint16_t* ones = reinterpret_cast<uint16_t*>(sm + pl.ones);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) ones[i] = 0x3F80u;  // BF16 1.0
  }
  // this CTA's gradient slot
  float* gW = part_g + (size_t)blockIdx.x * n_w;
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
  const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
  const uint32_t s0 = smem_u32(sm);
  uint32_t phase = 0;
  bool ok = true;
  auto wait_mma = [&]() {  // the same verdict in every thread
    if (threadIdx.x == 0) mma_commit(mbar);
    const bool done = mbar_wait(mbar, phase);
    phase ^= 1u;
    fence_after_sync();
    return __syncthreads_and(done ? 1 : 0) != 0;
  };
  auto sync_for_mma = [&]() {  // smem stores and TMEM loads before the next MMA
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  };

  // canonical offsets of the FP32 gradient
  const size_t ob0 = (size_t)C * F, oblk = ob0 + C, blk = 2 * (size_t)C * C + 2 * C;
  const size_t oWH = oblk + (size_t)R * blk, obH = oWH + (size_t)NO * C;
  const long long n_px = (long long)N * H * W, HW = (long long)H * W;
  const long long ntiles = (n_px + kTTM - 1) / kTTM;
  const float scale = 1.f / (0.6931471805599453f * 3.f * (float)n_px);
  const int CH = (C / 8 + 3) / 4;  // chunks of 8 columns per thread (<= 2)
  float loss = 0.f;
  unsigned char* U = sm + pl.u;
  const int tb = tile_bytes(C);

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long q0 = tile * kTTM;
    if (threadIdx.x < kTTM) {
      const long long q = q0 + threadIdx.x;
      int4 s = make_int4(0, 0, 0, 0);
      if (q < n_px) {
        const long long rr = q % HW;
        s = make_int4((int)(q / HW), (int)(rr / W), (int)(rr % W), 1);
      }
      slots[threadIdx.x] = s;
    }
    tt_gather(d, batch, H, W, n_px, q0, sm + pl.gx);
    sync_for_mma();

    // ---------------- forward ----------------
    float a[2][8];  // residual stream a_r (FP32), columns 8 (part + 4 i) .. + 7
    if (threadIdx.x == 0)
      tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, Fp), false, op_k(s0 + pl.w0, Fp), false, C, Fp / 16,
             false);
    ok &= wait_mma();
    auto fwd_epi = [&](const float* b, int mode, unsigned char* out) {
      // mode 0: a = acc + b; 1: a += acc + b; 2: hidden only.  out = ELU(.)
      uint32_t r[2][8];
#pragma unroll
      for (int i = 0; i < 2; i++)
        if (i < CH && part + 4 * i < C / 8) tmem_ld8_nw(tl + kColAcc + 8 * (part + 4 * i), r[i]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int c = part + 4 * i;
        if (i < CH && c < C / 8) {
          tmem_touch(r[i]);
          float u[8];
#pragma unroll
          for (int e = 0; e < 8; e++) {
            const float v = __fadd_rn(__uint_as_float(r[i][e]), b[8 * c + e]);
            if (mode == 0) a[i][e] = v;
            if (mode == 1) a[i][e] = __fadd_rn(a[i][e], v);
            u[e] = elu_t(mode == 2 ? v : a[i][e]);
          }
          tt_store8(out, C, row, c, u);
        }
      }
      sync_for_mma();
    };
    fwd_epi(sbias, 0, U);
    for (int r = 0; r < R && ok; r++) {
      const float* b1 = sbias + C + 2 * r * C;
      if (threadIdx.x == 0)
        tt_mma(tmem + kColAcc, op_k(s0 + pl.u + (2 * r) * tb, C), false, op_k(s0 + pl.w1[r], C),
               false, C, C / 16, false);
      ok &= wait_mma();
      fwd_epi(b1, 2, U + (2 * r + 1) * tb);
      if (threadIdx.x == 0)
        tt_mma(tmem + kColAcc, op_k(s0 + pl.u + (2 * r + 1) * tb, C), false,
               op_k(s0 + pl.w2[r], C), false, C, C / 16, false);
      ok &= wait_mma();
      fwd_epi(b1 + C, 1, U + (2 * r + 2) * tb);
    }
    if (threadIdx.x == 0)
      tt_mma(tmem + kColAcc, op_k(s0 + pl.u + (2 * R) * tb, C), false, op_k(s0 + pl.wh, C), false,
             NOp, C / 16, false);
    ok &= wait_mma();
    if (!ok) break;

    // ---------------- likelihood gradient dP -> BF16 tile [128][NOp] ----------------
    {
      const float* bh = sbias + C + 2 * R * C;
      uint16_t* DP = reinterpret_cast<uint16_t*>(sm + pl.gx);
      const int4 sl = slots[row];
      const bool valid = sl.w != 0;
      const long long q = q0 + row;
      float Pr[kCompPerThread][10];
      uint32_t raw[kCompPerThread][10];
#pragma unroll
      for (int t = 0; t < kCompPerThread; t++) {
        const int k = part + 4 * t;
        if (k < K) {
#pragma unroll
          for (int g = 0; g < 10; g++)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                         : "=r"(raw[t][g])
                         : "r"(tl + kColAcc + (uint32_t)(g * K + k))
                         : "memory");
        }
      }
      tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < kCompPerThread; t++) {
        const int k = part + 4 * t;
        if (k < K) {
#pragma unroll
          for (int g = 0; g < 10; g++) {
            uint32_t x = raw[t][g];
            asm volatile("" : "+r"(x));
            Pr[t][g] = __fadd_rn(__uint_as_float(x), bh[g * K + k]);
          }
        }
      }
      if (MODE == 0) {
        int v[3] = {0, 0, 0};
        if (valid) {
          const uint8_t* px = batch + ((long long)sl.x * HW + (long long)sl.y * W + sl.z) * 3;
          v[0] = px[0];
          v[1] = px[1];
          v[2] = px[2];
        }
        const float xr = __fdiv_rn((float)(2 * v[0] - 255), 255.f);
        const float xg = __fdiv_rn((float)(2 * v[1] - 255), 255.f);
        // log-sum-exp of the logits over the four threads of this pixel
        float mx = -INFINITY;
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++)
          if (part + 4 * t < K) mx = fmaxf(mx, Pr[t][0]);
        red[part * kTTM + row] = mx;
        __syncthreads();
        mx = fmaxf(fmaxf(red[row], red[kTTM + row]), fmaxf(red[2 * kTTM + row], red[3 * kTTM + row]));
        __syncthreads();
        float se = 0.f;
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++)
          if (part + 4 * t < K) se = __fadd_rn(se, expf(__fsub_rn(Pr[t][0], mx)));
        red[part * kTTM + row] = se;
        __syncthreads();
        se = __fadd_rn(__fadd_rn(red[row], red[kTTM + row]), __fadd_rn(red[2 * kTTM + row], red[3 * kTTM + row]));
        __syncthreads();
        const float lse_pi = __fadd_rn(mx, logf(se));
        // per component: log-likelihood l_k and the derivatives of its
        // channel terms with respect to the location and the log-scale
        float l[kCompPerThread], dlm[kCompPerThread][3], dll[kCompPerThread][3];
        float co[kCompPerThread][3];
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++) {
          const int k = part + 4 * t;
          l[t] = -INFINITY;
          if (k < K) {
            float lk = __fsub_rn(Pr[t][0], lse_pi);
#pragma unroll
            for (int c = 0; c < 3; c++) co[t][c] = tanh_f(Pr[t][7 + c]);
            const float m3[3] = {Pr[t][1], __fadd_rn(Pr[t][2], __fmul_rn(co[t][0], xr)),
                                 __fadd_rn(__fadd_rn(Pr[t][3], __fmul_rn(co[t][1], xr)),
                                           __fmul_rn(co[t][2], xg))};
#pragma unroll
            for (int c = 0; c < 3; c++) {
              const float ls = fmaxf(Pr[t][4 + c], -7.f);
              const float inv = expf(-ls), mc = m3[c];
              lk = __fadd_rn(lk, log_bin_mass_f(mc, inv, bin_log_width(ls, inv), v[c]));
              if (v[c] == 0) {
                const float aa = __fmul_rn(__fsub_rn(edge_f(1), mc), inv);
                const float sa = 1.f / (1.f + expf(aa));
                dlm[t][c] = -inv * sa;
                dll[t][c] = -aa * sa;
              } else if (v[c] == 255) {
                const float bb = __fmul_rn(__fsub_rn(edge_f(255), mc), inv);
                const float sb = 1.f / (1.f + expf(-bb));
                dlm[t][c] = inv * sb;
                dll[t][c] = bb * sb;
              } else {
                const float aa = __fmul_rn(__fsub_rn(edge_f(v[c] + 1), mc), inv);
                const float bb = __fmul_rn(__fsub_rn(edge_f(v[c]), mc), inv);
                const float dd = __fmul_rn(__fdiv_rn(2.f, 255.f), inv);
                const float gk = 1.f / expm1f(dd);
                const float sa = 1.f / (1.f + expf(aa)), sb = 1.f / (1.f + expf(-bb));
                dlm[t][c] = -inv * (sa - sb);
                dll[t][c] = -aa * sa + bb * sb - gk * dd;
              }
            }
            l[t] = lk;
          }
        }
        mx = -INFINITY;
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++) mx = fmaxf(mx, l[t]);
        red[part * kTTM + row] = mx;
        __syncthreads();
        mx = fmaxf(fmaxf(red[row], red[kTTM + row]), fmaxf(red[2 * kTTM + row], red[3 * kTTM + row]));
        __syncthreads();
        se = 0.f;
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++)
          if (part + 4 * t < K) se = __fadd_rn(se, expf(__fsub_rn(l[t], mx)));
        red[part * kTTM + row] = se;
        __syncthreads();
        se = __fadd_rn(__fadd_rn(red[row], red[kTTM + row]), __fadd_rn(red[2 * kTTM + row], red[3 * kTTM + row]));
        const float lse = __fadd_rn(mx, logf(se));
        if (valid && part == 0) loss = __fadd_rn(loss, -lse);
        const float sc = valid ? scale : 0.f;
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++) {
          const int k = part + 4 * t;
          if (k < K) {
            const float rho = valid ? expf(__fsub_rn(l[t], lse)) : 0.f;
            const float pi = expf(__fsub_rn(Pr[t][0], lse_pi));
            float gk[10];
            gk[0] = sc * (pi - rho);
            const float dmR = -rho * dlm[t][0], dmG = -rho * dlm[t][1], dmB = -rho * dlm[t][2];
            gk[1] = sc * dmR;
            gk[2] = sc * dmG;
            gk[3] = sc * dmB;
#pragma unroll
            for (int c = 0; c < 3; c++) gk[4 + c] = Pr[t][4 + c] > -7.f ? sc * (-rho * dll[t][c]) : 0.f;
            gk[7] = sc * dmG * xr * (1.f - co[t][0] * co[t][0]);
            gk[8] = sc * dmB * xr * (1.f - co[t][1] * co[t][1]);
            gk[9] = sc * dmB * xg * (1.f - co[t][2] * co[t][2]);
#pragma unroll
            for (int g = 0; g < 10; g++)
              DP[umma_off(row, g * K + k, NOp)] = __bfloat16_as_ushort(__float2bfloat16_rn(gk[g]));
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < kCompPerThread; t++) {
          const int k = part + 4 * t;
          if (k < K) {
#pragma unroll
            for (int g = 0; g < 10; g++) {
              const float gv = valid ? dparams[q * NO + g * K + k] : 0.f;
              DP[umma_off(row, g * K + k, NOp)] = __bfloat16_as_ushort(__float2bfloat16_rn(gv));
            }
          }
        }
      }
      if (part == 0)
        for (int c = NO; c < NOp; c++) DP[umma_off(row, c, NOp)] = 0;
    }
    sync_for_mma();

    // ---------------- adjoint ----------------
    // head: dH = dP WH, dWH = dP^T u_R, dbH = dP^T 1
    const uint32_t uoff = s0 + pl.u;
    if (threadIdx.x == 0) {
      tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, NOp), false, op_mn(s0 + pl.wh, C), true, C,
             NOp / 16, false);
      tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, NOp), true, op_mn(uoff + (2 * R) * tb, C), true, C,
             kTTM / 16, false);
      tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, NOp), true, SmOp{s0 + pl.ones, 128u, 256u, 0u},
             false, 16, kTTM / 16, false);
    }
    ok &= wait_mma();
    float ga[2][8];  // gradient of the residual stream (FP32)
    // g = acc * ELU'(act), act read from tile `act`; mode 0: ga = g (and G
    // = ga), 1: ga += g (G = ga), 2: G2 = g only
    auto bwd_epi = [&](const unsigned char* act, int mode, unsigned char* out) {
      uint32_t r[2][8];
#pragma unroll
      for (int i = 0; i < 2; i++)
        if (i < CH && part + 4 * i < C / 8) tmem_ld8_nw(tl + kColAcc + 8 * (part + 4 * i), r[i]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int c = part + 4 * i;
        if (i < CH && c < C / 8) {
          tmem_touch(r[i]);
          float u[8], o[8];
          tt_load8(act, C, row, c, u);
#pragma unroll
          for (int e = 0; e < 8; e++) {
            const float g = __fmul_rn(__uint_as_float(r[i][e]), elu_d_from_act(u[e]));
            if (mode == 0) ga[i][e] = g;
            if (mode == 1) ga[i][e] = __fadd_rn(ga[i][e], g);
            o[e] = mode == 2 ? g : ga[i][e];
          }
          tt_store8(out, C, row, c, o);
        }
      }
    };
    bwd_epi(U + (2 * R) * tb, 0, sm + pl.gx);
    tt_flush(tmem, NO, C, C, 1.f, gW + oWH, gW + obH);
    sync_for_mma();
    for (int r = R - 1; r >= 0 && ok; r--) {
      const size_t oW1 = oblk + r * blk, ob1 = oW1 + (size_t)C * C;
      const size_t oW2 = ob1 + C, ob2 = oW2 + (size_t)C * C;
      // dv = da W2, dW2 = da^T v_r, db2 = da^T 1  (da in G)
      if (threadIdx.x == 0) {
        tt_mma(tmem + kColAcc, op_k(s0 + pl.gx, C), false, op_mn(s0 + pl.w2[r], C), true, C,
               C / 16, false);
        tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, C), true, op_mn(uoff + (2 * r + 1) * tb, C), true,
               C, kTTM / 16, false);
        tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, C), true, SmOp{s0 + pl.ones, 128u, 256u, 0u},
               false, 16, kTTM / 16, false);
      }
      ok &= wait_mma();
      bwd_epi(U + (2 * r + 1) * tb, 2, sm + pl.g2);  // dz = dv * ELU'(z)
      tt_flush(tmem, C, C, C, 1.f, gW + oW2, gW + ob2);
      sync_for_mma();
      // du = dz W1, dW1 = dz^T u_r, db1 = dz^T 1  (dz in G2)
      if (threadIdx.x == 0) {
        tt_mma(tmem + kColAcc, op_k(s0 + pl.g2, C), false, op_mn(s0 + pl.w1[r], C), true, C,
               C / 16, false);
        tt_mma(tmem + kColDW, op_mn(s0 + pl.g2, C), true, op_mn(uoff + (2 * r) * tb, C), true, C,
               kTTM / 16, false);
        tt_mma(tmem + kColDB, op_mn(s0 + pl.g2, C), true, SmOp{s0 + pl.ones, 128u, 256u, 0u},
               false, 16, kTTM / 16, false);
      }
      ok &= wait_mma();
      bwd_epi(U + (2 * r) * tb, 1, sm + pl.gx);  // da_r = da_{r+1} + du * ELU'(a_r)
      tt_flush(tmem, C, C, C, 1.f, gW + oW1, gW + ob1);
      sync_for_mma();
    }
    if (!ok) break;
    // first layer: dW0 = da_0^T X / 255 (X gathered again), db0 = da_0^T 1
    tt_gather(d, batch, H, W, n_px, q0, sm + pl.xe);
    sync_for_mma();
    if (threadIdx.x == 0) {
      tt_mma(tmem + kColDW, op_mn(s0 + pl.gx, C), true, op_mn(s0 + pl.xe, Fp), true, Fp,
             kTTM / 16, false);
      tt_mma(tmem + kColDB, op_mn(s0 + pl.gx, C), true, SmOp{s0 + pl.ones, 128u, 256u, 0u}, false,
             16, kTTM / 16, false);
    }
    ok &= wait_mma();
    tt_flush(tmem, C, F, F, 1.f / 255.f, gW, gW + ob0);
    sync_for_mma();
  }
  if (!ok && threadIdx.x == 0) set_status(status, ST_TIMEOUT);
  // per-CTA loss (nats), fixed order over the 128 row owners
  if (MODE == 0) {
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
  float* part_g = reinterpret_cast<float*>(ws);
  float* part_l = part_g + (size_t)g * n_w;
  if (dparams)
    tc_train_kernel<1><<<g, kTT, pl.end, s>>>(d, umma, bias, batch, N, H, W, dparams, part_g,
                                              part_l, n_w, status);
  else
    tc_train_kernel<0><<<g, kTT, pl.end, s>>>(d, umma, bias, batch, N, H, W, nullptr, part_g,
                                              part_l, n_w, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_grad(part_g, dparams ? nullptr : part_l, g, n_w, n_px, grad, loss, s);
}

}  // namespace nlc
